"""Seeded synthetic lightcurves and templates for the Fast Template Periodogram.

These generators produce *inputs only*: observation times, values,
uncertainties, template Fourier coefficients and frequency grids.  They hold
none of the periodogram's arithmetic, so the CPU oracle and the CUDA library
can both be fed from them without sharing any of the method's code.

The shapes follow the paper's simulated workloads (Section 3: uniformly random
observation times, Gaussian uncorrelated uncertainties, a template given by a
truncated Fourier series of H harmonics, Section 2 first equation) and the five
workload recipes listed below.  Template coefficients are drawn as
a_h, b_h ~ N(0, 1)/h^2 and scaled to unit variance over phase,
(1/2) * sum_h (a_h^2 + b_h^2) = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Template:
    """Truncated Fourier template M(x) = sum_{n=1..H} c_n cos(n x) + s_n sin(n x)."""

    c: np.ndarray  # float64[H], coefficient of cos(n x), n = 1..H
    s: np.ndarray  # float64[H], coefficient of sin(n x)

    @property
    def H(self) -> int:
        return int(self.c.shape[0])

    def __call__(self, x: np.ndarray) -> np.ndarray:
        """Evaluate the series at phases x (radians).  Used only to synthesise
        signals, never by the periodogram itself."""
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        for n in range(1, self.H + 1):
            out += self.c[n - 1] * np.cos(n * x) + self.s[n - 1] * np.sin(n * x)
        return out


@dataclasses.dataclass
class Grid:
    """Trial frequencies f_k = (k0 + k) * df, k = 0..nf-1 (cycles per unit time)."""

    df: float
    k0: int
    nf: int

    def freqs(self) -> np.ndarray:
        return (self.k0 + np.arange(self.nf, dtype=np.float64)) * self.df


@dataclasses.dataclass
class Lightcurve:
    t: np.ndarray
    y: np.ndarray
    dy: np.ndarray


def make_template(H: int, seed: int) -> Template:
    """Template with a_h, b_h ~ N(0,1)/h^2, scaled so (1/2) sum(a^2+b^2) = 1."""
    rng = np.random.default_rng(seed)
    h = np.arange(1, H + 1, dtype=np.float64)
    a = rng.standard_normal(H) / h**2
    b = rng.standard_normal(H) / h**2
    scale = math.sqrt(0.5 * float(np.sum(a * a + b * b)))
    return Template(c=a / scale, s=b / scale)


def nightly_times(rng: np.random.Generator, nights: int, n_obs: int,
                  keep: float = 0.7, hours: float = 8.0) -> np.ndarray:
    """Times over `nights` nights: each night keeps an `hours`-long window with
    probability `keep`; n_obs times are drawn uniformly over the kept windows
    and sorted."""
    kept = np.flatnonzero(rng.random(nights) < keep).astype(np.float64)
    if kept.size == 0:
        kept = np.zeros(1)
    width = hours / 24.0
    night = rng.integers(0, kept.size, size=n_obs)
    t = kept[night] + width * rng.random(n_obs)
    return np.sort(t)


# --------------------------------------------------------------------------
# Workload 1: small single curve (N=200, H=3, 5000 frequencies)
# --------------------------------------------------------------------------
def small_curve(n_obs: int = 200, H: int = 3, nf: int = 5000, seed: int = 1001):
    """N=200 times uniform in [0, 30] d (sorted); y = 0.5*M(2 pi t/2.37 + 1.1)
    + N(0, sigma^2) with sigma ~ U(0.05, 0.15); grid f_k = k/150, k = 1..nf."""
    rng = np.random.default_rng(seed)
    tpl = make_template(H, 2000)
    t = np.sort(rng.uniform(0.0, 30.0, n_obs))
    dy = rng.uniform(0.05, 0.15, n_obs)
    y = 0.5 * tpl(2.0 * np.pi * t / 2.37 + 1.1) + dy * rng.standard_normal(n_obs)
    grid = Grid(df=1.0 / 150.0, k0=1, nf=nf)
    return Lightcurve(t, y, dy), tpl, grid


# --------------------------------------------------------------------------
# Workload 2: single long curve with nightly gaps (N=1e4, H=6, 2.5e5 freqs)
# --------------------------------------------------------------------------
def long_curve(n_obs: int = 10_000, H: int = 6, nf: int = 250_000, nights: int = 3000,
               seed: int = 1002):
    """3000 nights with 8 h windows, 30 % of nights dropped; N=1e4 sorted times;
    y = 0.1*M(2 pi t/0.63 - phi0) + N(0, 0.05^2); df = 1/(5*3000 d), k = 1..nf."""
    rng = np.random.default_rng(seed)
    tpl = make_template(H, 2000)
    t = nightly_times(rng, nights, n_obs)
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    dy = np.full(n_obs, 0.05)
    y = 0.1 * tpl(2.0 * np.pi * t / 0.63 - phi0) + 0.05 * rng.standard_normal(n_obs)
    grid = Grid(df=1.0 / (5.0 * nights), k0=1, nf=nf)
    return Lightcurve(t, y, dy), tpl, grid


# --------------------------------------------------------------------------
# Workload 5: template bank over one very long curve (N=1e5, 32 x H=10, 1e6 freqs)
# --------------------------------------------------------------------------
def bank_curve(n_obs: int = 100_000, H: int = 10, n_templates: int = 32, nf: int = 1_000_000,
               nights: int = 4000, seed: int = 1005):
    """As workload 2 but N=1e5 over 4000 nights, 32 seeded H=10 templates
    (seeds 2000+i), signal from template 0 at period 0.63 d; df = 1/(5*4000 d)."""
    rng = np.random.default_rng(seed)
    bank = [make_template(H, 2000 + i) for i in range(n_templates)]
    t = nightly_times(rng, nights, n_obs)
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    dy = np.full(n_obs, 0.05)
    y = 0.1 * bank[0](2.0 * np.pi * t / 0.63 - phi0) + 0.05 * rng.standard_normal(n_obs)
    grid = Grid(df=1.0 / (5.0 * nights), k0=1, nf=nf)
    return Lightcurve(t, y, dy), bank, grid


# --------------------------------------------------------------------------
# Workload 3: batched survey of many curves of uneven size
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Survey:
    obs_off: np.ndarray      # int64[ncurves+1]
    t: np.ndarray
    y: np.ndarray
    dy: np.ndarray
    grids: list              # list[Grid]
    bank: list               # list[Template]
    tpl_of_curve: np.ndarray  # int32[ncurves]
    injected: np.ndarray     # bool[ncurves]
    period: np.ndarray       # float64[ncurves] (nan if not injected)

    @property
    def ncurves(self) -> int:
        return int(self.obs_off.shape[0] - 1)

    def curve(self, c: int) -> Lightcurve:
        a, b = int(self.obs_off[c]), int(self.obs_off[c + 1])
        return Lightcurve(self.t[a:b], self.y[a:b], self.dy[a:b])


def survey(ncurves: int = 4096, n_bank: int = 16, median_obs: float = 1000.0,
           log_sigma: float = 1.0, min_obs: int = 50, max_obs: int = 20_000,
           f_max: float = 10.0, ofac: float = 5.0, baseline=(100.0, 3000.0),
           Hs=(2, 4, 6), seed: int = 1003) -> Survey:
    """N ~ lognormal(ln 1000, 1.0) clipped to [50, 20000]; baseline T ~ U(100,
    3000) d; t ~ U[0, T] sorted; sigma ~ U(0.05, 0.15); bank of 16 templates
    with H cycling through (2, 4, 6); curve c uses template c mod 16; even
    curves carry 0.5*M at a period log-uniform in [0.2, 50] d, odd curves are
    noise only; df = 1/(5T), f up to 10 /d (nf = floor(f_max/df))."""
    rng = np.random.default_rng(seed)
    bank = [make_template(Hs[i % len(Hs)], 2000 + i) for i in range(n_bank)]
    n = np.clip(np.round(rng.lognormal(np.log(median_obs), log_sigma, ncurves)),
                min_obs, max_obs).astype(np.int64)
    off = np.zeros(ncurves + 1, dtype=np.int64)
    off[1:] = np.cumsum(n)
    tot = int(off[-1])
    t = np.empty(tot)
    y = np.empty(tot)
    dy = np.empty(tot)
    grids = []
    tpl_of_curve = (np.arange(ncurves) % n_bank).astype(np.int32)
    injected = (np.arange(ncurves) % 2) == 0
    period = np.full(ncurves, np.nan)
    for c in range(ncurves):
        a, b = off[c], off[c + 1]
        T = rng.uniform(*baseline)
        tc = np.sort(rng.uniform(0.0, T, b - a))
        sc = rng.uniform(0.05, 0.15, b - a)
        yc = sc * rng.standard_normal(b - a)
        if injected[c]:
            P = float(np.exp(rng.uniform(np.log(0.2), np.log(50.0))))
            ph = rng.uniform(0.0, 2.0 * np.pi)
            yc = yc + 0.5 * bank[tpl_of_curve[c]](2.0 * np.pi * tc / P - ph)
            period[c] = P
        t[a:b], y[a:b], dy[a:b] = tc, yc, sc
        df = 1.0 / (ofac * T)
        grids.append(Grid(df=df, k0=1, nf=int(math.floor(f_max / df))))
    return Survey(off, t, y, dy, grids, bank, tpl_of_curve, injected, period)


def random_curve(rng: np.random.Generator, n_obs: int, T: float = 10.0,
                 signal: float = 0.0, tpl: Template | None = None, period: float = 1.3,
                 phase: float = 0.7, sigma=(0.05, 0.15), sort: bool = True) -> Lightcurve:
    """Small generic curve for tests: uniform times in [0, T], heteroscedastic
    Gaussian noise, optional injected template signal signal*M(2 pi t/period - phase)."""
    t = rng.uniform(0.0, T, n_obs)
    if sort:
        t = np.sort(t)
    dy = rng.uniform(sigma[0], sigma[1], n_obs)
    y = dy * rng.standard_normal(n_obs)
    if signal and tpl is not None:
        y = y + signal * tpl(2.0 * np.pi * t / period - phase)
    return Lightcurve(t, y, dy)
