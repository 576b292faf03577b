"""Plain FP64 CPU oracle for the Fast Template Periodogram (FTP).

TEST INFRASTRUCTURE ONLY.  This module is imported by the tests, by
``__graft_entry__.smoke()`` and by the benchmark's CPU-baseline leg, and by
nothing else.  It shares no code with the CUDA library: it computes the
trigonometric sums directly (O(N) per harmonic and frequency, no NFFT), builds
the polynomials exactly as Section 2 writes them, finds the zeros with
``numpy.polynomial.polynomial.polyroots`` (companion-matrix eigenvalues, the
routine Section 2 names) and evaluates the power at every normalised root
directly from the data.

Notation follows Section 2: weights w_i (sum w = 1), ybar = <y>,
YY = Var(y); template M(x) = sum_n c_n cos nx + s_n sin nx; model
y ~ theta1 * M(omega t - theta2) + theta3; alpha_n = (c_n + i s_n)/2;
psi = exp(i theta2); YM' = psi^H YM, MM' = psi^{2H} MM.

Readings of the paper taken here (the paper is silent or inconsistent):
  * The final polynomial 2 MM' d(YM') - YM' d(MM') has degree 6H-2, not
    6H-1 as Section 2.3 states: the psi^{6H-1} coefficient is identically zero
    ((2l - j) = 0 for j = 4H, l = 2H).  It is dropped after checking it is ~0.
  * P is evaluated at *all* 6H-2 roots after scaling them onto the unit circle
    (Section 2, end): a superset of the true stationary points; extra
    candidates are real phases and cannot raise the maximum above the truth.
  * Ties (within rel_tie * Pmax of the maximum): prefer theta1 > 0, then the
    smallest theta2 in [0, 2 pi).
  * MM <= 1e-14 * <M^2> at a candidate: that candidate has P = 0 and the
    frequency is flagged degenerate.
  * A vanishing final polynomial (|F| <= 1e-14 * scale) means P(theta2) is
    constant; the single candidate theta2 = 0 is used.
  * Weights: all sigma = 0 -> unit weights; a mix of zero and non-zero
    sigma, a negative or non-finite sigma, Var(y) = 0 or N < 2 are errors.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import polynomial as npoly

TWO_PI = 2.0 * math.pi

FLAG_NONCONVERGED = 1   # root solver hit its iteration cap (never set here)
FLAG_DEGENERATE_MM = 2  # MM ~ 0 at the chosen candidate
FLAG_CONSTANT_P = 4     # final polynomial vanishes: P independent of theta2
FLAG_NEGATIVE_AMP = 8   # best fit has theta1 < 0 (Section 2.1: allowed, reported)
FLAG_NO_POSITIVE = 64   # positive-amplitude mode: no candidate with theta1 > 0, P = 0


class OracleInputError(ValueError):
    """Invalid input per Section 2 (sigma and variance rules)."""


# ---------------------------------------------------------------------------
# Weights, weighted mean and variance (Eq. lsp and the paragraph after the
# chi^2 conditions in Section 2).
# ---------------------------------------------------------------------------
def normalized_weights(dy) -> np.ndarray:
    """w_i proportional to sigma_i^-2 with sum w = 1.

    All sigma_i = 0 -> uniform weights (Section 2).  Mixed zero / non-zero
    sigma is not considered by the paper and is rejected, as is sigma < 0 or a
    non-finite sigma."""
    dy = np.asarray(dy, dtype=np.float64)
    if dy.size < 2:
        raise OracleInputError("need at least two observations")
    if not np.all(np.isfinite(dy)) or np.any(dy < 0):
        raise OracleInputError("uncertainties must be finite and >= 0")
    if np.all(dy == 0):
        w = np.ones_like(dy)
    elif np.any(dy == 0):
        raise OracleInputError("mixed zero and non-zero uncertainties")
    else:
        w = dy ** -2.0
    return w / np.sum(w)


def data_moments(y, w):
    """ybar = <y> and YY = chi^2_0 = <(y - ybar)^2> (Eq. lsp and below)."""
    y = np.asarray(y, dtype=np.float64)
    if not np.all(np.isfinite(y)):
        raise OracleInputError("values must be finite")
    # Var(y) = 0 exactly when every value is equal (all weights are > 0).
    if np.min(y) == np.max(y):
        raise OracleInputError("zero variance: the periodogram is undefined")
    ybar = float(np.dot(w, y))
    YY = float(np.dot(w, (y - ybar) ** 2))
    return ybar, YY


def harmonic_phases(t, freq: float, H: int) -> np.ndarray:
    """Phases n * omega * t_i for n = 1..H, shape [H, N].  The product n f t is
    reduced modulo one cycle in FP64 before scaling by 2 pi."""
    t = np.asarray(t, dtype=np.float64)
    n = np.arange(1, H + 1, dtype=np.float64)[:, None]
    cyc = n * freq * t[None, :]
    return TWO_PI * (cyc - np.floor(cyc))


# ---------------------------------------------------------------------------
# Step (a): the trigonometric sums, Eqs. CCdef - YSdef, evaluated directly.
# ---------------------------------------------------------------------------
def direct_sums(t, y, w, ybar: float, freq: float, H: int) -> dict:
    """CC_nm, CS_nm, SS_nm = weighted covariances of cos(n wt), sin(m wt);
    YC_n, YS_n = <(y - ybar) cos(n wt)>, <(y - ybar) sin(n wt)>, n, m = 1..H.
    Also C_n = <cos n wt>, S_n = <sin n wt>."""
    ph = harmonic_phases(t, freq, H)
    cos, sin = np.cos(ph), np.sin(ph)
    C = cos @ w
    S = sin @ w
    CC = (cos * w) @ cos.T - np.outer(C, C)
    CS = (cos * w) @ sin.T - np.outer(C, S)
    SS = (sin * w) @ sin.T - np.outer(S, S)
    r = w * (np.asarray(y, dtype=np.float64) - ybar)
    YC = cos @ r
    YS = sin @ r
    return dict(C=C, S=S, CC=CC, CS=CS, SS=SS, YC=YC, YS=YS)


# ---------------------------------------------------------------------------
# Step (b): polynomial assembly (Section 2, MM_nm and YM_k, then Eq. finalpoly).
# ---------------------------------------------------------------------------
def template_alpha(c, s) -> np.ndarray:
    """alpha_n = (c_n + i s_n) / 2."""
    return (np.asarray(c, dtype=np.float64) + 1j * np.asarray(s, dtype=np.float64)) / 2.0


def mm_poly(alpha, CC, CS, SS) -> np.ndarray:
    """Coefficients of MM' = psi^{2H} MM, lowest power first (4H+1 entries).

    MM_nm = alpha_n alpha_m CCt_nm psi^{n+m} + 2 alpha_n alpha*_m CSt_nm psi^{n-m}
            + alpha*_n alpha*_m SSt_nm psi^{-(n+m)}, with
    CCt = (CC - SS) - i (CS + CS^T), CSt = (CC + SS) + i (CS - CS^T),
    SSt = (CC - SS) + i (CS + CS^T)."""
    H = alpha.shape[0]
    CCt = (CC - SS) - 1j * (CS + CS.T)
    CSt = (CC + SS) + 1j * (CS - CS.T)
    SSt = (CC - SS) + 1j * (CS + CS.T)
    out = np.zeros(4 * H + 1, dtype=np.complex128)
    for n in range(1, H + 1):
        an = alpha[n - 1]
        for m in range(1, H + 1):
            am = alpha[m - 1]
            out[2 * H + n + m] += an * am * CCt[n - 1, m - 1]
            out[2 * H + n - m] += 2.0 * an * np.conj(am) * CSt[n - 1, m - 1]
            out[2 * H - n - m] += np.conj(an) * np.conj(am) * SSt[n - 1, m - 1]
    return out


def ym_poly(alpha, YC, YS) -> np.ndarray:
    """Coefficients of YM' = psi^H YM (2H+1 entries):
    YM = sum_k alpha_k YCt_k psi^k + alpha*_k YCt*_k psi^{-k}, YCt = YC - i YS."""
    H = alpha.shape[0]
    YCt = YC - 1j * YS
    out = np.zeros(2 * H + 1, dtype=np.complex128)
    for k in range(1, H + 1):
        out[H + k] += alpha[k - 1] * YCt[k - 1]
        out[H - k] += np.conj(alpha[k - 1]) * np.conj(YCt[k - 1])
    return out


def final_poly(MMp, YMp):
    """F = 2 MM' d(YM') - YM' d(MM') (Eq. finalpoly), derivatives in psi.

    Returns (F with the identically-zero psi^{6H-1} term removed, that term)."""
    F = 2.0 * npoly.polymul(MMp, npoly.polyder(YMp)) - npoly.polymul(YMp, npoly.polyder(MMp))
    H = (len(YMp) - 1) // 2
    full = np.zeros(6 * H, dtype=np.complex128)
    full[: len(F)] = F
    return full[: 6 * H - 1], full[6 * H - 1]


# ---------------------------------------------------------------------------
# Step (c): roots, normalisation onto the unit circle, candidate evaluation.
# ---------------------------------------------------------------------------
def candidate_phases(F) -> np.ndarray:
    """Zeros of F by companion-matrix eigenvalues, scaled by their modulus onto
    the unit circle (Section 2, end), returned as theta2 in [0, 2 pi).

    A vanishing F (P independent of theta2) yields the single candidate 0."""
    scale = np.max(np.abs(F)) if len(F) else 0.0
    if scale == 0.0:
        return np.zeros(1)
    Fn = F / scale
    nz = np.flatnonzero(np.abs(Fn) > 1e-14)
    if nz.size == 0 or nz[-1] == 0:
        return np.zeros(1)
    roots = npoly.polyroots(Fn[: nz[-1] + 1])
    roots = roots[np.abs(roots) > 0]
    psi = roots / np.abs(roots)
    return np.mod(np.angle(psi), TWO_PI)


def fit_at_phase(t, y, w, ybar: float, YY: float, freq: float, c, s, theta2):
    """Closed-form optimum at fixed theta2, evaluated directly from the data
    (Section 2): M_i = M(omega t_i - theta2); MM = Var(M); YM = Cov(M, y);
    P = YM^2/(YY MM); theta1 = YM/MM; theta3 = ybar - theta1 <M>.

    theta2 may be an array; returns arrays (P, theta1, theta3, degenerate)."""
    theta2 = np.atleast_1d(np.asarray(theta2, dtype=np.float64))
    H = len(c)
    ph = harmonic_phases(t, freq, H)                        # [H, N]
    n = np.arange(1, H + 1, dtype=np.float64)[:, None, None]
    x = ph[:, None, :] - n * theta2[None, :, None]          # [H, K, N]
    M = np.tensordot(np.asarray(c, float), np.cos(x), axes=(0, 0)) + \
        np.tensordot(np.asarray(s, float), np.sin(x), axes=(0, 0))  # [K, N]
    Mbar = M @ w
    MMhat = (M * M) @ w
    MM = MMhat - Mbar ** 2
    YM = M @ (w * (np.asarray(y, float) - ybar))
    degenerate = ~(MM > 1e-14 * MMhat)
    safe = np.where(degenerate, 1.0, MM)
    P = np.where(degenerate, 0.0, YM * YM / (YY * safe))
    theta1 = np.where(degenerate, 0.0, YM / safe)
    theta3 = ybar - theta1 * Mbar
    return P, theta1, theta3, degenerate


def choose_best(P, theta1, theta2, rel_tie: float = 1e-12) -> int:
    """Index of the best candidate: maximal P; among candidates within
    rel_tie * Pmax of it prefer theta1 > 0, then the smallest theta2."""
    Pmax = np.max(P)
    near = np.flatnonzero(P >= Pmax - rel_tie * max(Pmax, 1e-300))
    pos = near[theta1[near] > 0]
    pool = pos if pos.size else near
    return int(pool[np.argmin(theta2[pool])])


def polynomials_at(t, y, dy, freq: float, c, s):
    """MM', YM' and F for one frequency (steps a-b), plus ybar, YY."""
    w = normalized_weights(dy)
    ybar, YY = data_moments(y, w)
    H = len(c)
    sm = direct_sums(t, y, w, ybar, freq, H)
    alpha = template_alpha(c, s)
    MMp = mm_poly(alpha, sm["CC"], sm["CS"], sm["SS"])
    YMp = ym_poly(alpha, sm["YC"], sm["YS"])
    F, top = final_poly(MMp, YMp)
    return dict(MMp=MMp, YMp=YMp, F=F, top=top, ybar=ybar, YY=YY, w=w, sums=sm)


def periodogram(t, y, dy, freqs, c, s, rel_tie: float = 1e-12, positive_only: bool = False):
    """FTP at each trial frequency (cycles per unit time).

    positive_only: the template amplitude is constrained to theta1 >= 0
    (Section 2.1 leaves the choice to the user).  At fixed theta2 the best
    theta1 >= 0 is YM/MM when YM > 0 and 0 otherwise (P = 0), so the
    constrained power is P(theta2) [YM(theta2) > 0]; P vanishes where YM does,
    so on each arc with YM > 0 its maximum is an interior stationary point - a
    candidate of the polynomial.  The best candidate with theta1 > 0 is
    therefore the constrained optimum; with none, P = 0, theta1 = 0,
    theta2 = 0, theta3 = ybar and FLAG_NO_POSITIVE is set.

    Returns dict of float64 arrays power, theta1, theta2, theta3 and uint8
    flags, all of shape [len(freqs)]."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if not np.all(np.isfinite(t)):
        raise OracleInputError("times must be finite")
    w = normalized_weights(dy)
    ybar, YY = data_moments(y, w)
    c = np.asarray(c, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    H = len(c)
    alpha = template_alpha(c, s)
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    nf = freqs.shape[0]
    out = {k: np.zeros(nf) for k in ("power", "theta1", "theta2", "theta3")}
    out["flags"] = np.zeros(nf, dtype=np.uint8)
    for k in range(nf):
        f = freqs[k]
        sm = direct_sums(t, y, w, ybar, f, H)
        MMp = mm_poly(alpha, sm["CC"], sm["CS"], sm["SS"])
        YMp = ym_poly(alpha, sm["YC"], sm["YS"])
        F, _ = final_poly(MMp, YMp)
        flag = 0
        if np.max(np.abs(F)) <= 1e-14 * max(np.max(np.abs(MMp)) * np.max(np.abs(YMp)), 1e-300) * H:
            th2 = np.zeros(1)
            flag |= FLAG_CONSTANT_P
        else:
            th2 = candidate_phases(F)
        P, th1, th3, deg = fit_at_phase(t, y, w, ybar, YY, f, c, s, th2)
        if positive_only:
            keep = th1 > 0
            if not np.any(keep):
                out["theta3"][k] = ybar
                out["flags"][k] = flag | FLAG_NO_POSITIVE
                continue
            P, th1, th2, th3, deg = P[keep], th1[keep], th2[keep], th3[keep], deg[keep]
        b = choose_best(P, th1, th2, rel_tie)
        if deg[b]:
            flag |= FLAG_DEGENERATE_MM
        if th1[b] < 0:
            flag |= FLAG_NEGATIVE_AMP
        out["power"][k] = P[b]
        out["theta1"][k] = th1[b]
        out["theta2"][k] = th2[b]
        out["theta3"][k] = th3[b]
        out["flags"][k] = flag
    return out


def best_candidate_margin(t, y, dy, freq: float, c, s, theta2_best: float,
                          sep: float = 0.05, rel_tie: float = 1e-9) -> float:
    """P(best) minus the best P among candidates more than `sep` rad away
    (mod 2 pi): used to decide whether the optimum is well separated, in which
    case the best phase is unique and comparable across implementations.

    A far candidate that ties with the best (within rel_tie * P) but has the
    opposite amplitude sign is resolved by the tie rule (theta1 > 0 first) and
    does not count: e.g. templates with only odd harmonics, where theta2 and
    theta2 + pi give the same P with opposite theta1."""
    pol = polynomials_at(t, y, dy, freq, c, s)
    th2 = candidate_phases(pol["F"])
    P, th1, _, _ = fit_at_phase(t, y, pol["w"], pol["ybar"], pol["YY"], freq, c, s, th2)
    d = np.abs(np.angle(np.exp(1j * (th2 - theta2_best))))
    Pb, th1b, _, _ = fit_at_phase(t, y, pol["w"], pol["ybar"], pol["YY"], freq, c, s,
                                  np.array([theta2_best]))
    Pbest = Pb[0]
    twin = (np.sign(th1) != np.sign(th1b[0])) & (np.abs(P - Pbest) <= rel_tie * max(Pbest, 1e-300))
    far = P[(d > sep) & ~twin]
    return float(Pbest - (far.max() if far.size else 0.0))


# ---------------------------------------------------------------------------
# Multi-band, multi-phase model (Section 2.2, Eq. multibandmultiphase)
# ---------------------------------------------------------------------------
def chi2_0(y, dy) -> float:
    """Weighted sum of squared residuals about the weighted mean, with the
    raw weights sigma^-2 (unit weights when every sigma is zero)."""
    y = np.asarray(y, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    wr = np.ones_like(dy) if np.all(dy == 0) else dy ** -2.0
    ybar = np.sum(wr * y) / np.sum(wr)
    return float(np.sum(wr * (y - ybar) ** 2))


def multiband_periodogram(bands, freqs, rel_tie: float = 1e-12):
    """Multi-phase multi-band template periodogram: every band k has its own
    amplitude, phase and offset (and template) at a shared frequency, and
    P = sum_k chi2_0,k P_k / sum_k chi2_0,k (Eq. multibandmultiphase).

    bands: sequence of (t, y, dy, c, s).  Returns dict(power [nf],
    band_power [K][nf], chi2_0 [K], bands: the per-band periodogram dicts)."""
    per = [periodogram(t, y, dy, freqs, c, s, rel_tie) for (t, y, dy, c, s) in bands]
    w = np.array([chi2_0(y, dy) for (_, y, dy, _, _) in bands])
    bp = np.array([p["power"] for p in per])
    return dict(power=(w[:, None] * bp).sum(axis=0) / w.sum(), band_power=bp, chi2_0=w,
                bands=per)


# ---------------------------------------------------------------------------
# Shared-phase multi-band template (Appendix A)
# ---------------------------------------------------------------------------
def shared_phase_multiband(bands, freqs, offsets=None, rel_tie: float = 1e-12):
    """Multi-band model with one amplitude, phase and offset shared by every
    band and a template per band (Appendix A):
        y_i^(k) ~ theta1 M^(k)(omega t_i - theta2) + theta3 + lambda_k,
    the fixed band offsets lambda_k subtracted from the data first.  Weights
    are normalised over all observations (sum_k W_k = 1, W_k the band's share).
    The polynomials pool the single-band ones:
        MM' = sum_k W_k <M^(k)2>' - (sum_k W_k Mbar^(k)')^2,
        YM' = sum_k W_k YM^(k)' with y centred on the pooled mean,
    and the candidates are evaluated directly from the pooled data.

    bands: sequence of (t, y, dy, c, s); templates shorter than the longest
    are padded with zero harmonics.  Returns dict of power, theta1, theta2,
    theta3, flags (as periodogram)."""
    K = len(bands)
    H = max(len(b[3]) for b in bands)
    lam = np.zeros(K) if offsets is None else np.asarray(offsets, dtype=np.float64)
    tb, yb, cb, sb, kb = [], [], [], [], []
    for k, (t, y, dy, c, s) in enumerate(bands):
        tb.append(np.asarray(t, dtype=np.float64))
        yb.append(np.asarray(y, dtype=np.float64) - lam[k])
        cp = np.zeros(H)
        sp = np.zeros(H)
        cp[:len(c)] = c
        sp[:len(s)] = s
        cb.append(cp)
        sb.append(sp)
        kb.append(np.full(len(t), k))
    t_all = np.concatenate(tb)
    y_all = np.concatenate(yb)
    k_all = np.concatenate(kb)
    w = normalized_weights(np.concatenate([np.asarray(b[2], dtype=np.float64) for b in bands]))
    ybar, YY = data_moments(y_all, w)
    Wk = np.array([w[k_all == k].sum() for k in range(K)])
    alphas = [template_alpha(cb[k], sb[k]) for k in range(K)]
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    out = {n: np.zeros(freqs.size) for n in ("power", "theta1", "theta2", "theta3")}
    out["flags"] = np.zeros(freqs.size, dtype=np.uint8)

    def fit(f, th2):
        th2 = np.atleast_1d(th2)
        M = np.zeros((th2.size, t_all.size))
        for k in range(K):
            sel = k_all == k
            ph = harmonic_phases(t_all[sel], f, H)
            n = np.arange(1, H + 1, dtype=np.float64)[:, None, None]
            x = ph[:, None, :] - n * th2[None, :, None]
            M[:, sel] = np.tensordot(cb[k], np.cos(x), axes=(0, 0)) + \
                np.tensordot(sb[k], np.sin(x), axes=(0, 0))
        Mbar = M @ w
        MMhat = (M * M) @ w
        MM = MMhat - Mbar ** 2
        YMv = M @ (w * (y_all - ybar))
        deg = ~(MM > 1e-14 * MMhat)
        safe = np.where(deg, 1.0, MM)
        P = np.where(deg, 0.0, YMv * YMv / (YY * safe))
        th1 = np.where(deg, 0.0, YMv / safe)
        return P, th1, ybar - th1 * Mbar, deg

    for q, f in enumerate(freqs):
        MMhat = np.zeros(4 * H + 1, dtype=np.complex128)
        Mbar = np.zeros(2 * H + 1, dtype=np.complex128)
        YMp = np.zeros(2 * H + 1, dtype=np.complex128)
        for k in range(K):
            sel = k_all == k
            sm = direct_sums(t_all[sel], y_all[sel], w[sel] / Wk[k], ybar, f, H)
            C, S = sm["C"], sm["S"]
            MMhat += Wk[k] * mm_poly(alphas[k], sm["CC"] + np.outer(C, C),
                                     sm["CS"] + np.outer(C, S), sm["SS"] + np.outer(S, S))
            Mbar += Wk[k] * ym_poly(alphas[k], C, S)
            YMp += Wk[k] * ym_poly(alphas[k], sm["YC"], sm["YS"])
        MMp = MMhat - npoly.polymul(Mbar, Mbar)
        F, _ = final_poly(MMp, YMp)
        flag = 0
        if np.max(np.abs(F)) <= 1e-14 * max(np.max(np.abs(MMp)) * np.max(np.abs(YMp)), 1e-300) * H:
            th2 = np.zeros(1)
            flag |= FLAG_CONSTANT_P
        else:
            th2 = candidate_phases(F)
        P, th1, th3, deg = fit(f, th2)
        b = choose_best(P, th1, th2, rel_tie)
        if deg[b]:
            flag |= FLAG_DEGENERATE_MM
        if th1[b] < 0:
            flag |= FLAG_NEGATIVE_AMP
        out["power"][q], out["theta1"][q] = P[b], th1[b]
        out["theta2"][q], out["theta3"][q] = th2[b], th3[b]
        out["flags"][q] = flag
    return out
