import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="session")
def orthogonal_grid():
    """The hand-derived closed-form case in golden/orthogonal_grid.json:
    uniform samples over whole cycles, so every harmonic product averages to
    zero and P, |theta1|, theta3 and the phase relation follow exactly."""
    import json

    import numpy as np

    with open(os.path.join(GOLDEN, "orthogonal_grid.json")) as fh:
        g = json.load(fh)
    N, T, sig = g["N"], g["T"], g["signal"]
    t = np.arange(N) * T / N
    y = sig["a"] * np.cos(2.0 * np.pi * sig["k_sig"] * t / T + sig["phi0"]) + sig["b"]
    dy = np.full(N, g["dy"])
    c = np.array(g["template"]["c"])
    s = np.array(g["template"]["s"])
    k0, nf = g["grid"]["k0"], g["grid"]["nf"]
    return dict(g=g, t=t, y=y, dy=dy, c=c, s=s, df=1.0 / T, k0=k0, nf=nf,
                freqs=(k0 + np.arange(nf)) / T, psi=np.arctan2(s, c), phi0=sig["phi0"])


def check_orthogonal_grid(case, res, tol_p, tol_amp, tol_phase):
    """Compare one template's outputs (arrays over the case's frequencies)
    with the closed form: P everywhere; |theta1|, theta3 and
    h theta2 + psi_h + phi0 = 0 (theta1 > 0) or pi (theta1 < 0), mod 2 pi,
    where a harmonic matches the signal."""
    import numpy as np

    for e in case["g"]["expected"]:
        q = e["k"] - case["k0"]
        assert abs(res["power"][q] - e["P"]) <= tol_p, (e["k"], res["power"][q], e["P"])
        if e["h"] is None:
            continue
        h = e["h"]
        th1 = res["theta1"][q]
        assert abs(abs(th1) - e["abs_theta1"]) <= tol_amp, (e["k"], th1)
        assert abs(res["theta3"][q] - e["theta3"]) <= tol_amp, (e["k"], res["theta3"][q])
        target = 0.0 if th1 > 0 else np.pi
        rel = h * res["theta2"][q] + case["psi"][h - 1] + case["phi0"] - target
        assert abs(np.angle(np.exp(1j * rel))) <= h * tol_phase, (e["k"], res["theta2"][q])


def shared_orthogonal_case():
    """tests/golden/shared_phase_orthogonal.json: two bands, each sampled
    uniformly over whole cycles, with the closed-form power, amplitude, offset
    and phase of the shared-phase fit at every trial frequency (derivation in
    the file)."""
    import json
    import math

    import numpy as np

    with open(os.path.join(GOLDEN, "shared_phase_orthogonal.json")) as fh:
        g = json.load(fh)
    T, ks, d = g["T"], g["k_sig"], g["d"]
    bands, lam, share = [], [], []
    for b in g["bands"]:
        t = b["t_start"] + np.arange(b["N"]) * T / b["N"]
        y = b["a"] * np.cos(2.0 * np.pi * ks * t / T + b["phi"]) + b["lambda"] + d
        bands.append((t, y, np.full(b["N"], b["dy"]), np.array(b["c"]), np.array(b["s"])))
        lam.append(b["lambda"])
        share.append(b["N"] / b["dy"] ** 2)
    W = np.array(share) / np.sum(share)
    YY = sum(W[i] * b["a"] ** 2 / 2 for i, b in enumerate(g["bands"]))
    MM = sum(W[i] * np.sum(np.array(b["c"]) ** 2 + np.array(b["s"]) ** 2) / 2
             for i, b in enumerate(g["bands"]))
    ks_grid = g["grid"]["k0"] + np.arange(g["grid"]["nf"])
    expect = []
    for k in ks_grid:
        h = ks // k if ks % k == 0 else 0
        Z = 0j
        matched = False
        for i, b in enumerate(g["bands"]):
            if 1 <= h <= len(b["c"]):
                matched = True
                A = math.hypot(b["c"][h - 1], b["s"][h - 1])
                psi = math.atan2(b["s"][h - 1], b["c"][h - 1])
                Z += W[i] * b["a"] * A * np.exp(1j * (psi + b["phi"])) / 2
        h = h if matched else 0
        expect.append(dict(h=h, P=abs(Z) ** 2 / (YY * MM), abs_theta1=abs(Z) / MM,
                           theta3=d, argZ=np.angle(Z)))
    return bands, np.array(lam), ks_grid / T, expect


def check_shared_orthogonal(expect, res, tol_p, tol_amp, tol_phase):
    """Compare shared-phase outputs with the closed form of
    shared_orthogonal_case: P everywhere; |theta1|, theta3 and
    h theta2 + arg Z = 0 (theta1 > 0) or pi (theta1 < 0), mod 2 pi, where a
    harmonic matches."""
    import numpy as np

    for q, e in enumerate(expect):
        assert abs(res["power"][q] - e["P"]) <= tol_p, (q, res["power"][q], e["P"])
        if e["h"] == 0:
            continue
        th1 = res["theta1"][q]
        assert abs(abs(th1) - e["abs_theta1"]) <= tol_amp, (q, th1)
        assert abs(res["theta3"][q] - e["theta3"]) <= tol_amp, (q, res["theta3"][q])
        rel = e["h"] * res["theta2"][q] + e["argZ"] - (0.0 if th1 > 0 else np.pi)
        assert abs(np.angle(np.exp(1j * rel))) <= e["h"] * tol_phase, (q, res["theta2"][q])


def multiphase_orthogonal_expect():
    """The multi-phase reading of the same two bands (derivation_multiphase
    in shared_phase_orthogonal.json): per-band closed-form powers P_b [K][nf]
    and the chi2_0-weighted combination P [nf]."""
    import json
    import math

    import numpy as np

    with open(os.path.join(GOLDEN, "shared_phase_orthogonal.json")) as fh:
        g = json.load(fh)
    ks = g["k_sig"]
    ks_grid = g["grid"]["k0"] + np.arange(g["grid"]["nf"])
    Pb = np.zeros((len(g["bands"]), ks_grid.size))
    chi0 = np.array([b["N"] / b["dy"] ** 2 * b["a"] ** 2 / 2 for b in g["bands"]])
    for i, b in enumerate(g["bands"]):
        A2 = np.array(b["c"]) ** 2 + np.array(b["s"]) ** 2
        for q, k in enumerate(ks_grid):
            h = ks // k if ks % k == 0 else 0
            if 1 <= h <= len(b["c"]):
                Pb[i, q] = A2[h - 1] / A2.sum()
    return Pb, (chi0[:, None] * Pb).sum(axis=0) / chi0.sum()
