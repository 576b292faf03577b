"""Pins of the screening oracle (features and network) to things other than
itself: the FTP oracle at H = 1, nesting of least-squares models, closed
forms, finite differences, and the BF16 conversion of an independent library.
Each planted-mistake test shows that a plausible error fails a pin."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import screen_oracle as so


def curve(seed=0, n=60, T=20.0, offset=3.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0, T, n))
    dy = rng.uniform(0.05, 0.2, n)
    y = offset + 0.8 * np.sin(2 * np.pi * t / 3.1 + 0.4) + dy * rng.standard_normal(n)
    return t, y, dy


# ------------------------------------------------------------------ features
def test_single_harmonic_power_is_ftp_with_a_pure_sinusoid_template():
    """FTP with the H = 1 template cos x is the floating-mean Lomb-Scargle
    periodogram (Section 2.1), reached by the polynomial route; the feature
    P_1 reaches it by a direct least-squares fit."""
    t, y, dy = curve(1)
    freqs = np.linspace(0.05, 2.0, 37)
    feat = so.screening_features(t, y, dy, freqs, 3)
    ftp = oracle.periodogram(t, y, dy, freqs, [1.0], [0.0])
    np.testing.assert_allclose(feat[:, 0], ftp["power"], atol=1e-10)


def test_harmonic_h_power_is_the_first_harmonic_at_h_times_the_frequency():
    t, y, dy = curve(2)
    freqs = np.linspace(0.05, 1.0, 11)
    f3 = so.screening_features(t, y, dy, freqs, 3)
    for h in (2, 3):
        f1 = so.screening_features(t, y, dy, h * freqs, 1)
        np.testing.assert_allclose(f3[:, h - 1], f1[:, 0], atol=1e-12)
        np.testing.assert_allclose(f3[:, 3 + h - 1], f1[:, 1], atol=1e-12)


def test_multiharmonic_power_bounds_ftp_and_reduces_to_one_harmonic():
    """The template model is the multi-harmonic model with tied amplitudes,
    so P_MHLS(H) >= P_FTP; with H = 1 both models are the same."""
    rng = np.random.default_rng(3)
    for seed in range(4):
        t, y, dy = curve(10 + seed, n=40)
        H = 1 + seed % 3
        tpl = synth.make_template(H, 500 + seed)
        freqs = rng.uniform(0.05, 2.0, 15)
        feat = so.screening_features(t, y, dy, freqs, H)
        ftp = oracle.periodogram(t, y, dy, freqs, tpl.c, tpl.s)
        assert np.all(feat[:, 2 * H] >= ftp["power"] - 1e-10)
        assert np.all(feat[:, 2 * H] >= feat[:, :H].max(axis=1) - 1e-10)
        if H == 1:
            np.testing.assert_allclose(feat[:, 2], feat[:, 0], atol=1e-12)
    assert np.all((feat[:, :2 * H + 1] >= -1e-12) & (feat[:, :2 * H + 1] <= 1 + 1e-12))


def test_noiseless_multiharmonic_signal_gives_unit_mhls_power():
    rng = np.random.default_rng(4)
    t = np.sort(rng.uniform(0, 10, 50))
    f0 = 0.37
    y = 1.0 + 0.3 * np.cos(2 * np.pi * f0 * t) - 0.2 * np.sin(4 * np.pi * f0 * t + 1.0)
    feat = so.screening_features(t, y, np.ones_like(t), [f0], 2)
    assert abs(feat[0, 4] - 1.0) < 1e-12
    assert abs(feat[0, 5] - math.log10(50)) < 1e-15


def test_harmonic_amplitude_closed_form():
    """Unit weights, N equispaced samples over whole cycles, y = cos(h w t):
    sum (1/N) y exp(i h w t) = 1/2 and Var(y) = 1/2, so A_h = 1/2 and the
    other harmonics vanish."""
    N, f = 64, 0.25
    t = np.arange(N) / (N * f) * 4  # four whole cycles
    for h in (1, 2, 3):
        y = np.cos(2 * np.pi * h * f * t)
        feat = so.screening_features(t, y, np.zeros(N), [f], 3)
        A = feat[0, 3:6]
        assert abs(A[h - 1] - 0.5) < 1e-12
        assert np.all(np.abs(np.delete(A, h - 1)) < 1e-12)


def test_planted_mistake_fit_without_offset_is_caught():
    """Fitting the single harmonic without the constant (the original,
    non-floating-mean periodogram) breaks the H = 1 FTP pin for data with an
    offset."""
    t, y, dy = curve(5, offset=2.0)
    freqs = np.linspace(0.05, 2.0, 9)
    w = oracle.normalized_weights(dy)
    ybar, _ = oracle.data_moments(y, w)
    yc, sw = y - ybar, np.sqrt(w)
    wrong = []
    for f in freqs:
        ph = 2 * np.pi * f * t
        X = np.column_stack([np.cos(ph), np.sin(ph)]) * sw[:, None]
        coef, *_ = np.linalg.lstsq(X, yc * sw, rcond=None)
        r = yc * sw - X @ coef
        wrong.append(1 - (r @ r) / ((yc * sw) @ (yc * sw)))
    ftp = oracle.periodogram(t, y, dy, freqs, [1.0], [0.0])
    assert np.max(np.abs(np.array(wrong) - ftp["power"])) > 1e-4


# ------------------------------------------------------------------ network
def test_bf16_rounding_matches_known_values_and_torch():
    one = 1.0
    assert so.bf16_round(one) == 1.0
    assert so.bf16_round(1 + 2 ** -8) == 1.0                  # tie -> even
    assert so.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6      # tie -> even (up)
    assert so.bf16_round(1 + 2 ** -8 + 2 ** -12) == 1 + 2 ** -7
    assert so.bf16_round(-3.0) == -3.0
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(6).standard_normal(10000) * 10.0 ** np.random.default_rng(7).uniform(-5, 5, 10000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(so.bf16_round(x), ref)


def finite_difference_check(p, X, tgt, nfeat, idx, h=1e-6):
    loss, g = so.loss_and_gradients(p, X, tgt, nfeat, bf16=False)
    num = np.empty(idx.size)
    for j, i in enumerate(idx):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num[j] = (so.loss_and_gradients(pp, X, tgt, nfeat, bf16=False)[0] -
                  so.loss_and_gradients(pm, X, tgt, nfeat, bf16=False)[0]) / (2 * h)
    return g[idx], num


def test_gradients_match_finite_differences():
    nfeat = 10
    rng = np.random.default_rng(8)
    p = so.init_params(nfeat, seed=1)
    X = rng.uniform(0, 1, (12, nfeat))
    tgt = rng.uniform(0, 1, 12)
    n = so.param_count(nfeat)
    # every W1, b1, b3 entry and a random subset of the large blocks
    head = np.arange(128 * nfeat + 128)
    idx = np.unique(np.concatenate([head[::7], rng.choice(n, 300, replace=False), [n - 1]]))
    ana, num = finite_difference_check(p, X, tgt, nfeat, idx)
    scale = np.max(np.abs(ana))
    assert np.max(np.abs(ana - num)) <= 1e-6 * scale


def test_planted_mistake_transposed_w2_in_backward_is_caught():
    """Back-propagating through W2^T instead of W2 fails the finite-difference pin."""
    nfeat = 6
    rng = np.random.default_rng(9)
    p = so.init_params(nfeat, seed=2)
    X = rng.uniform(0, 1, (8, nfeat))
    tgt = rng.uniform(0, 1, 8)
    fw = so.forward(p, X, nfeat, bf16=False)
    ds = 2 * (fw["s"] - tgt) / tgt.size
    dZ2 = np.outer(ds, fw["w3"]) * (fw["Z2"] > 0)
    wrong_dZ1 = (dZ2 @ fw["W2"].T) * (fw["Z1"] > 0)
    wrong_gW1 = (wrong_dZ1.T @ fw["Xb"]).ravel()
    idx = np.arange(128 * nfeat)
    _, num = finite_difference_check(p, X, tgt, nfeat, idx)
    assert np.max(np.abs(wrong_gW1 - num)) > 1e-3 * np.max(np.abs(num))


def test_bf16_network_stays_close_to_the_exact_one():
    nfeat = 10
    rng = np.random.default_rng(10)
    p = so.init_params(nfeat, seed=3)
    X = rng.uniform(0, 1, (64, nfeat))
    s_b = so.forward(p, X, nfeat, bf16=True)["s"]
    s_x = so.forward(p, X, nfeat, bf16=False)["s"]
    assert np.max(np.abs(s_b - s_x)) < 0.05 * (1 + np.max(np.abs(s_x)))
    assert np.max(np.abs(s_b - s_x)) > 0  # the rounding points are really applied


def test_bf16_gradient_stays_close_to_the_exact_one():
    """The BF16 network's gradient (rounded forward values and rounded error
    signals into the weight-gradient products) differs from the exact
    network's by rounding only: each rounding perturbs one factor by at most
    2^-8 relative, so the difference is a small fraction of the gradient, yet
    non-zero (the rounding points are really applied)."""
    nfeat = 10
    rng = np.random.default_rng(11)
    p = so.init_params(nfeat, seed=4)
    X = rng.uniform(0, 1, (256, nfeat))
    tgt = rng.uniform(0, 1, 256)
    _, gb = so.loss_and_gradients(p, X, tgt, nfeat, bf16=True)
    _, gx = so.loss_and_gradients(p, X, tgt, nfeat, bf16=False)
    rel = np.linalg.norm(gb - gx) / np.linalg.norm(gx)
    assert 0 < rel < 0.03
