"""FP64 CPU oracle for the learned screening surrogate (not part of the paper).

TEST INFRASTRUCTURE ONLY.  Imported by tests/ and nothing else; it shares no
code with the CUDA library.

Two things are defined here, each by its plain definition:

1. The per-frequency screening features, x in R^{2H+2}, read from the
   multi-harmonic extension of Lomb-Scargle that Section 2.1 describes
   (a constant plus H harmonics, fitted by weighted least squares):
     x[h-1]     P_h  = 1 - chi2_min / chi2_0 of  y ~ c0 + a cos(h w t) + b sin(h w t)
                       (the floating-mean single-harmonic periodogram at h*omega), h = 1..H
     x[H+h-1]   A_h  = |sum_i w_i (y_i - ybar) exp(i h w t_i)|^2 / YY,  h = 1..H
     x[2H]      P_MHLS(H) = 1 - chi2_min / chi2_0 of y ~ c0 + sum_h a_h cos + b_h sin
                       (Section 2.1, the multi-harmonic model with H harmonics)
     x[2H+1]    log10(N_obs)
   The fits are solved with numpy.linalg.lstsq on the sqrt(w)-scaled design
   matrix - the definition itself, no closed forms.  P_MHLS(H) bounds the FTP
   power from above (the template model is the multi-harmonic model with the
   harmonic amplitudes tied to the template).

2. The surrogate network 2H+2 -> 128 -> 128 -> 1 with BF16 weights and
   activations and FP32 accumulation, and its loss gradients.  The oracle
   computes in FP64 and applies BF16 rounding (round to nearest even, via
   FP32) at the points the network defines:
     Xb = bf16(X); W1b, W2b, w3b = bf16(W1, W2, w3); biases stay FP32
     Z1 = Xb W1b^T + b1;  A1 = bf16(relu(Z1))
     Z2 = A1 W2b^T + b2;  A2 = bf16(relu(Z2))
     s  = A2 w3b + b3
     loss = mean((s - target)^2)
   Gradients are taken with respect to the rounded weights (the master copy
   is FP32; rounding is treated as the identity in the backward pass), with
   relu'(z) = [z > 0].  The backward pass of the BF16 network rounds the two
   error signals where they enter a matrix product, as the tensor cores
   consume them:
     r = s - target, ds = 2 r / n, dZ2 = ds w3b^T * [Z2 > 0]
     g_w3 = A2^T ds, g_b3 = sum ds, g_b2 = column sums of dZ2
     g_W2 = bf16(dZ2)^T A1,  dZ1 = (bf16(dZ2) W2b) * [Z1 > 0]
     g_b1 = column sums of dZ1, g_W1 = bf16(dZ1)^T Xb
   With bf16=False every rounding is skipped and the function is an ordinary
   smooth network, which the tests pin by finite differences.

Flat parameter layout (shared with the C ABI as an interface):
   W1 [hidden][nfeat] row-major, b1 [hidden], W2 [hidden][hidden] row-major
   (W2[j][i]: output j, input i), b2 [hidden], w3 [hidden], b3 [1].
"""
from __future__ import annotations

import math

import numpy as np

from .ftp_oracle import data_moments, harmonic_phases, normalized_weights


# ---------------------------------------------------------------------------
# Features (Section 2.1 multi-harmonic least squares)
# ---------------------------------------------------------------------------
def _wls_power(sw, yc, cols) -> float:
    """1 - chi2_min/chi2_0 for the weighted fit of y (centred) on a constant
    and `cols`; sw = sqrt(w), yc = y - ybar."""
    X = np.column_stack([np.ones_like(sw)] + list(cols)) * sw[:, None]
    b = yc * sw
    coef, *_ = np.linalg.lstsq(X, b, rcond=None)
    r = b - X @ coef
    return 1.0 - float(r @ r) / float(b @ b)


def screening_features(t, y, dy, freqs, H: int) -> np.ndarray:
    """Features [len(freqs)][2H+2] as defined in the module docstring."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = normalized_weights(dy)
    ybar, YY = data_moments(y, w)
    yc = y - ybar
    sw = np.sqrt(w)
    freqs = np.atleast_1d(np.asarray(freqs, dtype=np.float64))
    out = np.zeros((freqs.size, 2 * H + 2))
    for k, f in enumerate(freqs):
        ph = harmonic_phases(t, f, H)  # [H, N], h * omega * t mod 2 pi
        cos, sin = np.cos(ph), np.sin(ph)
        for h in range(H):
            out[k, h] = _wls_power(sw, yc, [cos[h], sin[h]])
            z = np.sum(w * yc * np.exp(1j * ph[h]))
            out[k, H + h] = abs(z) ** 2 / YY
        cols = []
        for h in range(H):
            cols += [cos[h], sin[h]]
        out[k, 2 * H] = _wls_power(sw, yc, cols)
        out[k, 2 * H + 1] = math.log10(t.size)
    return out


# ---------------------------------------------------------------------------
# The network
# ---------------------------------------------------------------------------
def param_count(nfeat: int, hidden: int = 128) -> int:
    return hidden * nfeat + hidden + hidden * hidden + hidden + hidden + 1


def unflatten(flat, nfeat: int, hidden: int = 128) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == param_count(nfeat, hidden)
    o = 0
    out = {}
    for name, shape in (("W1", (hidden, nfeat)), ("b1", (hidden,)), ("W2", (hidden, hidden)),
                        ("b2", (hidden,)), ("w3", (hidden,)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.ravel(p[k]) for k in ("W1", "b1", "W2", "b2", "w3", "b3")])


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), through FP32 as the
    FP32 accumulators of the network are; returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(flat, X, nfeat: int, hidden: int = 128, bf16: bool = True) -> dict:
    """Scores s [n] and the intermediate values of the forward pass."""
    p = unflatten(flat, nfeat, hidden)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    Xb = rnd(np.asarray(X, dtype=np.float64))
    W1, W2, w3 = rnd(p["W1"]), rnd(p["W2"]), rnd(p["w3"])
    Z1 = Xb @ W1.T + p["b1"]
    A1 = rnd(np.maximum(Z1, 0.0))
    Z2 = A1 @ W2.T + p["b2"]
    A2 = rnd(np.maximum(Z2, 0.0))
    s = A2 @ w3 + p["b3"][0]
    return dict(s=s, Xb=Xb, W1=W1, W2=W2, w3=w3, Z1=Z1, A1=A1, Z2=Z2, A2=A2)


def loss_and_gradients(flat, X, target, nfeat: int, hidden: int = 128, bf16: bool = True):
    """(mean squared error, flat gradient) by backpropagation."""
    fw = forward(flat, X, nfeat, hidden, bf16)
    target = np.asarray(target, dtype=np.float64)
    n = target.size
    r = fw["s"] - target
    loss = float(np.mean(r * r))
    ds = 2.0 * r / n                                   # d loss / d s
    g = {}
    g["w3"] = fw["A2"].T @ ds
    g["b3"] = np.array([np.sum(ds)])
    rnd = bf16_round if bf16 else (lambda v: v)
    dZ2 = np.outer(ds, fw["w3"]) * (fw["Z2"] > 0)      # through relu
    g["b2"] = np.sum(dZ2, axis=0)
    dZ2 = rnd(dZ2)
    g["W2"] = dZ2.T @ fw["A1"]
    dZ1 = (dZ2 @ fw["W2"]) * (fw["Z1"] > 0)
    g["b1"] = np.sum(dZ1, axis=0)
    g["W1"] = rnd(dZ1).T @ fw["Xb"]
    return loss, flatten(g)


def init_params(nfeat: int, hidden: int = 128, seed: int = 0) -> np.ndarray:
    """Seeded uniform initialisation, U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for
    weights and biases of each layer (a test input, not the library's own
    initialisation)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, bname, fan_in, shape in (("W1", "b1", nfeat, (hidden, nfeat)),
                                       ("W2", "b2", hidden, (hidden, hidden)),
                                       ("w3", "b3", hidden, (hidden,))):
        a = 1.0 / math.sqrt(fan_in)
        p[name] = rng.uniform(-a, a, shape)
        p[bname] = rng.uniform(-a, a, (1,) if name == "w3" else (hidden,))
    return flatten(p)
