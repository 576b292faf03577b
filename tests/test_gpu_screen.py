"""Learned screening on the GPU, through the C ABI: features from the NFFT
sums against the FP64 oracle's least-squares definitions, the tcgen05 BF16
network (forward and gradient) against the oracle's network, training,
training-row selection, and the screened batch against the exhaustive one.

Tolerances.  Features: the mixed path's sums carry an absolute error of
~2e-6 (FP32 NFFT), so a least-squares power b^T G^-1 b / YY moves by about
(2|b| + |b|^2 / lambda_min) * 2e-6 / (lambda_min YY); on frequencies whose
basis covariance has lambda_min >= 0.02 that stays below 3e-4 (FP64 path:
1e-7, the FP32 storage of a feature in [0, 1] alone rounds by up to 6e-8).  Network: both sides round to BF16 at the same points, but the GPU
accumulates in FP32 (tensor cores) and the oracle in FP64, so a value within
~1e-6 relative of a BF16 rounding boundary can round the other way; one such
flip moves an activation by 2^-8 relative and a score by ~1e-3 at most, so
scores agree to 5e-3 everywhere and to 1e-4 on 99 % of rows, gradients to
3e-2 of the block's largest entry and 1e-2 in relative L2 norm."""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle
import synth
from oracle import screen_oracle as so
from paper_2101_12348_gb300 import screen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp as f
    f.load()
    return f


def small_survey(n=6, H=4, seed=21, f_max=2.0, baseline=(20.0, 100.0), median_obs=150):
    return synth.survey(ncurves=n, n_bank=2, median_obs=median_obs, min_obs=30, max_obs=600,
                        f_max=f_max, baseline=baseline, Hs=(H,), seed=seed)


def grids_of(sv):
    return [(g.df, g.k0, g.nf) for g in sv.grids]


def plan_for(ftp, sv, H, prec):
    g = max(sv.grids, key=lambda g: g.k0 + g.nf)
    nf = max(x.nf for x in sv.grids)
    return ftp.Plan(int(np.max(np.diff(sv.obs_off))), H, (g.df, g.k0, nf), 2, prec)


def lambda_min(t, dy, f, H):
    """Smallest eigenvalue of the weighted covariance of cos/sin(h w t), h <= H."""
    w = 1.0 / dy ** 2
    w /= w.sum()
    ph = 2 * np.pi * np.outer(np.arange(1, H + 1), f * t)
    X = np.concatenate([np.cos(ph), np.sin(ph)])
    Xc = X - (X @ w)[:, None]
    return float(np.linalg.eigvalsh((Xc * w) @ Xc.T)[0])


@pytest.mark.parametrize("prec,tol", [("mixed", 3e-4), ("fp64", 1e-7)])
def test_features_match_oracle(ftp, prec, tol):
    H = 4
    sv = small_survey(H=H)
    grids = grids_of(sv)
    off = np.zeros(len(grids) + 1, dtype=np.int64)
    off[1:] = np.cumsum([g[2] for g in grids])
    feats = torch.empty((int(off[-1]), 2 * H + 2), dtype=torch.float32, device="cuda")
    with plan_for(ftp, sv, H, prec) as plan:
        ftp.ftp_batch_features(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids, off, H, feats)
    F = feats.cpu().numpy()
    assert np.all(np.isfinite(F))
    compared = 0
    for c in range(sv.ncurves):
        lc = sv.curve(c)
        fr = sv.grids[c].freqs()
        sel = np.arange(c % 11, fr.size, 13)
        ref = so.screening_features(lc.t, lc.y, lc.dy, fr[sel], H)
        got = F[off[c] + sel]
        good = np.array([lambda_min(lc.t, lc.dy, f, H) >= 0.02 for f in fr[sel]])
        assert np.all((got[:, :2 * H + 1] > -1e-2) & (got[:, :2 * H + 1] < 1 + 1e-2))
        err = np.abs(got - ref)[good]
        assert err[:, :2 * H + 1].max(initial=0) <= tol, (c, err.max(axis=0))
        np.testing.assert_allclose(got[:, 2 * H + 1], math.log10(lc.t.size), rtol=1e-6)
        compared += int(good.sum())
    assert compared > 100


@pytest.mark.parametrize("nfeat,n", [(10, 1000), (18, 129), (4, 1)])
def test_mlp_forward_matches_oracle(ftp, nfeat, n):
    rng = np.random.default_rng(nfeat + n)
    p = so.init_params(nfeat, seed=nfeat).astype(np.float32)
    X = rng.uniform(0, 1, (n, nfeat)).astype(np.float32)
    h = ftp.ftp_mlp_create(nfeat, p, 0, 0)
    try:
        s_host = np.empty(n, dtype=np.float32)
        ftp.ftp_mlp_forward(h, X, n, s_host)                       # host arrays
        Xd = torch.from_numpy(X).cuda()
        sd = torch.empty(n, dtype=torch.float32, device="cuda")
        ftp.ftp_mlp_forward(h, Xd, n, sd)                           # device arrays
        q = np.empty(p.size, dtype=np.float32)
        ftp.ftp_mlp_get_params(h, q)
    finally:
        ftp.ftp_mlp_destroy(h)
    np.testing.assert_array_equal(q, p)
    np.testing.assert_array_equal(sd.cpu().numpy(), s_host)
    ref = so.forward(p.astype(np.float64), X.astype(np.float64), nfeat)["s"]
    err = np.abs(s_host - ref)
    assert err.max() <= 5e-3, err.max()
    assert np.quantile(err, 0.99) <= 1e-4, np.quantile(err, 0.99)


@pytest.mark.parametrize("nfeat,rows,n,use_idx", [(10, 500, 300, True), (18, 200, 200, False),
                                                  (10, 4000, 2600, True)])
def test_mlp_gradient_matches_oracle(ftp, nfeat, rows, n, use_idx):
    rng = np.random.default_rng(rows)
    p = so.init_params(nfeat, seed=3).astype(np.float32)
    X = rng.uniform(0, 1, (rows, nfeat)).astype(np.float32)
    tgt = rng.uniform(0, 1, rows).astype(np.float32)
    idx = rng.permutation(rows)[:n].astype(np.int64) if use_idx else None
    h = ftp.ftp_mlp_create(nfeat, p, 0, 0)
    try:
        g = np.empty(p.size, dtype=np.float32)
        loss = np.empty(1, dtype=np.float32)
        ftp.ftp_mlp_gradient(h, X, tgt, rows, idx, n, g, loss)
    finally:
        ftp.ftp_mlp_destroy(h)
    rows_used = idx if use_idx else np.arange(n)
    ref_loss, ref = so.loss_and_gradients(p.astype(np.float64), X[rows_used].astype(np.float64),
                                          tgt[rows_used].astype(np.float64), nfeat)
    assert abs(loss[0] - ref_loss) <= 1e-3 * ref_loss + 1e-6
    blocks = so.unflatten(np.arange(p.size), nfeat)
    for name, ix in blocks.items():
        ix = ix.ravel().astype(np.int64)
        scale = np.abs(ref[ix]).max()
        assert np.abs(g[ix] - ref[ix]).max() <= 3e-2 * scale, name
    assert np.linalg.norm(g - ref) <= 1e-2 * np.linalg.norm(ref)


def test_mlp_training_reduces_the_loss(ftp):
    nfeat, rows = 10, 20000
    rng = np.random.default_rng(9)
    X = rng.uniform(0, 1, (rows, nfeat)).astype(np.float32)
    y = (X[:, 0] * X[:, 1] + 0.5 * X[:, 2] ** 2).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    h = ftp.ftp_mlp_create(nfeat, None, 4, 0)
    try:
        losses = np.empty(1500, dtype=np.float32)
        ftp.ftp_mlp_train(h, Xd, yd, rows, 1500, 1024, 2e-3, 11, losses)
        s = np.empty(rows, dtype=np.float32)
        ftp.ftp_mlp_forward(h, X, rows, s)
    finally:
        ftp.ftp_mlp_destroy(h)
    assert np.all(np.isfinite(losses))
    assert losses[-100:].mean() < 0.05 * losses[:10].mean()
    assert np.mean((s - y) ** 2) < 2e-3


def splitmix64(x):
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(2 ** 64 - 1)
    x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(2 ** 64 - 1)
    x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(2 ** 64 - 1)
    return x ^ (x >> np.uint64(31))


def test_training_rows_selection(ftp):
    rng = np.random.default_rng(12)
    nf = [700, 1, 2500]
    off = np.zeros(4, dtype=np.int64)
    off[1:] = np.cumsum(nf)
    rows, nfeat = int(off[-1]), 6
    power = rng.permutation(rows).astype(np.float64) / rows
    feats = rng.standard_normal((rows, nfeat)).astype(np.float32)
    cap = rows
    Xo = torch.zeros((cap, nfeat), dtype=torch.float32, device="cuda")
    yo = torch.zeros(cap, dtype=torch.float32, device="cuda")
    top, nbr, rf, seed = 0.01, 3, 0.05, 5
    with np.errstate(over="ignore"):
        count = ftp.ftp_training_rows(torch.from_numpy(power).cuda(),
                                      torch.from_numpy(feats).cuda(), nfeat, off, top, nbr, rf,
                                      seed, Xo, yo, cap, 3)
        key = splitmix64(np.uint64(seed))
        hsh = splitmix64(key ^ np.arange(rows, dtype=np.uint64))
    thr = np.uint64(int(rf * 2.0 ** 64))
    sel = np.zeros(rows, dtype=bool)
    for c in range(3):
        pc = power[off[c]:off[c + 1]]
        K = max(1, math.ceil(top * pc.size))
        on = pc >= np.sort(pc)[-K]
        dil = np.zeros_like(on)
        for d in range(-nbr, nbr + 1):
            lo, hi = max(0, d), min(pc.size, pc.size + d)
            dil[lo:hi] |= on[lo - d:hi - d]
        sel[off[c]:off[c + 1]] = dil
    sel |= hsh < thr
    want = np.flatnonzero(sel)
    assert count == 3 + want.size
    np.testing.assert_array_equal(Xo[3:count].cpu().numpy(), feats[want])
    np.testing.assert_array_equal(yo[3:count].cpu().numpy(), power[want].astype(np.float32))


@pytest.mark.parametrize("prec,tol", [("mixed", 1e-4), ("fp64", 1e-9)])
def test_screened_batch_equals_exhaustive_where_evaluated(ftp, prec, tol):
    """Step (a) accumulates with atomics, so two runs agree to rounding, not
    bit for bit: evaluated powers match the exhaustive run within the path's
    parity tolerance, and the selection is checked away from its threshold
    (the scores of a separate features call may differ in the last bits)."""
    H = 4
    sv = small_survey(n=7, H=H, seed=33, f_max=3.0)
    grids = grids_of(sv)
    off = np.zeros(len(grids) + 1, dtype=np.int64)
    off[1:] = np.cumsum([g[2] for g in grids])
    rows = int(off[-1])
    bank = [(b.c, b.s) for b in sv.bank]
    top, nbr = 0.03, 3
    with plan_for(ftp, sv, H, prec) as plan, screen.Surrogate(H, seed=17) as net:
        ex = [torch.empty(rows, dtype=torch.float64, device="cuda") for _ in range(4)]
        exf = torch.empty(rows, dtype=torch.uint8, device="cuda")
        ftp.ftp_batch(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids, off[:-1].copy(), bank,
                      sv.tpl_of_curve, *ex, exf)
        sc = [torch.full((rows,), -7.0, dtype=torch.float64, device="cuda") for _ in range(4)]
        scf = torch.zeros(rows, dtype=torch.uint8, device="cuda")
        for _ in range(2):  # the second, identical call is captured into a CUDA graph
            ftp.ftp_batch_screened(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids,
                                   off[:-1].copy(), bank, sv.tpl_of_curve, net.h, top, nbr, *sc,
                                   scf)
        ftp.ftp_batch_screened(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids, off[:-1].copy(),
                               bank, sv.tpl_of_curve, net.h, top, nbr, *sc, scf)  # replay
        feats = torch.empty((rows, 2 * H + 2), dtype=torch.float32, device="cuda")
        ftp.ftp_batch_features(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids, off, H, feats)
        scores = net.forward(feats, rows, torch.empty(rows, dtype=torch.float32, device="cuda"))
    P_ex, P_sc = ex[0].cpu().numpy(), sc[0].cpu().numpy()
    f_sc, f_ex = scf.cpu().numpy(), exf.cpu().numpy()
    s = scores.cpu().numpy()
    evaluated = ~np.isnan(P_sc)
    assert np.all((f_sc[~evaluated] & ftp.FLAG_SCREENED_OUT) != 0)
    assert np.all((f_sc[evaluated] & ftp.FLAG_SCREENED_OUT) == 0)
    for i in range(4):
        a = sc[i].cpu().numpy()
        assert np.all(np.isnan(a[~evaluated]))
        assert np.all(np.isfinite(a[evaluated]))
    assert np.abs(P_sc[evaluated] - P_ex[evaluated]).max() <= tol
    assert evaluated.sum() > 0
    # the best-scored frequencies of each curve (the top half of the
    # selection, clear of its threshold) and their +-nbr neighbours were evaluated
    nsel = 0
    for c in range(len(grids)):
        sl = slice(off[c], off[c + 1])
        sc_c = s[sl].astype(np.float32)
        K = max(1, math.ceil(top * sc_c.size))
        nsel += min(sc_c.size, K * (2 * nbr + 1))
        on = sc_c >= np.sort(sc_c)[-max(1, K // 2)]
        dil = np.zeros_like(on)
        for d in range(-nbr, nbr + 1):
            lo, hi = max(0, d), min(on.size, on.size + d)
            dil[lo:hi] |= on[lo - d:hi - d]
        assert np.all(evaluated[sl][dil]), c
    assert evaluated.sum() <= 2 * nsel


HELDOUT = 1200


def test_screening_gains_over_exhaustive_with_high_recall(ftp):
    """Trained on exact FTP output of one set of curves, the surrogate keeps
    the best peak of held-out curves (recall >= 0.995, the screening target)
    while the exact solve runs on a small fraction of the frequencies; an
    untrained network keeps no more.

    With 1200 held-out curves the bar allows at most 6 misses, so one miss
    does not decide it: at a true miss rate of 1.5 % (three times the allowed
    0.5 %) the chance of 6 or fewer misses is about 1e-3 (binomial, mean 18),
    and at the 0.05 % rate measured on the full screening workload the chance
    of more than 6 is about 3e-6."""
    H = 4
    train = synth.survey(ncurves=1024, n_bank=8, median_obs=300, min_obs=50, max_obs=3000,
                         f_max=5.0, baseline=(50.0, 400.0), Hs=(H,), seed=404)
    test = synth.survey(ncurves=HELDOUT, n_bank=8, median_obs=300, min_obs=50, max_obs=3000,
                        f_max=5.0, baseline=(50.0, 400.0), Hs=(H,), seed=405)
    gmax = max(train.grids + test.grids, key=lambda g: g.k0 + g.nf)
    nfmax = max(g.nf for g in train.grids + test.grids)
    nmax = int(max(np.max(np.diff(train.obs_off)), np.max(np.diff(test.obs_off))))
    with ftp.Plan(nmax, H, (gmax.df, gmax.k0, nfmax), 8, "mixed") as plan:
        cap = 12_000_000
        Xt = torch.empty((cap, 2 * H + 2), dtype=torch.float32, device="cuda")
        yt = torch.empty(cap, dtype=torch.float32, device="cuda")
        bank = [(b.c, b.s) for b in train.bank]
        n = screen.training_rows(plan.h, train.obs_off, train.t, train.y, train.dy,
                                 grids_of(train), bank, train.tpl_of_curve, H, X_out=Xt,
                                 y_out=yt)
        assert 0 < n <= cap
        grids = grids_of(test)
        off = screen.row_offsets(grids)
        rows = int(off[-1])
        ex = [torch.empty(rows, dtype=torch.float64, device="cuda") for _ in range(4)]
        ftp.ftp_batch(plan.h, test.obs_off, test.t, test.y, test.dy, grids, off[:-1].copy(),
                      bank, test.tpl_of_curve, *ex)
        P_ex = ex[0].cpu().numpy()

        def recall(net):
            out = [torch.empty(rows, dtype=torch.float64, device="cuda") for _ in range(4)]
            ftp.ftp_batch_screened(plan.h, test.obs_off, test.t, test.y, test.dy, grids,
                                   off[:-1].copy(), bank, test.tpl_of_curve, net.h, 0.01, 3,
                                   *out)
            P = out[0].cpu().numpy()
            hit, evaluated = [], 0
            for c in range(test.ncurves):
                a, b = P[off[c]:off[c + 1]], P_ex[off[c]:off[c + 1]]
                hit.append(np.nanmax(a) >= b.max() - 1e-4)
                evaluated += int(np.sum(~np.isnan(a)))
            return float(np.mean(hit)), evaluated / rows

        with screen.Surrogate(H, seed=3) as raw:
            r_raw, _ = recall(raw)
        with screen.Surrogate(H, seed=3) as net:
            net.train(Xt, yt, n, steps=3000, batch=2048, lr=2e-3, seed=9)
            r_net, frac = recall(net)
    print(f"recall {r_net:.4f} on {test.ncurves} held-out curves (untrained {r_raw:.4f}), "
          f"{frac:.3%} of the frequencies solved exactly")
    assert frac < 0.15, frac
    assert r_net >= 0.995, (r_net, r_raw)
    assert r_net >= r_raw
