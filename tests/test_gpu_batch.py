"""ftp_batch: many curves through chunked persistent launches and a CUDA graph.

The batch path runs step (a) per curve into one chunk's sum tiles, then one
roots launch per harmonic count over every curve of the chunk (a segment
table maps work units to curves), a batched re-solve pass for ill-conditioned
frequencies, and - for repeated all-device calls - a captured CUDA graph.
Every result is compared with the FP64 oracle within the parity tolerances
(|dP| <= 1e-4 mixed, <= 1e-9 FP64)."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_P = {"mixed": 1e-4, "fp64": 1e-9}


@pytest.fixture(scope="module")
def ftp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp as f
    f.load()
    return f


def mixed_survey():
    """A small survey (uneven N and grids, bank H in {2, 4, 6}) plus two
    three-point curves whose clustered phases make MM ill-conditioned."""
    sv = synth.survey(ncurves=24, n_bank=6, median_obs=80, min_obs=20, max_obs=400,
                      f_max=1.5, baseline=(20, 120), seed=313)
    rng = np.random.default_rng(5)
    extra = [synth.random_curve(rng, 3, T=10.0, signal=0.6, tpl=sv.bank[0], period=3.0),
             synth.random_curve(rng, 3, T=8.0, signal=0.4, tpl=sv.bank[1], period=2.0)]
    t, y, dy = [sv.t], [sv.y], [sv.dy]
    off = list(sv.obs_off)
    grids = list(sv.grids)
    tpc = list(sv.tpl_of_curve)
    for i, lc in enumerate(extra):
        t.append(lc.t)
        y.append(lc.y)
        dy.append(lc.dy)
        off.append(off[-1] + lc.t.size)
        grids.append(synth.Grid(df=1 / 50.0, k0=1, nf=300))
        tpc.append(i)
    return (np.array(off, dtype=np.int64), np.concatenate(t), np.concatenate(y),
            np.concatenate(dy), grids, sv.bank, np.array(tpc, dtype=np.int32))


def plan_for(ftp, off, grids, bank, prec):
    maxnf = max(g.nf for g in grids)
    gj = max(grids, key=lambda g: g.k0 + g.nf)
    Hmax = max(b.H for b in bank)
    return ftp.Plan(int(np.max(np.diff(off))), Hmax, (gj.df, gj.k0, max(maxnf, gj.nf)),
                    len(bank), prec)


def variance_condition(t, dy, freqs, tp, theta2):
    """kappa = <M^2> / Var(M) at the given phases.  Var(M) evaluated in FP64
    as a difference of O(<M^2>) terms carries an absolute error ~eps <M^2>,
    so P = YM^2 / (YY Var(M)) is defined by any FP64 evaluation (the oracle's
    included) only to ~eps * kappa."""
    w = 1.0 / np.asarray(dy) ** 2
    w /= w.sum()
    kap = np.empty(len(freqs))
    for i, (f, th) in enumerate(zip(freqs, theta2)):
        M = tp(2 * np.pi * f * t - th)
        m2 = np.sum(w * M * M)
        kap[i] = m2 / max(m2 - np.sum(w * M) ** 2, 1e-300)
    return kap


def check_curves(off, t, y, dy, grids, bank, tpc, power, out_off, prec, every=7, theta2=None):
    """Every `every`-th frequency of each curve (all of the tiny ones) vs the
    oracle: |dP| <= the path's tolerance, widened by 8 eps kappa where Var(M)
    is ill-conditioned (three-point curves): such frequencies are solved from
    FP64 sums on both paths, and any FP64 evaluation (the oracle's included)
    defines P only to ~eps kappa.  kappa is taken at the oracle's phase and
    at the reported one: where P is flat (a three-point curve fits every
    phase exactly) the two may differ, and the larger conditioning decides
    how well either FP64 evaluation defines P."""
    for c in range(len(grids)):
        sl = slice(off[c], off[c + 1])
        g = grids[c]
        n = off[c + 1] - off[c]
        sel = np.arange(g.nf) if n <= 3 else np.arange(c % every, g.nf, every)
        tp = bank[tpc[c]]
        ref = oracle.periodogram(t[sl], y[sl], dy[sl], g.freqs()[sel], tp.c, tp.s)
        p = power[out_off[c]:out_off[c] + g.nf][sel]
        # the mixed path re-solves ill-conditioned frequencies from FP64 sums,
        # so the FP64 conditioning floor applies to it as well
        kap = variance_condition(t[sl], dy[sl], g.freqs()[sel], tp, ref["theta2"])
        if theta2 is not None:
            th = theta2[out_off[c]:out_off[c] + g.nf][sel]
            kap = np.maximum(kap, variance_condition(t[sl], dy[sl], g.freqs()[sel], tp, th))
        tol = TOL_P[prec] + 8 * np.finfo(np.float64).eps * kap
        bad = np.abs(p - ref["power"]) > tol
        assert not np.any(bad), (f"curve {c} (N={n}): |dP| = {np.abs(p - ref['power'])[bad]} "
                                 f"tol {tol[bad]}")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_chunks_graph_and_host_paths(ftp, prec):
    off, t, y, dy, grids, bank, tpc = mixed_survey()
    grid_t = [(g.df, g.k0, g.nf) for g in grids]
    out_off = np.zeros(len(grids) + 1, dtype=np.int64)
    out_off[1:] = np.cumsum([g.nf for g in grids])
    tot = int(out_off[-1])
    with plan_for(ftp, off, grids, bank, prec) as plan:
        # a budget of a few curves' sum tiles: several chunks
        ftp.ftp_set_batch_options(plan.h, 1 << 18, True)
        host = [np.full(tot, np.nan) for _ in range(4)]
        hflags = np.full(tot, 255, dtype=np.uint8)
        ftp.ftp_batch(plan.h, off, t, y, dy, grid_t, out_off[:-1], [(b.c, b.s) for b in bank],
                      tpc, *host, hflags)
        info = ftp.ftp_batch_info(plan.h)
        assert info["chunks"] >= 3 and info["graph"] == 0
        stats = plan.solver_stats()
        assert stats["resolved"] >= 1
        assert np.all(np.isfinite(host[0])) and np.all(hflags != 255)
        assert np.all((hflags & 16) == 0)  # nothing left unresolved
        check_curves(off, t, y, dy, grids, bank, tpc, host[0], out_off, prec, theta2=host[2])

        # the same batch from device memory: eager, then captured, then replayed
        dev = torch.device("cuda:0")
        dt, dyv, ddy = (torch.from_numpy(a).to(dev) for a in (t, y, dy))
        outs = [torch.empty(tot, dtype=torch.float64, device=dev) for _ in range(4)]
        fl = torch.empty(tot, dtype=torch.uint8, device=dev)
        modes = []
        for _ in range(3):
            for o in outs:
                o.fill_(float("nan"))
            fl.fill_(255)
            torch.cuda.synchronize()  # the plan works on its own stream
            ftp.ftp_batch(plan.h, off, dt, dyv, ddy, grid_t, out_off[:-1],
                          [(b.c, b.s) for b in bank], tpc, *outs, fl)
            modes.append(ftp.ftp_batch_info(plan.h)["graph"])
            p = outs[0].cpu().numpy()
            assert np.max(np.abs(p - host[0])) <= 2 * TOL_P[prec]
            assert np.all(fl.cpu().numpy() != 255)
        assert modes == [0, 1, 2]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_every_template_on_every_curve(ftp, prec):
    """tpl_of_curve = NULL: one launch per template group (H = 2, 4, 6) covers
    all curves; outputs are template-major per curve."""
    sv = synth.survey(ncurves=5, n_bank=3, median_obs=60, min_obs=20, max_obs=200,
                      f_max=1.0, baseline=(30, 80), seed=78)
    bank = [(b.c, b.s) for b in sv.bank]
    grid_t = [(g.df, g.k0, g.nf) for g in sv.grids]
    out_off = np.zeros(sv.ncurves + 1, dtype=np.int64)
    out_off[1:] = np.cumsum([len(bank) * g.nf for g in sv.grids])
    with plan_for(ftp, sv.obs_off, sv.grids, sv.bank, prec) as plan:
        o = [np.zeros(int(out_off[-1])) for _ in range(4)]
        ftp.ftp_batch(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grid_t, out_off[:-1], bank, None, *o)
    for c in range(sv.ncurves):
        lc = sv.curve(c)
        g = sv.grids[c]
        sel = np.arange(c, g.nf, 5)
        for i, tp in enumerate(sv.bank):
            ref = oracle.periodogram(lc.t, lc.y, lc.dy, g.freqs()[sel], tp.c, tp.s)
            a = out_off[c] + i * g.nf
            assert np.max(np.abs(o[0][a:a + g.nf][sel] - ref["power"])) <= TOL_P[prec]


def test_batch_survey_scale_sampled(ftp):
    """The batched survey at 512 curves (N lognormal around 1000, clipped to
    [50, 20000]; baselines 100-3000 d; f up to 10 /d), mixed precision, device
    arrays, replayed from the graph: sampled frequencies of sampled curves vs
    the oracle, and every power in [0, 1]."""
    sv = synth.survey(ncurves=512, seed=1003)
    bank = [(b.c, b.s) for b in sv.bank]
    grid_t = [(g.df, g.k0, g.nf) for g in sv.grids]
    out_off = np.zeros(sv.ncurves + 1, dtype=np.int64)
    out_off[1:] = np.cumsum([g.nf for g in sv.grids])
    tot = int(out_off[-1])
    dev = torch.device("cuda:0")
    dt, dyv, ddy = (torch.from_numpy(a).to(dev) for a in (sv.t, sv.y, sv.dy))
    outs = [torch.empty(tot, dtype=torch.float64, device=dev) for _ in range(4)]
    fl = torch.empty(tot, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()  # the plan works on its own stream
    with plan_for(ftp, sv.obs_off, sv.grids, sv.bank, "mixed") as plan:
        for _ in range(3):
            ftp.ftp_batch(plan.h, sv.obs_off, dt, dyv, ddy, grid_t, out_off[:-1], bank,
                          sv.tpl_of_curve, *outs, fl)
        assert ftp.ftp_batch_info(plan.h)["graph"] == 2
    p = outs[0].cpu().numpy()
    assert np.all((p >= -1e-6) & (p <= 1 + 1e-6))
    rng = np.random.default_rng(9)
    for c in rng.choice(sv.ncurves, 12, replace=False):
        lc = sv.curve(c)
        g = sv.grids[c]
        tp = sv.bank[sv.tpl_of_curve[c]]
        pc = p[out_off[c]:out_off[c + 1]]
        sel = np.unique(np.concatenate([rng.choice(g.nf, 20, replace=False),
                                        np.argsort(-pc)[:5]]))
        ref = oracle.periodogram(lc.t, lc.y, lc.dy, g.freqs()[sel], tp.c, tp.s)
        assert np.max(np.abs(pc[sel] - ref["power"])) <= TOL_P["mixed"]


def test_batch_full_survey_sampled(ftp, tmp_path):
    """The batched survey at its full size, in the launch configuration the
    benchmark times: 4096 curves from the same generator and seed, one mixed
    plan on its own stream, device-resident arrays, step (a) lanes and roots
    grid autotuned, then replayed from the captured graph.  Every power is
    finite and in [0, 1], no item is left at the iteration cap, and on 16
    sampled curves 20 random frequencies and the 3 highest peaks match the
    oracle within 1e-4."""
    sv = synth.survey(ncurves=4096, seed=1003)
    bank = [(b.c, b.s) for b in sv.bank]
    grid_t = [(g.df, g.k0, g.nf) for g in sv.grids]
    out_off = np.zeros(sv.ncurves + 1, dtype=np.int64)
    out_off[1:] = np.cumsum([g.nf for g in sv.grids])
    tot = int(out_off[-1])
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    dt, dyv, ddy = (torch.from_numpy(a).to(dev) for a in (sv.t, sv.y, sv.dy))
    outs = [torch.empty(tot, dtype=torch.float64, device=dev) for _ in range(4)]
    fl = torch.empty(tot, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    gj = max(sv.grids, key=lambda g: g.k0 + g.nf)
    plan_grid = (gj.df, gj.k0, max(g.nf for g in sv.grids))
    plan = ftp.ftp_plan(int(np.max(np.diff(sv.obs_off))), 6, plan_grid, len(bank), "mixed", 0,
                        stream.cuda_stream)
    try:
        args = (plan, sv.obs_off, dt, dyv, ddy, grid_t, out_off[:-1], bank, sv.tpl_of_curve)
        ftp.ftp_batch(*args, *outs, fl)
        ftp.ftp_batch_autotune(*args, *outs, cache_path=str(tmp_path / "tuning.json"))
        for _ in range(3):
            ftp.ftp_batch(*args, *outs, fl)
        assert ftp.ftp_batch_info(plan)["graph"] == 2
        stats = ftp.ftp_solver_stats(plan)
    finally:
        ftp.ftp_destroy(plan)
    assert stats["still_nonconverged"] == 0, stats
    p = outs[0]
    assert bool(torch.all(torch.isfinite(p)))
    assert bool(torch.all((p >= -1e-6) & (p <= 1 + 1e-6)))
    rng = np.random.default_rng(17)
    for c in rng.choice(sv.ncurves, 16, replace=False):
        lc = sv.curve(c)
        g = sv.grids[c]
        tp = sv.bank[sv.tpl_of_curve[c]]
        pc = p[out_off[c]:out_off[c + 1]].cpu().numpy()
        sel = np.unique(np.concatenate([rng.choice(g.nf, 20, replace=False),
                                        np.argsort(-pc)[:3]]))
        ref = oracle.periodogram(lc.t, lc.y, lc.dy, g.freqs()[sel], tp.c, tp.s)
        assert np.max(np.abs(pc[sel] - ref["power"])) <= TOL_P["mixed"], c


def test_batch_autotune_and_tuning_knobs(ftp, tmp_path):
    """ftp_batch_autotune times the step (a) lane count and the roots grid on
    the batch, keeps the fastest, writes them to the JSON cache, and a second
    plan applies the cached choice without timing; every setting gives results
    within the parity tolerance."""
    import json
    off, t, y, dy, grids, bank, tpc = mixed_survey()
    grid_t = [(g.df, g.k0, g.nf) for g in grids]
    out_off = np.zeros(len(grids) + 1, dtype=np.int64)
    out_off[1:] = np.cumsum([g.nf for g in grids])
    tot = int(out_off[-1])
    bk = [(b.c, b.s) for b in bank]
    cache = str(tmp_path / "ftp_tuning.json")
    outs = [np.empty(tot) for _ in range(4)]
    with plan_for(ftp, off, grids, bank, "mixed") as plan:
        assert ftp.ftp_get_batch_tuning(plan.h) == {"sum_lanes": 4, "roots_ctas_per_sm": 0}
        r1 = ftp.ftp_batch_autotune(plan.h, off, t, y, dy, grid_t, out_off[:-1], bk, tpc, *outs,
                                    cache_path=cache)
        assert not r1["from_cache"]
        assert r1["sum_lanes"] in (1, 2, 4, 8) and r1["roots_ctas_per_sm"] in (0, 2, 3, 4)
        entries = json.load(open(cache))
        assert len(entries) == 1
        (rec,) = entries.values()
        assert rec["sum_lanes"] == r1["sum_lanes"]
        assert set(rec["step_a_ms"]) == {"1", "2", "4", "8"}
        ftp.ftp_batch(plan.h, off, t, y, dy, grid_t, out_off[:-1], bk, tpc, *outs)
        check_curves(off, t, y, dy, grids, bank, tpc, outs[0], out_off, "mixed", theta2=outs[2])
        for lanes, ctas in ((1, 2), (8, 3)):
            ftp.ftp_set_batch_tuning(plan.h, lanes, ctas)
            o2 = [np.empty(tot) for _ in range(4)]
            ftp.ftp_batch(plan.h, off, t, y, dy, grid_t, out_off[:-1], bk, tpc, *o2)
            check_curves(off, t, y, dy, grids, bank, tpc, o2[0], out_off, "mixed", theta2=o2[2])
        with pytest.raises(ftp.FtpError):
            ftp.ftp_set_batch_tuning(plan.h, 9, 0)
    with plan_for(ftp, off, grids, bank, "mixed") as plan2:
        r2 = ftp.ftp_batch_autotune(plan2.h, off, t, y, dy, grid_t, out_off[:-1], bk, tpc, *outs,
                                    cache_path=cache)
        assert r2["from_cache"]
        assert (r2["sum_lanes"], r2["roots_ctas_per_sm"]) == (r1["sum_lanes"],
                                                              r1["roots_ctas_per_sm"])
