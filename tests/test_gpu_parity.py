"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: |dP| <= 1e-4 for mixed precision and <= 1e-9 for the FP64 path,
best phase within 1e-3 rad (mixed) / 1e-6 rad (FP64) at well-separated optima
(best P exceeds every candidate more than 0.05 rad away by >= 1e-3)."""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_P = {"mixed": 1e-4, "fp64": 1e-9}
TOL_PHASE = {"mixed": 1e-3, "fp64": 1e-6}
TOL_AMP = {"mixed": 1e-3, "fp64": 1e-7}


@pytest.fixture(scope="module")
def ftp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp as f
    f.load()
    return f


def phase_err(a, b):
    return np.abs(np.angle(np.exp(1j * (np.asarray(a) - np.asarray(b)))))


def compare(gpu, ref, sel, prec, lc, tpl, freqs, check_phase=True, max_phase_checks=60):
    dP = np.abs(gpu["power"][sel] - ref["power"])
    assert np.max(dP) <= TOL_P[prec], f"max|dP| = {np.max(dP)}"
    if not check_phase:
        return
    # phases / amplitudes only where the optimum is well separated
    order = np.argsort(-ref["power"])[:max_phase_checks]
    checked = 0
    for q in order:
        f = freqs[q]
        margin = oracle.best_candidate_margin(lc.t, lc.y, lc.dy, f, tpl.c, tpl.s, ref["theta2"][q])
        if margin < 1e-3:
            continue
        checked += 1
        k = sel[q]
        assert phase_err(gpu["theta2"][k], ref["theta2"][q]) <= TOL_PHASE[prec]
        assert abs(gpu["theta1"][k] - ref["theta1"][q]) <= TOL_AMP[prec] * max(1, abs(ref["theta1"][q]))
        assert abs(gpu["theta3"][k] - ref["theta3"][q]) <= TOL_AMP[prec] * max(1, abs(ref["theta3"][q]))
    assert checked > 0


@pytest.fixture(scope="module")
def small_workload():
    lc, tpl, grid = synth.small_curve()
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), tpl.c, tpl.s)
    return lc, tpl, grid, ref


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_golden_orthogonal_grid(ftp, orthogonal_grid, prec):
    """The hand-derived closed form in tests/golden/orthogonal_grid.json
    (uniform samples over whole cycles, H = 3): P = A_h^2 / sum A_n^2 where
    harmonic h of the template matches the signal, 0 elsewhere, with the
    matching |theta1|, theta3 and phase; the h-fold tie of the optimum may
    resolve to any of its members."""
    from conftest import check_orthogonal_grid

    cs = orthogonal_grid
    with ftp.Plan(cs["t"].size, 3, (cs["df"], cs["k0"], cs["nf"]), 1, prec) as plan:
        r = plan.periodogram(cs["t"], cs["y"], cs["dy"], [(cs["c"], cs["s"])])
    g = {k: v[0] for k, v in r.items()}
    check_orthogonal_grid(cs, g, TOL_P[prec], TOL_AMP[prec], TOL_PHASE[prec])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_small_workload_every_frequency(ftp, small_workload, prec):
    """N=200, H=3, 5000 frequencies: every frequency against the oracle."""
    lc, tpl, grid, ref = small_workload
    with ftp.Plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        r = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
    g = {k: v[0] for k, v in r.items()}
    sel = np.arange(grid.nf)
    compare(g, ref, sel, prec, lc, tpl, grid.freqs())
    assert np.all(g["power"] >= -1e-12) and np.all(g["power"] <= 1 + 1e-9)
    assert np.mean((g["flags"] & 1) != 0) < 1e-3  # root solver converged


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_sums_against_direct_definition(ftp, prec):
    """Step (a): NFFT sums vs sum_i w_i e^{i h omega t_i} evaluated directly."""
    rng = np.random.default_rng(5)
    lc = synth.random_curve(rng, 300, T=40.0)
    H = 4
    grid = synth.Grid(df=1 / (5 * 40.0), k0=3, nf=777)
    with ftp.Plan(lc.t.size, H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        s, (ybar, YY) = plan.sums(lc.t, lc.y, lc.dy, H)
    w = oracle.normalized_weights(lc.dy)
    yb, yy = oracle.data_moments(lc.y, w)
    assert abs(ybar - yb) <= 1e-14 * max(1, abs(yb)) and abs(YY - yy) <= 1e-13 * yy
    tol = 2e-6 if prec == "mixed" else 1e-12
    freqs = grid.freqs()
    for k in list(range(0, grid.nf, 37)) + [grid.nf - 1]:
        ph = oracle.harmonic_phases(lc.t, freqs[k], 2 * H)
        Z = np.exp(1j * ph) @ w
        Y = np.exp(1j * ph[:H]) @ (w * (lc.y - yb))
        assert np.max(np.abs(s[: 2 * H, k] - Z)) <= tol
        assert np.max(np.abs(s[2 * H:, k] - Y)) <= tol


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("H,n_obs,nf,k0", [(1, 40, 131, 1), (2, 35, 97, 5), (4, 60, 203, 2),
                                          (5, 50, 65, 1), (8, 80, 150, 7), (10, 90, 129, 1),
                                          (16, 120, 70, 3)])
def test_random_cases_across_H(ftp, prec, H, n_obs, nf, k0):
    """Several H (degrees D = 6H-2 from 4 to 94), ragged frequency tails."""
    rng = np.random.default_rng(100 + H)
    tpl = synth.make_template(H, 5000 + H)
    lc = synth.random_curve(rng, n_obs, T=20.0, signal=0.4, tpl=tpl, period=2.3, phase=1.0)
    grid = synth.Grid(df=1 / 100.0, k0=k0, nf=nf)
    with ftp.Plan(n_obs, H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        r = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
    g = {k: v[0] for k, v in r.items()}
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), tpl.c, tpl.s)
    compare(g, ref, np.arange(nf), prec, lc, tpl, grid.freqs(), max_phase_checks=15)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_template_bank_matches_single_calls(ftp, prec):
    """Several templates (mixed H) sharing one set of sums == one call each."""
    rng = np.random.default_rng(9)
    bank = [synth.make_template(H, 6000 + i) for i, H in enumerate((3, 2, 5, 3))]
    lc = synth.random_curve(rng, 70, T=15.0, signal=0.3, tpl=bank[0], period=1.9)
    grid = synth.Grid(df=1 / 75.0, k0=1, nf=333)
    with ftp.Plan(lc.t.size, 5, (grid.df, grid.k0, grid.nf), len(bank), prec) as plan:
        allr = plan.periodogram(lc.t, lc.y, lc.dy, [(b.c, b.s) for b in bank])
        for i, b in enumerate(bank):
            one = plan.periodogram(lc.t, lc.y, lc.dy, [(b.c, b.s)])
            # sums for the bank are built for H = 5; single calls for H_i: same
            # arithmetic on a different grid length, so compare within tolerance
            assert np.max(np.abs(allr["power"][i] - one["power"][0])) <= TOL_P[prec]
    for i in (0, 2):
        ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), bank[i].c, bank[i].s)
        assert np.max(np.abs(allr["power"][i] - ref["power"])) <= TOL_P[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_device_and_host_pointers_agree(ftp, prec):
    """Device-resident inputs/outputs give the host-pointer results.  Spreading
    accumulates in shared memory with atomics, so the two runs agree to
    rounding, not bit for bit."""
    lc, tpl, grid = synth.small_curve(nf=700)
    dev = torch.device("cuda:0")
    with ftp.Plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        host = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
        td = [torch.from_numpy(a).to(dev) for a in (lc.t, lc.y, lc.dy)]
        outs = [torch.empty(grid.nf, dtype=torch.float64, device=dev) for _ in range(4)]
        fl = torch.empty(grid.nf, dtype=torch.uint8, device=dev)
        ftp.ftp_periodogram(plan.h, *td, lc.t.size, [(tpl.c, tpl.s)], *outs, fl)
        torch.cuda.synchronize()
    p_dev = outs[0].cpu().numpy()
    tol = 1e-6 if prec == "mixed" else 1e-13
    assert np.max(np.abs(p_dev - host["power"][0])) <= tol
    same = phase_err(outs[2].cpu().numpy(), host["theta2"][0]) <= TOL_PHASE[prec]
    assert np.mean(same) >= 0.99


@pytest.mark.parametrize("n_obs", [300, 5000])
def test_stage_timing_and_both_preparation_paths(ftp, n_obs):
    """Stage events: the first root kernel's time is positive and inside the
    root stage.  300 observations take the single-CTA step (a) preparation,
    5000 the multi-kernel one; both agree with the oracle."""
    rng = np.random.default_rng(40 + n_obs)
    tpl = synth.make_template(4, 4040)
    lc = synth.random_curve(rng, n_obs, T=60.0, signal=0.3, tpl=tpl, period=3.1, phase=0.4)
    grid = synth.Grid(df=1 / (5 * 60.0), k0=1, nf=900)
    dev = torch.device("cuda:0")
    with ftp.Plan(n_obs, tpl.H, (grid.df, grid.k0, grid.nf), 1, "mixed") as plan:
        td = [torch.from_numpy(a).to(dev) for a in (lc.t, lc.y, lc.dy)]
        outs = [torch.empty(grid.nf, dtype=torch.float64, device=dev) for _ in range(4)]
        ftp.ftp_set_timing(plan.h, True)
        ftp.ftp_periodogram(plan.h, *td, n_obs, [(tpl.c, tpl.s)], *outs, None)
        torch.cuda.synchronize()
        st = ftp.ftp_stage_times(plan.h)
        first = ftp.ftp_roots_first_phase_ms(plan.h)
        ftp.ftp_set_timing(plan.h, False)
    assert all(v >= 0 for v in st) and st[4] > 0
    assert 0 < first <= st[4]
    sel = np.arange(0, grid.nf, 7)
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs()[sel], tpl.c, tpl.s)
    assert np.max(np.abs(outs[0].cpu().numpy()[sel] - ref["power"])) <= TOL_P["mixed"]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_input_errors(ftp, prec):
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 10, 50))
    y = rng.normal(size=50)
    dy = rng.uniform(0.1, 0.2, 50)
    tpl = [(np.array([1.0, 0.3]), np.array([0.2, 0.1]))]
    with ftp.Plan(64, 2, (0.01, 1, 100), 1, prec) as plan:
        cases = [
            ((t, np.full(50, 3.0), dy), 2),            # zero variance
            ((t, y, np.where(np.arange(50) == 7, 0.0, dy)), 3),  # mixed zero sigma
            ((t, np.where(np.arange(50) == 3, np.nan, y), dy), 4),
            ((t, y, np.where(np.arange(50) == 3, -0.1, dy)), 4),
        ]
        for (tt, yy, dd), code in cases:
            with pytest.raises(ftp.FtpError) as e:
                plan.periodogram(tt, yy, dd, tpl)
            assert e.value.status == code
        with pytest.raises(ftp.FtpError) as e:  # too many observations for the plan
            plan.periodogram(np.arange(70.0), np.arange(70.0), np.ones(70), tpl)
        assert e.value.status == 8
        with pytest.raises(ftp.FtpError) as e:  # H above the plan's
            plan.periodogram(t, y, dy, [(np.ones(3), np.ones(3))])
        assert e.value.status == 8
        with pytest.raises(ftp.FtpError) as e:  # single observation
            plan.periodogram(t[:1], y[:1], dy[:1], tpl)
        assert e.value.status == 1
        # the plan stays usable after errors; all-zero sigma = unit weights
        r0 = plan.periodogram(t, y, np.zeros(50), tpl)
        r1 = plan.periodogram(t, y, np.ones(50), tpl)
        np.testing.assert_allclose(r0["power"], r1["power"], rtol=0,
                                   atol=1e-6 if prec == "mixed" else 1e-12)
        ref = oracle.periodogram(t, y, np.ones(50), np.arange(1, 101) * 0.01, tpl[0][0], tpl[0][1])
        assert np.max(np.abs(r0["power"][0] - ref["power"])) <= TOL_P[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_two_points_and_unsorted_times(ftp, prec):
    """Degenerate sizes: N = 2 (P = 1 is reachable) and unsorted input times."""
    rng = np.random.default_rng(11)
    tpl = synth.make_template(3, 7000)
    lc = synth.random_curve(rng, 45, T=12.0, signal=0.5, tpl=tpl, sort=False)
    grid = synth.Grid(df=1 / 60.0, k0=1, nf=150)
    with ftp.Plan(45, 3, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        r = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
        order = np.argsort(lc.t)
        rs = plan.periodogram(lc.t[order], lc.y[order], lc.dy[order], [(tpl.c, tpl.s)])
        r2 = plan.periodogram(lc.t[:2], lc.y[:2], lc.dy[:2], [(tpl.c, tpl.s)])
    assert np.max(np.abs(r["power"] - rs["power"])) <= TOL_P[prec]
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), tpl.c, tpl.s)
    assert np.max(np.abs(r["power"][0] - ref["power"])) <= TOL_P[prec]
    ref2 = oracle.periodogram(lc.t[:2], lc.y[:2], lc.dy[:2], grid.freqs(), tpl.c, tpl.s)
    assert np.max(np.abs(r2["power"][0] - ref2["power"])) <= TOL_P[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_matches_oracle(ftp, prec):
    """ftp_batch over curves of uneven size and grid, one template per curve
    and all templates per curve."""
    sv = synth.survey(ncurves=6, n_bank=3, median_obs=60, min_obs=20, max_obs=200,
                      f_max=1.0, baseline=(30, 80), seed=77)
    bank = [(b.c, b.s) for b in sv.bank]
    grids = [(g.df, g.k0, g.nf) for g in sv.grids]
    maxnf = max(g.nf for g in sv.grids)
    maxJ_grid = max(sv.grids, key=lambda g: g.k0 + g.nf)
    plan_grid = (maxJ_grid.df, maxJ_grid.k0, maxnf)
    Hmax = max(b.H for b in sv.bank)
    with ftp.Plan(int(np.max(np.diff(sv.obs_off))), Hmax, plan_grid, len(bank), prec) as plan:
        # one template per curve
        out_off = np.zeros(sv.ncurves + 1, dtype=np.int64)
        out_off[1:] = np.cumsum([g.nf for g in sv.grids])
        tot = int(out_off[-1])
        o = [np.zeros(tot) for _ in range(4)]
        fl = np.zeros(tot, dtype=np.uint8)
        ftp.ftp_batch(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids, out_off[:-1], bank,
                      sv.tpl_of_curve, *o, fl)
        for c in range(sv.ncurves):
            lc = sv.curve(c)
            tp = sv.bank[sv.tpl_of_curve[c]]
            g = sv.grids[c]
            ref = oracle.periodogram(lc.t, lc.y, lc.dy, g.freqs(), tp.c, tp.s)
            p = o[0][out_off[c]:out_off[c + 1]]
            assert np.max(np.abs(p - ref["power"])) <= TOL_P[prec]
        # every template on every curve
        out2 = np.zeros(sv.ncurves + 1, dtype=np.int64)
        out2[1:] = np.cumsum([len(bank) * g.nf for g in sv.grids])
        o2 = [np.zeros(int(out2[-1])) for _ in range(4)]
        ftp.ftp_batch(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, grids, out2[:-1], bank, None, *o2)
        c = 2
        lc = sv.curve(c)
        g = sv.grids[c]
        for i, tp in enumerate(sv.bank):
            ref = oracle.periodogram(lc.t, lc.y, lc.dy, g.freqs(), tp.c, tp.s)
            a = out2[c] + i * g.nf
            assert np.max(np.abs(o2[0][a:a + g.nf] - ref["power"])) <= TOL_P[prec]
        # a curve whose grid reaches past the largest supported bin (here so
        # far that 2 H (k0 + nf - 1) would overflow) is rejected on the host
        # before any work is queued
        bad = list(grids)
        bad[1] = (grids[1][0], 2**62, grids[1][2])
        with pytest.raises(ftp.FtpError) as e:
            ftp.ftp_batch(plan.h, sv.obs_off, sv.t, sv.y, sv.dy, bad, out_off[:-1], bank,
                          sv.tpl_of_curve, *o, fl)
        assert e.value.status == 8


@pytest.fixture(scope="module")
def long_workload(ftp):
    """The full single-curve workload: N=1e4 over 3000 nights, H=6, 2.5e5 freqs."""
    lc, tpl, grid = synth.long_curve()
    res = {}
    for prec in ("mixed", "fp64"):
        with ftp.Plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
            res[prec] = {k: (v[0] if v is not None else None) for k, v in
                         plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)]).items()}
    rng = np.random.default_rng(0)
    sel = np.sort(np.concatenate([rng.choice(grid.nf, 60, replace=False),
                                  np.argsort(-res["mixed"]["power"])[:20]]))
    sel = np.unique(sel)
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs()[sel], tpl.c, tpl.s)
    return lc, tpl, grid, res, sel, ref


def test_long_workload_mixed_vs_fp64_every_frequency(long_workload):
    lc, tpl, grid, res, sel, ref = long_workload
    d = np.abs(res["mixed"]["power"] - res["fp64"]["power"])
    assert np.max(d) <= 1e-4, np.max(d)
    k = int(np.argmax(res["mixed"]["power"]))
    assert abs(grid.freqs()[k] - 1 / 0.63) <= 2 * grid.df


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_long_workload_sampled_against_oracle(long_workload, prec):
    lc, tpl, grid, res, sel, ref = long_workload
    compare(res[prec], ref, sel, prec, lc, tpl, grid.freqs()[sel], max_phase_checks=10)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_resolves_ill_conditioned_frequencies(ftp, prec):
    """With three observations MM = Var(M) is tiny wherever their phases
    cluster, a small difference of O(1) NFFT sums: the a-posteriori error
    estimate sends those frequencies to the direct-FP64 re-solve, and the
    result meets the path's tolerance everywhere."""
    rng = np.random.default_rng(21)
    tpl = synth.make_template(2, 8000)
    lc = synth.random_curve(rng, 3, T=10.0, signal=0.6, tpl=tpl, period=3.0)
    grid = synth.Grid(df=1 / 50.0, k0=1, nf=200)
    with ftp.Plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        r = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
        stats = plan.solver_stats()
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), tpl.c, tpl.s)
    assert np.max(np.abs(r["power"][0] - ref["power"])) <= TOL_P[prec]
    assert stats["resolved"] >= 1


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_positive_amplitude_mode(ftp, prec):
    """ftp_set_positive_amplitude: every frequency of a curve with a negative
    injected amplitude against the oracle's positive-amplitude periodogram
    (best candidate with theta1 > 0, else P = 0), in a single call and in a
    batch; the mode switches back off."""
    rng = np.random.default_rng(77)
    tpl = synth.make_template(3, 3200)
    lc = synth.random_curve(rng, 120, T=20.0, signal=-0.5, tpl=tpl, period=2.3, phase=0.6)
    nf = 900
    grid = synth.Grid(df=1 / 100.0, k0=1, nf=nf)
    freqs = grid.freqs()
    ref = oracle.periodogram(lc.t, lc.y, lc.dy, freqs, tpl.c, tpl.s, positive_only=True)
    free_ref = oracle.periodogram(lc.t, lc.y, lc.dy, freqs, tpl.c, tpl.s)
    assert np.any(free_ref["theta1"] < 0)
    with ftp.Plan(lc.t.size, tpl.H, (grid.df, grid.k0, nf), 1, prec) as plan:
        ftp.ftp_set_positive_amplitude(plan.h, True)
        r = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
        g = {k: v[0] for k, v in r.items()}
        out = [np.empty(nf) for _ in range(4)]
        fl = np.empty(nf, dtype=np.uint8)
        ftp.ftp_batch(plan.h, np.array([0, lc.t.size]), lc.t, lc.y, lc.dy,
                      [(grid.df, grid.k0, nf)], np.array([0]), [(tpl.c, tpl.s)], None, *out, fl)
        ftp.ftp_set_positive_amplitude(plan.h, False)
        r2 = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
    sel = np.arange(nf)
    compare(g, ref, sel, prec, lc, tpl, freqs, check_phase=False)
    assert np.max(np.abs(out[0] - ref["power"])) <= TOL_P[prec]
    assert np.all(g["theta1"][g["power"] > 0] > 0)
    none = (ref["flags"] & oracle.FLAG_NO_POSITIVE) != 0
    assert np.all((g["flags"][none] & ftp.FLAG_NO_POSITIVE) != 0)
    assert np.all(g["power"][none] == 0.0) and np.all(g["theta3"][none] == pytest.approx(
        np.average(lc.y, weights=lc.dy ** -2.0), abs=1e-9))
    assert np.max(np.abs(r2["power"][0] - free_ref["power"])) <= TOL_P[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_multiband_periodogram(ftp, prec):
    """ftp_multiband_periodogram: three bands of different size, noise level,
    offset and template (H = 2, 3, 4) on one grid, every frequency against the
    oracle's multi-phase combination (Eq. multibandmultiphase); per-band
    outputs against the single-band oracle; host and device outputs agree."""
    rng = np.random.default_rng(88)
    bands = []
    for b, (n, sig, H) in enumerate([(90, (0.05, 0.1), 3), (40, (0.1, 0.3), 2),
                                     (150, (0.02, 0.05), 4)]):
        tpl = synth.make_template(H, 3400 + b)
        lc = synth.random_curve(rng, n, T=25.0, signal=0.3 + 0.2 * b, tpl=tpl, period=3.1,
                                phase=0.5 * b, sigma=sig)
        bands.append((lc.t, lc.y + 1.5 * b, lc.dy, tpl))
    nf = 700
    grid = synth.Grid(df=1 / 125.0, k0=1, nf=nf)
    freqs = grid.freqs()
    ref = oracle.multiband_periodogram([(t, y, dy, tp.c, tp.s) for t, y, dy, tp in bands], freqs)
    off = np.cumsum([0] + [b[0].size for b in bands]).astype(np.int64)
    t = np.concatenate([b[0] for b in bands])
    y = np.concatenate([b[1] for b in bands])
    dy = np.concatenate([b[2] for b in bands])
    bank = [(tp.c, tp.s) for *_, tp in bands]
    with ftp.Plan(int(np.max(np.diff(off))), 4, (grid.df, grid.k0, nf), 3, prec) as plan:
        p = np.empty(nf)
        bp = np.empty((3, nf))
        ftp.ftp_multiband_periodogram(plan.h, off, t, y, dy, bank, np.arange(3), p, bp)
        pd = torch.empty(nf, dtype=torch.float64, device="cuda")
        ftp.ftp_multiband_periodogram(plan.h, off, torch.from_numpy(t).cuda(),
                                      torch.from_numpy(y).cuda(), torch.from_numpy(dy).cuda(),
                                      bank, np.arange(3), pd)
    assert np.max(np.abs(p - ref["power"])) <= TOL_P[prec]
    assert np.max(np.abs(bp - ref["band_power"])) <= TOL_P[prec]
    assert np.max(np.abs(pd.cpu().numpy() - p)) <= 2 * TOL_P[prec]
    assert np.all(p >= bp.min(axis=0) - 1e-12) and np.all(p <= bp.max(axis=0) + 1e-12)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_golden_shared_phase_orthogonal(ftp, prec):
    """ftp_shared_multiband on the hand-derived two-band closed form of
    tests/golden/shared_phase_orthogonal.json (Appendix A): P = |Z|^2/(YY MM)
    where a harmonic matches, 0 elsewhere, with |theta1|, theta3 and phase."""
    from conftest import check_shared_orthogonal, shared_orthogonal_case

    bands, lam, freqs, expect = shared_orthogonal_case()
    off = np.cumsum([0] + [b[0].size for b in bands]).astype(np.int64)
    t, y, dy = (np.concatenate([b[i] for b in bands]) for i in range(3))
    bank = [(b[3], b[4]) for b in bands]
    nf = freqs.size
    with ftp.Plan(int(np.max(np.diff(off))), 3, (freqs[0], 1, nf), 2, prec) as plan:
        out = [np.empty(nf) for _ in range(4)]
        ftp.ftp_shared_multiband(plan.h, off, t, y, dy, lam, bank, np.arange(2), *out)
    r = dict(zip(("power", "theta1", "theta2", "theta3"), out))
    check_shared_orthogonal(expect, r, TOL_P[prec], TOL_AMP[prec], TOL_PHASE[prec])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_golden_multiphase_orthogonal(ftp, prec):
    """ftp_multiband_periodogram on the same two orthogonal bands: per-band
    powers and the chi2_0-weighted combination (Eq. multibandmultiphase)
    equal the closed form."""
    from conftest import multiphase_orthogonal_expect, shared_orthogonal_case

    bands, _, freqs, _ = shared_orthogonal_case()
    Pb, P = multiphase_orthogonal_expect()
    off = np.cumsum([0] + [b[0].size for b in bands]).astype(np.int64)
    t, y, dy = (np.concatenate([b[i] for b in bands]) for i in range(3))
    bank = [(b[3], b[4]) for b in bands]
    nf = freqs.size
    with ftp.Plan(int(np.max(np.diff(off))), 3, (freqs[0], 1, nf), 2, prec) as plan:
        p = np.empty(nf)
        bp = np.empty((2, nf))
        ftp.ftp_multiband_periodogram(plan.h, off, t, y, dy, bank, np.arange(2), p, bp)
    assert np.max(np.abs(bp - Pb)) <= TOL_P[prec]
    assert np.max(np.abs(p - P)) <= TOL_P[prec]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_shared_phase_multiband(ftp, prec):
    """ftp_shared_multiband: three bands with their own templates (H = 2, 3, 3)
    and fixed offsets sharing one amplitude, phase and offset, every frequency
    against the oracle's pooled Appendix A periodogram; host and device
    arrays agree; a single band reproduces ftp_periodogram."""
    rng = np.random.default_rng(99)
    bands, lam = [], np.array([0.0, 1.1, -0.6])
    for b, (n, H) in enumerate([(80, 3), (50, 2), (120, 3)]):
        tpl = synth.make_template(H, 3600 + b)
        t = np.sort(rng.uniform(0, 30.0, n))
        dy = rng.uniform(0.05, 0.15, n)
        y = 0.5 * tpl(2 * np.pi * t / 2.9 - 0.4) + 0.1 + lam[b] + dy * rng.standard_normal(n)
        bands.append((t, y, dy, tpl))
    nf = 800
    grid = synth.Grid(df=1 / 150.0, k0=1, nf=nf)
    freqs = grid.freqs()
    ref = oracle.shared_phase_multiband([(t, y, dy, tp.c, tp.s) for t, y, dy, tp in bands], freqs,
                                        lam)
    off = np.cumsum([0] + [b[0].size for b in bands]).astype(np.int64)
    t = np.concatenate([b[0] for b in bands])
    y = np.concatenate([b[1] for b in bands])
    dy = np.concatenate([b[2] for b in bands])
    bank = [(tp.c, tp.s) for *_, tp in bands]
    with ftp.Plan(int(np.max(np.diff(off))), 3, (grid.df, grid.k0, nf), 3, prec) as plan:
        out = [np.empty(nf) for _ in range(4)]
        fl = np.empty(nf, dtype=np.uint8)
        ftp.ftp_shared_multiband(plan.h, off, t, y, dy, lam, bank, np.arange(3), *out, fl)
        dev = [torch.empty(nf, dtype=torch.float64, device="cuda") for _ in range(4)]
        ftp.ftp_shared_multiband(plan.h, off, *(torch.from_numpy(a).cuda() for a in (t, y, dy)),
                                 lam, bank, np.arange(3), *dev)
        one = [np.empty(nf) for _ in range(4)]
        ftp.ftp_shared_multiband(plan.h, off[:2], t, y, dy, None, bank, None, *one)
        single = plan.periodogram(bands[0][0], bands[0][1], bands[0][2], [bank[0]])
    dP = np.abs(out[0] - ref["power"])
    assert dP.max() <= TOL_P[prec], dP.max()
    g = {"power": out[0], "theta1": out[1], "theta2": out[2], "theta3": out[3]}
    k = int(np.argmax(ref["power"]))
    assert phase_err(g["theta2"][k], ref["theta2"][k]) <= TOL_PHASE[prec]
    assert abs(g["theta1"][k] - ref["theta1"][k]) <= TOL_AMP[prec] * max(1, abs(ref["theta1"][k]))
    assert abs(g["theta3"][k] - ref["theta3"][k]) <= TOL_AMP[prec] * max(1, abs(ref["theta3"][k]))
    assert np.max(np.abs(dev[0].cpu().numpy() - out[0])) <= 2 * TOL_P[prec]
    assert np.max(np.abs(one[0] - single["power"][0])) <= 2 * TOL_P[prec]
