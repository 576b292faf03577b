"""Early settling of off-circle Aberth roots (the mixed path's main root kernel
at H >= 8) against the FP64 oracle on every frequency.

Only zeros of F on the unit circle are stationary points of P (Section 2, end
of the method), so the kernel lets a root stop iterating once its correction
is a small Newton step and the root lies far off the circle.  A root wrongly
settled would leave a circle zero unfound, and the best power would then
miss that stationary point wherever it is the maximum.  These cases run the
settling kernel at H = 8, 12, 16 (D = 46, 70, 94) on a nightly-gap curve and
compare every frequency with the oracle (both precisions; the FP64 path never
settles, so mixed against FP64 at every frequency checks it independently
too), with phases, amplitudes and offsets at well-separated optima, and no
item left unconverged."""
import numpy as np
import pytest

import __graft_entry__
import synth
from oracle_pool import oracle_map
from test_gpu_parity import TOL_P, compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NIGHTS, NOBS = 300, 1000
K0, NF = 1800, 1200          # f in [1.2, 2.0] /d around the signal at 1/0.63 /d


def settle_case(H: int):
    rng = np.random.default_rng(3000 + H)
    tpl = synth.make_template(H, 2100 + H)
    t = synth.nightly_times(rng, NIGHTS, NOBS)
    dy = rng.uniform(0.05, 0.15, NOBS)
    y = 0.1 * tpl(2.0 * np.pi * t / 0.63 - 1.3) + dy * rng.standard_normal(NOBS)
    grid = synth.Grid(df=1.0 / (5.0 * NIGHTS), k0=K0, nf=NF)
    return synth.Lightcurve(t, y, dy), tpl, grid


@pytest.fixture(scope="module")
def ftp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp as f
    f.load()
    return f


@pytest.fixture(scope="module")
def settle_runs(ftp):
    cases = {H: settle_case(H) for H in (8, 12, 16)}
    # the oracle on every frequency, split in blocks over a spawn pool
    jobs, where = [], []
    for H, (lc, tpl, grid) in cases.items():
        f = grid.freqs()
        for blk in np.array_split(np.arange(NF), 24):
            jobs.append((lc.t, lc.y, lc.dy, f[blk], tpl.c, tpl.s))
            where.append((H, blk))
    parts = oracle_map(jobs)
    refs = {H: {k: np.zeros(NF) for k in ("power", "theta1", "theta2", "theta3")} for H in cases}
    for (H, blk), r in zip(where, parts):
        for k in refs[H]:
            refs[H][k][blk] = r[k]
    gpu = {}
    for H, (lc, tpl, grid) in cases.items():
        for prec in ("mixed", "fp64"):
            with ftp.Plan(lc.t.size, H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
                out = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
                stats = plan.solver_stats()
            gpu[H, prec] = ({k: (v[0] if v is not None else None) for k, v in out.items()}, stats)
    return cases, refs, gpu


@pytest.mark.parametrize("H", [8, 12, 16])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_settled_roots_every_frequency_against_oracle(ftp, settle_runs, H, prec):
    cases, refs, gpu = settle_runs
    lc, tpl, grid = cases[H]
    res, stats = gpu[H, prec]
    sel = np.arange(NF)
    compare(res, refs[H], sel, prec, lc, tpl, grid.freqs(), max_phase_checks=20)
    assert stats["still_nonconverged"] == 0, stats
    left = res["flags"] & (ftp.FLAG_NONCONVERGED | ftp.FLAG_UNRESOLVED)
    assert not np.any(left), "unresolved or non-converged items left"


@pytest.mark.parametrize("H", [8, 12, 16])
def test_settled_roots_mixed_vs_fp64_every_frequency(settle_runs, H):
    cases, refs, gpu = settle_runs
    d = np.abs(gpu[H, "mixed"][0]["power"] - gpu[H, "fp64"][0]["power"])
    assert np.max(d) <= TOL_P["mixed"], np.max(d)
