"""The template-bank path at the shape it has at full size, scaled only in the
number of frequencies: the N = 1e5 lightcurve over 4000 nights with nightly
gaps, all 32 seeded H = 10 templates (final polynomial of degree 58) sharing
one set of NFFT sums, N_f = 2e4 of its frequencies f_k = k / (5 * 4000 d).

Both precisions are compared with the FP64 oracle on a seeded sample of
(frequency, template) items, on the five highest peaks of four templates
(with phase, amplitude and offset where the optimum is well separated), and
on every item the solver re-solved (FTP_FLAG_RESOLVED: ill-conditioned, or an
item of the frequency hit the Aberth cap).  No item may be left unconverged,
since Section 2 takes every stationary point as a candidate.  Mixed and FP64
are also compared with each other on every item."""
import numpy as np
import pytest

import __graft_entry__
import synth
from oracle_pool import oracle_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_P = {"mixed": 1e-4, "fp64": 1e-9}
TOL_PHASE = {"mixed": 1e-3, "fp64": 1e-6}
TOL_AMP = {"mixed": 1e-3, "fp64": 1e-7}
NF = 20_000
MAX_RESOLVED_CHECKED = 48


@pytest.fixture(scope="module")
def ftp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp as f
    f.load()
    return f


@pytest.fixture(scope="module")
def bank_run(ftp):
    lc, bank, grid = synth.bank_curve()
    templates = [(b.c, b.s) for b in bank]
    res, stats = {}, {}
    for prec in ("mixed", "fp64"):
        with ftp.Plan(lc.t.size, 10, (grid.df, grid.k0, NF), len(bank), prec) as plan:
            res[prec] = plan.periodogram(lc.t, lc.y, lc.dy, templates)
            stats[prec] = plan.solver_stats()
    freqs = grid.df * (grid.k0 + np.arange(NF))
    rng = np.random.default_rng(55)
    items = {(int(rng.integers(len(bank))), int(k)) for k in rng.choice(NF, 16, replace=False)}
    peaks = set()
    for ti in range(4):
        for k in np.argsort(-res["mixed"]["power"][ti])[:5]:
            peaks.add((ti, int(k)))
    resolved = set()
    for prec in ("mixed", "fp64"):
        for ti, k in np.argwhere(res[prec]["flags"] & ftp.FLAG_RESOLVED):
            resolved.add((int(ti), int(k)))
    resolved = sorted(resolved)
    if len(resolved) > MAX_RESOLVED_CHECKED:
        pick = rng.choice(len(resolved), MAX_RESOLVED_CHECKED, replace=False)
        resolved = [resolved[i] for i in sorted(pick)]
    check = sorted(items | peaks | set(resolved))
    by_tpl = {}
    for ti, k in check:
        by_tpl.setdefault(ti, []).append(k)
    jobs, keys = [], []
    for ti, ks in sorted(by_tpl.items()):
        for k in ks:  # one job per item: the pool balances them
            jobs.append((lc.t, lc.y, lc.dy, freqs[[k]], bank[ti].c, bank[ti].s,
                         (ti, k) in peaks))
            keys.append((ti, k))
    refs = dict(zip(keys, oracle_map(jobs)))
    return lc, bank, grid, res, stats, refs, peaks, resolved


def phase_err(a, b):
    return float(np.abs(np.angle(np.exp(1j * (a - b)))))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_bank_full_shape_against_oracle(bank_run, prec):
    lc, bank, grid, res, stats, refs, peaks, resolved = bank_run
    st = stats[prec]
    assert st["items"] == len(bank) * NF
    assert st["still_nonconverged"] == 0, st
    r = res[prec]
    assert not np.any(r["flags"] & 1)  # FTP_FLAG_NONCONVERGED
    worst = 0.0
    phases = 0
    for (ti, k), ref in refs.items():
        d = abs(r["power"][ti, k] - ref["power"][0])
        worst = max(worst, d)
        assert d <= TOL_P[prec], ((ti, k), r["power"][ti, k], ref["power"][0])
        if (ti, k) in peaks and ref["margin"][0] >= 1e-3:
            phases += 1
            assert phase_err(r["theta2"][ti, k], ref["theta2"][0]) <= TOL_PHASE[prec]
            for q in ("theta1", "theta3"):
                assert abs(r[q][ti, k] - ref[q][0]) <= TOL_AMP[prec] * max(1, abs(ref[q][0]))
    assert phases > 0
    print(f"{prec}: {len(refs)} items vs oracle, max|dP| {worst:.2e}; {len(resolved)} "
          f"re-solved items checked; stats {st}")


def test_bank_full_shape_mixed_vs_fp64_every_item(bank_run):
    lc, bank, grid, res, stats, refs, peaks, resolved = bank_run
    d = np.abs(res["mixed"]["power"] - res["fp64"]["power"])
    assert np.max(d) <= TOL_P["mixed"], float(np.max(d))
    assert np.all((res["mixed"]["power"] >= 0) & (res["mixed"]["power"] <= 1))
