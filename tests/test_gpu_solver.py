"""The root solver's failure paths, made to fire without any GPU fault.

- An Aberth iteration cap of 1 leaves (nearly) every item unconverged: the
  items are counted, their frequencies re-solved from direct FP64 sums with
  the re-solve cap (Section 2 needs every stationary point as a candidate, so
  a root that did not converge is not just reported), and the results meet
  the oracle's tolerance.
- A cap of 1 in the re-solve too leaves FTP_FLAG_NONCONVERGED on the items
  and counts them as still unconverged; the plan works normally afterwards.
- Fault injection: the roots kernels arm their waits for the staged sum tiles
  but never issue the copies, so each bounded wait runs out (a short host-set
  poll limit), the call returns FTP_ERR_TIMEOUT, and the next call on the same
  plan succeeds.  No copy is ever in flight, nothing faults or hangs.
- The self-checking build (-DFTP_DEVICE_CHECKS: every guarded index and
  alignment check compiled in) runs the small workload to parity with no
  check failing."""
import os
import subprocess
import sys

import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_P = {"mixed": 1e-4, "fp64": 1e-9}
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ftp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2101_12348_gb300 import ftp as f
    f.load()
    return f


@pytest.fixture(scope="module")
def case():
    """Small curve (N = 200, H = 3) on 600 frequencies, and a second, H = 2
    template, with the oracle's results for both."""
    lc, tpl, grid = synth.small_curve(nf=600)
    bank = [tpl, synth.make_template(2, 9101)]
    refs = [oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), b.c, b.s) for b in bank]
    return lc, bank, grid, refs


def run(ftp, plan, lc, bank):
    return plan.periodogram(lc.t, lc.y, lc.dy, [(b.c, b.s) for b in bank])


def check_parity(r, refs, prec):
    for i, ref in enumerate(refs):
        d = np.abs(r["power"][i] - ref["power"])
        assert np.max(d) <= TOL_P[prec], (i, float(np.max(d)))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_iteration_cap_hits_are_resolved(ftp, case, prec):
    lc, bank, grid, refs = case
    with ftp.Plan(lc.t.size, 3, (grid.df, grid.k0, grid.nf), 2, prec) as plan:
        plan.set_solver_limits(maxit=1)
        r = run(ftp, plan, lc, bank)
        st = plan.solver_stats()
        items = 2 * grid.nf
        assert st["items"] == items
        # one iteration from the Newton-polygon start converges nothing
        assert st["nonconverged"] >= 0.9 * items, st
        assert st["resolved_nonconverged"] >= 0.9 * grid.nf, st
        assert st["resolved"] >= st["resolved_nonconverged"]
        assert st["still_nonconverged"] == 0, st
        fl = r["flags"]
        assert not np.any(fl & ftp.FLAG_NONCONVERGED)
        assert np.count_nonzero(np.any(fl & ftp.FLAG_RESOLVED, axis=0)) == st["resolved"]
        check_parity(r, refs, prec)
        # back to the default caps: the main pass converges on its own
        plan.set_solver_limits()
        r2 = run(ftp, plan, lc, bank)
        st2 = plan.solver_stats()
        assert st2["nonconverged"] == 0 and st2["still_nonconverged"] == 0, st2
        check_parity(r2, refs, prec)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cap_left_after_resolve_is_flagged_and_counted(ftp, case, prec):
    lc, bank, grid, refs = case
    with ftp.Plan(lc.t.size, 3, (grid.df, grid.k0, grid.nf), 2, prec) as plan:
        plan.set_solver_limits(maxit=1, redo_maxit=1)
        r = run(ftp, plan, lc, bank)
        st = plan.solver_stats()
        flagged = np.count_nonzero(r["flags"] & ftp.FLAG_NONCONVERGED)
        assert flagged > 0 and st["still_nonconverged"] == flagged, (flagged, st)
        assert np.all(np.isfinite(r["power"]))
        assert np.all((r["power"] >= -1e-12) & (r["power"] <= 1 + 1e-12))
        plan.set_solver_limits()
        check_parity(run(ftp, plan, lc, bank), refs, prec)


def test_solver_limits_are_validated(ftp, case):
    lc, bank, grid, _ = case
    with ftp.Plan(lc.t.size, 3, (grid.df, grid.k0, grid.nf), 2, "mixed") as plan:
        for bad in ((-1, 0, 0), (0, -1, 0), (0, 0, -5), (200000, 0, 0)):
            with pytest.raises(ftp.FtpError) as e:
                plan.set_solver_limits(*bad)
            assert e.value.status == 1
        with pytest.raises(ftp.FtpError) as e:
            ftp.ftp_set_fault_injection(plan.h, 2)
        assert e.value.status == 1


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_timeout_status_and_recovery(ftp, case, prec):
    lc, bank, grid, refs = case
    templates = [(b.c, b.s) for b in bank]
    with ftp.Plan(lc.t.size, 3, (grid.df, grid.k0, grid.nf), 2, prec) as plan:
        plan.set_solver_limits(wait_polls=256)
        ftp.ftp_set_fault_injection(plan.h, 1)
        with pytest.raises(ftp.FtpError) as e:
            plan.periodogram(lc.t, lc.y, lc.dy, templates)
        assert e.value.status == 7  # FTP_ERR_TIMEOUT
        # the batched path reports it the same way (host arrays: eager launches)
        off = np.array([0, lc.t.size], dtype=np.int64)
        outs = [np.empty(2 * grid.nf) for _ in range(4)]
        with pytest.raises(ftp.FtpError) as e:
            ftp.ftp_batch(plan.h, off, lc.t, lc.y, lc.dy, [(grid.df, grid.k0, grid.nf)],
                          np.zeros(1, dtype=np.int64), templates, None, *outs)
        assert e.value.status == 7
        ftp.ftp_set_fault_injection(plan.h, 0)
        plan.set_solver_limits()
        check_parity(plan.periodogram(lc.t, lc.y, lc.dy, templates), refs, prec)
        ftp.ftp_batch(plan.h, off, lc.t, lc.y, lc.dy, [(grid.df, grid.k0, grid.nf)],
                      np.zeros(1, dtype=np.int64), templates, None, *outs)
        for i, ref in enumerate(refs):
            assert np.max(np.abs(outs[0][i * grid.nf:(i + 1) * grid.nf] - ref["power"])) \
                <= TOL_P[prec]


_CHECKED_RUN = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle, synth
from paper_2101_12348_gb300 import ftp
assert ftp.LIB_PATH.endswith("libftp_gb300_checks.so"), ftp.LIB_PATH
lc, tpl, grid = synth.small_curve(nf=700)
ref = oracle.periodogram(lc.t, lc.y, lc.dy, grid.freqs(), tpl.c, tpl.s)
for prec, tol in (("mixed", 1e-4), ("fp64", 1e-9)):
    with ftp.Plan(lc.t.size, tpl.H, (grid.df, grid.k0, grid.nf), 1, prec) as plan:
        r = plan.periodogram(lc.t, lc.y, lc.dy, [(tpl.c, tpl.s)])
        off = np.array([0, lc.t.size], dtype=np.int64)
        outs = [np.empty(grid.nf) for _ in range(4)]
        ftp.ftp_batch(plan.h, off, lc.t, lc.y, lc.dy, [(grid.df, grid.k0, grid.nf)],
                      np.zeros(1, dtype=np.int64), [(tpl.c, tpl.s)], None, *outs)
    d = max(np.max(np.abs(r["power"][0] - ref["power"])), np.max(np.abs(outs[0] - ref["power"])))
    assert d <= tol, (prec, d)
    print(prec, "max|dP|", d)
"""


def test_self_checking_build_runs_to_parity(ftp):
    from paper_2101_12348_gb300 import build
    lib = build.build(checks=True)
    env = dict(os.environ, FTP_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", _CHECKED_RUN, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "device check failed" not in r.stderr, r.stderr
    assert "mixed max|dP|" in r.stdout and "fp64 max|dP|" in r.stdout
