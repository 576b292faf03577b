"""The allocation-free entry point agrees with the ordinary one.

ftp_periodogram_sums_noalloc exists for callers that cannot call cudaMalloc
(a process whose device memory belongs to another runtime's pool, a
latency-bound loop that cannot afford an allocation's implicit
synchronisation, a service under a hard memory cap): it runs the root stage on
sums the caller already holds, with its scratch in a fixed array inside the
library.  Here the sums come from ftp_sums, are copied into a padded device
buffer, and two consecutive allocation-free calls are compared with
ftp_periodogram on the same lightcurve, within the parity tolerances of the
other GPU tests.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

import __graft_entry__
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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_no_alloc_matches_periodogram_twice(ftp, prec):
    lc, tpl, grid = synth.small_curve(nf=3001)
    bank = [tpl, synth.make_template(2, 9100)]
    H = max(b.H for b in bank)
    templates = [(b.c, b.s) for b in bank]
    with ftp.Plan(lc.t.size, H, (grid.df, grid.k0, grid.nf), len(bank), prec) as plan:
        ref = plan.periodogram(lc.t, lc.y, lc.dy, templates)
        sums, (ybar, YY) = plan.sums(lc.t, lc.y, lc.dy, H)
    dev = torch.device("cuda:0")
    stride = (grid.nf + 63) // 64 * 64 + 64
    cdt = torch.complex64 if prec == "mixed" else torch.complex128
    dsums = torch.zeros((3 * H, stride), dtype=cdt, device=dev)
    dsums[:, : grid.nf] = torch.from_numpy(sums).to(dev)
    shape = (len(bank), grid.nf)
    previous = None
    for _ in range(2):
        outs = [torch.full(shape, np.nan, dtype=torch.float64, device=dev) for _ in range(4)]
        flags = torch.full(shape, 255, dtype=torch.uint8, device=dev)
        ftp.ftp_periodogram_sums_noalloc(dsums, stride, prec, grid.nf, H, ybar, YY, templates,
                                         *outs, flags, device=0)
        torch.cuda.synchronize()
        power = outs[0].cpu().numpy()
        assert np.all(np.isfinite(power))
        assert np.max(np.abs(power - ref["power"])) <= TOL_P[prec]
        assert np.all(flags.cpu().numpy() != 255)
        if previous is not None:
            # the same sums give the same answer on the second call
            np.testing.assert_array_equal(power, previous)
        previous = power


def test_no_alloc_rejects_requests_beyond_its_scratch(ftp):
    dev = torch.device("cuda:0")
    nf, H = 100, 2
    dsums = torch.zeros((3 * H, 128), dtype=torch.complex64, device=dev)
    outs = [torch.empty(nf, dtype=torch.float64, device=dev) for _ in range(4)]
    many = [(np.ones(H), np.zeros(H))] * 65
    with pytest.raises(ftp.FtpError) as e:
        ftp.ftp_periodogram_sums_noalloc(dsums, 128, "mixed", nf, H, 0.0, 1.0, many, *outs)
    assert e.value.status == 8
    with pytest.raises(ftp.FtpError) as e:  # row stride too short for whole work units
        ftp.ftp_periodogram_sums_noalloc(dsums, 100, "mixed", nf, H, 0.0, 1.0, many[:1], *outs)
    assert e.value.status == 1
    host = [np.empty(nf) for _ in range(4)]
    with pytest.raises(ftp.FtpError) as e:  # outputs must be device memory
        ftp.ftp_periodogram_sums_noalloc(dsums, 128, "mixed", nf, H, 0.0, 1.0, many[:1], *host)
    assert e.value.status == 1
