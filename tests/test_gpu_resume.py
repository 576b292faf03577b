"""Checkpoint and resume on the GPU.

- A survey run through resume.SurveyRun with ftp_batch, stopped after its
  second chunk (an exception raised on the host between chunks, with no
  kernel in flight), resumes with the finished chunks skipped; the combined
  results match the oracle on sampled frequencies of every curve within the
  parity tolerances and agree with a single ftp_batch call over the whole
  survey.
- The surrogate's training state (parameters, Adam moments, step count)
  saved part-way and loaded into a new handle continues bit for bit as an
  uninterrupted run, both through ftp_mlp_get_state / ftp_mlp_set_state and
  through Surrogate.train_to's checkpoint file."""
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


class Stop(Exception):
    pass


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_survey_resumes_after_a_stop(ftp, prec, tmp_path):
    from paper_2101_12348_gb300 import resume
    sv = synth.survey(ncurves=24, n_bank=6, median_obs=80, min_obs=20, max_obs=400, f_max=1.5,
                      baseline=(20, 120), seed=314)
    grids = [(g.df, g.k0, g.nf) for g in sv.grids]
    bank = [(b.c, b.s) for b in sv.bank]
    args = (sv.obs_off, sv.t, sv.y, sv.dy, grids, bank, sv.tpl_of_curve)
    gj = max(sv.grids, key=lambda g: g.k0 + g.nf)
    nfmax = max(g.nf for g in sv.grids)
    with ftp.Plan(int(np.max(np.diff(sv.obs_off))), max(b.H for b in sv.bank),
                  (gj.df, gj.k0, nfmax), len(bank), prec) as plan:
        compute = resume.ftp_batch_compute(plan.h)
        d = str(tmp_path / prec)

        def stop(i):
            if i == 1:
                raise Stop()

        r1 = resume.SurveyRun(d, *args, precision=prec, chunk_curves=7)
        with pytest.raises(Stop):
            r1.run(compute, on_chunk=stop)
        assert r1.computed == [0, 1]
        r2 = resume.SurveyRun(d, *args, precision=prec, chunk_curves=7)
        out = r2.run(compute)
        assert r2.computed == [2, 3]
        whole = compute(*args)
    off = out["out_off"]
    assert np.all((out["flags"] & ftp.FLAG_NONCONVERGED) == 0)
    assert np.max(np.abs(out["power"] - whole["power"])) <= TOL_P[prec]
    for c in range(sv.ncurves):
        g, tp = sv.grids[c], sv.bank[sv.tpl_of_curve[c]]
        sel = np.arange(c % 11, g.nf, 11)
        lc = sv.curve(c)
        ref = oracle.periodogram(lc.t, lc.y, lc.dy, g.freqs()[sel], tp.c, tp.s)
        d_p = np.abs(out["power"][off[c]:off[c + 1]][sel] - ref["power"])
        assert np.max(d_p) <= TOL_P[prec], (c, float(np.max(d_p)))


def _data(rows=8000, nfeat=10, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (rows, nfeat)).astype(np.float32)
    y = (X[:, 0] * X[:, 1] + 0.5 * X[:, 2] ** 2).astype(np.float32)
    return torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), rows


def test_training_state_resumes_bit_for_bit(ftp):
    X, y, rows = _data()
    n = ftp.ftp_mlp_param_count(10)
    straight = ftp.ftp_mlp_create(10, None, 4, 0)
    first = ftp.ftp_mlp_create(10, None, 4, 0)
    second = ftp.ftp_mlp_create(10, None, 99, 0)  # other initial weights: all overwritten
    try:
        ftp.ftp_mlp_train(straight, X, y, rows, 70, 512, 2e-3, 11)
        ftp.ftp_mlp_train(first, X, y, rows, 25, 512, 2e-3, 11)
        st = [np.empty(n, dtype=np.float32) for _ in range(3)]
        steps = ftp.ftp_mlp_get_state(first, *st)
        assert steps == 25
        assert np.all(st[2] >= 0) and np.any(st[1] != 0)
        # device arrays are accepted as well
        ftp.ftp_mlp_set_state(second, *[torch.from_numpy(a).cuda() for a in st], steps)
        ftp.ftp_mlp_train(second, X, y, rows, 45, 512, 2e-3, 11)
        a = [np.empty(n, dtype=np.float32) for _ in range(3)]
        b = [np.empty(n, dtype=np.float32) for _ in range(3)]
        assert ftp.ftp_mlp_get_state(straight, *a) == ftp.ftp_mlp_get_state(second, *b) == 70
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)
        # set_params restarts Adam: the moments are zero and the count is 0
        ftp.ftp_mlp_set_params(second, a[0])
        c = [np.empty(n, dtype=np.float32) for _ in range(3)]
        assert ftp.ftp_mlp_get_state(second, *c) == 0 and not np.any(c[1]) and not np.any(c[2])
        for bad in (-1, 2 ** 31):
            with pytest.raises(ftp.FtpError) as e:
                ftp.ftp_mlp_set_state(second, *a, bad)
            assert e.value.status == 1
        with pytest.raises(ftp.FtpError):
            ftp.ftp_mlp_set_state(second, a[0], None, a[2], 3)
    finally:
        for h in (straight, first, second):
            ftp.ftp_mlp_destroy(h)


def test_train_to_continues_from_its_checkpoint(ftp, tmp_path):
    from paper_2101_12348_gb300.screen import Surrogate
    X, y, rows = _data(nfeat=8, seed=4)
    ck = str(tmp_path / "surrogate.npz")
    with Surrogate(3, seed=5) as ref:
        ref.train(X, y, rows, 50, batch=512, lr=2e-3, seed=9)
        want = ref.state()
    with Surrogate(3, seed=5) as s1:  # "interrupted" after 30 of 50 steps
        assert s1.train_to(X, y, rows, 30, ck, every=20, batch=512, lr=2e-3, seed=9) == 30
    with Surrogate(3, seed=123) as s2:  # a new process would start like this
        assert s2.train_to(X, y, rows, 50, ck, every=20, batch=512, lr=2e-3, seed=9) == 20
        got = s2.state()
    assert got["steps"] == want["steps"] == 50
    for k in ("params", "adam_m", "adam_v"):
        np.testing.assert_array_equal(got[k], want[k])
    loaded = Surrogate.load(ck)
    try:
        np.testing.assert_array_equal(loaded.params(), want["params"])
        assert loaded.state()["steps"] == 50
    finally:
        loaded.close()
