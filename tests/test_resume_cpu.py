"""Resumable survey runs (paper_2101_12348_gb300/resume.py) on the CPU.

The chunk computation is a stand-in here (a deterministic function of each
curve's own inputs, so chunking cannot change it): what is tested is the
host logic around it - results written per chunk, the manifest listing only
complete chunks, a run stopped part-way resuming from the first unfinished
chunk with the same final results as an uninterrupted run, altered or
missing chunk files recomputed, and a directory refusing another survey's
inputs.  The GPU test of the same driver with ftp_batch is in
test_gpu_resume.py."""
import json
import os

import numpy as np
import pytest

import synth
from paper_2101_12348_gb300 import resume


def fake_compute(calls):
    def compute(obs_off, t, y, dy, grids, bank, tpl_of_curve):
        calls.append(len(grids))
        out = {k: [] for k in resume.FIELDS}
        for c, g in enumerate(grids):
            sl = slice(obs_off[c], obs_off[c + 1])
            k = np.arange(int(g[2]))
            base = float(np.sum(t[sl] * y[sl] / dy[sl]))
            out["power"].append(np.abs(np.sin(base + 0.01 * k)))
            out["theta1"].append(base + k * g[0])
            out["theta2"].append(np.mod(base * k, 2 * np.pi))
            out["theta3"].append(np.full(k.size, float(len(bank[tpl_of_curve[c]][0]))))
            out["flags"].append((k % 5).astype(np.uint8))
        return {kk: np.concatenate(v) for kk, v in out.items()}
    return compute


@pytest.fixture(scope="module")
def survey():
    sv = synth.survey(ncurves=23, n_bank=4, median_obs=40, min_obs=10, max_obs=100, f_max=0.5,
                      baseline=(20, 60), seed=77)
    grids = [(g.df, g.k0, g.nf) for g in sv.grids]
    bank = [(b.c, b.s) for b in sv.bank]
    return sv.obs_off, sv.t, sv.y, sv.dy, grids, bank, sv.tpl_of_curve


class Stop(Exception):
    pass


def stop_after(n):
    def on_chunk(i):
        if i == n:
            raise Stop(i)
    return on_chunk


def test_chunks_cover_the_survey_in_order():
    assert resume.chunk_bounds(10, 4) == [(0, 4), (4, 8), (8, 10)]
    assert resume.chunk_bounds(8, 4) == [(0, 4), (4, 8)]
    assert resume.chunk_bounds(0, 4) == []
    with pytest.raises(ValueError):
        resume.chunk_bounds(5, 0)


def test_interrupted_run_resumes_from_the_first_unfinished_chunk(survey, tmp_path):
    calls = []
    ref = resume.SurveyRun(str(tmp_path / "ref"), *survey, chunk_curves=5).run(fake_compute(calls))
    assert calls == [5, 5, 5, 5, 3]
    d = str(tmp_path / "run")
    r1 = resume.SurveyRun(d, *survey, chunk_curves=5)
    with pytest.raises(Stop):
        r1.run(fake_compute([]), on_chunk=stop_after(1))
    assert r1.computed == [0, 1]
    with open(os.path.join(d, "manifest.json")) as f:
        m = json.load(f)
    assert sorted(m["chunks"]) == ["0", "1"] and m["chunks"]["1"]["curves"] == [5, 10]
    with pytest.raises(RuntimeError):  # the survey is not complete yet
        r1.results()
    calls2 = []
    r2 = resume.SurveyRun(d, *survey, chunk_curves=5)
    assert r2.finished() == [0, 1]
    out = r2.run(fake_compute(calls2))
    assert r2.computed == [2, 3, 4] and calls2 == [5, 5, 3]
    for k in resume.FIELDS + ("out_off",):
        np.testing.assert_array_equal(out[k], ref[k])
    # a third run finds everything done
    r3 = resume.SurveyRun(d, *survey, chunk_curves=5)
    r3.run(fake_compute([]))
    assert r3.computed == []


def test_altered_or_missing_chunk_files_are_recomputed(survey, tmp_path):
    d = str(tmp_path / "run")
    ref = resume.SurveyRun(d, *survey, chunk_curves=6).run(fake_compute([]))
    p0 = os.path.join(d, "chunk_000000.npz")
    with open(p0, "r+b") as f:  # flip a byte of chunk 0
        f.seek(100)
        b = f.read(1)
        f.seek(100)
        f.write(bytes([b[0] ^ 0xFF]))
    os.remove(os.path.join(d, "chunk_000002.npz"))
    with open(os.path.join(d, "chunk_000003.npz.tmp-1"), "wb") as f:  # a crash's leftover
        f.write(b"partial")
    r = resume.SurveyRun(d, *survey, chunk_curves=6)
    assert r.finished() == [1, 3]
    out = r.run(fake_compute([]))
    assert r.computed == [0, 2]
    for k in resume.FIELDS:
        np.testing.assert_array_equal(out[k], ref[k])


def test_directory_refuses_other_inputs_or_chunking(survey, tmp_path):
    d = str(tmp_path / "run")
    resume.SurveyRun(d, *survey, chunk_curves=5).run(fake_compute([]))
    off, t, y, dy, grids, bank, tpc = survey
    y2 = y.copy()
    y2[7] += 1e-9
    with pytest.raises(ValueError, match="fingerprint"):
        resume.SurveyRun(d, off, t, y2, dy, grids, bank, tpc, chunk_curves=5)
    with pytest.raises(ValueError, match="fingerprint"):
        resume.SurveyRun(d, *survey, chunk_curves=4)
    with pytest.raises(ValueError, match="fingerprint"):
        resume.SurveyRun(d, *survey, precision="fp64", chunk_curves=5)


def test_a_chunk_of_the_wrong_shape_is_not_recorded(survey, tmp_path):
    d = str(tmp_path / "run")

    def bad(*args):
        res = fake_compute([])(*args)
        res["theta2"] = res["theta2"][:-1]
        return res

    r = resume.SurveyRun(d, *survey, chunk_curves=5)
    with pytest.raises(ValueError, match="theta2"):
        r.run(bad)
    assert r.finished() == [] and not os.path.exists(os.path.join(d, "chunk_000000.npz"))
