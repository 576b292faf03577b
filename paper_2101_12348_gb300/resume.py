"""Resumable survey runs: ftp_batch over a survey chunk by chunk of curves,
each chunk's results written to its own file and listed in a manifest once
complete, so that a run stopped part-way (a crash, a pre-empted job, a lost
GPU) restarts from the first unfinished chunk instead of from curve 0.

The paper has no such machinery; its periodograms are independent per curve
(Section 2: everything after the sums is per frequency and template), so a
chunk of curves is a unit of work that can be redone or skipped on its own.

Layout of `out_dir`:
  manifest.json     {"version", "fingerprint", "ncurves", "chunk_curves",
                     "chunks": {"<i>": {"curves": [c0, c1], "file", "sha256"}}}
  chunk_<i>.npz     power, theta1, theta2, theta3 (float64) and flags (uint8)
                    of curves c0 .. c1-1, frequencies stacked curve by curve
Every file is written to a temporary name, flushed and renamed, and the
manifest is rewritten (the same way) only after its chunk file is in place:
a chunk listed in the manifest is complete, and anything else is redone.  The
fingerprint (SHA-256 of the inputs and the chunking) ties a directory to one
survey; resuming with other inputs raises instead of mixing results.  A
listed chunk whose file is missing or does not match its recorded hash is
recomputed.

This module only sequences calls and files; the periodograms come from the
CUDA library (`compute` defaults to ftp_batch on the chunk's host arrays).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

VERSION = 1
FIELDS = ("power", "theta1", "theta2", "theta3", "flags")


def _sha256_file(path: str) -> str:
    h = hashlib.sha256()
    with open(path, "rb") as f:
        for block in iter(lambda: f.read(1 << 20), b""):
            h.update(block)
    return h.hexdigest()


def _write_atomic(path: str, write) -> None:
    tmp = f"{path}.tmp-{os.getpid()}"
    with open(tmp, "wb") as f:
        write(f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def fingerprint(obs_off, t, y, dy, grids, bank, tpl_of_curve, precision: str,
                chunk_curves: int) -> str:
    h = hashlib.sha256()
    for a in (obs_off, t, y, dy):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(np.asarray([tuple(g) for g in grids], dtype=np.float64).tobytes())
    for c, s in bank:
        h.update(np.ascontiguousarray(c, dtype=np.float64).tobytes())
        h.update(np.ascontiguousarray(s, dtype=np.float64).tobytes())
        h.update(b"|")
    if tpl_of_curve is not None:
        h.update(np.ascontiguousarray(tpl_of_curve, dtype=np.int32).tobytes())
    h.update(f"{precision}|{int(chunk_curves)}|{VERSION}".encode())
    return h.hexdigest()


def chunk_bounds(ncurves: int, chunk_curves: int) -> list:
    """[(c0, c1)] covering 0..ncurves in order, chunk_curves curves each
    (the last one shorter)."""
    if chunk_curves < 1:
        raise ValueError("chunk_curves must be >= 1")
    return [(c0, min(c0 + chunk_curves, ncurves)) for c0 in range(0, ncurves, chunk_curves)]


def ftp_batch_compute(plan: int):
    """The default `compute`: ftp_batch of one chunk, host arrays in and out."""
    from . import ftp

    def compute(obs_off, t, y, dy, grids, bank, tpl_of_curve):
        nfs = np.array([int(g[2]) for g in grids], dtype=np.int64)
        out_off = np.zeros(len(grids), dtype=np.int64)
        out_off[1:] = np.cumsum(nfs)[:-1]
        tot = int(nfs.sum())
        res = {k: np.empty(tot, dtype=np.float64) for k in FIELDS[:4]}
        res["flags"] = np.empty(tot, dtype=np.uint8)
        ftp.ftp_batch(plan, obs_off, t, y, dy, grids, out_off, bank, tpl_of_curve,
                      res["power"], res["theta1"], res["theta2"], res["theta3"], res["flags"])
        return res

    return compute


class SurveyRun:
    """A survey bound to an output directory.  run() computes the chunks the
    manifest does not list as complete and returns the whole survey's
    results; `computed` lists the chunk indices this object computed."""

    def __init__(self, out_dir: str, obs_off, t, y, dy, grids, bank, tpl_of_curve=None,
                 precision: str = "mixed", chunk_curves: int = 256):
        self.out_dir = out_dir
        self.obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
        self.t, self.y, self.dy = (np.ascontiguousarray(a, dtype=np.float64) for a in (t, y, dy))
        self.grids = [tuple(g) for g in grids]
        self.bank = list(bank)
        self.tpl_of_curve = (None if tpl_of_curve is None
                             else np.ascontiguousarray(tpl_of_curve, dtype=np.int32))
        self.ncurves = self.obs_off.size - 1
        if len(self.grids) != self.ncurves:
            raise ValueError("one grid per curve required")
        self.chunk_curves = int(chunk_curves)
        self.bounds = chunk_bounds(self.ncurves, self.chunk_curves)
        self.fp = fingerprint(self.obs_off, self.t, self.y, self.dy, self.grids, self.bank,
                              self.tpl_of_curve, precision, self.chunk_curves)
        self.computed: list = []
        os.makedirs(out_dir, exist_ok=True)
        self.manifest_path = os.path.join(out_dir, "manifest.json")
        self.manifest = self._read_manifest()

    # manifest -------------------------------------------------------------
    def _read_manifest(self) -> dict:
        if not os.path.exists(self.manifest_path):
            return {"version": VERSION, "fingerprint": self.fp, "ncurves": self.ncurves,
                    "chunk_curves": self.chunk_curves, "chunks": {}}
        with open(self.manifest_path) as f:
            m = json.load(f)
        if m.get("version") != VERSION or m.get("fingerprint") != self.fp:
            raise ValueError(f"{self.out_dir} holds the results of another survey or chunking "
                             "(fingerprint mismatch); use a new directory")
        return m

    def _write_manifest(self) -> None:
        data = json.dumps(self.manifest, indent=1, sort_keys=True).encode()
        _write_atomic(self.manifest_path, lambda f: f.write(data))

    def finished(self) -> list:
        """Indices of the chunks listed as complete whose files check out."""
        ok = []
        for key, ent in self.manifest["chunks"].items():
            path = os.path.join(self.out_dir, ent["file"])
            if os.path.exists(path) and _sha256_file(path) == ent["sha256"]:
                ok.append(int(key))
        return sorted(ok)

    # work -----------------------------------------------------------------
    def _chunk_inputs(self, i: int):
        c0, c1 = self.bounds[i]
        a, b = int(self.obs_off[c0]), int(self.obs_off[c1])
        off = self.obs_off[c0:c1 + 1] - a
        tpc = None if self.tpl_of_curve is None else self.tpl_of_curve[c0:c1]
        return (off, self.t[a:b], self.y[a:b], self.dy[a:b], self.grids[c0:c1], self.bank, tpc)

    def run(self, compute, on_chunk=None) -> dict:
        """compute(obs_off, t, y, dy, grids, bank, tpl_of_curve) -> dict of
        the FIELDS arrays of one chunk; on_chunk(i), if given, is called
        after chunk i is recorded (a test uses it to stop a run part-way)."""
        done = set(self.finished())
        for key in [k for k in self.manifest["chunks"] if int(k) not in done]:
            del self.manifest["chunks"][key]  # listed, but its file is gone or altered
        for i, (c0, c1) in enumerate(self.bounds):
            if i in done:
                continue
            res = compute(*self._chunk_inputs(i))
            nrows = sum(int(g[2]) for g in self.grids[c0:c1])
            for k in FIELDS:
                if np.asarray(res[k]).shape != (nrows,):
                    raise ValueError(f"chunk {i}: {k} has shape {np.asarray(res[k]).shape}, "
                                     f"expected ({nrows},)")
            name = f"chunk_{i:06d}.npz"
            path = os.path.join(self.out_dir, name)
            _write_atomic(path, lambda f: np.savez(f, **{k: np.asarray(res[k]) for k in FIELDS}))
            self.manifest["chunks"][str(i)] = {"curves": [c0, c1], "file": name,
                                               "sha256": _sha256_file(path)}
            self._write_manifest()
            self.computed.append(i)
            if on_chunk is not None:
                on_chunk(i)
        return self.results()

    def results(self) -> dict:
        """The whole survey's results in curve order, from the chunk files;
        out_off[c] is curve c's first row."""
        missing = [i for i in range(len(self.bounds)) if str(i) not in self.manifest["chunks"]]
        if missing:
            raise RuntimeError(f"chunks {missing} are not complete")
        parts = {k: [] for k in FIELDS}
        for i in range(len(self.bounds)):
            with np.load(os.path.join(self.out_dir, self.manifest["chunks"][str(i)]["file"])) as z:
                for k in FIELDS:
                    parts[k].append(z[k])
        out = {k: np.concatenate(v) if v else np.empty(0) for k, v in parts.items()}
        off = np.zeros(self.ncurves + 1, dtype=np.int64)
        off[1:] = np.cumsum([int(g[2]) for g in self.grids])
        out["out_off"] = off
        return out
