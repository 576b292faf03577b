"""Learned screening of trial frequencies: a thin driver of the C ABI's
ftp_mlp_* / ftp_batch_features / ftp_training_rows / ftp_batch_screened.

The surrogate is not part of the paper.  It reads 2H+2 features per frequency
(single-harmonic and multi-harmonic least-squares powers of Section 2.1,
harmonic amplitudes, log10 N) computed from the NFFT sums, predicts the
template power, and lets the exact solve run on the top-ranked frequencies
and their neighbours only.  Everything that computes runs in the CUDA
library; this module allocates device tensors (torch, as plain device memory)
and sequences the calls.
"""
from __future__ import annotations

import os

import numpy as np

from . import ftp


class Surrogate:
    """Owner of an ftp_mlp_t handle: nfeat = 2 H_feat + 2 inputs."""

    def __init__(self, H_feat: int, params=None, seed: int = 0, device: int = 0):
        self.H_feat = int(H_feat)
        self.nfeat = 2 * self.H_feat + 2
        self.h = ftp.ftp_mlp_create(self.nfeat, params, seed, device)

    @property
    def nparams(self) -> int:
        return ftp.ftp_mlp_param_count(self.nfeat)

    def params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        ftp.ftp_mlp_get_params(self.h, out)
        return out

    def set_params(self, p) -> None:
        ftp.ftp_mlp_set_params(self.h, np.ascontiguousarray(p, dtype=np.float32))

    def state(self) -> dict:
        """Parameters, Adam moments and the Adam step count (host copies)."""
        st = {k: np.empty(self.nparams, dtype=np.float32) for k in ("params", "adam_m", "adam_v")}
        st["steps"] = ftp.ftp_mlp_get_state(self.h, st["params"], st["adam_m"], st["adam_v"])
        return st

    def set_state(self, st: dict) -> None:
        f32 = [np.ascontiguousarray(st[k], dtype=np.float32) for k in ("params", "adam_m", "adam_v")]
        if any(a.shape != (self.nparams,) for a in f32):
            raise ValueError(f"training state of {self.nparams} parameters expected")
        ftp.ftp_mlp_set_state(self.h, *f32, int(st["steps"]))

    def save(self, path: str) -> None:
        """Checkpoint of the whole training state (.npz), written to a
        temporary file and renamed, so a crash leaves the old one intact."""
        st = self.state()
        tmp = f"{path}.tmp-{os.getpid()}"
        with open(tmp, "wb") as f:
            np.savez(f, H_feat=np.int64(self.H_feat), steps=np.int64(st["steps"]),
                     params=st["params"], adam_m=st["adam_m"], adam_v=st["adam_v"])
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)

    @classmethod
    def load(cls, path: str, device: int = 0) -> "Surrogate":
        with np.load(path) as z:
            sur = cls(int(z["H_feat"]), params=z["params"], device=device)
            sur.set_state({k: z[k] for k in ("params", "adam_m", "adam_v", "steps")})
        return sur

    def train_to(self, X, y, rows: int, total_steps: int, checkpoint: str, every: int,
                 batch: int = 2048, lr: float = 2e-3, seed: int = 1) -> int:
        """Train until `total_steps` Adam steps have been taken in all,
        writing the training state to `checkpoint` every `every` steps and
        at the end.  If `checkpoint` exists it is loaded first, so calling
        this again with the same arguments after an interruption continues
        where the last checkpoint left off and ends in the same state as an
        uninterrupted run.  Returns the steps taken by this call."""
        if every < 1 or total_steps < 0:
            raise ValueError("every >= 1 and total_steps >= 0 required")
        if os.path.exists(checkpoint):
            with np.load(checkpoint) as z:
                if int(z["H_feat"]) != self.H_feat:
                    raise ValueError(f"{checkpoint} holds a network of H_feat = {int(z['H_feat'])}")
                self.set_state({k: z[k] for k in ("params", "adam_m", "adam_v", "steps")})
        done = self.state()["steps"]
        if done > total_steps:
            raise ValueError(f"{checkpoint} is already past {total_steps} steps ({done})")
        taken = 0
        while done < total_steps:
            k = min(every, total_steps - done)
            self.train(X, y, rows, k, batch, lr, seed)
            done += k
            taken += k
            self.save(checkpoint)
        return taken

    def forward(self, X, n=None, scores=None):
        n = X.shape[0] if n is None else n
        if scores is None:
            scores = np.empty(n, dtype=np.float32)
        ftp.ftp_mlp_forward(self.h, X, n, scores)
        return scores

    def train(self, X, y, rows: int, steps: int, batch: int = 2048, lr: float = 2e-3,
              seed: int = 1, losses=None):
        ftp.ftp_mlp_train(self.h, X, y, rows, steps, batch, lr, seed, losses)

    def close(self):
        if self.h:
            ftp.ftp_mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def row_offsets(grids) -> np.ndarray:
    """First row of each curve when every curve's frequencies are stacked."""
    off = np.zeros(len(grids) + 1, dtype=np.int64)
    off[1:] = np.cumsum([int(g[2]) for g in grids])
    return off


def training_rows(plan, obs_off, t, y, dy, grids, bank, tpl_of_curve, H_feat: int,
                  top_frac: float = 0.02, neighbours: int = 3, rand_frac: float = 0.02,
                  seed: int = 7, X_out=None, y_out=None, count: int = 0):
    """Exact template powers (ftp_batch, exhaustive) and features of every
    frequency of the given curves, reduced to training rows on the device:
    the top_frac best powers of each curve with their +-neighbours plus a
    random rand_frac of all rows.  Appends to (X_out, y_out) (torch device
    tensors) from row `count` on and returns the new count."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    grids = [tuple(g) for g in grids]
    off = row_offsets(grids)
    rows = int(off[-1])
    nfeat = 2 * H_feat + 2
    feats = torch.empty((rows, nfeat), dtype=torch.float32, device=dev)
    ftp.ftp_batch_features(plan, obs_off, t, y, dy, grids, off, H_feat, feats)
    outs = [torch.empty(rows, dtype=torch.float64, device=dev) for _ in range(4)]
    ftp.ftp_batch(plan, obs_off, t, y, dy, grids, off[:-1].copy(), bank, tpl_of_curve, *outs)
    cap = X_out.shape[0]
    return ftp.ftp_training_rows(outs[0], feats, nfeat, off, top_frac, neighbours, rand_frac,
                                 seed, X_out, y_out, cap, count, dev.index or 0)
