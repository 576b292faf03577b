"""Parallel evaluation of the FP64 oracle for the GPU tests.

A spawn pool of single-threaded workers: spawn rather than fork, because a
process forked after the first CUDA call can hang.  Each job is
(t, y, dy, freqs, c, s[, margins]) and returns oracle.periodogram's dict, plus
`margin` (oracle.best_candidate_margin at each frequency's best phase) when
margins is true."""
import multiprocessing as mp
import os

_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _work(job):
    import numpy as np

    import oracle
    t, y, dy, freqs, c, s = job[:6]
    r = oracle.periodogram(t, y, dy, freqs, c, s)
    if len(job) > 6 and job[6]:
        r["margin"] = np.array([oracle.best_candidate_margin(t, y, dy, f, c, s, th)
                                for f, th in zip(freqs, r["theta2"])])
    return r


def oracle_map(jobs, cores=None):
    """oracle.periodogram of every job, in order, on a spawn pool."""
    if not jobs:
        return []
    try:
        avail = len(os.sched_getaffinity(0))
    except Exception:
        avail = os.cpu_count() or 1
    cores = max(1, min(len(jobs), cores or avail))
    saved = {k: os.environ.get(k) for k in _THREAD_ENV}
    for k in _THREAD_ENV:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            return pool.map(_work, jobs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
