"""Thin ctypes binding of the C ABI in include/ftp.h.

Argument marshalling only: every step of the periodogram runs in the CUDA
library.  Functions keep the C names (ftp_plan, ftp_sums, ftp_periodogram,
ftp_batch, ftp_destroy, ftp_status_string, ftp_plan_info, ftp_set_timing,
ftp_stage_times).  Arrays may be NumPy arrays (host memory) or torch tensors
(host or CUDA); pointers are passed through unchanged and the library decides
whether they are host or device memory.  If the shared library is missing the
import of this module succeeds but every call raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FTP_GB300_LIB selects another build of the same library (e.g. the
# self-checking libftp_gb300_checks.so); it must exist like the default one.
LIB_PATH = os.environ.get("FTP_GB300_LIB") or os.path.join(_HERE, "libftp_gb300.so")

FTP_OK = 0
FTP_FP64 = 0
FTP_MIXED = 1
FTP_MAX_H = 16
FLAG_NONCONVERGED = 1
FLAG_DEGENERATE_MM = 2
FLAG_CONSTANT_P = 4
FLAG_NEGATIVE_AMP = 8
FLAG_UNRESOLVED = 16
FLAG_SCREENED_OUT = 32
FLAG_NO_POSITIVE = 64
FLAG_RESOLVED = 128

STATUS_NAMES = {0: "FTP_OK", 1: "FTP_ERR_INVALID_ARG", 2: "FTP_ERR_ZERO_VARIANCE",
                3: "FTP_ERR_MIXED_ZERO_SIGMA", 4: "FTP_ERR_NONFINITE", 5: "FTP_ERR_OOM",
                6: "FTP_ERR_CUDA", 7: "FTP_ERR_TIMEOUT", 8: "FTP_ERR_UNSUPPORTED"}

# every symbol include/ftp.h declares
EXPORTS = ("ftp_plan", "ftp_sums", "ftp_periodogram", "ftp_batch", "ftp_destroy",
           "ftp_status_string", "ftp_plan_info", "ftp_solver_stats", "ftp_set_timing",
           "ftp_stage_times", "ftp_periodogram_sums_noalloc", "ftp_set_batch_options",
           "ftp_batch_info", "ftp_mlp_param_count", "ftp_mlp_create", "ftp_mlp_destroy",
           "ftp_mlp_get_params", "ftp_mlp_set_params", "ftp_mlp_forward", "ftp_mlp_gradient",
           "ftp_mlp_train", "ftp_batch_features", "ftp_batch_screened", "ftp_training_rows",
           "ftp_set_batch_tuning", "ftp_get_batch_tuning", "ftp_batch_autotune",
           "ftp_set_positive_amplitude", "ftp_multiband_periodogram",
           "ftp_shared_multiband", "ftp_roots_first_phase_ms", "ftp_set_solver_limits",
           "ftp_set_fault_injection", "ftp_alu_peak", "ftp_mlp_get_state",
           "ftp_mlp_set_state")


class FtpGrid(C.Structure):
    _fields_ = [("df", C.c_double), ("k0", C.c_int64), ("nf", C.c_int64)]


class FtpTemplate(C.Structure):
    _fields_ = [("H", C.c_int), ("c", C.POINTER(C.c_double)), ("s", C.POINTER(C.c_double))]


class FtpError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{STATUS_NAMES.get(self.status, self.status)}: {what}")


_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load (once) and return the CUDA library; raises if it is not built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} is not built: run __graft_entry__.build() "
                                "(the periodogram has no CPU fallback)")
    lib = C.CDLL(p)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    lib.ftp_plan.argtypes = [C.POINTER(vp), i64, i32, FtpGrid, i32, i32, i32, vp]
    lib.ftp_sums.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp]
    lib.ftp_periodogram.argtypes = [vp, vp, vp, vp, i64, C.POINTER(FtpTemplate), i32,
                                    vp, vp, vp, vp, vp]
    lib.ftp_batch.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(FtpGrid), vp,
                              C.POINTER(FtpTemplate), i32, vp, vp, vp, vp, vp, vp]
    lib.ftp_destroy.argtypes = [vp]
    lib.ftp_destroy.restype = None
    lib.ftp_status_string.argtypes = [i32]
    lib.ftp_status_string.restype = C.c_char_p
    lib.ftp_plan_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i64),
                                  C.POINTER(i32)]
    lib.ftp_solver_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(dbl), C.POINTER(i64),
                                     C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.ftp_set_solver_limits.argtypes = [vp, i32, i32, i32]
    lib.ftp_set_fault_injection.argtypes = [vp, i32]
    lib.ftp_alu_peak.argtypes = [i32, i32, i32, C.POINTER(dbl), C.POINTER(C.c_float)]
    lib.ftp_set_timing.argtypes = [vp, i32]
    lib.ftp_periodogram_sums_noalloc.argtypes = [vp, i64, i32, i64, i32, dbl, dbl,
                                                 C.POINTER(FtpTemplate), i32, vp, vp, vp, vp,
                                                 vp, i32, vp]
    lib.ftp_stage_times.argtypes = [vp, C.POINTER(C.c_float)]
    lib.ftp_roots_first_phase_ms.argtypes = [vp, C.POINTER(C.c_float)]
    lib.ftp_set_batch_options.argtypes = [vp, i64, i32]
    lib.ftp_batch_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32)]
    u64, f32 = C.c_uint64, C.c_float
    lib.ftp_mlp_param_count.argtypes = [i32]
    lib.ftp_mlp_create.argtypes = [C.POINTER(vp), i32, vp, u64, i32, vp]
    lib.ftp_mlp_destroy.argtypes = [vp]
    lib.ftp_mlp_destroy.restype = None
    lib.ftp_mlp_get_params.argtypes = [vp, vp]
    lib.ftp_mlp_set_params.argtypes = [vp, vp]
    lib.ftp_mlp_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(i64)]
    lib.ftp_mlp_set_state.argtypes = [vp, vp, vp, vp, i64]
    lib.ftp_mlp_forward.argtypes = [vp, vp, i64, vp]
    lib.ftp_mlp_gradient.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp]
    lib.ftp_mlp_train.argtypes = [vp, vp, vp, i64, i64, i64, f32, u64, vp]
    lib.ftp_batch_features.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(FtpGrid), vp, i32, vp]
    lib.ftp_batch_screened.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(FtpGrid), vp,
                                       C.POINTER(FtpTemplate), i32, vp, vp, dbl, i32, vp, vp, vp,
                                       vp, vp]
    lib.ftp_training_rows.argtypes = [vp, vp, i32, i64, vp, dbl, i32, dbl, u64, vp, vp, i64,
                                      C.POINTER(i64), i32, vp]
    lib.ftp_set_batch_tuning.argtypes = [vp, i32, i32]
    lib.ftp_set_positive_amplitude.argtypes = [vp, i32]
    lib.ftp_shared_multiband.argtypes = [vp, i32, vp, vp, vp, vp, vp, C.POINTER(FtpTemplate), i32,
                                         vp, vp, vp, vp, vp, vp]
    lib.ftp_multiband_periodogram.argtypes = [vp, i32, vp, vp, vp, vp, C.POINTER(FtpTemplate),
                                              i32, vp, vp, vp, vp, vp, vp, vp]
    lib.ftp_get_batch_tuning.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    lib.ftp_batch_autotune.argtypes = [vp, i64, vp, vp, vp, vp, C.POINTER(FtpGrid), vp,
                                       C.POINTER(FtpTemplate), i32, vp, vp, vp, vp, vp,
                                       C.c_char_p, C.POINTER(i32)]
    for name in EXPORTS:
        if name not in ("ftp_destroy", "ftp_status_string", "ftp_mlp_destroy"):
            getattr(lib, name).restype = i64 if name == "ftp_mlp_param_count" else i32
    if path is None:
        _lib = lib
    return lib


def _ptr(a) -> int | None:
    """Raw address of a NumPy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _check(st: int, what: str):
    if st != FTP_OK:
        raise FtpError(st, what)


def ftp_status_string(status: int) -> str:
    return load().ftp_status_string(int(status)).decode()


def ftp_plan(max_nobs: int, max_H: int, grid, max_templates: int = 1, precision: str = "mixed",
             device: int = 0, stream: int | None = None) -> int:
    """Create a plan; grid = (df, k0, nf).  Returns the opaque plan handle."""
    lib = load()
    prec = {"mixed": FTP_MIXED, "fp64": FTP_FP64}[precision]
    h = C.c_void_p()
    g = FtpGrid(float(grid[0]), int(grid[1]), int(grid[2]))
    _check(lib.ftp_plan(C.byref(h), int(max_nobs), int(max_H), g, int(max_templates), prec,
                        int(device), stream), "ftp_plan")
    return h.value


def ftp_destroy(plan: int) -> None:
    load().ftp_destroy(plan)


def _templates(tpls):
    keep = []
    arr = (FtpTemplate * len(tpls))()
    for i, (c, s) in enumerate(tpls):
        c = np.ascontiguousarray(c, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        if c.shape != s.shape or c.ndim != 1:
            raise ValueError("template c and s must be 1-D arrays of equal length")
        keep += [c, s]
        arr[i].H = c.shape[0]
        arr[i].c = c.ctypes.data_as(C.POINTER(C.c_double))
        arr[i].s = s.ctypes.data_as(C.POINTER(C.c_double))
    return arr, keep


def ftp_sums(plan: int, t, y, dy, nobs: int, H_sums: int, sums_out, moments_out=None) -> None:
    _check(load().ftp_sums(plan, _ptr(t), _ptr(y), _ptr(dy), int(nobs), int(H_sums),
                           _ptr(sums_out), _ptr(moments_out)), "ftp_sums")


def ftp_periodogram(plan: int, t, y, dy, nobs: int, templates, power, theta1, theta2, theta3,
                    flags=None) -> None:
    """templates: sequence of (c, s) coefficient arrays."""
    arr, keep = _templates(templates)
    _check(load().ftp_periodogram(plan, _ptr(t), _ptr(y), _ptr(dy), int(nobs), arr, len(keep) // 2,
                                  _ptr(power), _ptr(theta1), _ptr(theta2), _ptr(theta3),
                                  _ptr(flags)), "ftp_periodogram")


def ftp_batch(plan: int, obs_off, t, y, dy, grids, out_off, bank, tpl_of_curve, power, theta1,
              theta2, theta3, flags=None) -> None:
    """obs_off/out_off: int64 host arrays; grids: sequence of (df, k0, nf);
    bank: sequence of (c, s); tpl_of_curve: int32 host array or None."""
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    g = _grids(grids)
    arr, keep = _templates(bank)
    tpc = None if tpl_of_curve is None else np.ascontiguousarray(tpl_of_curve, dtype=np.int32)
    _check(load().ftp_batch(plan, obs_off.shape[0] - 1, _ptr(obs_off), _ptr(t), _ptr(y), _ptr(dy),
                            g, _ptr(out_off), arr, len(keep) // 2, _ptr(tpc), _ptr(power),
                            _ptr(theta1), _ptr(theta2), _ptr(theta3), _ptr(flags)), "ftp_batch")


def _grids(grids):
    g = (FtpGrid * len(grids))()
    for i, (df, k0, nf) in enumerate(grids):
        g[i] = FtpGrid(float(df), int(k0), int(nf))
    return g


def ftp_batch_features(plan: int, obs_off, t, y, dy, grids, row_off, H_feat: int,
                       features) -> None:
    """Screening features of every frequency of every curve; features is a
    device tensor [rows][2 H_feat + 2] (float32); row_off an int64 host array."""
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    row_off = np.ascontiguousarray(row_off, dtype=np.int64)
    _check(load().ftp_batch_features(plan, obs_off.shape[0] - 1, _ptr(obs_off), _ptr(t), _ptr(y),
                                     _ptr(dy), _grids(grids), _ptr(row_off), int(H_feat),
                                     _ptr(features)), "ftp_batch_features")


def ftp_batch_screened(plan: int, obs_off, t, y, dy, grids, out_off, bank, tpl_of_curve,
                       mlp: int, top_frac: float, neighbours: int, power, theta1, theta2, theta3,
                       flags=None) -> None:
    """ftp_batch with surrogate screening (arguments as ftp_batch plus the
    network handle, the selected fraction and the neighbour half-width)."""
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    arr, keep = _templates(bank)
    tpc = None if tpl_of_curve is None else np.ascontiguousarray(tpl_of_curve, dtype=np.int32)
    _check(load().ftp_batch_screened(plan, obs_off.shape[0] - 1, _ptr(obs_off), _ptr(t), _ptr(y),
                                     _ptr(dy), _grids(grids), _ptr(out_off), arr, len(keep) // 2,
                                     _ptr(tpc), mlp, float(top_frac), int(neighbours),
                                     _ptr(power), _ptr(theta1), _ptr(theta2), _ptr(theta3),
                                     _ptr(flags)), "ftp_batch_screened")


def ftp_mlp_param_count(nfeat: int) -> int:
    return int(load().ftp_mlp_param_count(int(nfeat)))


def ftp_mlp_create(nfeat: int, params=None, seed: int = 0, device: int = 0,
                   stream: int | None = None) -> int:
    h = C.c_void_p()
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    _check(load().ftp_mlp_create(C.byref(h), int(nfeat), _ptr(p), int(seed) & (2**64 - 1),
                                 int(device), stream), "ftp_mlp_create")
    return h.value


def ftp_mlp_destroy(mlp: int) -> None:
    load().ftp_mlp_destroy(mlp)


def ftp_mlp_get_params(mlp: int, out) -> None:
    _check(load().ftp_mlp_get_params(mlp, _ptr(out)), "ftp_mlp_get_params")


def ftp_mlp_set_params(mlp: int, params) -> None:
    _check(load().ftp_mlp_set_params(mlp, _ptr(params)), "ftp_mlp_set_params")


def ftp_mlp_get_state(mlp: int, params, adam_m, adam_v) -> int:
    """Fills the three arrays; returns the number of Adam steps taken."""
    steps = C.c_int64(0)
    _check(load().ftp_mlp_get_state(mlp, _ptr(params), _ptr(adam_m), _ptr(adam_v),
                                    C.byref(steps)), "ftp_mlp_get_state")
    return int(steps.value)


def ftp_mlp_set_state(mlp: int, params, adam_m, adam_v, steps: int) -> None:
    _check(load().ftp_mlp_set_state(mlp, _ptr(params), _ptr(adam_m), _ptr(adam_v), int(steps)),
           "ftp_mlp_set_state")


def ftp_mlp_forward(mlp: int, X, n: int, scores) -> None:
    _check(load().ftp_mlp_forward(mlp, _ptr(X), int(n), _ptr(scores)), "ftp_mlp_forward")


def ftp_mlp_gradient(mlp: int, X, target, rows: int, idx, n: int, grad=None, loss=None) -> None:
    _check(load().ftp_mlp_gradient(mlp, _ptr(X), _ptr(target), int(rows), _ptr(idx), int(n),
                                   _ptr(grad), _ptr(loss)), "ftp_mlp_gradient")


def ftp_mlp_train(mlp: int, X, target, rows: int, steps: int, batch: int, lr: float, seed: int,
                  losses=None) -> None:
    _check(load().ftp_mlp_train(mlp, _ptr(X), _ptr(target), int(rows), int(steps), int(batch),
                                float(lr), int(seed) & (2**64 - 1), _ptr(losses)),
           "ftp_mlp_train")


def ftp_training_rows(power, features, nfeat: int, row_off, top_frac: float, neighbours: int,
                      rand_frac: float, seed: int, X_out, y_out, cap: int, count: int,
                      device: int = 0, stream: int | None = None) -> int:
    """Appends training rows (see include/ftp.h); returns the new row count."""
    row_off = np.ascontiguousarray(row_off, dtype=np.int64)
    c = C.c_int64(int(count))
    _check(load().ftp_training_rows(_ptr(power), _ptr(features), int(nfeat), row_off.shape[0] - 1,
                                    _ptr(row_off), float(top_frac), int(neighbours),
                                    float(rand_frac), int(seed) & (2**64 - 1), _ptr(X_out),
                                    _ptr(y_out), int(cap), C.byref(c), int(device), stream),
           "ftp_training_rows")
    return c.value


def ftp_multiband_periodogram(plan: int, obs_off, t, y, dy, bank, tpl_of_band, power,
                              band_power=None, band_theta1=None, band_theta2=None,
                              band_theta3=None, band_flags=None) -> None:
    """Multi-phase multi-band periodogram over the plan's grid (see include/ftp.h)."""
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    arr, keep = _templates(bank)
    tob = None if tpl_of_band is None else np.ascontiguousarray(tpl_of_band, dtype=np.int32)
    _check(load().ftp_multiband_periodogram(plan, obs_off.shape[0] - 1, _ptr(obs_off), _ptr(t),
                                            _ptr(y), _ptr(dy), arr, len(keep) // 2, _ptr(tob),
                                            _ptr(power), _ptr(band_power), _ptr(band_theta1),
                                            _ptr(band_theta2), _ptr(band_theta3),
                                            _ptr(band_flags)), "ftp_multiband_periodogram")


def ftp_shared_multiband(plan: int, obs_off, t, y, dy, offsets, bank, tpl_of_band, power,
                         theta1, theta2, theta3, flags=None) -> None:
    """Shared-phase multi-band template periodogram (see include/ftp.h)."""
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    lam = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.float64)
    arr, keep = _templates(bank)
    tob = None if tpl_of_band is None else np.ascontiguousarray(tpl_of_band, dtype=np.int32)
    _check(load().ftp_shared_multiband(plan, obs_off.shape[0] - 1, _ptr(obs_off), _ptr(t), _ptr(y),
                                       _ptr(dy), _ptr(lam), arr, len(keep) // 2, _ptr(tob),
                                       _ptr(power), _ptr(theta1), _ptr(theta2), _ptr(theta3),
                                       _ptr(flags)), "ftp_shared_multiband")


def ftp_set_positive_amplitude(plan: int, enable: bool) -> None:
    _check(load().ftp_set_positive_amplitude(plan, 1 if enable else 0),
           "ftp_set_positive_amplitude")


def ftp_set_batch_tuning(plan: int, sum_lanes: int, roots_ctas_per_sm: int = 0) -> None:
    _check(load().ftp_set_batch_tuning(plan, int(sum_lanes), int(roots_ctas_per_sm)),
           "ftp_set_batch_tuning")


def ftp_get_batch_tuning(plan: int) -> dict:
    a, b = C.c_int(), C.c_int()
    _check(load().ftp_get_batch_tuning(plan, C.byref(a), C.byref(b)), "ftp_get_batch_tuning")
    return {"sum_lanes": a.value, "roots_ctas_per_sm": b.value}


def ftp_batch_autotune(plan: int, obs_off, t, y, dy, grids, out_off, bank, tpl_of_curve, power,
                       theta1, theta2, theta3, cache_path: str | None = None) -> dict:
    """Times the batch tuning choices on this batch (outputs are scratch) or
    applies a cached result; returns the chosen settings and whether they
    came from the cache."""
    obs_off = np.ascontiguousarray(obs_off, dtype=np.int64)
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    arr, keep = _templates(bank)
    tpc = None if tpl_of_curve is None else np.ascontiguousarray(tpl_of_curve, dtype=np.int32)
    fc = C.c_int()
    _check(load().ftp_batch_autotune(plan, obs_off.shape[0] - 1, _ptr(obs_off), _ptr(t), _ptr(y),
                                     _ptr(dy), _grids(grids), _ptr(out_off), arr, len(keep) // 2,
                                     _ptr(tpc), _ptr(power), _ptr(theta1), _ptr(theta2),
                                     _ptr(theta3), None if cache_path is None else
                                     os.fsencode(cache_path), C.byref(fc)), "ftp_batch_autotune")
    r = ftp_get_batch_tuning(plan)
    r["from_cache"] = bool(fc.value)
    return r


def ftp_set_batch_options(plan: int, chunk_bytes: int = 0, use_graph: bool = True) -> None:
    _check(load().ftp_set_batch_options(plan, int(chunk_bytes), 1 if use_graph else 0),
           "ftp_set_batch_options")


def ftp_batch_info(plan: int) -> dict:
    n, g = C.c_int64(), C.c_int()
    _check(load().ftp_batch_info(plan, C.byref(n), C.byref(g)), "ftp_batch_info")
    return {"chunks": n.value, "graph": g.value}


def ftp_plan_info(plan: int) -> dict:
    n, nt = C.c_int64(), C.c_int64()
    m, la = C.c_int(), C.c_int()
    _check(load().ftp_plan_info(plan, C.byref(n), C.byref(m), C.byref(nt), C.byref(la)),
           "ftp_plan_info")
    return {"grid_len": n.value, "half_width": m.value, "ntiles": nt.value,
            "last_launches": la.value}


def ftp_solver_stats(plan: int) -> dict:
    n, nc, rs, rn, sn = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    it = C.c_double()
    _check(load().ftp_solver_stats(plan, C.byref(n), C.byref(it), C.byref(nc), C.byref(rs),
                                   C.byref(rn), C.byref(sn)), "ftp_solver_stats")
    return {"items": n.value, "mean_iterations": it.value, "nonconverged": nc.value,
            "resolved": rs.value, "resolved_nonconverged": rn.value,
            "still_nonconverged": sn.value}


def ftp_set_solver_limits(plan: int, maxit: int = 0, redo_maxit: int = 0,
                          wait_polls: int = 0) -> None:
    _check(load().ftp_set_solver_limits(plan, int(maxit), int(redo_maxit), int(wait_polls)),
           "ftp_set_solver_limits")


def ftp_alu_peak(device: int, kind: int, iters: int) -> tuple:
    """(flops, ms) of one FMA-chain launch: kind 0 FP32, 1 FP32 pairs, 2 FP64."""
    f, ms = C.c_double(), C.c_float()
    _check(load().ftp_alu_peak(int(device), int(kind), int(iters), C.byref(f), C.byref(ms)),
           "ftp_alu_peak")
    return f.value, float(ms.value)


def ftp_set_fault_injection(plan: int, mode: int) -> None:
    _check(load().ftp_set_fault_injection(plan, int(mode)), "ftp_set_fault_injection")


def ftp_set_timing(plan: int, enable: bool) -> None:
    _check(load().ftp_set_timing(plan, 1 if enable else 0), "ftp_set_timing")


def ftp_stage_times(plan: int) -> list:
    a = (C.c_float * 6)()
    _check(load().ftp_stage_times(plan, a), "ftp_stage_times")
    return list(a)


def ftp_roots_first_phase_ms(plan: int) -> float:
    v = C.c_float()
    _check(load().ftp_roots_first_phase_ms(plan, C.byref(v)), "ftp_roots_first_phase_ms")
    return float(v.value)


def ftp_periodogram_sums_noalloc(sums, row_stride: int, precision: str, nf: int, H_sums: int,
                                 ybar: float, YY: float, templates, power, theta1, theta2,
                                 theta3, flags=None, device: int = 0,
                                 stream: int | None = None) -> None:
    """Root stage on device-resident sums without any allocation (see
    include/ftp.h); all arrays must be device memory."""
    prec = {"mixed": FTP_MIXED, "fp64": FTP_FP64}[precision]
    arr, keep = _templates(templates)
    _check(load().ftp_periodogram_sums_noalloc(
        _ptr(sums), int(row_stride), prec, int(nf), int(H_sums), float(ybar), float(YY), arr,
        len(keep) // 2, _ptr(power), _ptr(theta1), _ptr(theta2), _ptr(theta3), _ptr(flags),
        int(device), stream), "ftp_periodogram_sums_noalloc")


class Plan:
    """Convenience owner of a plan handle (closes it on exit)."""

    def __init__(self, max_nobs, max_H, grid, max_templates=1, precision="mixed", device=0,
                 stream=None):
        self.grid = (float(grid[0]), int(grid[1]), int(grid[2]))
        self.precision = precision
        self.h = ftp_plan(max_nobs, max_H, self.grid, max_templates, precision, device, stream)

    @property
    def nf(self) -> int:
        return self.grid[2]

    def close(self):
        if self.h:
            ftp_destroy(self.h)
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

    def periodogram(self, t, y, dy, templates, flags=True) -> dict:
        """Host arrays in, host arrays out: dict(power, theta1, theta2, theta3, flags)."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        dy = np.ascontiguousarray(dy, dtype=np.float64)
        nt = len(templates)
        out = {k: np.empty((nt, self.nf)) for k in ("power", "theta1", "theta2", "theta3")}
        out["flags"] = np.empty((nt, self.nf), dtype=np.uint8) if flags else None
        ftp_periodogram(self.h, t, y, dy, t.shape[0], templates, out["power"], out["theta1"],
                        out["theta2"], out["theta3"], out["flags"])
        return out

    def sums(self, t, y, dy, H):
        """Host arrays in: returns (complex sums [3H][nf], (ybar, YY))."""
        t = np.ascontiguousarray(t, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        dy = np.ascontiguousarray(dy, dtype=np.float64)
        dt = np.complex64 if self.precision == "mixed" else np.complex128
        s = np.empty((3 * H, self.nf), dtype=dt)
        mo = np.empty(2)
        ftp_sums(self.h, t, y, dy, t.shape[0], H, s, mo)
        return s, (float(mo[0]), float(mo[1]))

    def info(self) -> dict:
        return ftp_plan_info(self.h)

    def solver_stats(self) -> dict:
        return ftp_solver_stats(self.h)

    def set_solver_limits(self, maxit: int = 0, redo_maxit: int = 0, wait_polls: int = 0):
        ftp_set_solver_limits(self.h, maxit, redo_maxit, wait_polls)
