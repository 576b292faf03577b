"""GB300 (sm_103a) Fast Template Periodogram: a CUDA library behind a C ABI
(include/ftp.h) and a thin ctypes binding (``paper_2101_12348_gb300.ftp``).

Importing the package does not load the shared library; the first call does,
and raises if it has not been built."""
from . import ftp
from .ftp import (FtpError, Plan, ftp_batch, ftp_destroy, ftp_periodogram, ftp_plan,
                  ftp_plan_info, ftp_set_timing, ftp_solver_stats, ftp_stage_times, ftp_status_string, ftp_sums)

__all__ = ["ftp", "FtpError", "Plan", "ftp_batch", "ftp_destroy", "ftp_periodogram", "ftp_plan",
           "ftp_plan_info", "ftp_set_timing", "ftp_solver_stats", "ftp_stage_times", "ftp_status_string", "ftp_sums"]
