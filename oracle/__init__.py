"""FP64 CPU oracle for the Fast Template Periodogram.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg; never by the CUDA library or its binding."""
from .ftp_oracle import (FLAG_CONSTANT_P, FLAG_DEGENERATE_MM, FLAG_NEGATIVE_AMP,
                         FLAG_NO_POSITIVE, FLAG_NONCONVERGED, OracleInputError, best_candidate_margin,
                         candidate_phases, choose_best, data_moments, direct_sums,
                         final_poly, fit_at_phase, harmonic_phases, mm_poly,
                         normalized_weights, periodogram, polynomials_at, template_alpha,
                         ym_poly)
from .ftp_oracle import chi2_0, multiband_periodogram, shared_phase_multiband
from . import screen_oracle
