"""Seeded synthetic inputs (lightcurves, templates, frequency grids) shared by
the CPU oracle tests, the CUDA parity tests and the benchmark.  Inputs only:
no periodogram arithmetic lives here."""
from .lightcurves import (Grid, Lightcurve, Survey, Template, bank_curve, long_curve,
                          make_template, nightly_times, random_curve, small_curve, survey)

__all__ = ["Grid", "Lightcurve", "Survey", "Template", "bank_curve", "long_curve",
           "make_template", "nightly_times", "random_curve", "small_curve", "survey"]
