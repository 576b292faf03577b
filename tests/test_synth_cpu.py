"""The seeded input generators match the recipe they document (sizes, ranges,
grids, template normalisation) and give the same arrays for the same seed."""
import numpy as np

import synth


def test_templates_are_seeded_and_unit_variance():
    a, b = synth.make_template(6, 2000), synth.make_template(6, 2000)
    np.testing.assert_array_equal(a.c, b.c)
    np.testing.assert_array_equal(a.s, b.s)
    for H in (1, 3, 10, 16):
        tp = synth.make_template(H, 7 + H)
        assert tp.H == H
        assert abs(0.5 * np.sum(tp.c ** 2 + tp.s ** 2) - 1.0) < 1e-12
        x = np.linspace(0, 2 * np.pi, 4096, endpoint=False)
        assert abs(np.mean(tp(x))) < 1e-12          # no constant term
        assert abs(np.mean(tp(x) ** 2) - 1.0) < 1e-12


def test_small_curve_recipe():
    lc, tpl, grid = synth.small_curve()
    lc2, _, _ = synth.small_curve()
    np.testing.assert_array_equal(lc.y, lc2.y)
    assert lc.t.size == 200 and tpl.H == 3
    assert np.all(np.diff(lc.t) >= 0) and lc.t.min() >= 0 and lc.t.max() <= 30
    assert np.all((lc.dy >= 0.05) & (lc.dy <= 0.15))
    assert (grid.k0, grid.nf) == (1, 5000) and abs(grid.df - 1 / 150) < 1e-15
    np.testing.assert_allclose(grid.freqs()[[0, -1]], [1 / 150, 5000 / 150])


def test_long_curve_recipe():
    lc, tpl, grid = synth.long_curve()
    assert lc.t.size == 10_000 and tpl.H == 6
    assert np.all(np.diff(lc.t) >= 0) and lc.t.max() < 3000
    assert np.all(lc.t - np.floor(lc.t) <= 8 / 24 + 1e-12)      # 8 h nightly windows
    kept = np.unique(np.floor(lc.t)).size
    assert 0.6 * 3000 < kept <= 0.7 * 3000 * 1.05                 # ~30 % of nights dropped
    assert np.all(lc.dy == 0.05)
    assert (grid.k0, grid.nf) == (1, 250_000) and abs(grid.df - 1 / 15000) < 1e-18


def test_survey_recipe():
    sv = synth.survey(ncurves=64)
    sv2 = synth.survey(ncurves=64)
    np.testing.assert_array_equal(sv.t, sv2.t)
    n = np.diff(sv.obs_off)
    assert sv.ncurves == 64 and np.all((n >= 50) & (n <= 20_000))
    np.testing.assert_array_equal(sv.tpl_of_curve, np.arange(64) % 16)
    assert [tp.H for tp in sv.bank] == [(2, 4, 6)[i % 3] for i in range(16)]
    assert np.all(sv.injected == (np.arange(64) % 2 == 0))
    per = sv.period[sv.injected]
    assert np.all((per >= 0.2) & (per <= 50)) and np.all(np.isnan(sv.period[~sv.injected]))
    for c in range(sv.ncurves):
        lc, g = sv.curve(c), sv.grids[c]
        T = 1.0 / (5.0 * g.df)
        assert 100 <= T <= 3000 and lc.t.max() <= T and g.k0 == 1
        assert g.nf == int(np.floor(10.0 / g.df))
        assert np.all((lc.dy >= 0.05) & (lc.dy <= 0.15))


def test_bank_curve_recipe():
    lc, bank, grid = synth.bank_curve()
    assert lc.t.size == 100_000 and len(bank) == 32 and all(tp.H == 10 for tp in bank)
    np.testing.assert_array_equal(bank[5].c, synth.make_template(10, 2005).c)
    assert np.all(np.diff(lc.t) >= 0) and lc.t.max() < 4000
    assert np.all(lc.t - np.floor(lc.t) <= 8 / 24 + 1e-12)
    assert (grid.k0, grid.nf) == (1, 1_000_000) and abs(grid.df - 1 / 20000) < 1e-18
