"""Pins for the oracle's E_1 and E_1-difference routines (definition below Eq. 2).

E_1 is checked against two independent library implementations (scipy, mpmath at 40
digits) and the A&S 5.1.20 bounds; the difference is checked against mpmath at 40
digits, including differences that cancel to 1e-9 of the values.
"""
import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
sp = pytest.importorskip("scipy.special")


def test_e1_matches_scipy_over_range():
    x = np.logspace(-12, np.log10(700.0), 600)
    got = oracle.e1(x)
    ref = sp.exp1(x)
    assert np.max(np.abs(got / ref - 1.0)) < 1e-14


def test_e1_matches_mpmath():
    mp.mp.dps = 40
    xs = [1e-10, 1e-3, 0.1, 0.5, 0.99, 1.0, 1.01, 2.0, 5.0, 10.0, 50.0, 200.0, 700.0]
    for x in xs:
        ref = float(mp.e1(mp.mpf(x)))
        assert abs(float(oracle.e1(x)) / ref - 1.0) < 1e-14, x


def test_e1_special_values():
    assert np.isinf(oracle.e1(0.0))              # E1(0) = +inf
    assert oracle.e1(800.0) == 0.0               # below FP64 range
    assert np.isnan(oracle.e1(-1.0))


def test_e1_as_bounds():
    # A&S 5.1.20: 1/2 ln(1 + 2/x) < e^x E1(x) < ln(1 + 1/x)
    x = np.logspace(-6, 2.5, 300)
    g = np.exp(x) * oracle.e1(x)
    assert np.all(0.5 * np.log1p(2.0 / x) < g)
    assert np.all(g < np.log1p(1.0 / x))


@pytest.mark.parametrize("a", [1e-12, 1e-6, 1e-3, 0.05, 0.5, 1.0, 1.5, 3.0, 10.0, 40.0, 120.0, 600.0])
def test_e1_difference_matches_mpmath(a):
    mp.mp.dps = 40
    for ell in [1e-12, 1e-9, 1e-6, 1e-3, 0.05, 0.5, 2.0, 8.0, 30.0]:
        b = mp.mpf(a) * mp.e ** mp.mpf(ell)
        ref = mp.e1(mp.mpf(a)) - mp.e1(b)
        if ref == 0 or float(ref) < 1e-300:
            continue
        q = float(oracle.e1_diff_log(a, ell))
        assert abs(q / float(ref) - 1.0) < 2e-14, (a, ell, q, float(ref))
        if float(b) < 1e300:
            d = float(oracle.e1_diff(a, float(b)))
            # two-number interface: b carries its own rounding, relative ~ u / ell
            tol = max(3e-13, 4e-16 / ell * (1 + a))
            assert abs(d / float(ref) - 1.0) < tol, (a, ell, d, float(ref))


def test_quadrature_agrees_with_value_difference_where_well_conditioned():
    rng = np.random.default_rng(11)
    a = 10.0 ** rng.uniform(-8, 2, 200)
    b = a * (1.0 + 10.0 ** rng.uniform(0, 2, 200))
    q = oracle.e1_diff_quad(a, b)
    d = oracle.e1(a) - oracle.e1(b)
    assert np.max(np.abs(q / d - 1.0)) < 1e-13


def test_tabulated_values():
    """The oracle's E1 against tabulated values (tests/golden/e1_table.txt, 10 significant
    digits): agreement to the table's last digit."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "e1_table.txt")
    rows = np.loadtxt(path, comments="#")
    assert rows.shape == (9, 2)
    for x, v in rows:
        got = float(oracle.e1(x))
        assert abs(got / v - 1.0) <= 5e-10, (x, got, v)
