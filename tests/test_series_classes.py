"""Truncation of the FP32 field kernel's exponent-series classes (the pair term of Eq. 1/2).

E1(a) - E1(b) = e^{-a} P(h) with P(h) = int_0^1 e^{-hs} r / (1 + r s) ds, h = b - a and
r = b/a - 1 (the substitution u = a (1 + r s) in the definition of E1 below Eq. 2).  The
kernel evaluates ln P(h) as ln c_0 + sum_{m<=d} l_m h^m, where the l_m are the coefficients
of the power series of ln(P(h)/c_0) (the cumulant recurrence l_m = p_m - (1/m) sum_{k<m}
k l_k p_{m-k}, p_m = c_m / c_0, c_m = (-1)^m J_m / m!, J_m = int_0^1 r s^m / (1 + r s) ds),
and picks the degree d per (warp, visit) from the largest h of its pairs.  This test takes
each class's largest h from the kernel header and checks, against FP64 adaptive quadrature
of P(h) itself (independent of the kernel's recurrences), that the truncated series stays
within the stated bound for r across twelve decades.
"""
import math
import os
import re

import numpy as np
import pytest

integrate = pytest.importorskip("scipy.integrate")

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2507_00294_gb300", "csrc", "dd_field_impl.cuh")
BOUND = 2.5e-7          # as the header states; the quadrature itself is good to ~1e-13


def class_limits():
    text = open(HEADER).read()
    m = re.search(r"constexpr float kL2H = ([0-9.]+)f, kL4H = ([0-9.]+)f, kL8H = ([0-9.]+)f, kL12H = ([0-9.]+)f;", text)
    assert m, "class limits not found in the kernel header"
    return {2: float(m.group(1)), 4: float(m.group(2)), 8: float(m.group(3)), 12: float(m.group(4))}


def quad(f, r):
    pts = [1.0 / r] if r > 1.0 else None
    v, err = integrate.quad(f, 0.0, 1.0, points=pts, epsabs=0.0, epsrel=1e-13, limit=400)
    return v


def log_series_coeffs(r, M=12):
    J = [math.log1p(r)] + [quad(lambda s, m=m: r * s ** m / (1.0 + r * s), r) for m in range(1, M + 1)]
    c = [(-1) ** m * J[m] / math.factorial(m) for m in range(M + 1)]
    p = [cm / c[0] for cm in c]
    l = [0.0] * (M + 1)
    for m in range(1, M + 1):
        l[m] = p[m] - sum(k * l[k] * p[m - k] for k in range(1, m)) / m
    return c, l


@pytest.mark.parametrize("degree", [2, 4, 8, 12])
def test_truncation_within_bound_at_class_limit(degree):
    h = class_limits()[degree]
    worst = 0.0
    for r in 10.0 ** np.arange(-12.0, 6.01, 0.5):
        c, l = log_series_coeffs(r)
        exact = math.log(quad(lambda s: math.exp(-h * s) * r / (1.0 + r * s), r))
        approx = math.log(c[0]) + sum(l[m] * h ** m for m in range(1, degree + 1))
        worst = max(worst, abs(exact - approx))
    assert worst <= BOUND, (degree, h, worst)


def test_class_limits_increase_and_series_converge():
    lim = class_limits()
    assert lim[2] < lim[4] < lim[8] < lim[12] < 2.0 * math.pi      # the series' radius is 2 pi
    # the cumulant coefficients shrink like (2 pi)^-m: the bound that makes the classes work
    for r in (1e-12, 1e-9, 1e-6, 1e-2, 1.0, 1e2, 1e6):
        _, l = log_series_coeffs(r)
        for m in range(2, 13):
            assert abs(l[m]) <= 0.6 * (2.0 * math.pi) ** (1 - m), (r, m, l[m])
