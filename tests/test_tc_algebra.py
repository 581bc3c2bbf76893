"""The algebra of the tensor-core contraction (dd_field_tc.cuh), in FP64 on the CPU: with
x = dx^2 and y = dy^2 (rho^2 = x + y), a pair term 2^G, G = g_0 + sum_m g_m (x + y)^m, is
summed as a rank-2 (degree 2) or rank-4 (degree 4) bilinear form of column factors (x
only) and row factors (y only).  These tests check that the stated forms reproduce 2^G
within the series classes' budget at every point where the class holds (h = rho^2 dq up to
0.04 and 0.33), for coefficients spanning the exponent series' range (|g_m| up to
log2(e) l_m dq^m with the largest |l_m|)."""
import math

import numpy as np

LN2 = math.log(2.0)
LOG2E = 1.0 / LN2
# largest |l_m| of the exponent series (cumulants of s on [0, 1] under r/(1+rs)): m = 1..4
L_MAX = (0.5, 0.042, 3.9e-3, 4.0e-4)


def draw(rng, n, h_max, deg):
    """Random records and points with h = (x + y) dq <= h_max: g_1 carries the -a term
    (-q1 log2 e) plus log2(e) l_1 dq, the higher g_m = log2(e) l_m dq^m."""
    dq = 10.0 ** rng.uniform(-6, 0, n)
    q1 = dq * 10.0 ** rng.uniform(-1, 3, n)              # a = rho^2 q1 >= h / 10
    l = [rng.uniform(-L_MAX[m], L_MAX[m], n) for m in range(deg)]
    g = [rng.uniform(-20, 0, n)]                         # g_0: log2 of ln(w1/w0)
    g.append(LOG2E * (l[0] * dq - q1))
    for m in range(2, deg + 1):
        g.append(LOG2E * l[m - 1] * dq ** m)
    rho2 = rng.uniform(0, 1, n) * h_max / dq
    frac = rng.uniform(0, 1, n)
    return g, rho2 * frac, rho2 * (1 - frac)


def exact(g, x, y):
    r = x + y
    G = g[0] + sum(g[m] * r ** m for m in range(1, len(g)))
    return np.exp2(G)


def test_degree2_form():
    """term = X Y + A B, X = 2^(g_1 x + g_2 x^2), Y = 2^(g_0 + g_1 y + g_2 y^2),
    A = X (2 ln2 g_2) x, B = Y y: within 2.5e-7 of 2^G wherever h <= 0.04."""
    rng = np.random.default_rng(1)
    g, x, y = draw(rng, 200_000, 0.04, 2)
    X = np.exp2(g[1] * x + g[2] * x * x)
    Y = np.exp2(g[0] + g[1] * y + g[2] * y * y)
    A = X * (2 * LN2 * g[2]) * x
    B = Y * y
    t = exact(g, x, y)
    rel = np.abs(X * Y + A * B - t) / t
    assert rel.max() <= 2.5e-7, rel.max()
    # and the leading product alone misses by the cross term 2 g_2 x y (log2 units)
    assert np.max(np.abs(X * Y / t - 1)) > 1e-6


def test_degree4_form():
    """term = X Y + A_1 B_1 + A_2 B_2 + A_3 B_3 with B_k = y^k Y,
    A_1 = X ln2 x (2 g_2 + 3 g_3 x + 4 g_4 x^2),
    A_2 = X x (3 ln2 g_3 + (6 ln2 g_4 + 2 ln2^2 g_2^2) x), A_3 = X ln2 4 g_4 x:
    within 3e-7 of 2^G wherever h <= 0.33."""
    rng = np.random.default_rng(2)
    g, x, y = draw(rng, 200_000, 0.33, 4)
    X = np.exp2(g[1] * x + g[2] * x ** 2 + g[3] * x ** 3 + g[4] * x ** 4)
    Y = np.exp2(g[0] + g[1] * y + g[2] * y ** 2 + g[3] * y ** 3 + g[4] * y ** 4)
    c1, c2, c3 = 2 * LN2 * g[2], 3 * LN2 * g[3], 4 * LN2 * g[4]
    c6 = 6 * LN2 * g[4] + 2 * LN2 ** 2 * g[2] ** 2
    A1 = X * x * (c1 + x * (c2 + x * c3))
    A2 = X * x * (c2 + x * c6)
    A3 = X * x * c3
    B1, B2, B3 = Y * y, Y * y * y, Y * y ** 3
    t = exact(g, x, y)
    rel = np.abs(X * Y + A1 * B1 + A2 * B2 + A3 * B3 - t) / t
    assert rel.max() <= 3e-7, rel.max()
    # the dropped second-order cross terms matter only beyond that budget: keeping just
    # the first-order part (z) misses by (2 ln2 g_2 x y)^2 / 2
    first = X * Y * (1 + LN2 * (2 * g[2] * x * y + g[3] * (3 * x * x * y + 3 * x * y * y)
                                 + g[4] * (4 * x ** 3 * y + 6 * x * x * y * y + 4 * x * y ** 3)))
    assert np.max(np.abs(first / t - 1)) > rel.max()


def test_bf16_three_piece_split():
    """v = h + m + l in BF16 pieces (each the round-to-nearest BF16 of what the earlier
    leave): |v - h - m - l| <= 2^-24 |v|, and the six products of two such splits keep
    X Y to about 4 2^-24."""
    rng = np.random.default_rng(3)

    def bf16(v):
        b = v.astype(np.float32).view(np.uint32).astype(np.uint64)
        r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16            # round to nearest even
        return r.astype(np.uint32).view(np.float32).astype(np.float64)

    def split3(v):
        v = v.astype(np.float32).astype(np.float64)
        h = bf16(v)
        m = bf16(v - h)
        return h, m, bf16(v - h - m)

    X = 10.0 ** rng.uniform(-30, 0, 100_000)
    Y = 10.0 ** rng.uniform(-30, 0, 100_000)
    xh, xm, xl = split3(X)
    yh, ym, yl = split3(Y)
    Xf, Yf = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
    assert np.max(np.abs(Xf - xh - xm - xl) / Xf) <= 2.0 ** -24
    six = xh * yh + xh * ym + xm * yh + xh * yl + xl * yh + xm * ym
    assert np.max(np.abs(six - Xf * Yf) / (Xf * Yf)) <= 4 * 2.0 ** -24
