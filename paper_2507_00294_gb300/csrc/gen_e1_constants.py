"""Generate the constants of dd_e1.cuh (run by hand; output is pasted into the header).

1. Ein(x) = sum_{k>=1} (-1)^(k+1) x^k / (k k!)  (the entire part of E1, A&S 5.1.11):
   the coefficients are exact rationals, printed as FP32 and FP64.
2. F(z) = x e^x E1(x) with z = 1/x, on z in [0, 1] (x >= 1): a (4,4) rational fit in
   z minimising the relative error, by linearised least squares (Sanathanan-Koerner
   reweighting) on Chebyshev nodes, followed by Lawson reweighting toward minimax.
   Values of F come from mpmath at 30 digits.  The device evaluates
   E1(x) = e^-x P*(x) / (x Q*(x)) with P*(x) = x^4 P(1/x), Q*(x) = x^4 Q(1/x).
"""
import math
from fractions import Fraction

import mpmath as mp
import numpy as np


def ein_coefficients(K):
    return [Fraction((-1) ** (k + 1), k * math.factorial(k)) for k in range(1, K + 1)]


def fit_rational(p=4, q=4, n=3000):
    mp.mp.dps = 30
    z = 0.5 + 0.5 * np.cos(np.pi * (np.arange(n) + 0.5) / n)

    def F(zz):
        if zz == 0:
            return 1.0
        x = 1 / mp.mpf(zz)
        return float(x * mp.e ** x * mp.e1(x))
    f = np.array([F(v) for v in z])
    Vp = np.vander(z, p + 1, increasing=True)
    Vq = np.vander(z, q + 1, increasing=True)[:, 1:]
    w = np.ones(n)
    lawson = np.ones(n)
    best = None
    for it in range(60):
        A = np.hstack([Vp, -f[:, None] * Vq]) * (w * lawson / f)[:, None]
        rhs = f * (w * lawson / f)
        c, *_ = np.linalg.lstsq(A, rhs, rcond=None)
        P, Q = c[:p + 1], np.concatenate([[1.0], c[p + 1:]])
        Qv = np.polyval(Q[::-1], z)
        err = (np.polyval(P[::-1], z) / Qv - f) / f
        m = np.max(np.abs(err))
        if best is None or m < best[0]:
            best = (m, P.copy(), Q.copy())
        w = 1.0 / np.abs(Qv)
        if it >= 10:
            lawson = lawson * (np.abs(err) / m + 1e-3)
            lawson /= lawson.sum() / n
    return best


if __name__ == "__main__":
    for k, c in enumerate(ein_coefficients(12), 1):
        print("ein c%-2d = % .17e" % (k, float(c)))
    m, P, Q = fit_rational()
    print("max rel err of the (4,4) fit: %.3e" % m)
    # reversed (x-form) coefficients, highest power first for Horner in x
    print("P* (x^4..x^0):", ", ".join("%.9ef" % v for v in P))
    print("Q* (x^4..x^0):", ", ".join("%.9ef" % v for v in Q))
