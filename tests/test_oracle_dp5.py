"""Pins for the oracle's embedded 5(4) pairs (Dormand-Prince, Cash-Karp,
Fehlberg; Sec. 3.2): the Butcher order conditions (so a mistyped coefficient
fails), the local orders of the solution and of the error estimate, and the
global order on a harmonic oscillator."""
from fractions import Fraction as Fr
import itertools

import numpy as np
import pytest


def _frac(x):
    return Fr(x).limit_denominator(10 ** 7)


METHODS = [0, 1, 2]      # Dormand-Prince, Cash-Karp, Fehlberg


@pytest.mark.parametrize("method", METHODS)
def test_order_conditions(orc, method):
    c, A, b, bh = orc.tableau(method)
    c = [_frac(x) for x in c]
    A = [[_frac(x) for x in row] for row in A]
    b = [_frac(x) for x in b]
    bh = [_frac(x) for x in bh]
    s = len(c)
    assert s == (7 if method == 0 else 6)
    # row-sum condition and explicitness
    for i in range(s):
        assert sum(A[i]) == c[i]
        assert all(A[i][j] == 0 for j in range(i, s))
    Ac = [sum(A[i][j] * c[j] for j in range(s)) for i in range(s)]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in range(s)) for i in range(s)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(s)) for i in range(s)]
    Ac3 = [sum(A[i][j] * c[j] ** 3 for j in range(s)) for i in range(s)]
    AcAc = [sum(A[i][j] * c[j] * Ac[j] for j in range(s)) for i in range(s)]
    AAc2 = [sum(A[i][j] * Ac2[j] for j in range(s)) for i in range(s)]
    AAAc = [sum(A[i][j] * AAc[j] for j in range(s)) for i in range(s)]

    def conds(w):
        d = lambda v: sum(wi * vi for wi, vi in zip(w, v))
        one = [1] * s
        return [
            (d(one), Fr(1)),
            (d(c), Fr(1, 2)),
            (d([x ** 2 for x in c]), Fr(1, 3)), (d(Ac), Fr(1, 6)),
            (d([x ** 3 for x in c]), Fr(1, 4)), (d([ci * a for ci, a in zip(c, Ac)]), Fr(1, 8)),
            (d(Ac2), Fr(1, 12)), (d(AAc), Fr(1, 24)),
            (d([x ** 4 for x in c]), Fr(1, 5)), (d([ci ** 2 * a for ci, a in zip(c, Ac)]), Fr(1, 10)),
            (d([a * a for a in Ac]), Fr(1, 20)), (d([ci * a for ci, a in zip(c, Ac2)]), Fr(1, 15)),
            (d(Ac3), Fr(1, 20)), (d([ci * a for ci, a in zip(c, AAc)]), Fr(1, 30)),
            (d(AcAc), Fr(1, 40)), (d(AAc2), Fr(1, 60)), (d(AAAc), Fr(1, 120)),
        ]

    for got, want in conds(b):                 # all 17 conditions of order 5
        assert got == want
    for got, want in conds(bh)[:8]:            # the 8 conditions of order 4
        assert got == want
    # the embedded pair really differs at order 5
    assert any(g != w for g, w in conds(bh)[8:])
    if method == 0:
        # first-same-as-last: the last stage is evaluated at the solution
        assert A[6][:6] == b[:6] and b[6] == 0 and c[6] == 1


def test_tableau_values(orc):
    """A few coefficients as printed by the pairs' authors (Cash & Karp 1990,
    Fehlberg 1969), beyond what the order conditions fix."""
    c, A, b, bh = orc.tableau(1)
    assert _frac(c[5]) == Fr(7, 8) and _frac(A[5][3]) == Fr(44275, 110592)
    assert _frac(b[5]) == Fr(512, 1771) and _frac(bh[4]) == Fr(277, 14336)
    c, A, b, bh = orc.tableau(2)
    assert _frac(c[3]) == Fr(12, 13) and _frac(A[3][1]) == Fr(-7200, 2197)
    assert _frac(b[3]) == Fr(28561, 56430) and _frac(bh[4]) == Fr(-1, 5)


@pytest.mark.parametrize("method", METHODS)
def test_fnew_is_rhs_at_solution(orc, method):
    f = lambda y: [y[1], -y[0] + 0.1 * y[0] ** 3]
    yn, fn, _ = orc.dp5_step(f, np.array([0.3, -0.2]), 0.07, method)
    assert np.allclose(fn, f(yn), rtol=0, atol=1e-15)


@pytest.mark.parametrize("method", METHODS)
def test_local_orders(orc, method):
    lam = -0.7 + 0.3j

    def f(y):
        z = complex(y[0], y[1]) * lam
        return [z.real, z.imag]

    errs, ests = [], []
    for h in (0.2, 0.1, 0.05):
        yn, _, e = orc.dp5_step(f, np.array([1.0, 0.0]), h, method)
        ex = np.exp(lam * h)
        errs.append(abs(complex(*yn) - ex))
        ests.append(abs(complex(*e)))
    # solution local error O(h^6), error estimate O(h^5)
    for k in range(2):
        assert 2 ** 5.6 < errs[k] / errs[k + 1] < 2 ** 6.4
        assert 2 ** 4.6 < ests[k] / ests[k + 1] < 2 ** 5.4


@pytest.mark.parametrize("method", METHODS)
def test_global_order_harmonic_oscillator(orc, method):
    f = lambda y: [y[1], -y[0]]
    res = []
    for n in (20, 40, 80):
        h = 2 * np.pi / n
        y = np.array([1.0, 0.0])
        for _ in range(n):
            y, _, _ = orc.dp5_step(f, y, h, method)
        res.append(np.hypot(y[0] - 1.0, y[1]))
    for k in range(2):
        order = np.log2(res[k] / res[k + 1])
        assert 4.7 < order < 5.5
