"""Pins for oracle/quadrature.py against closed forms.

The rule must integrate every monomial of total degree <= 2m-1 exactly on the
reference n-simplex; the exact value is the Dirichlet moment formula
    int_{simplex} x^alpha dx = prod(alpha_i!) / (|alpha| + n)!
The 1D Legendre rule must coincide with the textbook Gauss-Legendre rule."""
import itertools
import math

import numpy as np
import pytest

from oracle import quadrature as q


def dirichlet_moment(alpha):
    return math.prod(math.factorial(a) for a in alpha) / math.factorial(sum(alpha) + len(alpha))


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7])
def test_simplex_moments_exact(n, m):
    pts, w, bary = q.simplex_rule(n, m)
    assert pts.shape == (m ** n, n)
    assert np.all(w > 0)
    assert np.all(bary >= -1e-15) and np.allclose(bary.sum(axis=1), 1.0)
    for deg in range(2 * m):
        for alpha in itertools.product(range(deg + 1), repeat=n):
            if sum(alpha) != deg:
                continue
            val = float(np.sum(w * np.prod(pts ** np.array(alpha), axis=1)))
            ex = dirichlet_moment(alpha)
            assert abs(val - ex) <= 2e-15 * max(1.0, ex) + 1e-16, (n, m, alpha, val, ex)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_degree_not_exceeded(n):
    """The rule is not exact beyond degree 2m-1 (so the test above is sharp)."""
    m = 3
    pts, w, _ = q.simplex_rule(n, m)
    alpha = (2 * m,) + (0,) * (n - 1)
    val = float(np.sum(w * pts[:, 0] ** (2 * m)))
    assert abs(val - dirichlet_moment(alpha)) > 1e-8


@pytest.mark.parametrize("m", [1, 2, 5, 8])
def test_legendre_matches_textbook(m):
    x, w = q.gauss_jacobi(m, 0.0, 0.0)
    xr, wr = np.polynomial.legendre.leggauss(m)
    assert np.allclose(x, xr, atol=1e-14, rtol=0) and np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("a", [1, 2])
def test_jacobi_weighted_moments(a):
    """Gauss-Jacobi on [0,1] with weight (1-x)^a integrates x^k exactly:
    int_0^1 (1-x)^a x^k dx = a! k! / (a+k+1)!"""
    m = 4
    x, w = q.gauss_jacobi01(m, a)
    for k in range(2 * m):
        ex = math.factorial(a) * math.factorial(k) / math.factorial(a + k + 1)
        assert abs(np.sum(w * x ** k) - ex) < 1e-15
