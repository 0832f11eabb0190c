"""Pins for oracle/basis.py (the recursion eq. (3.1)).

* every basis polynomial solves -Lap U + U_tt = 0 exactly (rational check);
* the dimensions equal the paper's formula (golden file, Section 3);
* the recursion started from x^beta (type 0) / t x^beta (type 1) equals the
  closed form sum_j t^(2j+type)/(2j+type)! Lap^j x^beta (Taylor series in t of
  the solution with U(.,0) = x^beta, U_t(.,0) = 0 resp. U = 0, U_t = x^beta);
* the functions are linearly independent;
* the float evaluation tables differentiate correctly (finite differences).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import basis as bz

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "trefftz_dims.txt")


def _laplacian(poly, n):
    """poly: {(k, alpha): coef} -> Lap poly (space variables only)."""
    out = {}
    for (k, al), cf in poly.items():
        for m in range(n):
            if al[m] >= 2:
                a2 = list(al)
                a2[m] -= 2
                key = (k, tuple(a2))
                out[key] = out.get(key, Fraction(0)) + cf * al[m] * (al[m] - 1)
    return {k: v for k, v in out.items() if v != 0}


def _dtt(poly):
    out = {}
    for (k, al), cf in poly.items():
        if k >= 2:
            key = (k - 2, al)
            out[key] = out.get(key, Fraction(0)) + cf * k * (k - 1)
    return {k: v for k, v in out.items() if v != 0}


CASES = [(1, p) for p in range(1, 7)] + [(2, p) for p in range(1, 6)] + [(3, p) for p in range(1, 5)]


@pytest.mark.parametrize("n,p", CASES)
def test_trefftz_property_exact(n, p):
    for poly in bz.trefftz_coefficients(n, p):
        lap = _laplacian(poly, n)
        tt = _dtt(poly)
        keys = set(lap) | set(tt)
        for key in keys:
            assert tt.get(key, 0) - lap.get(key, 0) == 0
        assert all(k + sum(al) <= p for (k, al) in poly)


def test_dimensions_match_paper():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert rows
    for n, p, dU, dW in (map(int, r) for r in rows):
        assert len(bz.trefftz_coefficients(n, p)) == dU == bz.dim_U(n, p)
        assert bz.dim_U(n, p + 1) - 1 == dW


@pytest.mark.parametrize("n,p", [(1, 5), (2, 4), (3, 3)])
def test_closed_form_taylor_series(n, p):
    funcs = bz.trefftz_coefficients(n, p)
    i = 0
    for typ, deg0 in ((0, p), (1, p - 1)):
        for beta in bz.multi_indices(n, deg0):
            expect = {}
            term = {(0, beta): Fraction(1)}
            j = 0
            while term:
                k = 2 * j + typ
                for (_, al), cf in term.items():
                    if k + sum(al) <= p:
                        expect[(k, al)] = cf / math.factorial(k)
                term = _laplacian(term, n)
                j += 1
            got = {k: v for k, v in funcs[i].items() if v != 0}
            assert got == expect, (typ, beta)
            i += 1
    assert i == len(funcs)


@pytest.mark.parametrize("n,p", [(1, 4), (2, 4), (2, 5), (3, 3)])
def test_linear_independence(n, p):
    B = bz.TrefftzBasis(n, p)
    assert np.linalg.matrix_rank(B.coef) == B.nb == bz.dim_U(n, p)


@pytest.mark.parametrize("n,p", [(1, 3), (2, 4), (3, 3)])
def test_derivative_tables_fd(n, p):
    B = bz.TrefftzBasis(n, p)
    rng = np.random.default_rng(0)
    xh = rng.uniform(-0.5, 0.5, size=(7, n))
    th = rng.uniform(-0.5, 0.5, size=7)
    U, Ut, G = B.eval_ref(xh, th)
    eps = 1e-6
    Up, _, _ = B.eval_ref(xh, th + eps)
    Um, _, _ = B.eval_ref(xh, th - eps)
    assert np.allclose((Up - Um) / (2 * eps), Ut, atol=1e-8)
    for m in range(n):
        d = np.zeros(n)
        d[m] = eps
        Up, _, _ = B.eval_ref(xh + d, th)
        Um, _, _ = B.eval_ref(xh - d, th)
        assert np.allclose((Up - Um) / (2 * eps), G[:, m, :], atol=1e-8)
