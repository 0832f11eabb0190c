"""Section 6.3: the recursion eq. (3.1) may start from any basis of the
spatial polynomials; the paper compares monomials, Legendre and Chebyshev
polynomials and finds that only the monomials keep the system well
conditioned at high degree.  Pinned here on the oracle: every start gives
exact Trefftz functions spanning the same U^p (same dimension, same front
after a sweep up to rounding), and on a 1+1D tent sweep the tent matrices'
condition numbers grow with p fastest for Chebyshev, then Legendre, slowest
for the monomials -- the paper's finding."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import basis as ob
from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs


def test_legendre_and_chebyshev_polynomials_exact():
    assert ob.poly1d("legendre", 3) == [0, Fraction(-3, 2), 0, Fraction(5, 2)]
    assert ob.poly1d("chebyshev", 4) == [1, 0, -8, 0, 8]
    # a 2D index is the tensor product: P_2(x) P_1(y) = (3x^2 - 1)/2 * y
    assert ob.initial_polynomial("legendre", (2, 1)) == {(0, 1): Fraction(-1, 2), (2, 1): Fraction(3, 2)}
    assert ob.initial_polynomial("chebyshev", (1, 2)) == {(1, 0): Fraction(-1), (1, 2): Fraction(2)}


@pytest.mark.parametrize("init", ["legendre", "chebyshev"])
@pytest.mark.parametrize("n,p", [(1, 5), (2, 4), (3, 3)])
def test_every_start_gives_trefftz_functions_of_the_same_space(init, n, p):
    funcs = ob.trefftz_coefficients(n, p, init=init)
    assert len(funcs) == ob.dim_U(n, p)
    monos = [(k, al) for k in range(p + 1) for al in ob.multi_indices(n, p - k)]
    idx = {mm: i for i, mm in enumerate(monos)}
    for a in funcs:                        # -Lap U + U_tt = 0 coefficient by coefficient, exactly
        for (k, al) in monos:
            if k + 2 > p:
                continue
            lap = sum((al[m] + 1) * (al[m] + 2) * a.get((k, tuple(al[:m] + (al[m] + 2,) + al[m + 1:])), 0)
                      for m in range(n)) if k + sum(al) + 2 <= p else 0
            assert (k + 2) * (k + 1) * a.get((k + 2, al), 0) == lap
    # same span as the monomial start: the stacked coefficient matrix has rank dim U^p
    def mat(fs):
        M = np.zeros((len(fs), len(monos)))
        for j, a in enumerate(fs):
            for key, v in a.items():
                M[j, idx[key]] = float(v)
        return M
    A, B = mat(funcs), mat(ob.trefftz_coefficients(n, p))
    assert np.linalg.matrix_rank(np.vstack([A, B]), tol=1e-9) == ob.dim_U(n, p)


def test_same_front_and_the_papers_conditioning_order():
    mesh = inputs.mesh_interval(4)
    w = inputs.workload("plane1d")
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, 0.9, 0.5)
    kappas = {}
    for p in (3, 7, 11):
        fronts = {}
        for init in ("monomial", "legendre", "chebyshev"):
            ks = []
            F, _ = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, w.init, w.dirichlet, basis_init=init,
                             record=lambda it, d: ks.append(np.linalg.cond(d["A"])))
            fronts[init] = F
            kappas[(p, init)] = max(ks)
        if p <= 7:                           # the same discrete solution while rounding stays small
            for init in ("legendre", "chebyshev"):
                assert np.linalg.norm(fronts[init] - fronts["monomial"]) <= 1e-11 * np.linalg.norm(fronts["monomial"])
    for p in (7, 11):
        assert kappas[(p, "monomial")] < kappas[(p, "legendre")] < kappas[(p, "chebyshev")]
    # and the gap widens with p (Section 6.3: the other starts fail at high degree)
    assert kappas[(11, "chebyshev")] / kappas[(11, "monomial")] > kappas[(3, "chebyshev")] / kappas[(3, "monomial")]
