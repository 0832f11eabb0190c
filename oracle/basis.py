"""Trefftz basis of U^p (TEST INFRASTRUCTURE; see oracle/__init__.py).

Section 3: U^p(K) = { U in P^p : -Lap U + c^-2 U_tt = 0 }.  A polynomial
U = sum_{|alpha| + k <= p} a_{k,alpha} x^alpha t^k is Trefftz iff the
coefficients satisfy the recursion eq. (3.1)

    a_{k,alpha} = c^2 / (k (k-1)) * sum_m (alpha_m + 1)(alpha_m + 2) a_{k-2, alpha + 2 e_m}.

The recursion is started from a basis of P^p (k = 0 data, dU/dt(.,0) = 0) and
a basis of P^{p-1} (k = 1 data, U(.,0) = 0); dim U^p = C(p+n, n) + C(p-1+n, n).
Monomials are the initial bases (Section 6.3: monomials behave best); the
Legendre and Chebyshev starts of that comparison are available too.
Coefficients are computed once for c = 1 (Remark 3.1) as exact rationals and
rounded to binary64 once.

Remark 3.1 maps the c = 1 basis to a tent: xhat = (x - x_c)/h,
that = c (t - t_c)/h, so U = Uhat, dU/dt = (c/h) dUhat/dthat,
grad U = (1/h) grad_hat Uhat.

Basis order (internal to the oracle; results never depend on it): type-0
functions before type-1 functions, each by graded order of beta
(total degree ascending, then exponent tuples descending).
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from math import comb

import numpy as np


def multi_indices(n: int, deg: int):
    """All alpha in N_0^n with |alpha| <= deg; total degree ascending, then
    exponent tuples in descending lexicographic order."""
    out = []
    for d in range(deg + 1):
        level = [a for a in itertools.product(range(d + 1), repeat=n) if sum(a) == d]
        level.sort(reverse=True)
        out.extend(level)
    return out


def dim_U(n: int, p: int) -> int:
    """dim U^p = C(p+n, n) + C(p-1+n, n) (Section 3)."""
    return comb(p + n, n) + (comb(p - 1 + n, n) if p >= 1 else 0)


def poly1d(kind: str, k: int):
    """Exact ascending-power coefficients of the degree-k Legendre polynomial
    ((j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}) or Chebyshev polynomial of the
    first kind (T_{j+1} = 2x T_j - T_{j-1}) on [-1, 1]."""
    P = [[Fraction(1)], [Fraction(0), Fraction(1)]]
    for j in range(1, k):
        xp = [Fraction(0)] + P[j]
        prev = P[j - 1] + [Fraction(0), Fraction(0)]
        if kind == "legendre":
            P.append([(Fraction(2 * j + 1) * xp[i] - Fraction(j) * prev[i]) / (j + 1) for i in range(j + 2)])
        elif kind == "chebyshev":
            P.append([2 * xp[i] - prev[i] for i in range(j + 2)])
        else:
            raise ValueError(kind)
    return P[k]


def initial_polynomial(kind: str, beta):
    """{alpha: coefficient} of the initial spatial polynomial with index beta:
    the monomial x^beta, or the tensor product prod_m P_{beta_m}(x_m) of
    Legendre / Chebyshev polynomials (Section 6.3 compares the three)."""
    if kind == "monomial":
        return {tuple(beta): Fraction(1)}
    terms = {(): Fraction(1)}
    for b in beta:
        cm = poly1d(kind, b)
        new = {}
        for key, v in terms.items():
            for e, cf in enumerate(cm):
                if cf:
                    new[key + (e,)] = new.get(key + (e,), Fraction(0)) + v * cf
        terms = new
    return terms


def trefftz_coefficients(n: int, p: int, c: Fraction = Fraction(1), init: str = "monomial"):
    """Exact coefficients of the basis: list of dicts {(k, alpha): Fraction}.
    init: the initial spatial polynomials the recursion eq. (3.1) starts from
    (k = 0 data for type 0, k = 1 data for type 1): "monomial" (the path's
    choice), "legendre" or "chebyshev" (Section 6.3); all span U^p."""
    c2 = Fraction(c) * Fraction(c)
    funcs = []
    for typ, deg0 in ((0, p), (1, p - 1)):
        if deg0 < 0:
            continue
        for beta in multi_indices(n, deg0):
            a = {}
            for al, v in initial_polynomial(init, beta).items():
                a[(typ, al)] = v
            for k in range(2, p + 1):
                for alpha in multi_indices(n, p - k):
                    s = Fraction(0)
                    for m in range(n):
                        up = list(alpha)
                        up[m] += 2
                        prev = a.get((k - 2, tuple(up)))
                        if prev:
                            s += (alpha[m] + 1) * (alpha[m] + 2) * prev
                    if s:
                        a[(k, tuple(alpha))] = c2 / (k * (k - 1)) * s
            funcs.append(a)
    return funcs


class TrefftzBasis:
    """Float tables for evaluating the c = 1 basis and its first derivatives."""

    def __init__(self, n: int, p: int, init: str = "monomial"):
        self.n, self.p, self.init = n, p, init
        self.exact = trefftz_coefficients(n, p, init=init)
        self.nb = len(self.exact)
        # monomials t^k x^alpha with k + |alpha| <= p
        self.monos = [(k, alpha) for k in range(p + 1) for alpha in multi_indices(n, p - k)]
        index = {m: i for i, m in enumerate(self.monos)}
        nm = len(self.monos)
        self.coef = np.zeros((self.nb, nm))
        for j, a in enumerate(self.exact):
            for key, val in a.items():
                self.coef[j, index[key]] = float(val)
        self.exps = np.array([[k] + list(al) for (k, al) in self.monos], dtype=np.int64)

    def _derivative_table(self, var: int) -> np.ndarray:
        """Coefficients of d/d(var) of every basis function in the monomial
        list (var 0 = that, var m+1 = xhat_m): exponent rule d(s^e) = e s^(e-1)."""
        index = {m: i for i, m in enumerate(self.monos)}
        D = np.zeros_like(self.coef)
        for i, (k, al) in enumerate(self.monos):
            e = [k] + list(al)
            if e[var] == 0:
                continue
            f = float(e[var])
            e[var] -= 1
            D[:, index[(e[0], tuple(e[1:]))]] += f * self.coef[:, i]
        return D

    def monomials(self, xh: np.ndarray, th: np.ndarray) -> np.ndarray:
        """t^k x^alpha at the points, shape (Q, n_mono)."""
        def powers(s):
            P = np.ones((s.shape[0], self.p + 1))
            for e in range(1, self.p + 1):
                P[:, e] = P[:, e - 1] * s
            return P
        M = powers(th)[:, self.exps[:, 0]]
        for m in range(self.n):
            M = M * powers(xh[:, m])[:, self.exps[:, m + 1]]
        return M

    def eval_ref(self, xh: np.ndarray, th: np.ndarray):
        """Uhat, dUhat/dthat, grad_hat Uhat at reference points:
        shapes (Q, nb), (Q, nb), (Q, n, nb)."""
        if not hasattr(self, "_dt"):
            self._dt = self._derivative_table(0).T.copy()
            self._dx = [self._derivative_table(m + 1).T.copy() for m in range(self.n)]
            self._c = self.coef.T.copy()
        M = self.monomials(xh, th)
        U = M @ self._c
        Ut = M @ self._dt
        G = np.stack([M @ d for d in self._dx], axis=1)
        return U, Ut, G

    def eval_phys(self, x: np.ndarray, t: np.ndarray, xc, tc: float, h: float, c: float):
        """Remark 3.1 mapping: U, v = dU/dt, sigma = -grad U at physical points
        (x (Q, n), t (Q,)) for the tent centred at (xc, tc) with scale h."""
        xh = (x - np.asarray(xc)[None, :]) / h
        th = c * (t - tc) / h
        U, Ut, G = self.eval_ref(xh, th)
        return U, (c / h) * Ut, -(1.0 / h) * G
