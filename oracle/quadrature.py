"""Quadrature on the reference n-simplex (TEST INFRASTRUCTURE; see oracle/__init__.py).

Section 4.1: the method integrates only over n-dimensional faces, so one rule
on the spatial n-simplex is built once and mapped onto the tent faces.  The
paper does not name the rule (reading: the collapsed conical-product rule with
m = p + 1 Gauss-Jacobi points per direction, exact for total degree 2p + 1,
enough for every polynomial integrand of the local system).

Gauss-Jacobi nodes/weights come from the Golub-Welsch eigenproblem of the
symmetric Jacobi matrix (numpy.linalg.eigvalsh/eigh as the library step).

Point order convention (shared with any implementation that must produce the
same front layout): nested loops over the collapsed coordinates xi_1 (outer),
..., xi_n (inner), each ascending; xi_1 carries the Jacobi weight
(1 - xi)^(n-1), xi_2 the weight (1 - xi)^(n-2), ..., xi_n the Legendre weight;
reference point x_1 = xi_1, x_2 = (1 - xi_1) xi_2,
x_3 = (1 - xi_1)(1 - xi_2) xi_3; barycentric (1 - sum x, x_1, ..., x_n).
Weights sum to 1/n! (the reference simplex volume).
"""
from __future__ import annotations

import math

import numpy as np


def gauss_jacobi(m: int, a: float, b: float = 0.0):
    """m-point Gauss rule on [-1, 1] for the weight (1-x)^a (1+x)^b
    (Golub-Welsch: nodes are eigenvalues of the Jacobi matrix, weights are
    mu0 times the squared first eigenvector components)."""
    k = np.arange(m, dtype=np.float64)
    s = 2.0 * k + a + b
    diag = np.empty(m)
    for i in range(m):
        if i == 0:
            diag[i] = (b - a) / (a + b + 2.0)
        else:
            diag[i] = (b * b - a * a) / (s[i] * (s[i] + 2.0))
    off = np.empty(max(m - 1, 0))
    for i in range(1, m):
        num = 4.0 * i * (i + a) * (i + b) * (i + a + b)
        den = (2.0 * i + a + b) ** 2 * (2.0 * i + a + b + 1.0) * (2.0 * i + a + b - 1.0)
        off[i - 1] = math.sqrt(num / den)
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    nodes, vecs = np.linalg.eigh(J)
    mu0 = 2.0 ** (a + b + 1.0) * math.gamma(a + 1.0) * math.gamma(b + 1.0) / math.gamma(a + b + 2.0)
    weights = mu0 * vecs[0, :] ** 2
    order = np.argsort(nodes)
    return nodes[order], weights[order]


def gauss_jacobi01(m: int, a: int):
    """Rule on [0, 1] for the weight (1 - xi)^a."""
    x, w = gauss_jacobi(m, float(a), 0.0)
    return 0.5 * (x + 1.0), w / 2.0 ** (a + 1)


def simplex_rule(n: int, m: int):
    """Collapsed rule on the reference n-simplex {x >= 0, sum x <= 1}.

    Returns (pts (Q, n), weights (Q,), bary (Q, n+1)) with Q = m^n."""
    rules = [gauss_jacobi01(m, n - 1 - d) for d in range(n)]
    pts, wts = [], []
    for idx in np.ndindex(*([m] * n)):
        xi = [rules[d][0][idx[d]] for d in range(n)]
        w = 1.0
        for d in range(n):
            w *= rules[d][1][idx[d]]
        x = []
        scale = 1.0
        for d in range(n):
            x.append(scale * xi[d])
            scale *= (1.0 - xi[d])
        pts.append(x)
        wts.append(w)
    pts = np.array(pts, dtype=np.float64)
    wts = np.array(wts, dtype=np.float64)
    bary = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    return pts, wts, bary
