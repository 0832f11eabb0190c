"""Energy and error functionals (TEST INFRASTRUCTURE; see oracle/__init__.py).

Section 6.5: E(w, tau) = 1/2 int (c^-2 w^2 + |tau|^2) on a time slice.  On a
tent front t = tau(x) (not flat) the conserved flux through the front is
1/2 (c^-2 v^2 + |sigma|^2) - v sigma.grad tau per unit dx (from
d/dt e + div(v sigma) = 0), which reduces to E when the front is flat.
Section 6: e(v, sigma) = (c^-2 ||v - v_h||^2 + ||sigma - sigma_h||^2)^(1/2) at T.
"""
from __future__ import annotations

import numpy as np


def element_gradients(coords, elems, tau):
    """Gradient of the piecewise-linear front time over each element, (E, n)."""
    X = coords[elems]
    J = X[:, 1:, :] - X[:, :1, :]
    tv = tau[elems]
    return np.linalg.solve(J, (tv[:, 1:] - tv[:, :1])[..., None])[..., 0]


def front_energy(front, wq, c, grad=None):
    """1/2 sum_K sum_q w_q (c_K^-2 v^2 + |sigma|^2 - 2 v sigma.g_K).

    front (E, Q, n+2), wq (E, Q), c (E,), grad (E, n) or None for a flat front."""
    v = front[:, :, 1]
    s = front[:, :, 2:]
    dens = v * v / (c[:, None] ** 2) + np.sum(s * s, axis=2)
    if grad is not None:
        dens = dens - 2.0 * v * np.einsum("eqd,ed->eq", s, grad)
    return 0.5 * float(np.sum(wq * dens))


def error_e(front, exact, wq, c):
    """Section 6: e = (c^-2 ||v - v_h||^2 + ||sigma - sigma_h||^2)^(1/2)."""
    d = front - exact
    dens = d[:, :, 1] ** 2 / (c[:, None] ** 2) + np.sum(d[:, :, 2:] ** 2, axis=2)
    return float(np.sqrt(np.sum(wq * dens)))


def error_U(front, exact, wq):
    """||U - U_h||_{L2} at T (Section 6.6 reports the L2 error of U)."""
    d = front[:, :, 0] - exact[:, :, 0]
    return float(np.sqrt(np.sum(wq * d * d)))
