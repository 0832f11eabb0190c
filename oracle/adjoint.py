"""Adjoint of the tent sweep (TEST INFRASTRUCTURE; see oracle/__init__.py).

With the space-time mesh fixed and g_D = 0, every tent maps the stored front
values at its bottom points linearly to the values at its top points
(Section 4.1, eq. (4.1) with the Section 5 recovery terms):

    b = B f_bot,    A x = b,    f_top = E x,

B the bottom-face bilinear form of eq. (4.1) as a map from the stored
(U, v, sigma) values to the right-hand side, E the evaluation of
(U_h, dU_h/dt, -grad U_h) at the top points.  The sweep is the composition
of these maps in the pitched order, so its adjoint runs the tents in reverse
order with

    mu = A^-T (E^T lambda_top),    lambda_bot = B^T mu

(the top and bottom points of a tent are the same stored front points, so
lambda_bot overwrites lambda_top there).  The paper has no adjoint; this
module writes the transpose of the oracle's own tent maps explicitly, and
tests pin it with the dot-product identity <lambda, F f> = <F^* lambda, f>
against oracle.tdg and with finite differences.
"""
from __future__ import annotations

import numpy as np

from . import basis as _basis
from . import tdg as _tdg
from . import quadrature as _quad


def _tent_maps(coords, elems, c, p, lay, B, star, vfac, tau, v, t_top, alpha):
    """A (nb x nb), Bmat (nb x P*Q*C), Emat (P*Q*C x nb) of one tent."""
    n = coords.shape[1]
    Q = lay.wq.shape[1]
    t_bot = float(tau[v])
    patch = star[v]
    if np.any(c[patch] != c[patch][0]):
        raise NotImplementedError("adjoint of interface tents")
    ct = float(c[patch][0])
    c2 = 1.0 / (ct * ct)
    pv = sorted({a for k in patch for a in elems[k].tolist()} - {v})
    tv = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
    tv += [np.append(coords[w], tau[w]) for w in pv]
    h = _tdg.anisotropic_diameter(np.array(tv), ct)
    xc, tc = coords[v], 0.5 * (t_bot + t_top)
    ids = elems[patch]
    tb = tau[ids]
    tt = np.where(ids == v, t_top, tb)
    Xk = coords[ids]
    J = Xk[:, 1:, :] - Xk[:, :1, :]
    g_b = np.linalg.solve(J, (tb[:, 1:] - tb[:, :1])[..., None])[..., 0]
    g_t = np.linalg.solve(J, (tt[:, 1:] - tt[:, :1])[..., None])[..., 0]
    x = lay.xq[patch].reshape(-1, n)
    w = lay.wq[patch].reshape(-1)
    gb = np.repeat(g_b, Q, axis=0)
    gt = np.repeat(g_t, Q, axis=0)
    Ut, Vt, St = B.eval_phys(x, (tt @ lay.bary.T).reshape(-1), xc, tc, h, ct)
    Ub, Vb, Sb = B.eval_phys(x, (tb @ lay.bary.T).reshape(-1), xc, tc, h, ct)
    Sgt = np.einsum("qdj,qd->qj", St, gt)
    A = (w[:, None] * c2 * Vt).T @ Vt + np.einsum("q,qdi,qdj->ij", w, St, St)
    A -= (w[:, None] * Sgt).T @ Vt + (w[:, None] * Vt).T @ Sgt
    A += (w[:, None] * Ub).T @ Ub
    _, wref_face, bary_face = _quad.simplex_rule(n, p + 1)
    for (fac, nrm, _k) in vfac[v]:
        others = [a for a in fac if a != v]
        Pf = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
        Pf += [np.append(coords[a], tau[a]) for a in others]
        Pf = np.array(Pf)
        Ed = (Pf[1:] - Pf[0]).T
        xt = bary_face @ Pf
        wf = wref_face * np.sqrt(abs(np.linalg.det(Ed.T @ Ed)))
        _, Vd, Sd = B.eval_phys(xt[:, :n], xt[:, n], xc, tc, h, ct)
        Sn = np.einsum("qdj,d->qj", Sd, nrm)
        A += np.einsum("q,qi,qj->ij", wf, Vd, Sn + alpha * Vd)
    # B: d b_i / d(U_b, v_b, sigma_b) at every bottom point (eq. 4.1 bottom face + recovery)
    C = n + 2
    NP = x.shape[0]
    Bm = np.zeros((B.nb, NP, C))
    Sgb = np.einsum("qdj,qd->qj", Sb, gb)
    Bm[:, :, 0] = (w[:, None] * Ub).T
    Bm[:, :, 1] = (w[:, None] * (c2 * Vb - Sgb)).T
    for m in range(n):
        Bm[:, :, 2 + m] = (w[:, None] * (Sb[:, m, :] - gb[:, m:m + 1] * Vb)).T
    # E: (U, v, sigma) at the top points
    Em = np.zeros((NP, C, B.nb))
    Em[:, 0, :] = Ut
    Em[:, 1, :] = Vt
    Em[:, 2:, :] = St
    return A, Bm.reshape(B.nb, NP * C), Em.reshape(NP * C, B.nb), patch


def adjoint_sweep(coords, elems, c, p, tents, lam_T, alpha=0.5):
    """lambda_0 = F^* lambda_T for the sweep with g_D = 0.

    lam_T: (E, Q, n+2) array (the same layout as the front).  Returns lambda_0."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    n = coords.shape[1]
    nv = coords.shape[0]
    lay = _tdg.front_layout(coords, elems, p)
    B = _basis.TrefftzBasis(n, p)
    star = _tdg.vertex_star(elems, nv)
    vfac = [[] for _ in range(nv)]
    for (f, nrm, k) in _tdg.boundary_facets(coords, elems):
        for a in f:
            vfac[a].append((f, nrm, k))
    # front times before every tent (the geometry does not depend on the data)
    tau = np.zeros(nv)
    before = []
    for it in range(len(tents["vert"])):
        before.append(tau.copy())
        tau[int(tents["vert"][it])] = float(tents["t_top"][it])
    lam = np.array(lam_T, dtype=np.float64).copy()
    E, Q, C = lam.shape
    for it in reversed(range(len(tents["vert"]))):
        v = int(tents["vert"][it])
        A, Bm, Em, patch = _tent_maps(coords, elems, c, p, lay, B, star, vfac, before[it], v,
                                      float(tents["t_top"][it]), alpha)
        lt = lam[patch].reshape(-1)
        mu = np.linalg.solve(A.T, Em.T @ lt)
        lam[patch] = (Bm.T @ mu).reshape(len(patch), Q, C)
    return lam


def misfit_gradient(front_T, obs_T, wq):
    """J = 1/2 sum_q w_q (U_h - U_obs)^2 at T (L2 misfit of U); returns (J, dJ/dfront_T)."""
    d = front_T[:, :, 0] - obs_T[:, :, 0]
    J = 0.5 * float(np.sum(wq * d * d))
    g = np.zeros_like(front_T)
    g[:, :, 0] = wq * d
    return J, g


def speed_gradient(coords, elems, c, p, tents, init, lam_T, rel_step=1e-6, **sweep_kw):
    """Gradient of J(c) = <lam_T, front_T(c)> with respect to the wave speed
    of each material (the distinct values of c, every element of a material
    moving together), the pitched tents held fixed: central differences of
    the oracle's own sweep, dJ/dc_m ~ (J(c_m (1 + s)) - J(c_m (1 - s))) /
    (2 s c_m) with s = rel_step.  The paper has no gradient; this is the
    definition of the derivative written out (truncation O(s^2), rounding
    O(u / s)).  sweep_kw goes to oracle.tdg.sweep (boundary data and kinds).
    Returns (speeds (M,), dJ/dc (M,))."""
    c = np.asarray(c, dtype=np.float64)
    speeds = np.unique(c)
    grad = np.zeros(len(speeds))
    lam = np.asarray(lam_T, dtype=np.float64)
    for m, cm in enumerate(speeds):
        J = []
        for sgn in (1.0, -1.0):
            cp = c.copy()
            cp[c == cm] = cm * (1.0 + sgn * rel_step)
            F, _ = _tdg.sweep(coords, elems, cp, p, tents, init, **sweep_kw)
            J.append(float(np.sum(lam.reshape(F.shape) * F)))
        grad[m] = (J[0] - J[1]) / (2.0 * rel_step * cm)
    return speeds, grad


def _global_system(coords, elems, c, p, tents, alpha=0.5):
    """The whole space-time system of the sweep at once (g_D = 0, single-material
    tents).  Unknowns: the coefficients x_t of every tent, stacked in the
    pitched order.  Block row t: A_t x_t = B_t f_t, where f_t holds, for each
    element K of the tent's patch, the front on K just before tent t: the
    top values E_t' x_t' of the last earlier tent t' over K, or the initial
    data on K.  Moving the E_t' x_t' terms to the left gives M x = R f_0 with
    M block lower triangular; the final front is S x + P f_0 (P keeps the
    initial data on elements no tent touches).
    Returns (M, R, S, P, nb) as dense arrays."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    n = coords.shape[1]
    nv, ne = coords.shape[0], elems.shape[0]
    lay = _tdg.front_layout(coords, elems, p)
    Bas = _basis.TrefftzBasis(n, p)
    star = _tdg.vertex_star(elems, nv)
    vfac = [[] for _ in range(nv)]
    for (f, nrm, k) in _tdg.boundary_facets(coords, elems):
        for a in f:
            vfac[a].append((f, nrm, k))
    Q = lay.wq.shape[1]
    C = n + 2
    blk = Q * C                                     # front values of one element
    nb = Bas.nb
    nt = len(tents["vert"])
    M = np.zeros((nt * nb, nt * nb))
    R = np.zeros((nt * nb, ne * blk))
    tau = np.zeros(nv)
    last = [None] * ne                              # (tent, E rows of K) of the last tent over K
    for it in range(nt):
        v = int(tents["vert"][it])
        A, Bm, Em, patch = _tent_maps(coords, elems, c, p, lay, Bas, star, vfac, tau.copy(), v,
                                      float(tents["t_top"][it]), alpha)
        rows = slice(it * nb, (it + 1) * nb)
        M[rows, rows] += A
        for j, K in enumerate(np.asarray(patch).tolist()):
            cols = slice(j * blk, (j + 1) * blk)
            if last[K] is None:
                R[rows, K * blk:(K + 1) * blk] += Bm[:, cols]
            else:
                tp, Ep = last[K]
                M[rows, tp * nb:(tp + 1) * nb] -= Bm[:, cols] @ Ep
        for j, K in enumerate(np.asarray(patch).tolist()):
            last[K] = (it, Em[j * blk:(j + 1) * blk, :])
        tau[v] = float(tents["t_top"][it])
    S = np.zeros((ne * blk, nt * nb))
    P = np.zeros((ne * blk, ne * blk))
    for K in range(ne):
        if last[K] is None:
            P[K * blk:(K + 1) * blk, K * blk:(K + 1) * blk] = np.eye(blk)
        else:
            tp, Ep = last[K]
            S[K * blk:(K + 1) * blk, tp * nb:(tp + 1) * nb] = Ep
    return M, R, S, P, nb


def global_solve(coords, elems, c, p, tents, front0, alpha=0.5):
    """Final front of the sweep from one dense LU of the whole space-time
    system (see _global_system).  front0: (E, Q, n+2).  Returns (E, Q, n+2)."""
    M, R, S, P, _ = _global_system(coords, elems, c, p, tents, alpha)
    f0 = np.asarray(front0, dtype=np.float64).reshape(-1)
    x = np.linalg.solve(M, R @ f0)
    return (S @ x + P @ f0).reshape(np.shape(front0))


def global_adjoint(coords, elems, c, p, tents, lam_T, alpha=0.5):
    """F^* lambda_T from the transposed whole system:
    R^T M^-T S^T lambda + P^T lambda.  lam_T: (E, Q, n+2)."""
    M, R, S, P, _ = _global_system(coords, elems, c, p, tents, alpha)
    lt = np.asarray(lam_T, dtype=np.float64).reshape(-1)
    y = np.linalg.solve(M.T, S.T @ lt)
    return (R.T @ y + P.T @ lt).reshape(np.shape(lam_T))


def speed_gradient_transposed(coords, elems, c, p, tents, front0, lam_T, rel_step=1e-6, alpha=0.5):
    """dJ/dc of J = <lam_T, front_T> on a single-material mesh (every element
    at the speed c_0), the tents held fixed and g_D = 0, through the
    transposed whole system (see _global_system): with M x = R f_0 and
    front_T = S x + P f_0,

        dJ/dc = lam^T S' x + y^T (R' f_0 - M' x),    y = M^-T S^T lam,

    M', R', S' the derivatives of the assembled system with respect to c
    (central differences of the assembly with step rel_step * c_0).  A second
    route to the speed gradient besides differencing whole sweeps
    (speed_gradient).  Returns dJ/dc_0."""
    c = np.asarray(c, dtype=np.float64)
    c0 = float(c[0])
    if np.any(c != c0):
        raise NotImplementedError("speed_gradient_transposed needs a single material")
    f0 = np.asarray(front0, dtype=np.float64).reshape(-1)
    lt = np.asarray(lam_T, dtype=np.float64).reshape(-1)
    M, R, S, _, _ = _global_system(coords, elems, c, p, tents, alpha)
    x = np.linalg.solve(M, R @ f0)
    y = np.linalg.solve(M.T, S.T @ lt)
    Mp, Rp, Sp, _, _ = _global_system(coords, elems, c * (1.0 + rel_step), p, tents, alpha)
    Mm, Rm, Sm, _, _ = _global_system(coords, elems, c * (1.0 - rel_step), p, tents, alpha)
    d = 2.0 * rel_step * c0
    dM, dR, dS = (Mp - Mm) / d, (Rp - Rm) / d, (Sp - Sm) / d
    return float(lt @ (dS @ x) + y @ (dR @ f0 - dM @ x))
