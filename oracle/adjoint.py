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


def _tent_maps(coords, elems, c, p, lay, B, star, vfac, tau, v, t_top, alpha, beta=0.5, bnd_type=None):
    """A (N x N), Bmat (N x P*Q*C), Emat (P*Q*C x N) of one tent, N = ng nb:
    one polynomial of U^p per material of the patch (Section 4.2, the same
    grouping by bitwise-equal c as oracle.tdg.sweep), eq. (4.1) with the
    Section 5 recovery terms, Dirichlet and Neumann facets (zero data) and
    the time-like interface terms of eq. (2.5)."""
    n = coords.shape[1]
    Q = lay.wq.shape[1]
    C = n + 2
    nb = B.nb
    t_bot = float(tau[v])
    patch = star[v]
    speeds = []
    for k in patch:
        if float(c[k]) not in speeds:
            speeds.append(float(c[k]))
    grp = {k: speeds.index(float(c[k])) for k in patch}
    ng = len(speeds)
    pv = sorted({a for k in patch for a in elems[k].tolist()} - {v})
    tv = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
    tv += [np.append(coords[w], tau[w]) for w in pv]
    h = _tdg.anisotropic_diameter(np.array(tv), max(speeds))
    xc, tc = coords[v], 0.5 * (t_bot + t_top)
    A = np.zeros((ng * nb, ng * nb))
    Bm = np.zeros((ng * nb, len(patch), Q, C))
    Em = np.zeros((len(patch), Q, C, ng * nb))
    for j, k in enumerate(patch):
        g = grp[k]
        ck = speeds[g]
        c2 = 1.0 / (ck * ck)
        blk = slice(g * nb, (g + 1) * nb)
        ids = elems[k]
        tb = tau[ids]
        tt = np.where(ids == v, t_top, tb)
        J = coords[ids][1:] - coords[ids][0]
        g_b = np.linalg.solve(J, tb[1:] - tb[0])
        g_t = np.linalg.solve(J, tt[1:] - tt[0])
        x, w = lay.xq[k], lay.wq[k]
        Ut, Vt, St = B.eval_phys(x, lay.bary @ tt, xc, tc, h, ck)
        Ub, Vb, Sb = B.eval_phys(x, lay.bary @ tb, xc, tc, h, ck)
        Sgt = np.einsum("qdj,d->qj", St, g_t)
        Ak = (w[:, None] * c2 * Vt).T @ Vt + np.einsum("q,qdi,qdj->ij", w, St, St)
        Ak -= (w[:, None] * Sgt).T @ Vt + (w[:, None] * Vt).T @ Sgt
        Ak += (w[:, None] * Ub).T @ Ub
        A[blk, blk] += Ak
        # b = Bm f_bot: the bottom form of eq. (4.1) and the recovery term
        Sgb = np.einsum("qdj,d->qj", Sb, g_b)
        Bm[blk, j, :, 0] = (w[:, None] * Ub).T
        Bm[blk, j, :, 1] = (w[:, None] * (c2 * Vb - Sgb)).T
        for m in range(n):
            Bm[blk, j, :, 2 + m] = (w[:, None] * (Sb[:, m, :] - g_b[m] * Vb)).T
        # f_top = Em x: (U, v, sigma) at the top points
        Em[j, :, 0, blk] = Ut
        Em[j, :, 1, blk] = Vt
        Em[j, :, 2:, blk] = St
    _, wref_face, bary_face = _quad.simplex_rule(n, p + 1)

    def face(fac):
        others = [a for a in fac if a != v]
        Pf = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
        Pf += [np.append(coords[a], tau[a]) for a in others]
        Pf = np.array(Pf)
        Ed = (Pf[1:] - Pf[0]).T
        return bary_face @ Pf, wref_face * np.sqrt(abs(np.linalg.det(Ed.T @ Ed)))

    for (fac, nrm, kf) in vfac[v]:
        g = grp[kf]
        blk = slice(g * nb, (g + 1) * nb)
        xt, wf = face(fac)
        _, Vd, Sd = B.eval_phys(xt[:, :n], xt[:, n], xc, tc, h, speeds[g])
        Sn = np.einsum("qdj,d->qj", Sd, nrm)
        if _tdg.facet_is_neumann(fac, kf, elems, bnd_type):
            A[blk, blk] += np.einsum("q,qi,qj->ij", wf, Sn, Vd + beta * Sn)
        else:
            A[blk, blk] += np.einsum("q,qi,qj->ij", wf, Vd, Sn + alpha * Vd)
    for (fac, kp, km, nrm) in _tdg.interface_facets(coords, elems, patch, v, grp):
        xt, wf = face(fac)
        side = {}
        for sgn, kk in ((1.0, kp), (-1.0, km)):
            g = grp[kk]
            _, Vf, Sf = B.eval_phys(xt[:, :n], xt[:, n], xc, tc, h, speeds[g])
            side[sgn] = (g, Vf, np.einsum("qdj,d->qj", Sf, nrm))
        for st in (1.0, -1.0):
            gt, Vt_, Snt = side[st]
            for ss in (1.0, -1.0):
                gs, Vs_, Sns = side[ss]
                blk = (slice(gt * nb, (gt + 1) * nb), slice(gs * nb, (gs + 1) * nb))
                A[blk] += 0.5 * st * (np.einsum("q,qi,qj->ij", wf, Snt, Vs_)
                                      + np.einsum("q,qi,qj->ij", wf, Vt_, Sns))
                A[blk] += st * ss * (alpha * np.einsum("q,qi,qj->ij", wf, Vt_, Vs_)
                                     + beta * np.einsum("q,qi,qj->ij", wf, Snt, Sns))
    N = ng * nb
    return A, Bm.reshape(N, len(patch) * Q * C), Em.reshape(len(patch) * Q * C, N), patch


def _boundary_lists(coords, elems, nv):
    vfac = [[] for _ in range(nv)]
    for (f, nrm, k) in _tdg.boundary_facets(coords, elems):
        for a in f:
            vfac[a].append((f, nrm, k))
    return vfac


def adjoint_sweep(coords, elems, c, p, tents, lam_T, alpha=0.5, beta=0.5, bnd_type=None):
    """lambda_0 = F^* lambda_T for the sweep with zero boundary data
    (interface tents and Neumann facets included).

    lam_T: (E, Q, n+2) array (the same layout as the front).  Returns lambda_0."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    n = coords.shape[1]
    nv = coords.shape[0]
    lay = _tdg.front_layout(coords, elems, p)
    B = _basis.TrefftzBasis(n, p)
    star = _tdg.vertex_star(elems, nv)
    vfac = _boundary_lists(coords, elems, nv)
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
                                      float(tents["t_top"][it]), alpha, beta, bnd_type)
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


def _global_system(coords, elems, c, p, tents, alpha=0.5, beta=0.5, bnd_type=None):
    """The whole space-time system of the sweep at once (zero boundary data).
    Unknowns: the coefficients x_t of every tent (ng_t dim U^p of them, one
    polynomial per material of the tent), stacked in the pitched order.
    Block row t: A_t x_t = B_t f_t, where f_t holds, for each element K of
    the tent's patch, the front on K just before tent t: the top values
    E_t' x_t' of the last earlier tent t' over K, or the initial data on K.
    Moving the E_t' x_t' terms to the left gives M x = R f_0 with M block
    lower triangular; the final front is S x + P f_0 (P keeps the initial
    data on elements no tent touches).
    Returns (M, R, S, P, offsets) as dense arrays and the tents' unknown offsets."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    n = coords.shape[1]
    nv, ne = coords.shape[0], elems.shape[0]
    lay = _tdg.front_layout(coords, elems, p)
    Bas = _basis.TrefftzBasis(n, p)
    star = _tdg.vertex_star(elems, nv)
    vfac = _boundary_lists(coords, elems, nv)
    Q = lay.wq.shape[1]
    C = n + 2
    blk = Q * C                                     # front values of one element
    nt = len(tents["vert"])
    maps = []
    tau = np.zeros(nv)
    for it in range(nt):
        v = int(tents["vert"][it])
        maps.append(_tent_maps(coords, elems, c, p, lay, Bas, star, vfac, tau.copy(), v,
                               float(tents["t_top"][it]), alpha, beta, bnd_type))
        tau[v] = float(tents["t_top"][it])
    off = np.zeros(nt + 1, dtype=np.int64)
    for it, (A, _, _, _) in enumerate(maps):
        off[it + 1] = off[it] + A.shape[0]
    NX = int(off[-1])
    M = np.zeros((NX, NX))
    R = np.zeros((NX, ne * blk))
    last = [None] * ne                              # (tent, E rows of K) of the last tent over K
    for it, (A, Bm, Em, patch) in enumerate(maps):
        rows = slice(off[it], off[it + 1])
        M[rows, rows] += A
        for j, K in enumerate(np.asarray(patch).tolist()):
            cols = slice(j * blk, (j + 1) * blk)
            if last[K] is None:
                R[rows, K * blk:(K + 1) * blk] += Bm[:, cols]
            else:
                tp, Ep = last[K]
                M[rows, off[tp]:off[tp + 1]] -= Bm[:, cols] @ Ep
        for j, K in enumerate(np.asarray(patch).tolist()):
            last[K] = (it, Em[j * blk:(j + 1) * blk, :])
    S = np.zeros((ne * blk, NX))
    P = np.zeros((ne * blk, ne * blk))
    for K in range(ne):
        if last[K] is None:
            P[K * blk:(K + 1) * blk, K * blk:(K + 1) * blk] = np.eye(blk)
        else:
            tp, Ep = last[K]
            S[K * blk:(K + 1) * blk, off[tp]:off[tp + 1]] = Ep
    return M, R, S, P, off


def global_solve(coords, elems, c, p, tents, front0, alpha=0.5, beta=0.5, bnd_type=None):
    """Final front of the sweep from one dense LU of the whole space-time
    system (see _global_system).  front0: (E, Q, n+2).  Returns (E, Q, n+2)."""
    M, R, S, P, _ = _global_system(coords, elems, c, p, tents, alpha, beta, bnd_type)
    f0 = np.asarray(front0, dtype=np.float64).reshape(-1)
    x = np.linalg.solve(M, R @ f0)
    return (S @ x + P @ f0).reshape(np.shape(front0))


def global_adjoint(coords, elems, c, p, tents, lam_T, alpha=0.5, beta=0.5, bnd_type=None):
    """F^* lambda_T from the transposed whole system:
    R^T M^-T S^T lambda + P^T lambda.  lam_T: (E, Q, n+2)."""
    M, R, S, P, _ = _global_system(coords, elems, c, p, tents, alpha, beta, bnd_type)
    lt = np.asarray(lam_T, dtype=np.float64).reshape(-1)
    y = np.linalg.solve(M.T, S.T @ lt)
    return (R.T @ y + P.T @ lt).reshape(np.shape(lam_T))


def speed_gradient_transposed(coords, elems, c, p, tents, front0, lam_T, rel_step=1e-4, alpha=0.5,
                              beta=0.5, bnd_type=None):
    """dJ/dc_m of J = <lam_T, front_T> for every material m (the distinct
    values of c; all elements of a material move together), the tents held
    fixed and zero boundary data, through the transposed whole system (see
    _global_system): with M x = R f_0 and front_T = S x + P f_0,

        dJ/dc_m = lam^T S'_m x + y^T (R'_m f_0 - M'_m x),    y = M^-T S^T lam,

    M'_m, R'_m, S'_m the derivatives of the assembled system with respect to
    c_m, by the five-point central difference
    (-f(c + 2s) + 8 f(c + s) - 8 f(c - s) + f(c - 2s)) / (12 s), s = rel_step * c_m
    (truncation O(s^4) ~ 1e-16 and rounding O(u / s) ~ 1e-12 relative, against
    1e-8 for a two-point difference at s = 1e-6 c_m on ill-conditioned 3D
    assemblies); the mesh of tents, and so the block structure, does not
    move.  A second route to the speed gradient besides differencing whole
    sweeps (speed_gradient).  Returns (speeds (M,), dJ/dc (M,))."""
    c = np.asarray(c, dtype=np.float64)
    f0 = np.asarray(front0, dtype=np.float64).reshape(-1)
    lt = np.asarray(lam_T, dtype=np.float64).reshape(-1)
    M, R, S, _, _ = _global_system(coords, elems, c, p, tents, alpha, beta, bnd_type)
    x = np.linalg.solve(M, R @ f0)
    y = np.linalg.solve(M.T, S.T @ lt)
    speeds = np.unique(c)
    grad = np.zeros(len(speeds))
    for m, cm in enumerate(speeds):
        sys_ = {}
        for j in (2, 1, -1, -2):
            cp = c.copy()
            cp[c == cm] = cm * (1.0 + j * rel_step)
            sys_[j] = _global_system(coords, elems, cp, p, tents, alpha, beta, bnd_type)
        d = 12.0 * rel_step * cm
        dM, dR, dS = ((-sys_[2][i] + 8.0 * sys_[1][i] - 8.0 * sys_[-1][i] + sys_[-2][i]) / d for i in range(3))
        grad[m] = float(lt @ (dS @ x) + y @ (dR @ f0 - dM @ x))
    return speeds, grad
