"""Tent-by-tent Trefftz-DG sweep (TEST INFRASTRUCTURE; see oracle/__init__.py).

For each tent (vertex v, bottom time t_bot = tau_v, top time t_top) in the
pitched order, with U_h = sum_j x_j b_j in U^p (one polynomial per tent,
constant wave speed c on the patch), the local system eq. (4.1) is assembled
with the second-order recovery terms of Section 5 and solved:

  LHS  A_ij =  int_top [ c^-2 v_j w_i + s_j.t_i - v_j (t_i.g) - (s_j.g) w_i ] dx
             + int_bot  U_j V_i dx                                   (Section 5)
             + int_D   (s_j.n + alpha v_j) w_i dS                    (eq. 4.1)
             + int_N   v_j (t_i.n) + beta (s_j.n)(t_i.n) dS          (eq. 4.1)
  RHS  b_i  =  int_bot [ c^-2 v_b w_i + s_b.t_i - v_b (t_i.g_b) - (s_b.g_b) w_i ] dx
             + int_bot  U_b V_i dx                                   (Section 5)
             + int_D   g_D (alpha w_i - t_i.n) dS                    (eq. 4.1)
             + int_N   g_N (beta t_i.n - w_i) dS                     (eq. 4.1)

with trial fields (v_j, s_j) = (dU_j/dt, -grad U_j), test fields
(w_i, t_i) = (dV_i/dt, -grad V_i), g the gradient of the top (resp. bottom)
front time over each element, (U_b, v_b, s_b) the stored front values.  The
face integrals become spatial integrals through n_t dS = dx, n_x dS = -g dx on
the top and n_t dS = -dx, n_x dS = g dx on the bottom (graph faces
t = tau(x)).  Section 4.1: one spatial rule is mapped onto the faces; after
the solve (U, v, sigma) at the top points overwrite the stored front values.

Readings of the paper taken here (each listed in the design notes):
  * the recovery terms sit on the bottom face with measure dx (the jump form
    -[[U]]_t V^+ of Section 5 gives both the LHS and the RHS term there);
  * the Dirichlet terms follow eq. (4.1) / A and l of eq. (2.5), i.e. the
    dissipative sign sigma + alpha (v - g_D) n, not the sign printed in the
    flux table;
  * basis centre x_c = x_v, t_c = (t_bot + t_top)/2, scale h = anisotropic
    diameter eq. (3.3) over the tent vertices with the tent's largest speed
    (affects only rounding);
  * piecewise-constant c (Section 4.2): one polynomial per material of the
    tent (its own c in the Remark 3.1 map), coupled on the time-like facets
    through v by the F^time terms of eq. (2.5); the facet's + side is the
    element with the lower index in the vertex star, n its outward normal.

Parity unpinned: none of the above beyond what tests/test_oracle_*.py pin
(polynomial reproduction, energy identity, convergence rates).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import basis as _basis
from . import quadrature as _quad


# ----------------------------------------------------------------------------
# mesh topology
# ----------------------------------------------------------------------------
def vertex_star(elems: np.ndarray, nv: int):
    """Elements containing each vertex, ascending."""
    star = [[] for _ in range(nv)]
    for k, el in enumerate(elems.tolist()):
        for a in el:
            star[a].append(k)
    return star


def boundary_facets(coords: np.ndarray, elems: np.ndarray):
    """Facets that belong to one element only: list of (sorted vertex tuple,
    outward unit normal (n,), element)."""
    n = coords.shape[1]
    owner: dict = {}
    for k, el in enumerate(elems.tolist()):
        for o in range(n + 1):
            f = tuple(sorted(el[:o] + el[o + 1:]))
            owner.setdefault(f, []).append((k, el[o]))
    out = []
    for f, lst in sorted(owner.items()):
        if len(lst) != 1:
            continue
        k, opp = lst[0]
        P = coords[list(f)]
        if n == 1:
            nrm = np.array([1.0])
        elif n == 2:
            t = P[1] - P[0]
            nrm = np.array([t[1], -t[0]])
        else:
            nrm = np.cross(P[1] - P[0], P[2] - P[0])
        nrm = nrm / np.linalg.norm(nrm)
        if np.dot(coords[opp] - P[0], nrm) > 0:
            nrm = -nrm
        out.append((f, nrm, k))
    return out


@dataclass
class FrontLayout:
    """Front points: xq (E, Q, n), wq (E, Q) physical weights, bary (Q, n+1)."""
    xq: np.ndarray
    wq: np.ndarray
    bary: np.ndarray
    wref: np.ndarray


def front_layout(coords: np.ndarray, elems: np.ndarray, p: int) -> FrontLayout:
    n = coords.shape[1]
    _, wref, bary = _quad.simplex_rule(n, p + 1)
    X = coords[elems]                                   # (E, n+1, n)
    xq = np.einsum("qi,eid->eqd", bary, X)
    J = X[:, 1:, :] - X[:, :1, :]                       # rows = edges from vertex 0
    detJ = np.abs(np.linalg.det(J))
    wq = wref[None, :] * detJ[:, None]                  # wref sums to 1/n!
    return FrontLayout(xq, wq, bary, wref)


def anisotropic_diameter(pts_xt: np.ndarray, c: float) -> float:
    """eq. (3.3): sup over pairs of (|x-y|^2 + c^2 |t-s|^2)^(1/2) (attained at
    vertices of the tent)."""
    best = 0.0
    m = pts_xt.shape[0]
    for i in range(m):
        for j in range(i + 1, m):
            d = pts_xt[i] - pts_xt[j]
            val = math.sqrt(float(np.dot(d[:-1], d[:-1])) + c * c * d[-1] * d[-1])
            best = max(best, val)
    return best


# ----------------------------------------------------------------------------
# the sweep
# ----------------------------------------------------------------------------
def facet_is_neumann(facet, k, elems, bnd_type) -> bool:
    """Boundary facet `facet` of element k is Neumann when bnd_type[k, o] == 1,
    o the local index of the element's vertex opposite the facet (None: all
    boundary facets are Dirichlet)."""
    if bnd_type is None:
        return False
    el = list(elems[k])
    o = [i for i, a in enumerate(el) if a not in facet][0]
    return int(bnd_type[k][o]) == 1


def solve_refined(A, b, steps=3):
    """A x = b by LU with partial pivoting, then `steps` corrections
    x += A^-1 (b - A x) whose residual is formed in the platform's extended
    precision (numpy longdouble: 64-bit significand on x86, 113-bit on
    aarch64).  For the ill-conditioned tent systems of high degree
    (kappa(A) ~ 1e8 at p = 5) this removes the ~kappa(A) u error that a plain
    binary64 LU leaves in the oracle's own result."""
    x = np.linalg.solve(A, b)
    Al, bl = A.astype(np.longdouble), b.astype(np.longdouble)
    for _ in range(steps):
        r = (bl - Al @ x.astype(np.longdouble)).astype(np.float64)
        x = x + np.linalg.solve(A, r)
    return x


def sweep(coords, elems, c, p, tents, init, dirichlet=None, alpha=0.5,
          record=None, front0=None, tau0=None, tent_range=None, beta=0.5,
          bnd_type=None, neumann=None, refine=False, basis_init="monomial"):
    """Run the tent sweep.

    coords (Nv, n), elems (E, n+1), c (E,), p: Trefftz degree of U^p,
    tents: dict from oracle.pitching.pitch (sorted), init: callable x -> (N, n+2)
    initial (U, v, sigma) (ignored when front0 is given), dirichlet: callable
    (x (N, n), t (N,)) -> (N,) values g_D of v on the Dirichlet boundary, or
    None for 0.  bnd_type (E, n+1), optional: 1 marks the boundary facet
    opposite local vertex o of element k as Neumann (sigma.n = g_N), else
    Dirichlet; neumann: callable (x, t, n) -> (N,) values g_N, n the facet's
    outward unit normal, or None for 0.
    record: optional callable(tent_index, dict) receiving the local data.
    refine: solve every tent system with solve_refined instead of one LU.
    basis_init: initial polynomials of the basis recursion (Section 6.3).
    Returns (front (E, Q, n+2), tau (Nv,)).
    """
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    n = coords.shape[1]
    nv = coords.shape[0]
    lay = front_layout(coords, elems, p)
    B = _basis.TrefftzBasis(n, p, basis_init)
    star = vertex_star(elems, nv)
    bfac = boundary_facets(coords, elems)
    vfac = [[] for _ in range(nv)]
    for (f, nrm, k) in bfac:
        for a in f:
            vfac[a].append((f, nrm, k))
    E, Q = lay.wq.shape
    if front0 is None:
        front = np.asarray(init(lay.xq.reshape(-1, n)), dtype=np.float64).reshape(E, Q, n + 2).copy()
    else:
        front = np.array(front0, dtype=np.float64).reshape(E, Q, n + 2).copy()
    tau = np.zeros(nv) if tau0 is None else np.array(tau0, dtype=np.float64)
    _, wref_face, bary_face = _quad.simplex_rule(n, p + 1)

    idx = range(len(tents["vert"])) if tent_range is None else range(*tent_range)
    for it in idx:
        v = int(tents["vert"][it])
        t_top = float(tents["t_top"][it])
        t_bot = float(tau[v])
        patch = star[v]
        # Section 4.2: one Trefftz polynomial per material (bitwise-equal c) of the tent
        speeds = []
        for k in patch:
            if float(c[k]) not in speeds:
                speeds.append(float(c[k]))
        grp = {k: speeds.index(float(c[k])) for k in patch}
        ng = len(speeds)
        cmax = max(speeds)
        # Remark 3.1: centre and anisotropic diameter (with the largest speed of the tent)
        pv = sorted({a for k in patch for a in elems[k].tolist()} - {v})
        tv = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
        tv += [np.append(coords[w], tau[w]) for w in pv]
        h = anisotropic_diameter(np.array(tv), cmax)
        xc, tc = coords[v], 0.5 * (t_bot + t_top)

        nb = B.nb
        A = np.zeros((ng * nb, ng * nb))
        b = np.zeros(ng * nb)
        tops = []
        for k in patch:
            g = grp[k]
            ck = speeds[g]
            c2 = 1.0 / (ck * ck)
            blk = slice(g * nb, (g + 1) * nb)
            ids = elems[k]
            tb = tau[ids]                                   # bottom front times at the vertices
            tt = np.where(ids == v, t_top, tb)              # top: tau_v -> t_top
            Xk = coords[ids]
            J = Xk[1:] - Xk[0]
            g_b = np.linalg.solve(J, tb[1:] - tb[0])
            g_t = np.linalg.solve(J, tt[1:] - tt[0])
            x = lay.xq[k]
            w = lay.wq[k]
            Ut, Vt, St = B.eval_phys(x, lay.bary @ tt, xc, tc, h, ck)
            Ub, Vb, Sb = B.eval_phys(x, lay.bary @ tb, xc, tc, h, ck)
            # top face (LHS): c^-2 v_j w_i + s_j.t_i - v_j (t_i.g) - (s_j.g) w_i
            Sgt = np.einsum("qdj,d->qj", St, g_t)
            Ak = (w[:, None] * c2 * Vt).T @ Vt
            Ak += np.einsum("q,qdi,qdj->ij", w, St, St)
            Ak -= (w[:, None] * Sgt).T @ Vt
            Ak -= (w[:, None] * Vt).T @ Sgt
            # recovery on the bottom face (LHS): U_j V_i
            Ak += (w[:, None] * Ub).T @ Ub
            A[blk, blk] += Ak
            # bottom face data (RHS)
            f = front[k]
            Uf, vf, sf = f[:, 0], f[:, 1], f[:, 2:]
            Sgb = np.einsum("qdj,d->qj", Sb, g_b)
            bk = (w * c2 * vf) @ Vb
            bk += np.einsum("q,qd,qdi->i", w, sf, Sb)
            bk -= (w * vf) @ Sgb
            bk -= (w * (sf @ g_b)) @ Vb
            bk += (w * Uf) @ Ub
            b[blk] += bk
            tops.append((k, g, Ut, Vt, St))

        def face_simplex(fac):
            # the n-simplex {x in F, tau_bot(x) <= t <= tau_top(x)} with vertices
            # (x_v, t_bot), (x_v, t_top), (x_w, tau_w) for the other facet vertices w
            others = [a for a in fac if a != v]
            Pf = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
            Pf += [np.append(coords[a], tau[a]) for a in others]
            Pf = np.array(Pf)                                # (n+1, n+1)
            Ed = (Pf[1:] - Pf[0]).T                          # (n+1, n)
            scale = math.sqrt(abs(np.linalg.det(Ed.T @ Ed)))  # n! * n-volume
            xt = bary_face @ Pf
            return xt, wref_face * scale

        # Dirichlet and Neumann vertical faces through v (eq. 4.1)
        for (fac, nrm, kf) in vfac[v]:
            g = grp[kf]
            blk = slice(g * nb, (g + 1) * nb)
            xt, wf = face_simplex(fac)
            Ud, Vd, Sd = B.eval_phys(xt[:, :n], xt[:, n], xc, tc, h, speeds[g])
            Sn = np.einsum("qdj,d->qj", Sd, nrm)
            if facet_is_neumann(fac, kf, elems, bnd_type):
                A[blk, blk] += np.einsum("q,qi,qj->ij", wf, Sn, Vd + beta * Sn)  # v_j (t_i.n) + beta (s_j.n)(t_i.n)
                gn = np.zeros(len(wf)) if neumann is None else np.asarray(neumann(xt[:, :n], xt[:, n], nrm))
                b[blk] += np.einsum("q,qi->i", wf * gn, beta * Sn - Vd)        # g_N (beta t_i.n - w_i)
                continue
            A[blk, blk] += np.einsum("q,qi,qj->ij", wf, Vd, Sn + alpha * Vd)     # (s_j.n + alpha v_j) w_i
            gd = np.zeros(len(wf)) if dirichlet is None else np.asarray(dirichlet(xt[:, :n], xt[:, n]))
            b[blk] += np.einsum("q,qi->i", wf * gd, alpha * Vd - Sn)           # g_D (alpha w_i - t_i.n)

        # time-like interface faces between materials (Section 4.2, A of eq. 2.5):
        # {v}[[t]]_N + {s}.[[w]]_N + alpha [[v]]_N.[[w]]_N + beta [[s]]_N [[t]]_N
        for (fac, kp, km, nrm) in interface_facets(coords, elems, patch, v, grp):
            xt, wf = face_simplex(fac)
            side = {}
            for sgn, kk in ((1.0, kp), (-1.0, km)):
                g = grp[kk]
                _, Vf, Sf = B.eval_phys(xt[:, :n], xt[:, n], xc, tc, h, speeds[g])
                side[sgn] = (g, Vf, np.einsum("qdj,d->qj", Sf, nrm))
            for st in (1.0, -1.0):            # test side
                gt, Vt_, Snt = side[st]
                for ss in (1.0, -1.0):        # trial side
                    gs, Vs_, Sns = side[ss]
                    blk = (slice(gt * nb, (gt + 1) * nb), slice(gs * nb, (gs + 1) * nb))
                    A[blk] += 0.5 * st * (np.einsum("q,qi,qj->ij", wf, Snt, Vs_)
                                          + np.einsum("q,qi,qj->ij", wf, Vt_, Sns))
                    A[blk] += st * ss * (alpha * np.einsum("q,qi,qj->ij", wf, Vt_, Vs_)
                                         + beta * np.einsum("q,qi,qj->ij", wf, Snt, Sns))

        xs = solve_refined(A, b) if refine else np.linalg.solve(A, b)
        if record is not None:
            record(it, dict(v=v, t_bot=t_bot, t_top=t_top, A=A, b=b, x=xs, h=h,
                            xc=xc, tc=tc, c=speeds[0], speeds=speeds, groups=grp, patch=list(patch),
                            front_before={k: front[k].copy() for k in patch},
                            tau_before=tau.copy(), basis=B))
        for (k, g, Ut, Vt, St) in tops:
            xg = xs[g * nb:(g + 1) * nb]
            front[k][:, 0] = Ut @ xg
            front[k][:, 1] = Vt @ xg
            front[k][:, 2:] = np.einsum("qdj,j->qd", St, xg)
        tau[v] = t_top
    return front, tau


def interface_facets(coords, elems, patch, v, grp):
    """Facets through v shared by two patch elements of different materials:
    list of (facet vertices, K+, K-, unit normal pointing out of K+)."""
    n = coords.shape[1]
    out = []
    pl = list(patch)
    for a in range(len(pl)):
        for bb in range(a + 1, len(pl)):
            ka, kb = pl[a], pl[bb]
            if grp[ka] == grp[kb]:
                continue
            common = sorted(set(elems[ka].tolist()) & set(elems[kb].tolist()))
            if len(common) != n or v not in common:
                continue
            opp = [x for x in elems[ka].tolist() if x not in common][0]
            P = coords[common]
            if n == 1:
                nrm = np.array([1.0])
            elif n == 2:
                t = P[1] - P[0]
                nrm = np.array([t[1], -t[0]])
            else:
                nrm = np.cross(P[1] - P[0], P[2] - P[0])
            nrm = nrm / np.linalg.norm(nrm)
            if np.dot(coords[opp] - P[0], nrm) > 0:
                nrm = -nrm
            out.append((tuple(common), ka, kb, nrm))
    return out


def front_points(coords, elems, p):
    """(xq (E*Q, n), wq (E*Q,)) in the front layout order."""
    lay = front_layout(np.asarray(coords, dtype=np.float64), np.asarray(elems), p)
    n = coords.shape[1]
    return lay.xq.reshape(-1, n), lay.wq.reshape(-1)
