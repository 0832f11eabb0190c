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


def tent_dissipation(coords, elems, c, p, rec, alpha=0.5, beta=0.5, bnd_type=None,
                     dirichlet=None, neumann=None):
    """Energy lost in one tent, from point values of its solution (Section 6.5,
    eq. 2.5 and eq. 4.1 tested with V = U_h, the tent's own solution u):

        D = 1/2 int_bot Q_{g_b}(u - u_b) dx + int_bot (U - U_b) U dx
          + int_{F^D} [alpha v^2 - g_D (alpha v - sigma.n)] dS
          + int_{F^N} [beta (sigma.n)^2 - g_N (beta sigma.n - v)] dS
          + int_{F^time} [alpha (v+ - v-)^2 + beta ((sigma+ - sigma-).n)^2] dS,

    Q_g(w) = c^-2 w_v^2 + |w_s|^2 - 2 w_v (w_s . g), u_b the stored front
    below the tent, g_b the gradient of the bottom front on each element.
    Inside a Trefftz tent d/dt e + div(v sigma) = 0, so the tent's energy
    flux satisfies 1/2 int_top Q_{g_t}(u) = 1/2 int_bot Q_{g_b}(u_b) - D;
    summed over the sweep E(T) = E(0) - sum D.  With zero boundary data D is
    a sum of squares plus the recovery term of Section 5.

    rec: the dict oracle.tdg.sweep passes to its `record` callback; the
    vertical faces are the n-simplices {(x_v, t_bot), (x_v, t_top),
    (x_w, tau_w)} over the boundary and interface facets through v, with the
    same collapsed rule as the sweep (exact for these polynomial integrands).
    dirichlet(x, t), neumann(x, t, n): boundary data as for the sweep (None: 0).
    Returns D (float)."""
    import math

    from . import quadrature as _quad
    from . import tdg as _tdg

    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    n = coords.shape[1]
    lay = _tdg.front_layout(coords, elems, p)
    Bas, v, nb = rec["basis"], rec["v"], rec["basis"].nb
    tau = rec["tau_before"]
    t_bot, t_top = rec["t_bot"], rec["t_top"]
    xc, tc, h = rec["xc"], rec["tc"], rec["h"]
    grp, speeds, xs = rec["groups"], rec["speeds"], rec["x"]

    def fields(g, x, t):
        U, V, S = Bas.eval_phys(x, t, xc, tc, h, speeds[g])
        xg = xs[g * nb:(g + 1) * nb]
        return U @ xg, V @ xg, np.einsum("qdj,j->qd", S, xg)

    D = 0.0
    # bottom face: jump to the stored front and the recovery term
    for k in rec["patch"]:
        g = grp[k]
        ck = speeds[g]
        ids = elems[k]
        tb = tau[ids]
        gb = np.linalg.solve(coords[ids][1:] - coords[ids][0], tb[1:] - tb[0])
        U, V, S = fields(g, lay.xq[k], lay.bary @ tb)
        fb = rec["front_before"][k]
        dv = V - fb[:, 1]
        ds = S - fb[:, 2:]
        q = dv * dv / (ck * ck) + np.sum(ds * ds, axis=1) - 2.0 * dv * (ds @ gb)
        D += float(np.sum(lay.wq[k] * (0.5 * q + (U - fb[:, 0]) * U)))

    _, wref, bary = _quad.simplex_rule(n, p + 1)

    def face(fac):
        others = [a for a in fac if a != v]
        P = [np.append(coords[v], t_bot), np.append(coords[v], t_top)]
        P += [np.append(coords[a], tau[a]) for a in others]
        P = np.array(P)
        E = (P[1:] - P[0]).T
        xt = bary @ P
        return xt, wref * math.sqrt(abs(np.linalg.det(E.T @ E)))

    star = _tdg.vertex_star(elems, coords.shape[0])
    for (fac, nrm, kf) in _tdg.boundary_facets(coords, elems):
        if v not in fac:
            continue
        xt, wf = face(fac)
        _, V, S = fields(grp[kf], xt[:, :n], xt[:, n])
        sn = S @ nrm
        if _tdg.facet_is_neumann(fac, kf, elems, bnd_type):
            gn = np.zeros(len(wf)) if neumann is None else np.asarray(neumann(xt[:, :n], xt[:, n], nrm))
            D += float(np.sum(wf * (beta * sn * sn - gn * (beta * sn - V))))
        else:
            gd = np.zeros(len(wf)) if dirichlet is None else np.asarray(dirichlet(xt[:, :n], xt[:, n]))
            D += float(np.sum(wf * (alpha * V * V - gd * (alpha * V - sn))))
    for (fac, kp, km, nrm) in _tdg.interface_facets(coords, elems, star[v], v, grp):
        xt, wf = face(fac)
        _, Vp, Sp = fields(grp[kp], xt[:, :n], xt[:, n])
        _, Vm, Sm = fields(grp[km], xt[:, :n], xt[:, n])
        dsn = (Sp - Sm) @ nrm
        D += float(np.sum(wf * (alpha * (Vp - Vm) ** 2 + beta * dsn * dsn)))
    return D


def sweep_dissipation(coords, elems, c, p, tents, init, alpha=0.5, beta=0.5, bnd_type=None,
                      dirichlet=None, neumann=None, tent_range=None):
    """Run oracle.tdg.sweep and sum tent_dissipation over its tents.
    Returns (front (E, Q, n+2), tau, sum D, list of per-tent D)."""
    from . import tdg as _tdg
    per = []

    def rec(it, d):
        per.append(tent_dissipation(coords, elems, c, p, d, alpha, beta, bnd_type, dirichlet, neumann))

    F, tau = _tdg.sweep(coords, elems, c, p, tents, init, dirichlet, alpha=alpha, record=rec,
                        beta=beta, bnd_type=bnd_type, neumann=neumann, tent_range=tent_range)
    return F, tau, float(np.sum(per)), per


def locate(coords, elems, points):
    """Element of each point (the first whose barycentric coordinates are all
    >= -1e-12) and the point's barycentric coordinates there: (el (N,), bary (N, n+1))."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    n = coords.shape[1]
    X = coords[elems]                                   # (E, n+1, n)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # columns = edges
    pts = np.asarray(points, dtype=np.float64).reshape(-1, n)
    el = np.full(len(pts), -1)
    bary = np.zeros((len(pts), n + 1))
    for j, x in enumerate(pts):
        lam = np.linalg.solve(J, (x[None, :] - X[:, 0, :])[..., None])[..., 0]
        full = np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)
        ok = np.nonzero(np.all(full >= -1e-12, axis=1))[0]
        if len(ok) == 0:
            raise ValueError(f"point {j} lies in no element")
        el[j] = ok[0]
        bary[j] = full[ok[0]]
    return el, bary


def probe_values(coords, elems, c, p, tents, init, points, times, **sweep_kw):
    """U_h at the samples (x_j, t_k) (Section 6.7's point output U_C(t) is an
    integral of |U_h(., t)| over a box): each sample lies in the tent at a
    vertex of x_j's element whose bottom and top fronts enclose it there,
    t_bot(x_j) <= t_k < t_top(x_j) (at the final time: the tent whose top
    reaches it, with t_bot < t_top), and takes that tent's U_h (Remark 3.1
    map).  Returns (values (n_t, n_pts), the tent of every sample (n_t, n_pts))."""
    from . import tdg as _tdg
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    times = np.asarray(times, dtype=np.float64)
    el, bary = locate(coords, elems, points)
    pts = np.asarray(points, dtype=np.float64).reshape(len(el), -1)
    T = float(np.max(tents["t_top"]))
    vals = np.full((len(times), len(el)), np.nan)
    owner = np.full((len(times), len(el)), -1)
    at = {}
    for j, k in enumerate(el):
        at.setdefault(int(k), []).append(j)

    def rec(it, d):
        B, nb, v = d["basis"], d["basis"].nb, d["v"]
        for k in d["patch"]:
            for j in at.get(int(k), []):
                ids = elems[k]
                tb = float(bary[j] @ d["tau_before"][ids])
                tt = float(bary[j] @ np.where(ids == v, d["t_top"], d["tau_before"][ids]))
                for kt, t in enumerate(times):
                    if (tb <= t < tt) or (t == T and tb < tt == T):
                        g = d["groups"][k]
                        U, _, _ = B.eval_phys(pts[j:j + 1], np.array([t]), d["xc"], d["tc"], d["h"], d["speeds"][g])
                        vals[kt, j] = float(U[0] @ d["x"][g * nb:(g + 1) * nb])
                        owner[kt, j] = it

    _tdg.sweep(coords, elems, c, p, tents, init, record=rec, **sweep_kw)
    return vals, owner
