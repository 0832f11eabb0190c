"""Pins for oracle/tdg.py (the tent sweep, eq. (4.1) + Section 5).

* polynomial reproduction: the method is consistent (Section 2.4; Section 5
  notes the recovery terms preserve consistency) and any U in U^p lies in the
  discrete space, so exact initial/Dirichlet data give U_h = U up to rounding
  at every front point, for n = 1, 2, 3 and several p;
* energy identity: testing a tent system with V = U_h and using
  d/dt e + div(v sigma) = 0 inside the tent gives, with g_D = 0,
      1/2 int_top Q_g(u) = 1/2 int_bot Q_gb(u_b) - 1/2 int_bot Q_gb(u - u_b)
                           - int_bot (U - U_b) U dx - alpha int_D v^2 dS,
  Q_g(u) = c^-2 v^2 + |sigma|^2 - 2 v sigma.g; so the sweep is dissipative
  (Section 6.5: the numerical energy decreases);
* h-convergence of e(v, sigma) at the rate p (fields in W^(p-1), Section 6.4
  observes O(h^(q+1)) for W^q) and p-convergence faster than geometric.
"""
import math

import numpy as np
import pytest

from oracle import energy, pitching, tdg
from paper_1907_02367_gb300 import inputs


def _run(mesh, p, T, sol, kappa, dirichlet=True, record=None):
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, kappa, T)
    dfun = (lambda x, t: sol(x, t)[:, 1]) if dirichlet else None
    F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: sol(x, 0.0), dfun,
                       record=record)
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    ex = sol(lay.xq.reshape(-1, mesh.dim), T).reshape(F.shape)
    return F, tau, ex, lay, r


REPRO = [(1, 2, 0), (1, 3, 1), (1, 5, 1), (2, 2, 0), (2, 3, 1), (2, 4, 1), (2, 5, 0),
         (3, 2, 0), (3, 3, 1)]


@pytest.mark.parametrize("dim,p,which", REPRO)
def test_polynomial_reproduction(dim, p, which):
    mesh = {1: inputs.mesh_interval(6), 2: inputs.mesh_square(3, 0.2, seed=5),
            3: inputs.mesh_cube(1, 0.0, seed=3)}[dim]
    sol = inputs.polynomial_solution(dim, which)
    T = 0.3 if dim < 3 else 0.15
    F, tau, ex, _, _ = _run(mesh, p, T, sol, inputs.pitch_kappa(mesh))
    assert np.all(tau == T)
    scale = np.abs(ex).max()
    assert np.abs(F - ex).max() <= 1e-12 * max(1.0, scale) * (10 if dim == 3 else 1)


def test_reproduction_fails_for_degree_above_p():
    """Sanity: a solution outside U^p (degree 3 with p = 2) is not reproduced."""
    mesh = inputs.mesh_interval(6)
    sol = inputs.polynomial_solution(1, 1)
    F, _, ex, _, _ = _run(mesh, 2, 0.3, sol, 0.9)
    assert np.abs(F - ex).max() > 1e-6


def _energy_identity_check(mesh, p, T, sol, alpha=0.5, neumann=False, beta=0.5):
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    n = mesh.dim
    nodes, wts = np.polynomial.legendre.leggauss(12)
    bverts = {0, mesh.n_vert - 1} if n == 1 else set()
    worst = [0.0]
    checked = [0]

    def rec(it, d):
        v, patch, B = d["v"], d["patch"], d["basis"]
        tau = d["tau_before"]
        ids = mesh.elems[patch]
        tb = tau[ids]
        tt = np.where(ids == v, d["t_top"], tb)
        X = mesh.coords[ids]
        J = X[:, 1:, :] - X[:, :1, :]
        gb = np.linalg.solve(J, (tb[:, 1:] - tb[:, :1])[..., None])[..., 0]
        gt = np.linalg.solve(J, (tt[:, 1:] - tt[:, :1])[..., None])[..., 0]
        Q = lay.wq.shape[1]
        x = lay.xq[patch].reshape(-1, n)
        w = lay.wq[patch].reshape(-1)
        cK = np.repeat(mesh.c[patch], Q)

        def fields(t):
            U, V, S = B.eval_phys(x, t, d["xc"], d["tc"], d["h"], d["c"])
            return U @ d["x"], V @ d["x"], np.einsum("qdj,j->qd", S, d["x"])

        def Qg(vv, ss, g):
            return vv * vv / cK ** 2 + np.sum(ss * ss, axis=1) - 2 * vv * np.sum(ss * g, axis=1)

        Ut, Vt, St = fields((tt @ lay.bary.T).reshape(-1))
        Ub, Vb, Sb = fields((tb @ lay.bary.T).reshape(-1))
        fb = np.concatenate([d["front_before"][k] for k in patch])
        g_t = np.repeat(gt, Q, axis=0)
        g_b = np.repeat(gb, Q, axis=0)
        top = 0.5 * np.sum(w * Qg(Vt, St, g_t))
        rhs = 0.5 * np.sum(w * Qg(fb[:, 1], fb[:, 2:], g_b))
        rhs -= 0.5 * np.sum(w * Qg(Vb - fb[:, 1], Sb - fb[:, 2:], g_b))
        rhs -= np.sum(w * (Ub - fb[:, 0]) * Ub)
        if v in bverts:
            tq = d["t_bot"] + (d["t_top"] - d["t_bot"]) * 0.5 * (nodes + 1)
            xv = np.full((len(tq), 1), mesh.coords[v, 0])
            _, Vd, Sd = B.eval_phys(xv, tq, d["xc"], d["tc"], d["h"], d["c"])
            if neumann:                     # g_N = 0: dissipation beta int (sigma.n)^2
                sd = Sd[:, 0, :] @ d["x"]
                rhs -= beta * np.sum(0.5 * (d["t_top"] - d["t_bot"]) * wts * sd * sd)
            else:                           # g_D = 0: dissipation alpha int v^2
                vd = Vd @ d["x"]
                rhs -= alpha * np.sum(0.5 * (d["t_top"] - d["t_bot"]) * wts * vd * vd)
        elif n > 1 and _on_boundary(mesh, v):
            return
        scale = abs(top) + abs(0.5 * np.sum(w * Qg(fb[:, 1], fb[:, 2:], g_b))) + 1e-30
        worst[0] = max(worst[0], abs(top - rhs) / scale)
        checked[0] += 1

    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    marker = inputs.boundary_marker(mesh, lambda x: True) if neumann else None
    F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: sol(x, 0.0), None,
                       alpha=alpha, record=rec, bnd_type=marker, beta=beta)
    return worst[0], checked[0], F, lay


def _on_boundary(mesh, v):
    x = mesh.coords[v]
    return bool(np.any(np.isclose(x, 0.0) | np.isclose(x, 1.0)))


def _sinsin_1d(x, t):
    """Section 6.5 model problem U = sin(pi x) sin(pi t) (v = 0 at x = 0, 1)."""
    x = np.asarray(x).reshape(-1)
    t = np.broadcast_to(t, x.shape)
    pi = math.pi
    return np.stack([np.sin(pi * x) * np.sin(pi * t), pi * np.sin(pi * x) * np.cos(pi * t),
                     -pi * np.cos(pi * x) * np.sin(pi * t)], axis=1)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_energy_identity_1d_with_dirichlet(p):
    mesh = inputs.mesh_interval(5)           # Section 6.5: 5 elements
    worst, checked, F, lay = _energy_identity_check(mesh, p, 0.7, _sinsin_1d)
    assert checked > 10
    assert worst < 1e-12


@pytest.mark.parametrize("p,beta", [(2, 0.5), (3, 0.5), (3, 1.7)])
def test_energy_identity_1d_with_neumann(p, beta):
    """Per-tent energy identity with Neumann walls (g_N = 0): the boundary
    term of eq. (4.1) tested with the tent's own solution leaves the
    dissipation beta int (sigma.n)^2 on the vertical faces, in place of the
    Dirichlet alpha int v^2; pins the size of the Neumann penalty, which
    exact solutions (sigma.n = g_N) cannot see."""
    mesh = inputs.mesh_interval(5)
    worst, checked, F, lay = _energy_identity_check(mesh, p, 0.7, _sinsin_1d, neumann=True, beta=beta)
    assert checked > 10
    assert worst < 1e-12


def test_energy_identity_2d_interior():
    mesh = inputs.mesh_square(4, 0.2, seed=9)
    worst, checked, F, lay = _energy_identity_check(mesh, 3, 0.3, inputs.standing_wave_2d)
    assert checked > 10
    assert worst < 1e-12


def test_energy_identity_3d_interior():
    """The per-tent energy identity on the interior tents of a 3D mesh
    (jittered 3^3 hexes, six tetrahedra each, p = 2)."""
    mesh = inputs.mesh_cube(3, 0.1, seed=4)
    worst, checked, F, lay = _energy_identity_check(mesh, 2, 0.3, inputs.standing_wave_3d)
    assert checked > 10
    assert worst < 1e-12


def test_energy_decreases_1d():
    """Section 6.5: with exact (constant-energy) data the numerical energy at
    the flat final front is below the initial one."""
    mesh = inputs.mesh_interval(5)
    p = 3
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    E0 = energy.front_energy(_sinsin_1d(lay.xq.reshape(-1, 1), 0.0).reshape(5, -1, 3),
                             lay.wq, mesh.c)
    Es = []
    for T in (0.5, 1.0, 2.0):
        F, tau, ex, _, _ = _run(mesh, p, T, _sinsin_1d, 0.9, dirichlet=False)
        Es.append(energy.front_energy(F, lay.wq, mesh.c))
    assert E0 > Es[0] > Es[1] > Es[2]


@pytest.mark.parametrize("p", [2, 3, 4])
def test_h_convergence_1d(p):
    es = []
    for ne in (8, 16, 32):
        F, _, ex, lay, _ = _run(inputs.mesh_interval(ne), p, 1.0, inputs.plane_wave_1d, 0.9)
        es.append(energy.error_e(F, ex, lay.wq, np.ones(ne)))
    slopes = np.log2(np.array(es[:-1]) / np.array(es[1:]))
    assert np.all(slopes > p - 0.3) and np.all(slopes < p + 0.6), slopes


@pytest.mark.parametrize("p", [2, 3])
def test_h_convergence_2d(p):
    es = []
    for nx in (4, 8, 16):
        m = inputs.mesh_square(nx, 0.2, seed=11)
        F, _, ex, lay, _ = _run(m, p, 0.5, inputs.standing_wave_2d, inputs.pitch_kappa(m),
                                dirichlet=False)
        es.append(energy.error_e(F, ex, lay.wq, m.c))
    slopes = np.log2(np.array(es[:-1]) / np.array(es[1:]))
    assert np.all(slopes > p - 0.3) and np.all(slopes < p + 0.6), slopes


def test_p_convergence_1d():
    es = []
    for p in range(1, 8):
        F, _, ex, lay, _ = _run(inputs.mesh_interval(4), p, 1.0, inputs.plane_wave_1d, 0.9)
        es.append(energy.error_e(F, ex, lay.wq, np.ones(4)))
    ratios = np.array(es[:-1]) / np.array(es[1:])
    assert np.all(ratios > 4.0), ratios


@pytest.mark.parametrize("dim,p,which,cval", [(1, 3, 1, 2.5), (2, 3, 1, 0.4), (2, 4, 0, 3.0),
                                              (3, 2, 0, 1.7)])
def test_polynomial_reproduction_wave_speed(dim, p, which, cval):
    """U_c(x, t) = U_1(x, c t) solves -Lap U + c^-2 U_tt = 0 when U_1 solves the
    c = 1 equation; v = c dU_1/dt(x, ct), sigma = sigma_1(x, ct)."""
    mesh = {1: inputs.mesh_interval(6), 2: inputs.mesh_square(3, 0.2, seed=5),
            3: inputs.mesh_cube(1, 0.0, seed=3)}[dim]
    mesh.c[:] = cval
    base = inputs.polynomial_solution(dim, which)

    def sol(x, t):
        out = base(x, cval * np.asarray(t, dtype=np.float64))
        out[:, 1] *= cval
        return out

    T = 0.3 / cval
    F, tau, ex, _, _ = _run(mesh, p, T, sol, inputs.pitch_kappa(mesh))
    assert np.all(tau == T)
    assert np.abs(F - ex).max() <= 1e-11 * max(1.0, np.abs(ex).max())


@pytest.mark.parametrize("dim,p,c1,c2", [(1, 2, 1.0, 2.5), (1, 4, 3.0, 1.0), (2, 2, 1.0, 3.0),
                                         (2, 3, 2.0, 1.0)])
def test_interface_reproduction(dim, p, c1, c2):
    """Section 4.2: tents that straddle a jump of c carry one polynomial per
    material, coupled on the time-like facets; an exact piecewise-quadratic
    solution with continuous U and sigma.n is reproduced to rounding."""
    mesh = inputs.mesh_interval(6) if dim == 1 else inputs.mesh_square(4, 0.0, seed=1)
    sol, speed = inputs.interface_solution(dim, 0.5, c1, c2)
    mesh.c[:] = speed(mesh.coords[mesh.elems].mean(axis=1))
    T = 0.2
    F, tau, ex, _, _ = _run(mesh, p, T, sol, inputs.pitch_kappa(mesh))
    assert np.all(tau == T)
    assert np.abs(F - ex).max() <= 1e-11 * max(1.0, np.abs(ex).max())


def test_interface_mismatched_speed_not_reproduced():
    """Sanity for the test above: with speeds that do not match the solution
    the piecewise quadratic is not a discrete solution and is not reproduced."""
    mesh = inputs.mesh_interval(6)
    sol, speed = inputs.interface_solution(1, 0.5, 1.0, 2.5)
    mesh.c[:] = speed(mesh.coords[mesh.elems].mean(axis=1))
    mesh.c[mesh.c > 1.5] = 2.0          # speeds no longer match the solution
    F, tau, ex, _, _ = _run(mesh, 2, 0.2, sol, inputs.pitch_kappa(mesh))
    assert np.abs(F - ex).max() > 1e-6


def test_interface_energy_decreases():
    """With interface tents the sweep stays dissipative (Section 6.5)."""
    mesh = inputs.mesh_square(4, 0.2, seed=3)
    cen = mesh.coords[mesh.elems].mean(axis=1)
    mesh.c[:] = np.where(np.linalg.norm(cen - 0.5, axis=1) < 0.3, 3.0, 1.0)
    p = 3
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    f0 = inputs.gaussian_pulse((0.5, 0.5), 0.2)
    E0 = energy.front_energy(f0(lay.xq.reshape(-1, 2)).reshape(lay.wq.shape + (4,)), lay.wq, mesh.c)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), 0.3)
    F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, f0, None)
    E1 = energy.front_energy(F, lay.wq, mesh.c)
    assert E1 < E0


def test_interface_energy_identity_1d():
    """Energy identity of an interface tent (V = U_h, g_D = 0): the centred
    interface terms reproduce the physical flux v+ s+ - v- s-, so
        1/2 int_top Q(u) = 1/2 int_bot Q(u_b) - 1/2 int_bot Q(u - u_b)
                           - int_bot (U - U_b) U - alpha int_F [[v]]^2 - beta int_F [[s]]^2
    on the time-like face F = {x_v} x [t_bot, t_top] (Section 4.2)."""
    mesh = inputs.mesh_interval(6)
    cen = mesh.coords[mesh.elems].mean(axis=1)[:, 0]
    mesh.c[:] = np.where(cen < 0.5, 1.0, 2.5)
    p, alpha, beta = 3, 0.5, 0.5
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    nodes, wts = np.polynomial.legendre.leggauss(12)
    checked = []

    def rec(it, d):
        if len(d["speeds"]) < 2:
            return
        B, v, nb = d["basis"], d["v"], d["basis"].nb
        tau = d["tau_before"]
        top = rhs = 0.0
        for k in d["patch"]:
            g = d["groups"][k]
            ck = d["speeds"][g]
            xg = d["x"][g * nb:(g + 1) * nb]
            ids = mesh.elems[k]
            tb = tau[ids]
            tt = np.where(ids == v, d["t_top"], tb)
            X = mesh.coords[ids]
            gb = (tb[1] - tb[0]) / (X[1, 0] - X[0, 0])
            gt = (tt[1] - tt[0]) / (X[1, 0] - X[0, 0])
            x, w = lay.xq[k], lay.wq[k]

            def f(t):
                U, V, S = B.eval_phys(x, t, d["xc"], d["tc"], d["h"], ck)
                return U @ xg, V @ xg, S[:, 0, :] @ xg

            Ut, Vt, St = f(lay.bary @ tt)
            Ub, Vb, Sb = f(lay.bary @ tb)
            fb = d["front_before"][k]

            def Qg(vv, ss, gg):
                return vv * vv / ck ** 2 + ss * ss - 2 * vv * ss * gg

            top += 0.5 * np.sum(w * Qg(Vt, St, gt))
            rhs += 0.5 * np.sum(w * Qg(fb[:, 1], fb[:, 2], gb))
            rhs -= 0.5 * np.sum(w * Qg(Vb - fb[:, 1], Sb - fb[:, 2], gb))
            rhs -= np.sum(w * (Ub - fb[:, 0]) * Ub)
        tq = d["t_bot"] + (d["t_top"] - d["t_bot"]) * 0.5 * (nodes + 1)
        xv = np.full((len(tq), 1), mesh.coords[v, 0])
        vals = {}
        for k in d["patch"]:
            g = d["groups"][k]
            _, V, S = B.eval_phys(xv, tq, d["xc"], d["tc"], d["h"], d["speeds"][g])
            vals[k] = (V @ d["x"][g * nb:(g + 1) * nb], S[:, 0, :] @ d["x"][g * nb:(g + 1) * nb])
        kl, kr = sorted(d["patch"])
        jw = 0.5 * (d["t_top"] - d["t_bot"]) * wts
        rhs -= alpha * np.sum(jw * (vals[kl][0] - vals[kr][0]) ** 2)
        rhs -= beta * np.sum(jw * (vals[kl][1] - vals[kr][1]) ** 2)
        checked.append(abs(top - rhs) / (abs(top) + 1e-30))

    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, 0.9, 0.5)
    tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, _sinsin_1d_init, None, alpha=alpha, beta=beta,
              record=rec)
    assert len(checked) >= 3
    assert max(checked) < 1e-12


def _sinsin_1d_init(x):
    return _sinsin_1d(x, 0.3)


@pytest.mark.parametrize("dim,p,neumann", [(1, 3, False), (2, 3, False), (2, 3, True)])
def test_tent_matrix_symmetric_part_positive_definite(dim, p, neumann):
    """For Trefftz trial functions the tent form tested with the trial function
    itself is 1/2 int_top Q + 1/2 int_bot Q + int_bot U^2 + alpha int_D v^2 +
    the interface jumps (the energy flux through the tent's boundary, eq. (2.5)
    with the upwind and Dirichlet fluxes of Section 4): the symmetric part of
    every tent matrix, interior, Dirichlet and interface tents alike, is
    positive definite, so elimination without row interchanges cannot break
    down on it.  On Neumann facets the term is beta int_N (sigma.n)^2."""
    mesh = inputs.mesh_interval(6) if dim == 1 else inputs.mesh_square(4, 0.2, seed=3)
    cen = mesh.coords[mesh.elems].mean(axis=1)
    mesh.c[:] = np.where(np.linalg.norm(cen - 0.5, axis=1) < 0.3, 3.0, 1.0)
    kinds, worst = set(), np.inf
    bnd = np.isclose(mesh.coords, 0.0).any(axis=1) | np.isclose(mesh.coords, 1.0).any(axis=1)

    def rec(it, d):
        nonlocal worst
        A = d["A"]
        lam = np.linalg.eigvalsh(0.5 * (A + A.T))
        worst = min(worst, lam[0] / lam[-1])
        kinds.add(("dirichlet" if bnd[d["v"]] else "interior", len(d["speeds"])))

    sol = inputs.polynomial_solution(dim, 0)
    if neumann:
        marker = inputs.boundary_marker(mesh, lambda x: x[0] < 1e-12 or x[1] < 1e-12)
        r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), 0.2)
        tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: sol(x, 0.0), None,
                  bnd_type=marker, record=rec)
    else:
        _run(mesh, p, 0.2, sol, inputs.pitch_kappa(mesh), record=rec)
    assert ("dirichlet", 1) in kinds and ("interior", 2) in kinds and ("interior", 1) in kinds
    assert worst > 0.0, worst


def _neumann_data(sol):
    """g_N = sigma.n of a closed-form solution on a facet with outward normal n."""
    return lambda x, t, nrm: sol(x, t)[:, 2:] @ np.asarray(nrm)


@pytest.mark.parametrize("dim,p,which", [(1, 3, 1), (2, 3, 1), (2, 4, 0)])
def test_polynomial_reproduction_with_neumann_faces(dim, p, which):
    """eq. (4.1) with Neumann facets (sigma.n = g_N): a polynomial solution of
    degree <= p with exact Dirichlet and Neumann data is reproduced to
    rounding; the left (1D) or the left and top sides (2D) are Neumann."""
    mesh = inputs.mesh_interval(6) if dim == 1 else inputs.mesh_square(3, 0.2, seed=5)
    sol = inputs.polynomial_solution(dim, which)
    if dim == 1:
        marker = inputs.boundary_marker(mesh, lambda x: x[0] < 1e-12)
    else:
        marker = inputs.boundary_marker(mesh, lambda x: x[0] < 1e-12 or x[1] > 1 - 1e-12)
    assert marker.sum() >= (1 if dim == 1 else 4)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), 0.3)
    F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: sol(x, 0.0),
                       lambda x, t: sol(x, t)[:, 1], bnd_type=marker, neumann=_neumann_data(sol))
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    ex = sol(lay.xq.reshape(-1, dim), 0.3).reshape(F.shape)
    assert np.all(tau == 0.3)
    assert np.abs(F - ex).max() <= 1e-12 * max(1.0, np.abs(ex).max())
    # the Neumann data matter: dropping them breaks the reproduction
    F0, _ = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: sol(x, 0.0),
                      lambda x, t: sol(x, t)[:, 1], bnd_type=marker, neumann=None)
    assert np.abs(F0 - ex).max() > 1e-6


def test_energy_decreases_with_neumann_walls():
    """With g_N = 0 on every wall the only energy flux out of a tent is the
    beta (sigma.n)^2 dissipation of eq. (4.1): the front energy decreases."""
    mesh = inputs.mesh_square(4, 0.2, seed=3)
    marker = inputs.boundary_marker(mesh, lambda x: True)
    p = 3
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    init = lambda x: inputs.standing_wave_2d(x, 0.0)
    E0 = energy.front_energy(init(lay.xq.reshape(-1, 2)).reshape(mesh.n_elem, -1, 4), lay.wq, mesh.c)
    Es = []
    for T in (0.1, 0.2):
        r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
        F, _ = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, init, None, bnd_type=marker)
        Es.append(energy.front_energy(F, lay.wq, mesh.c))
    assert E0 > Es[0] > Es[1] > 0.5 * E0


def test_lshape_bessel_solution_converges():
    """Section 6.6 on the L-shape, p = 3, T = 1: with the singular solution
    cos(10 t) sin(2 phi / 3) J_2/3(10 r) as initial and Dirichlet data, the L2
    error of U at t = T against the closed form falls when the uniform mesh
    is halved, and on the finer mesh it is of the size the paper's Table 1
    reports near h = 0.07 (about 2e-2)."""
    sol = inputs.bessel_corner_solution()
    err = []
    for h in (0.25, 0.125):
        m = inputs.mesh_lshape(h, 1.0)
        F, _, ex, lay, _ = _run(m, 3, 1.0, sol, inputs.pitch_kappa(m))
        err.append(math.sqrt(float(np.sum(lay.wq * (F[..., 0] - ex[..., 0]) ** 2))))
    assert err[1] < err[0] / 3.0, err
    assert err[1] < 0.06, err


def test_long_time_energy_dissipation():
    """Section 6.5: U = sin(pi x) sin(pi t) on 5 elements (energy pi^2/4 at
    every t).  The numerical energy at T lies below the exact one, the gap
    grows about linearly in T (doubling T doubles it within 25 %), and it
    falls by more than 10x per degree from p = 2 to p = 4."""
    m = inputs.mesh_interval(5)
    E0 = math.pi ** 2 / 4.0
    rel = {}
    for p in (2, 3, 4):
        for T in (4.0, 8.0):
            F, _, _, lay, _ = _run(m, p, T, inputs.sine_product_1d, 0.9)
            rel[p, T] = (E0 - energy.front_energy(F, lay.wq, m.c)) / E0
    for p in (2, 3, 4):
        assert rel[p, 4.0] > 0 and rel[p, 8.0] > 0
        assert 1.5 <= rel[p, 8.0] / rel[p, 4.0] <= 2.5, (p, rel[p, 8.0] / rel[p, 4.0])
    assert rel[3, 8.0] < rel[2, 8.0] / 10 and rel[4, 8.0] < rel[3, 8.0] / 10


def test_long_time_energy_at_the_paper_times():
    """Section 6.5 at the paper's final times, on the oracle's values stored by
    tests/golden/make_energy_oracle.py (5 elements, T = 100, 1000, 10 000,
    p = 2 ... 8): the numerical energy stays below the exact pi^2/4; for
    p >= 4 the relative error grows linearly in T (x10 per decade, within
    20 %) and falls by more than 4x per degree at every T."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energy_oracle.json")
    with open(path) as f:
        rows = json.load(f)["rows"]
    err = {(r["p"], r["T"]): r["rel_energy_error"] for r in rows}
    assert all(e > 0 for e in err.values())
    for p in range(4, 9):
        for T0, T1 in ((100.0, 1000.0), (1000.0, 10000.0)):
            assert 8.0 <= err[p, T1] / err[p, T0] <= 12.0, (p, T0, err[p, T1] / err[p, T0])
    for T in (100.0, 1000.0, 10000.0):
        for p in range(3, 8):
            assert err[p + 1, T] < err[p, T] / 4.0, (p, T)


def test_multi_material_tent_matrix_is_block_sparse():
    """With one speed per element (a log-normal-like medium), a 2D tent over
    vertex v has one polynomial per element of its star (Section 4.2).  The
    block of A coupling two materials is nonzero exactly when they share an
    edge through v (an interface facet, eq. 2.5); around an interior vertex
    the elements form a cycle, so every material has two neighbours and A is
    block cyclic tridiagonal.  Tents here hold up to 8 materials."""
    m = inputs.mesh_square(4, 0.2, seed=9)
    m.c[:] = np.exp(np.random.default_rng(3).normal(0.0, 0.3, m.n_elem))
    p = 2
    nb = (p + 1) ** 2
    kappa = inputs.pitch_kappa(m)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, 0.1)
    seen = []

    def rec(it, d):
        seen.append(d)

    tdg.sweep(m.coords, m.elems, m.c, p, r, inputs.gaussian_pulse((0.5, 0.5), 0.3), None, record=rec)
    nmax, checked_interior = 0, 0
    for d in seen:
        v, A, grp = d["v"], d["A"], d["groups"]
        ng = len(d["speeds"])
        nmax = max(nmax, ng)
        adj = np.zeros((ng, ng), dtype=bool)
        patch = d["patch"]
        for i, ka in enumerate(patch):
            for kb in patch[i + 1:]:
                shared = set(m.elems[ka].tolist()) & set(m.elems[kb].tolist())
                if v in shared and len(shared) == 2 and grp[ka] != grp[kb]:
                    adj[grp[ka], grp[kb]] = adj[grp[kb], grp[ka]] = True
        for a in range(ng):
            for b in range(ng):
                if a == b:
                    continue
                blk = A[a * nb:(a + 1) * nb, b * nb:(b + 1) * nb]
                assert (np.abs(blk).max() > 0) == adj[a, b], (v, a, b)
        if ng == len(patch) and adj.sum(axis=1).min() == 2:
            checked_interior += 1
            assert np.all(adj.sum(axis=1) == 2)
    assert nmax > 4 and checked_interior > 0


@pytest.mark.parametrize("cval", [1.0, 2.0])
def test_energy_through_a_curved_front_is_conserved_for_exact_solutions(cval):
    """energy.front_energy on a front t = tau(x) that is not flat: for an exact
    solution the energy crossing any space-like front equals the energy at
    t = 0 when nothing crosses the walls (here v = 0 there).  The flux
    through the front is 1/2 int (c^-2 v^2 + |sigma|^2 - 2 v sigma.grad tau) dx
    (n dS = (-grad tau, 1) dx, Section 6.5's density on a graph); the front is
    the one the pitching leaves after 9 levels.  Standing wave at speed c:
    U = cos(sqrt2 pi c t) sin(pi x) sin(pi y)."""
    m = inputs.mesh_square(6, 0.2, seed=7)
    m.c[:] = cval
    p = 8
    lay = tdg.front_layout(m.coords, m.elems, p)
    r = pitching.pitch(m.coords, m.elems, m.c, inputs.pitch_kappa(m), 1.0)
    tau = np.zeros(m.n_vert)
    for it in range(len(r["vert"])):
        if r["level"][it] > 9:
            break
        tau[r["vert"][it]] = r["t_top"][it]
    assert tau.max() > tau.min() > 0

    def sol(x, t):
        f = inputs.standing_wave_2d(x, cval * np.asarray(t))
        f[:, 1] *= cval
        return f

    tq = np.einsum("qi,ei->eq", lay.bary, tau[m.elems]).reshape(-1)
    F = sol(lay.xq.reshape(-1, 2), tq).reshape(m.n_elem, -1, 4)
    F0 = sol(lay.xq.reshape(-1, 2), 0.0).reshape(m.n_elem, -1, 4)
    g = energy.element_gradients(m.coords, m.elems, tau)
    assert np.all(cval * np.linalg.norm(g, axis=1) < 1.0)
    E0 = energy.front_energy(F0, lay.wq, m.c)
    assert abs(E0 - np.pi ** 2 / 4) < 1e-10
    assert abs(energy.front_energy(F, lay.wq, m.c, g) - E0) <= 1e-10 * E0
    assert abs(energy.front_energy(F, lay.wq, m.c) - E0) > 1e-3 * E0     # the gradient term matters


def test_refined_solve_removes_the_lu_error_at_degree_5():
    """The tent systems at p = 5 reach kappa(A) ~ 1e8, so one binary64 LU
    leaves an error of a few 1e-12 in the sweep; solving each system with
    the extended-precision refinement agrees with an exact rational solve
    of a tent system far better than the plain LU does, and changes the
    sweep by about that amount (less at p = 4)."""
    from fractions import Fraction
    w = inputs.workload("inclusion_small")
    m = w.mesh
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    systems = []
    tdg.sweep(m.coords, m.elems, m.c, 5, r, w.init, None, tent_range=(0, 40),
              record=lambda it, d: systems.append((d["A"], d["b"])) if len(d["speeds"]) == 2 else None)
    A, b = systems[0]
    n = len(b)
    # exact solve of the binary64 system in rationals (Gauss-Jordan)
    M = [[Fraction(float(A[i, j])) for j in range(n)] + [Fraction(float(b[i]))] for i in range(n)]
    for k in range(n):
        piv = max(range(k, n), key=lambda i: abs(M[i][k]))
        M[k], M[piv] = M[piv], M[k]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k] / M[k][k]
                M[i] = [a - f * c for a, c in zip(M[i], M[k])]
    x_exact = np.array([float(M[i][n] / M[i][i]) for i in range(n)])
    e_lu = np.linalg.norm(np.linalg.solve(A, b) - x_exact) / np.linalg.norm(x_exact)
    e_ref = np.linalg.norm(tdg.solve_refined(A, b) - x_exact) / np.linalg.norm(x_exact)
    assert e_ref <= 1e-14 and e_ref * 10.0 < e_lu, (e_ref, e_lu)
    F0, _ = tdg.sweep(m.coords, m.elems, m.c, 5, r, w.init, None)
    F1, _ = tdg.sweep(m.coords, m.elems, m.c, 5, r, w.init, None, refine=True)
    assert np.linalg.norm(F1 - F0) <= 1e-10 * np.linalg.norm(F1)
