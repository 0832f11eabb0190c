"""Pins for oracle/adjoint.py.

* dot-product identity with the forward oracle: for the linear sweep F
  (g_D = 0, fixed tents), <lambda, F f> = <F^* lambda, f> for random f, lambda;
* finite differences of the L2 misfit J(f0) = 1/2 ||U_h(T) - U_obs||^2;
* the speed gradient against a closed form and a second, wider difference;
* brute force: the whole space-time system solved at once equals the sweep,
  and its transpose the reverse sweep.
"""
import numpy as np
import pytest

from oracle import adjoint, pitching, tdg
from paper_1907_02367_gb300 import inputs


def _setup(dim):
    if dim == 1:
        m, p, T = inputs.mesh_interval(5), 3, 0.4
    elif dim == 2:
        m, p, T = inputs.mesh_square(3, 0.2, seed=4), 3, 0.25
    else:
        m, p, T = inputs.mesh_cube(1, 0.0, seed=3), 2, 0.15
    kappa = inputs.pitch_kappa(m)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    return m, p, r


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_dot_product_identity(dim):
    m, p, r = _setup(dim)
    lay = tdg.front_layout(m.coords, m.elems, p)
    shape = lay.wq.shape + (dim + 2,)
    rng = np.random.default_rng(dim)
    f = rng.standard_normal(shape)
    lam = rng.standard_normal(shape)
    Ff, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None, front0=f)
    Fl = adjoint.adjoint_sweep(m.coords, m.elems, m.c, p, r, lam)
    lhs = float(np.sum(lam * Ff))
    rhs = float(np.sum(Fl * f))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), np.linalg.norm(lam) * np.linalg.norm(Ff))


def test_misfit_gradient_finite_differences():
    m, p, r = _setup(2)
    lay = tdg.front_layout(m.coords, m.elems, p)
    x = lay.xq.reshape(-1, 2)
    f0 = inputs.gaussian_pulse((0.5, 0.5), 0.3)(x).reshape(lay.wq.shape + (4,))
    obs, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None,
                       front0=inputs.gaussian_pulse((0.45, 0.55), 0.3)(x).reshape(f0.shape))

    def J(f):
        F, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None, front0=f)
        return adjoint.misfit_gradient(F, obs, lay.wq)

    j0, gT = J(f0)
    g0 = adjoint.adjoint_sweep(m.coords, m.elems, m.c, p, r, gT)
    rng = np.random.default_rng(7)
    d = rng.standard_normal(f0.shape)
    eps = 1e-5
    fd = (J(f0 + eps * d)[0] - J(f0 - eps * d)[0]) / (2 * eps)
    an = float(np.sum(g0 * d))
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12)


def test_speed_gradient_closed_form():
    """U = x^2 + c^2 t^2 on [0, 1] (v = 2 c^2 t, sigma = -2x) has initial data
    U0 = x^2, v0 = 0, sigma0 = -2x and Neumann data sigma.n = 0 at x = 0, -2
    at x = 1, none of which depend on c; at p >= 2 the sweep reproduces it for
    every c, so J(c) = sum lam . (x^2 + c^2 T^2, 2 c^2 T, -2x) and
    dJ/dc = sum 2 c T^2 lam_U + 4 c T lam_v exactly."""
    mesh = inputs.mesh_interval(5)
    cval, T, p = 1.3, 0.4, 3
    mesh.c[:] = cval
    marker = inputs.boundary_marker(mesh, lambda x: True)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)

    def init(x):
        x = np.asarray(x).reshape(-1)
        return np.stack([x * x, 0.0 * x, -2.0 * x], axis=1)

    def neumann(x, t, nrm):
        return -2.0 * np.asarray(x)[:, 0] * float(nrm[0])

    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    rng = np.random.default_rng(8)
    lam = rng.standard_normal((mesh.n_elem, lay.wq.shape[1], 3))
    speeds, g = adjoint.speed_gradient(mesh.coords, mesh.elems, mesh.c, p, r, init, lam,
                                       bnd_type=marker, neumann=neumann)
    exact = np.sum(2.0 * cval * T * T * lam[..., 0] + 4.0 * cval * T * lam[..., 1])
    assert speeds.tolist() == [cval]
    assert abs(g[0] - exact) <= 1e-7 * max(1.0, abs(exact))


def test_speed_gradient_two_materials_matches_swept_difference():
    """Two materials: each component equals the slope of J along that
    material's speed alone over a wider step (a second, independent
    difference), and the components differ (each material moves alone)."""
    mesh = inputs.mesh_interval(6)
    cen = mesh.coords[mesh.elems].mean(axis=1)[:, 0]
    mesh.c[:] = np.where(cen > 0.5, 2.0, 1.0)
    p, T = 3, 0.2
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    pulse = inputs.gaussian_pulse(np.array([0.4]), 0.15)
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    lam = np.random.default_rng(3).standard_normal((mesh.n_elem, lay.wq.shape[1], 3))
    speeds, g = adjoint.speed_gradient(mesh.coords, mesh.elems, mesh.c, p, r, pulse, lam)
    assert speeds.tolist() == [1.0, 2.0]
    for m, cm in enumerate(speeds):
        J = []
        for d in (1e-4, -1e-4):
            cp = mesh.c.copy()
            cp[mesh.c == cm] = cm + d
            F, _ = tdg.sweep(mesh.coords, mesh.elems, cp, p, r, pulse)
            J.append(float(np.sum(lam.reshape(F.shape) * F)))
        slope = (J[0] - J[1]) / 2e-4
        assert abs(g[m] - slope) <= 1e-6 * max(1.0, abs(slope)), (m, g[m], slope)
    assert abs(g[0] - g[1]) > 1e-6 * max(abs(g[0]), abs(g[1]))


GLOBAL_CASES = [
    (1, lambda: inputs.mesh_interval(5), 3, 1.0),
    (2, lambda: inputs.mesh_square(3, 0.2, seed=3), 2, 0.5),
    (3, lambda: inputs.mesh_cube(1, 0.1, seed=3), 2, 1.5),
]


@pytest.mark.parametrize("dim,mk,p,T", GLOBAL_CASES, ids=["1d", "2d", "3d"])
def test_global_space_time_solve_equals_sweep(dim, mk, p, T):
    """Brute force: the whole space-time system of all tents (each tent's
    eq. (4.1) block, coupled to the earlier tents whose top faces form its
    bottom), assembled densely and solved by one LU, gives the tent-by-tent
    sweep's final front to round-off; its transpose gives the reverse
    sweep's F^* lambda.  The matrix is block lower triangular in the pitched
    order (causality), and every vertex carries several tents."""
    m = mk()
    r = pitching.pitch(m.coords, m.elems, m.c, inputs.pitch_kappa(m), T)
    nt = len(r["vert"])
    assert nt >= 2 * m.n_vert
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(dim)
    f0 = rng.standard_normal((m.n_elem, lay.wq.shape[1], dim + 2))
    lam = rng.standard_normal(f0.shape)
    M, _, _, _, off = adjoint._global_system(m.coords, m.elems, m.c, p, r)
    nb = int(off[1] - off[0])
    assert np.all(np.diff(off) == nb)               # one material: every tent has dim U^p unknowns
    assert M.shape == (nt * nb, nt * nb)
    for t in range(nt - 1):
        assert not np.any(M[t * nb:(t + 1) * nb, (t + 1) * nb:])
    assert np.any(M[nb:, :nb])                      # later tents read earlier ones
    Fg = adjoint.global_solve(m.coords, m.elems, m.c, p, r, f0)
    Fs, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None, front0=f0)
    assert np.linalg.norm(Fg - Fs) <= 1e-12 * np.linalg.norm(Fs)
    Lg = adjoint.global_adjoint(m.coords, m.elems, m.c, p, r, lam)
    Ls = adjoint.adjoint_sweep(m.coords, m.elems, m.c, p, r, lam)
    assert np.linalg.norm(Lg - Ls) <= 1e-12 * np.linalg.norm(Ls)


@pytest.mark.parametrize("dim", [1, 2])
def test_speed_gradient_transposed_system_equals_swept_difference(dim):
    """Two routes to dJ/dc on one material with the tents fixed: the adjoint
    state of the whole space-time system contracted with the derivative of
    its assembly, and central differences of whole sweeps; they agree to
    1e-8 relative (both carry O(s^2) truncation)."""
    if dim == 1:
        m, p, T, cv = inputs.mesh_interval(5), 3, 0.6, 1.3
    else:
        m, p, T, cv = inputs.mesh_square(3, 0.2, seed=3), 2, 0.3, 0.8
    m.c[:] = cv
    r = pitching.pitch(m.coords, m.elems, m.c, inputs.pitch_kappa(m), T)
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(5)
    f0 = rng.standard_normal((m.n_elem, lay.wq.shape[1], dim + 2))
    lam = rng.standard_normal(f0.shape)
    _, g_t = adjoint.speed_gradient_transposed(m.coords, m.elems, m.c, p, r, f0, lam)
    _, g_d = adjoint.speed_gradient(m.coords, m.elems, m.c, p, r, None, lam, front0=f0)
    assert abs(g_t[0] - g_d[0]) <= 1e-8 * abs(g_d[0]), (g_t, g_d[0])


def _materials(case):
    """Meshes with several wave speeds (interface tents, Section 4.2)."""
    if case == "1d_per_element":
        m = inputs.mesh_interval(5)
        m.c[:] = np.exp(np.random.default_rng(8).normal(0.0, 0.3, m.n_elem))
        return m, 3, 0.4, None
    if case == "2d_two_materials":
        m = inputs.mesh_square(3, 0.2, seed=4)
        cen = m.coords[m.elems].mean(axis=1)
        m.c[:] = np.where(cen[:, 0] + 0.3 * cen[:, 1] < 0.55, 1.0, 1.8)
        return m, 2, 0.2, None
    m = inputs.mesh_square(3, 0.2, seed=4)           # two materials and Neumann walls on the left
    cen = m.coords[m.elems].mean(axis=1)
    m.c[:] = np.where(cen[:, 1] < 0.5, 1.0, 0.7)
    bnd = np.zeros((m.n_elem, 3), np.int8)
    bnd[cen[:, 0] < 0.5] = 1
    return m, 2, 0.2, bnd


CASES = ["1d_per_element", "2d_two_materials", "2d_neumann_two_materials"]


@pytest.mark.parametrize("case", CASES)
def test_multi_material_adjoint_dot_product_and_whole_system(case):
    """Interface tents and Neumann facets: the reverse sweep is the transpose
    of oracle.tdg.sweep (dot-product identity) and the whole space-time
    system solved at once reproduces the sweep and its adjoint."""
    m, p, T, bnd = _materials(case)
    r = pitching.pitch(m.coords, m.elems, m.c, inputs.pitch_kappa(m), T)
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(11)
    f = rng.standard_normal(lay.wq.shape + (m.dim + 2,))
    lam = rng.standard_normal(f.shape)
    Ff, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None, front0=f, bnd_type=bnd)
    Fl = adjoint.adjoint_sweep(m.coords, m.elems, m.c, p, r, lam, bnd_type=bnd)
    lhs, rhs = float(np.sum(lam * Ff)), float(np.sum(Fl * f))
    assert abs(lhs - rhs) <= 1e-11 * np.linalg.norm(lam) * np.linalg.norm(Ff)
    Fg = adjoint.global_solve(m.coords, m.elems, m.c, p, r, f, bnd_type=bnd)
    assert np.linalg.norm(Fg - Ff) <= 1e-11 * np.linalg.norm(Ff)
    Lg = adjoint.global_adjoint(m.coords, m.elems, m.c, p, r, lam, bnd_type=bnd)
    assert np.linalg.norm(Lg - Fl) <= 1e-11 * np.linalg.norm(Fl)


@pytest.mark.parametrize("case", CASES)
def test_per_material_speed_gradient_two_routes(case):
    """dJ/dc_m for every material (in 1D every element its own speed): the
    transposed whole system contracted with the derivative of its assembly
    equals central differences of whole sweeps to 1e-7 relative (both carry
    O(s^2) truncation and O(u/s) rounding)."""
    m, p, T, bnd = _materials(case)
    r = pitching.pitch(m.coords, m.elems, m.c * 1.1, inputs.pitch_kappa(m), T)   # room for the steps
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(21)
    f0 = rng.standard_normal(lay.wq.shape + (m.dim + 2,))
    lam = rng.standard_normal(f0.shape)
    sp_t, g_t = adjoint.speed_gradient_transposed(m.coords, m.elems, m.c, p, r, f0, lam, bnd_type=bnd)
    sp_d, g_d = adjoint.speed_gradient(m.coords, m.elems, m.c, p, r, None, lam, front0=f0, bnd_type=bnd)
    assert np.array_equal(sp_t, sp_d) and len(sp_t) >= 2
    assert np.all(np.abs(g_t - g_d) <= 1e-7 * np.abs(g_d).max()), (g_t, g_d)
