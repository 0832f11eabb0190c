"""GPU parity with Neumann facets (eq. 4.1: v (tau.n) + beta (sigma.n)(tau.n) on
the left, g_N (beta tau.n - w) on the right): exact polynomial solutions with
Dirichlet and Neumann data are reproduced, sweeps with Neumann walls match the
oracle element by element, and the adjoint of a sweep with Neumann facets
satisfies the dot-product identity."""
import numpy as np
import pytest

from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _solver(mesh, p, T, marker, precision="fp64", nrhs=1):
    import paper_1907_02367_gb300 as pkg
    return pkg.Solver(mesh.coords, mesh.elems, mesh.c, p, T, inputs.pitch_kappa(mesh), nrhs=nrhs,
                      precision=precision, bnd_type=marker)


def _run(s, init, sol_bnd=None):
    """Sweep from init(x); boundary data from sol_bnd(x, t) (U, v, sigma):
    g_D = v on Dirichlet points, g_N = sigma.n on Neumann points."""
    import torch
    xq, _ = s.front_points()
    front0 = torch.tensor(np.asarray(init(xq))[None], dtype=torch.float64, device="cuda").contiguous()
    gD = None
    if sol_bnd is not None and s.n_bnd:
        xt = s.boundary_points()
        nrm, kind = s.boundary_kinds()
        f = np.asarray(sol_bnd(xt[:, :-1], xt[:, -1]))
        g = np.where(kind == 1, np.einsum("qd,qd->q", f[:, 2:], nrm), f[:, 1])
        gD = torch.tensor(g[None], dtype=torch.float64, device="cuda").contiguous()
    s.set_state(front0, gD)
    s.advance()
    front, tau = s.get_state()
    return front.cpu().numpy(), tau.cpu().numpy(), s.sync_status()


def _neumann_data(sol):
    return lambda x, t, nrm: sol(x, t)[:, 2:] @ np.asarray(nrm)


MARKERS = {1: lambda x: x[0] < 1e-12, 2: lambda x: x[0] < 1e-12 or x[1] > 1 - 1e-12,
           3: lambda x: x[2] < 1e-12}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-9)])
@pytest.mark.parametrize("dim,p,which", [(1, 3, 1), (2, 3, 1), (2, 4, 0), (3, 3, 1)])
def test_polynomial_reproduction_with_neumann_faces(cuda_device, precision, tol, dim, p, which):
    mesh = {1: inputs.mesh_interval(6), 2: inputs.mesh_square(3, 0.2, seed=5),
            3: inputs.mesh_cube(1, 0.0, seed=3)}[dim]
    marker = inputs.boundary_marker(mesh, MARKERS[dim])
    assert marker.sum() > 0
    sol = inputs.polynomial_solution(dim, which)
    T = 0.3 if dim < 3 else 0.15
    s = _solver(mesh, p, T, marker, precision)
    _, kind = s.boundary_kinds()
    assert (kind == 1).any() and (kind == 0).any()
    got, tau, st = _run(s, lambda x: sol(x, 0.0), sol)
    assert st == (0, 0)
    assert np.all(tau == T)
    xq, _ = s.front_points()
    ex = sol(xq, T)
    assert np.abs(got.reshape(ex.shape) - ex).max() <= tol * max(1.0, np.abs(ex).max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_neumann_walls_match_oracle(cuda_device, precision, tol):
    """A Gaussian pulse in the unit square with g_N = 0 on every wall (a
    closed room), p = 4: the front after the sweep against the oracle."""
    mesh = inputs.mesh_square(5, 0.2, seed=7)
    marker = inputs.boundary_marker(mesh, lambda x: True)
    pulse = inputs.gaussian_pulse(np.array([0.35, 0.6]), 0.2)
    p, T = 4, 0.4
    s = _solver(mesh, p, T, marker, precision)
    got, tau, st = _run(s, pulse)
    assert st == (0, 0)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    ref, tau_ref = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, pulse, None, bnd_type=marker)
    assert np.array_equal(tau, tau_ref)
    assert _rel(got.reshape(ref.shape), ref) <= tol


def test_mixed_boundaries_with_data_match_oracle(cuda_device):
    """Dirichlet on two sides, Neumann on the others, non-polynomial data
    (the standing wave's v and sigma.n): element-by-element parity."""
    mesh = inputs.mesh_square(4, 0.15, seed=2)
    marker = inputs.boundary_marker(mesh, lambda x: x[0] < 1e-12 or x[1] < 1e-12)
    sol = inputs.standing_wave_2d
    p, T = 3, 0.3
    s = _solver(mesh, p, T, marker)
    got, _, st = _run(s, lambda x: sol(x, 0.0), sol)
    assert st == (0, 0)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    ref, _ = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: sol(x, 0.0),
                       lambda x, t: sol(x, t)[:, 1], bnd_type=marker, neumann=_neumann_data(sol))
    assert _rel(got.reshape(ref.shape), ref) <= 1e-11


def test_neumann_adjoint_dot_product(cuda_device):
    import torch
    mesh = inputs.mesh_square(4, 0.2, seed=3)
    marker = inputs.boundary_marker(mesh, lambda x: x[1] > 1 - 1e-12 or x[0] > 1 - 1e-12)
    s = _solver(mesh, 3, 0.3, marker)
    rng = np.random.default_rng(11)
    f = torch.tensor(rng.standard_normal(s.front_shape()), device="cuda")
    lam = torch.tensor(rng.standard_normal(s.front_shape()), device="cuda")
    s.set_state(f)
    s.advance()
    Ff, _ = s.get_state()
    Fl = s.adjoint(lam)
    assert s.sync_status() == (0, 0)
    lhs = float(torch.sum(lam * Ff))
    rhs = float(torch.sum(Fl * f))
    assert abs(lhs - rhs) <= 1e-11 * float(torch.linalg.norm(lam) * torch.linalg.norm(Ff))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_interface_meeting_neumann_and_dirichlet_walls(cuda_device, precision, tol):
    """Two materials (c = 1 left of x = 1/2, c = 2.5 right of it) whose interface
    meets a Neumann wall (y = 0) and a Dirichlet wall (y = 1): tents at the
    junctions carry interface, Neumann and Dirichlet facets and two
    polynomials at once; against the oracle."""
    mesh = inputs.mesh_square(4, 0.0, seed=1)
    cen = mesh.coords[mesh.elems].mean(axis=1)
    mesh.c[:] = np.where(cen[:, 0] > 0.5, 2.5, 1.0)
    marker = inputs.boundary_marker(mesh, lambda x: x[1] < 1e-12)
    pulse = inputs.gaussian_pulse(np.array([0.45, 0.3]), 0.25)
    p, T = 3, 0.2
    s = _solver(mesh, p, T, marker, precision)
    got, tau, st = _run(s, pulse)
    assert st == (0, 0)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    ref, tau_ref = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, pulse, None, bnd_type=marker)
    assert np.array_equal(tau, tau_ref)
    assert _rel(got.reshape(ref.shape), ref) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_penalty_beta_other_than_half(cuda_device, precision, tol):
    """beta = 1.7 (eq. 2.5) instead of the paper's 0.5: Neumann walls in 1D, and
    the inclusion's interface facets in 2D (with Dirichlet walls), against the
    oracle with the same beta."""
    import paper_1907_02367_gb300 as pkg
    beta = 1.7
    # 1D, Neumann walls, g_N = 0
    mesh = inputs.mesh_interval(5)
    marker = inputs.boundary_marker(mesh, lambda x: True)
    init = lambda x: inputs.sine_product_1d(x, 0.3)          # noqa: E731
    p, T = 3, 0.7
    s = pkg.Solver(mesh.coords, mesh.elems, mesh.c, p, T, 0.9, precision=precision, bnd_type=marker,
                   beta=beta)
    got, tau, st = _run(s, init)
    assert st == (0, 0)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, 0.9, T)
    ref, tau_ref = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, init, None, bnd_type=marker, beta=beta)
    assert np.array_equal(tau, tau_ref)
    assert _rel(got.reshape(ref.shape), ref) <= tol
    # 2D, interface facets (c = 3 in the disc, 1 outside)
    w = inputs.workload("inclusion_small")
    m = w.mesh
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, precision=precision, beta=beta)
    got, tau, st = _run(s, w.init)
    assert st == (0, 0)
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    ref, tau_ref = tdg.sweep(m.coords, m.elems, m.c, w.p, r, w.init, None, beta=beta)
    assert np.array_equal(tau, tau_ref)
    assert _rel(got.reshape(ref.shape), ref) <= tol
