"""The wave-speed gradient of the reverse tent sweep (tp_adjoint's d_dJ_dc)
against the oracle: J = <lambda, front(T)> with the tents held fixed.

References, both CPU-only and independent of the kernel's formula:
  * oracle.adjoint.speed_gradient_transposed: the adjoint state of the whole
    space-time system contracted with central differences of its assembly
    (per material; 1e-8 relative);
  * oracle.adjoint.speed_gradient / finite differences of whole sweeps
    (1e-6 relative, the bar for the adjoint against differences);
  * a closed form: U = x^2 + c^2 t^2 reproduced for every c.
The GPU returns one value per element; summed over the elements of a
material it is that material's derivative (with one speed per element it is
the derivative per element)."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _per_material(m, g):
    speeds = np.unique(m.c)
    return speeds, np.array([g[m.c == s].sum() for s in speeds])


def _case(name):
    if name == "1d_per_element":
        m = inputs.mesh_interval(6)
        m.c[:] = np.exp(np.random.default_rng(8).normal(0.0, 0.3, m.n_elem))
        return m, 3, 0.4, None
    if name == "2d_two_materials":
        m = inputs.mesh_square(3, 0.2, seed=4)
        cen = m.coords[m.elems].mean(axis=1)
        m.c[:] = np.where(cen[:, 0] + 0.3 * cen[:, 1] < 0.55, 1.0, 1.8)
        return m, 3, 0.2, None
    if name == "2d_neumann_two_materials":
        m = inputs.mesh_square(3, 0.2, seed=4)
        cen = m.coords[m.elems].mean(axis=1)
        m.c[:] = np.where(cen[:, 1] < 0.5, 1.0, 0.7)
        bnd = np.zeros((m.n_elem, 3), np.int8)
        bnd[cen[:, 0] < 0.5] = 1
        return m, 2, 0.2, bnd
    m = inputs.mesh_cube(1, 0.1, seed=3)
    cen = m.coords[m.elems].mean(axis=1)
    m.c[:] = np.where(cen[:, 2] < 0.5, 1.0, 1.4)
    return m, 2, 0.12, None


def _gpu_grad(m, p, T, tents, f0, lam, bnd=None, precision="fp64", stride=3, nrhs=1, rhs_split=0):
    import torch
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, 1.0, tents=tents, bnd_type=bnd, precision=precision,
                   ckpt_stride=stride, nrhs=nrhs, rhs_split=rhs_split)
    s.set_state(torch.tensor(f0, dtype=torch.float64, device="cuda").reshape(s.front_shape()).contiguous())
    s.advance()
    lam_t = torch.tensor(lam, dtype=torch.float64, device="cuda").reshape(s.front_shape()).contiguous()
    g = s.speed_gradient(lam_t).cpu().numpy()
    assert s.sync_status() == (0, 0)
    return s, g


@pytest.mark.parametrize("name", ["1d_per_element", "2d_two_materials", "2d_neumann_two_materials", "3d_two_materials"])
def test_speed_gradient_matches_transposed_system(cuda_device, name):
    import paper_1907_02367_gb300 as pkg
    m, p, T, bnd = _case(name)
    kappa = inputs.pitch_kappa(m)
    r = pitching.pitch(m.coords, m.elems, m.c * 1.1, kappa, T)          # room for the oracle's steps
    tents = pkg.Tents(m.coords, m.elems, m.c * 1.1, kappa, T)
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(21)
    f0 = rng.standard_normal(lay.wq.shape + (m.dim + 2,))
    lam = rng.standard_normal(f0.shape)
    _, g = _gpu_grad(m, p, T, tents, f0, lam, bnd)
    sp, gm = _per_material(m, g)
    sp_t, g_t = oadj.speed_gradient_transposed(m.coords, m.elems, m.c, p, r, f0, lam, bnd_type=bnd)
    assert np.array_equal(sp, sp_t) and len(sp) >= 2
    assert np.all(np.abs(gm - g_t) <= 1e-8 * np.abs(g_t).max()), (gm, g_t)


def test_speed_gradient_per_element_against_swept_differences(cuda_device):
    """One speed per element in 1D (every tent is an interface tent): each
    element's dJ/dc_K against central differences of whole oracle sweeps."""
    import paper_1907_02367_gb300 as pkg
    m, p, T, _ = _case("1d_per_element")
    kappa = inputs.pitch_kappa(m)
    r = pitching.pitch(m.coords, m.elems, m.c * 1.1, kappa, T)
    tents = pkg.Tents(m.coords, m.elems, m.c * 1.1, kappa, T)
    pulse = inputs.gaussian_pulse(np.array([0.45]), 0.2)
    lay = tdg.front_layout(m.coords, m.elems, p)
    f0 = pulse(lay.xq.reshape(-1, 1)).reshape(lay.wq.shape + (3,))
    lam = np.random.default_rng(4).standard_normal(f0.shape)
    _, g = _gpu_grad(m, p, T, tents, f0, lam)
    sp, g_fd = oadj.speed_gradient(m.coords, m.elems, m.c, p, r, pulse, lam)
    order = np.argsort(m.c)
    assert np.array_equal(sp, m.c[order])
    assert np.all(np.abs(g[order] - g_fd) <= 1e-6 * np.abs(g_fd).max()), (g[order], g_fd)


def test_speed_gradient_closed_form_with_neumann_walls(cuda_device):
    """U = x^2 + c^2 t^2 on [0, 1] with c-independent initial data and Neumann
    data sigma.n = -2x n: the sweep reproduces it for every c (p = 3), so
    dJ/dc = sum 2 c T^2 lam_U + 4 c T lam_v exactly."""
    import torch
    import paper_1907_02367_gb300 as pkg
    mesh = inputs.mesh_interval(5)
    cval, T, p = 1.3, 0.4, 3
    mesh.c[:] = cval
    marker = inputs.boundary_marker(mesh, lambda x: True)
    kappa = inputs.pitch_kappa(mesh)
    s = pkg.Solver(mesh.coords, mesh.elems, mesh.c, p, T, kappa, bnd_type=marker, ckpt_stride=4)
    xq, _ = s.front_points()
    x = xq[:, 0]
    f0 = torch.tensor(np.stack([x * x, 0 * x, -2 * x], 1)[None], dtype=torch.float64, device="cuda").contiguous()
    xt = s.boundary_points()
    nrm, kind = s.boundary_kinds()
    assert np.all(kind == 1)
    gN = torch.tensor((-2.0 * xt[:, 0] * nrm[:, 0])[None], dtype=torch.float64, device="cuda").contiguous()
    s.set_state(f0, gN)
    lam = np.random.default_rng(8).standard_normal(s.front_shape())
    g = s.speed_gradient(torch.tensor(lam, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert s.sync_status() == (0, 0)
    lam = lam.reshape(-1, 3)
    exact = float(np.sum(2.0 * cval * T * T * lam[:, 0] + 4.0 * cval * T * lam[:, 1]))
    assert abs(g.sum() - exact) <= 1e-9 * max(1.0, abs(exact)), (g.sum(), exact)


def test_checkpoint_stride_and_split_do_not_change_the_gradient(cuda_device):
    """The checkpoints only decide what is recomputed: strides 1, 2 and 7 give
    the same gradient bit for bit; eight right-hand sides split over 4 CTAs
    give the unsplit gradient to rounding, and the gradient is linear in lambda
    across columns."""
    import paper_1907_02367_gb300 as pkg
    m, p, T, _ = _case("2d_two_materials")
    kappa = inputs.pitch_kappa(m)
    tents = pkg.Tents(m.coords, m.elems, m.c, kappa, T)
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(2)
    f0 = rng.standard_normal((8,) + lay.wq.shape + (4,))
    lam = rng.standard_normal(f0.shape)
    gs = [_gpu_grad(m, p, T, tents, f0[:1], lam[:1], stride=st)[1] for st in (1, 2, 7)]
    assert np.array_equal(gs[0], gs[1]) and np.array_equal(gs[0], gs[2])
    _, g_all = _gpu_grad(m, p, T, tents, f0, lam, nrhs=8, rhs_split=1)
    _, g_split = _gpu_grad(m, p, T, tents, f0, lam, nrhs=8, rhs_split=4)
    assert np.abs(g_split - g_all).max() <= 1e-12 * np.abs(g_all).max()
    g_cols = sum(_gpu_grad(m, p, T, tents, f0[i:i + 1], lam[i:i + 1])[1] for i in range(8))
    assert np.abs(g_cols - g_all).max() <= 1e-11 * np.abs(g_all).max()


def test_mixed_forward_gradient_close_to_binary64(cuda_device):
    """The forward solutions of the gradient come from the context's own
    precision: with the mixed forward the gradient stays within 1e-8."""
    import paper_1907_02367_gb300 as pkg
    m, p, T, _ = _case("2d_two_materials")
    kappa = inputs.pitch_kappa(m)
    tents = pkg.Tents(m.coords, m.elems, m.c, kappa, T)
    lay = tdg.front_layout(m.coords, m.elems, p)
    rng = np.random.default_rng(9)
    f0 = rng.standard_normal(lay.wq.shape + (4,))
    lam = rng.standard_normal(f0.shape)
    _, g64 = _gpu_grad(m, p, T, tents, f0, lam)
    _, gmx = _gpu_grad(m, p, T, tents, f0, lam, precision="mixed")
    assert np.linalg.norm(gmx - g64) <= 1e-8 * np.linalg.norm(g64)


def test_autograd_speed_gradient_against_gpu_differences(cuda_device):
    """TentSweep.apply(front0, solver, c): the backward pass gives dJ/dc of an
    L2 misfit; its contraction with a random direction matches central
    differences of two GPU sweeps over the same tents (1e-6)."""
    import torch
    import paper_1907_02367_gb300 as pkg
    m, p, T, _ = _case("2d_two_materials")
    kappa = inputs.pitch_kappa(m)
    tents = pkg.Tents(m.coords, m.elems, m.c * 1.1, kappa, T)
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, tents=tents, ckpt_stride=5)
    xq, wq = s.front_points()
    f0 = torch.tensor(inputs.gaussian_pulse((0.45, 0.5), 0.25)(xq)[None], dtype=torch.float64,
                      device="cuda").contiguous()
    obs = torch.tensor(inputs.gaussian_pulse((0.5, 0.45), 0.25)(xq)[None], dtype=torch.float64, device="cuda")
    w = torch.tensor(wq, dtype=torch.float64, device="cuda").reshape(1, m.n_elem, -1)

    def misfit(front):
        d = front[..., 0] - obs.reshape(front.shape)[..., 0]
        return 0.5 * torch.sum(w * d * d)

    c = torch.tensor(m.c, dtype=torch.float64, device="cuda", requires_grad=True)
    J = misfit(pkg.TentSweep.apply(f0, s, c))
    J.backward()
    g = c.grad.cpu().numpy()
    d = np.random.default_rng(6).standard_normal(m.n_elem)
    d = np.where(m.c == m.c[0], d[0], d[1])            # a direction that keeps the materials intact
    eps = 1e-6

    def J_at(cv):
        s2 = pkg.Solver(m.coords, m.elems, cv, p, T, kappa, tents=tents)
        s2.set_state(f0)
        s2.advance()
        F, _ = s2.get_state()
        assert s2.sync_status() == (0, 0)
        return float(misfit(F))

    fd = (J_at(m.c * (1 + eps * d)) - J_at(m.c * (1 - eps * d))) / (2 * eps)
    an = float(np.sum(g * m.c * d))
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), (fd, an)
