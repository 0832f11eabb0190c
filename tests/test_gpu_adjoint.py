"""GPU adjoint sweep (tp_adjoint) against the oracle's transposed tent maps,
the dot-product identity <lambda, F f> = <F^* lambda, f> of the GPU forward
and adjoint sweeps (at full size too), and the autograd wrapper's gradient
against finite differences of an L2 misfit."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _setup(dim):
    if dim == 1:
        m, p, T = inputs.mesh_interval(7), 3, 0.5
    elif dim == 2:
        m, p, T = inputs.mesh_square(5, 0.2, seed=4), 4, 0.3
    else:
        m, p, T = inputs.mesh_cube(2, 0.1, seed=3), 3, 0.15
    return m, p, T, inputs.pitch_kappa(m)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_adjoint_matches_oracle(cuda_device, dim):
    import torch
    import paper_1907_02367_gb300 as pkg
    m, p, T, kappa = _setup(dim)
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa)
    rng = np.random.default_rng(11 + dim)
    lam = rng.standard_normal(s.front_shape())
    got = s.adjoint(torch.tensor(lam, device="cuda")).cpu().numpy()
    assert s.sync_status() == (0, 0)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    ref = oadj.adjoint_sweep(m.coords, m.elems, m.c, p, r, lam[0])
    assert _rel(got[0], ref) <= 1e-11


@pytest.mark.parametrize("name", ["small2d", "standing2d", "standing3d_small"])
def test_dot_product_identity_gpu(cuda_device, name):
    import torch
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload(name)
    m = w.mesh
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa)
    rng = np.random.default_rng(5)
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


def test_dot_product_identity_rhs_groups(cuda_device):
    """64 right-hand sides in 3D at p = 3 kept together in each CTA
    (rhs_split = 1) run as two groups of 32 in both the forward and the
    reverse sweep: the identity holds for every column."""
    import torch
    import paper_1907_02367_gb300 as pkg
    m = inputs.mesh_cube(2, 0.1, seed=4)
    s = pkg.Solver(m.coords, m.elems, m.c, 3, 0.1, inputs.pitch_kappa(m), nrhs=64, rhs_split=1)
    rng = np.random.default_rng(5)
    f = torch.tensor(rng.standard_normal(s.front_shape()), device="cuda")
    lam = torch.tensor(rng.standard_normal(s.front_shape()), device="cuda")
    s.set_state(f)
    s.advance()
    Ff, _ = s.get_state()
    Fl = s.adjoint(lam)
    assert s.sync_status() == (0, 0)
    for r in (0, 31, 40, 63):
        lhs = float(torch.sum(lam[r] * Ff[r]))
        rhs = float(torch.sum(Fl[r] * f[r]))
        assert abs(lhs - rhs) <= 1e-11 * float(torch.linalg.norm(lam[r]) * torch.linalg.norm(Ff[r]))


def test_autograd_gradient_finite_differences(cuda_device):
    import torch
    import paper_1907_02367_gb300 as pkg
    m, p, T, kappa = _setup(2)
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa)
    xq, wq = s.front_points()
    f0 = torch.tensor(inputs.gaussian_pulse((0.5, 0.5), 0.3)(xq), device="cuda").reshape(s.front_shape())
    obs = torch.tensor(inputs.gaussian_pulse((0.45, 0.55), 0.25)(xq), device="cuda").reshape(s.front_shape())
    w = torch.tensor(wq, device="cuda").reshape(1, m.n_elem, -1)

    def J(front0):
        out = pkg.TentSweep.apply(front0, s)
        return 0.5 * torch.sum(w * (out[..., 0] - obs[..., 0]) ** 2)

    x = f0.clone().requires_grad_(True)
    j = J(x)
    j.backward()
    g = x.grad.detach()
    d = torch.tensor(np.random.default_rng(3).standard_normal(s.front_shape()), device="cuda")
    eps = 1e-5
    with torch.no_grad():
        fd = (J(f0 + eps * d) - J(f0 - eps * d)) / (2 * eps)
    an = float(torch.sum(g * d))
    assert abs(float(fd) - an) <= 1e-6 * max(abs(an), 1e-12)
