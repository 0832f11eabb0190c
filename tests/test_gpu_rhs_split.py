"""Right-hand sides split over a tent's cluster (tp_params.rhs_split): every
CTA of the cluster owns a slice of the right-hand sides at every point of the
patch (data moments, solve, outflow) while the tent matrix is assembled once
from the points split over the same CTAs.  Each split must reproduce the
oracle column by column (FP64 1e-11, mixed 1e-8 relative L2), on interior,
Dirichlet, interface (two materials) and Neumann tents, and the adjoint
sweep must stay the transpose of the forward one."""
import numpy as np
import pytest

from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pulses(dim, n, seed):
    rng = np.random.default_rng(seed)
    return [inputs.gaussian_pulse(rng.uniform(0.3, 0.7, dim), rng.uniform(0.15, 0.3)) for _ in range(n)]


def _run(m, p, T, kappa, inits, precision, rhs_split, bnd_type=None, gN=None, schedule="dataflow"):
    import torch
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, nrhs=len(inits), precision=precision,
                   rhs_split=rhs_split, bnd_type=bnd_type, schedule=schedule)
    xq, _ = s.front_points()
    f0 = torch.tensor(np.stack([f(xq) for f in inits]), dtype=torch.float64, device="cuda").contiguous()
    g = None
    if gN is not None and s.n_bnd:
        xt = s.boundary_points()
        nrm, kind = s.boundary_kinds()
        g = torch.tensor(np.stack([np.where(kind == 1, gN(xt[:, :-1], xt[:, -1], nrm) * (r + 1), 0.0)
                                   for r in range(len(inits))]), dtype=torch.float64, device="cuda").contiguous()
    s.set_state(f0, g)
    s.advance()
    front, tau = s.get_state()
    return s, front.cpu().numpy(), tau.cpu().numpy(), s.sync_status()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
@pytest.mark.parametrize("split", [2, 4, 8])
@pytest.mark.parametrize("name", ["small2d", "inclusion_small"])
def test_split_columns_match_oracle(cuda_device, name, split, precision, tol):
    w = inputs.workload(name)
    m = w.mesh
    inits = _pulses(2, 16, 91)
    s, got, tau, st = _run(m, w.p, w.T, w.kappa, inits, precision, split)
    assert st == (0, 0)
    got = got.reshape(len(inits), m.n_elem, -1, 4)
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    for col in (0, 5, 15):
        ref, rtau = tdg.sweep(m.coords, m.elems, m.c, w.p, r, inits[col], None)
        assert _rel(got[col], ref) <= tol, col
    assert np.array_equal(tau, rtau)


@pytest.mark.parametrize("schedule", ["dataflow", "levels"])
def test_split_equals_unsplit_3d(cuda_device, schedule):
    """3D p = 3, 32 pulses: split over 4 and 8 CTAs equals the unsplit
    sweep to rounding (the moments are summed in another order)."""
    m = inputs.mesh_cube(2, 0.1, seed=4)
    kappa = inputs.pitch_kappa(m)
    inits = _pulses(3, 32, 44)
    _, a, ta, sa = _run(m, 3, 0.1, kappa, inits, "fp64", 1, schedule=schedule)
    for split in (4, 8):
        _, b, tb, sb = _run(m, 3, 0.1, kappa, inits, "fp64", split, schedule=schedule)
        assert sa == sb == (0, 0)
        assert np.array_equal(ta, tb)
        assert _rel(b, a) <= 1e-13, split
    ref, _ = tdg.sweep(m.coords, m.elems, m.c, 3, pitching.pitch(m.coords, m.elems, m.c, kappa, 0.1),
                       inits[31], None)
    assert _rel(b.reshape(32, m.n_elem, -1, 5)[31], ref) <= 1e-11


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_split_neumann_data(cuda_device, precision, tol):
    """Neumann walls with data g_N (different per column) under a split of 4."""
    m = inputs.mesh_square(4, 0.2, seed=6)
    bnd = np.zeros((m.n_elem, 3), np.int8)
    cen = m.coords[m.elems].mean(axis=1)
    bnd[cen[:, 0] < 0.5] = 1                      # the left half's boundary facets are Neumann
    kappa = inputs.pitch_kappa(m)
    inits = _pulses(2, 8, 7)

    def gN(x, t, n):   # n: one facet normal (oracle) or one per point (library)
        return np.sin(2.0 * x[:, 0] + x[:, 1]) * (1.0 + t) * np.atleast_2d(n)[:, 0]

    s, got, tau, st = _run(m, 3, 0.2, kappa, inits, precision, 4, bnd_type=bnd, gN=gN)
    assert st == (0, 0)
    got = got.reshape(len(inits), m.n_elem, -1, 4)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, 0.2)
    for col in (0, 3, 7):
        ref, _ = tdg.sweep(m.coords, m.elems, m.c, 3, r, inits[col], None, bnd_type=bnd,
                           neumann=lambda x, t, n, c=col: gN(x, t, n) * (c + 1))
        assert _rel(got[col], ref) <= tol, col


def test_split_adjoint_is_transpose(cuda_device):
    """<lambda, F f> = <F* lambda, f> column by column with the right-hand
    sides split over 4 CTAs (inclusion workload: interface tents)."""
    import torch
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload("inclusion_small")
    m = w.mesh
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, nrhs=8, rhs_split=4)
    g = torch.Generator(device="cpu").manual_seed(3)
    f = torch.randn(s.front_shape(), generator=g, dtype=torch.float64).cuda().contiguous()
    lam = torch.randn(s.front_shape(), generator=g, dtype=torch.float64).cuda().contiguous()
    s.set_state(f)
    s.advance()
    Ff, _ = s.get_state()
    Fl = s.adjoint(lam)
    assert s.sync_status() == (0, 0)
    for r in range(8):
        lhs = float(torch.sum(lam[r] * Ff[r]))
        rhs = float(torch.sum(Fl[r] * f[r]))
        assert abs(lhs - rhs) <= 1e-11 * float(torch.linalg.norm(lam[r]) * torch.linalg.norm(Ff[r])), r
