"""Accumulated energy loss on the GPU (tp_energy's second column, contexts
created with dissipation tracking): every forward tent adds the jump terms
of eq. (2.5)/(4.1) tested with its own solution (Section 6.5).  Checked:
the GPU's sum equals the oracle's (oracle.energy.tent_dissipation summed
over the same tents), and the GPU's own energy balance closes,
E(now) = E(0) - D, after the whole sweep and after a part of it (curved
front), on Dirichlet walls with and without data, Neumann walls with data,
interface tents and in 3D, in binary64 and in the mixed path, with
right-hand sides split over the cluster."""
import numpy as np
import pytest

from oracle import energy, pitching
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _neumann_half(m):
    bnd = np.zeros((m.n_elem, m.dim + 1), np.int8)
    bnd[m.coords[m.elems].mean(axis=1)[:, 0] < 0.5] = 1
    return bnd


def _gN(x, t, n):
    return np.sin(2.0 * x[:, 0] + x[:, 1]) * (1.0 + t) * np.atleast_2d(n)[:, 0]


def _case(name):
    if name == "2d_dirichlet":
        w = inputs.workload("small2d")
        return w.mesh, 3, 0.2, w.kappa, w.init, {}
    if name == "1d_dirichlet_data":
        w = inputs.workload("plane1d")
        return w.mesh, 3, 0.3, 0.9, w.init, {"dirichlet": w.dirichlet}
    if name == "2d_interface":
        w = inputs.workload("inclusion_small")
        return w.mesh, 3, 0.1, w.kappa, w.init, {}
    if name == "2d_neumann_data":
        m = inputs.mesh_square(4, 0.2, seed=6)
        return m, 3, 0.2, inputs.pitch_kappa(m), inputs.gaussian_pulse((0.4, 0.5), 0.2), \
            {"bnd_type": _neumann_half(m), "neumann": _gN, "beta": 1.7}
    m = inputs.mesh_cube(2, 0.1, seed=4)
    return m, 2, 0.1, inputs.pitch_kappa(m), inputs.gaussian_pulse((0.5, 0.45, 0.5), 0.3), {}


def _gpu(m, p, T, kappa, inits, kw, precision="fp64", levels=None, rhs_split=0):
    import torch
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, nrhs=len(inits), precision=precision,
                   bnd_type=kw.get("bnd_type"), beta=kw.get("beta", 0.5), rhs_split=rhs_split,
                   track_dissipation=True)
    xq, _ = s.front_points()
    f0 = torch.tensor(np.stack([f(xq) for f in inits]), dtype=torch.float64, device="cuda").contiguous()
    g = None
    if s.n_bnd and ("dirichlet" in kw or "neumann" in kw):
        xt = s.boundary_points()
        nrm, kind = s.boundary_kinds()
        gd = kw["dirichlet"](xt[:, :-1], xt[:, -1]) if "dirichlet" in kw else np.zeros(len(xt))
        gn = kw["neumann"](xt[:, :-1], xt[:, -1], nrm) if "neumann" in kw else np.zeros(len(xt))
        g = torch.tensor(np.stack([np.where(kind == 1, gn, gd)] * len(inits)), dtype=torch.float64,
                         device="cuda").contiguous()
    s.set_state(f0, g)
    ed0 = s.energy_and_dissipation().cpu().numpy()
    s.advance(1, (s.n_levels + 1) if levels is None else levels)
    ed1 = s.energy_and_dissipation().cpu().numpy()
    assert s.sync_status() == (0, 0)
    return s, ed0, ed1


CASES = ["2d_dirichlet", "1d_dirichlet_data", "2d_interface", "2d_neumann_data", "3d_dirichlet"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
@pytest.mark.parametrize("name", CASES)
def test_dissipation_matches_oracle_and_balance_closes(cuda_device, name, precision, tol):
    m, p, T, kappa, init, kw = _case(name)
    s, ed0, ed1 = _gpu(m, p, T, kappa, [init], kw, precision)
    E0, D0 = ed0[0]
    E1, D1 = ed1[0]
    assert D0 == 0.0 and D1 > 0.0
    assert abs(E1 - (E0 - D1)) <= tol * E0, (E0, E1, D1)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    okw = {k: v for k, v in kw.items()}
    _, _, Dref, _ = energy.sweep_dissipation(m.coords, m.elems, m.c, p, r, init, **okw)
    assert abs(D1 - Dref) <= tol * max(abs(Dref), E0 * 1e-3), (D1, Dref)


def test_balance_on_a_curved_front(cuda_device):
    """After 7 of the levels the front is not flat: the flux through it and
    the loss so far still add up to the initial energy, and the loss equals
    the oracle's over the same tents."""
    m, p, T, kappa, init, kw = _case("2d_dirichlet")
    L = 7
    s, ed0, ed1 = _gpu(m, p, T, kappa, [init], kw, levels=L)
    E0, E1, D1 = ed0[0][0], ed1[0][0], ed1[0][1]
    assert abs(E1 - (E0 - D1)) <= 1e-11 * E0
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    nt = int(np.sum(r["level"] < L))
    _, _, Dref, _ = energy.sweep_dissipation(m.coords, m.elems, m.c, p, r, init, tent_range=(0, nt))
    assert abs(D1 - Dref) <= 1e-11 * E0


@pytest.mark.parametrize("split", [1, 4])
def test_dissipation_per_column_with_many_rhs(cuda_device, split):
    """Sixteen pulses on the interface workload, kept together or split over
    4 CTAs: each column's loss equals that column's own single run."""
    m, p, T, kappa, _, kw = _case("2d_interface")
    rng = np.random.default_rng(12)
    inits = [inputs.gaussian_pulse(rng.uniform(0.3, 0.7, 2), rng.uniform(0.1, 0.25)) for _ in range(16)]
    s, ed0, ed1 = _gpu(m, p, T, kappa, inits, kw, rhs_split=split)
    assert np.all(np.abs(ed1[:, 0] - (ed0[:, 0] - ed1[:, 1])) <= 1e-11 * ed0[:, 0])
    for col in (0, 9, 15):
        _, e0, e1 = _gpu(m, p, T, kappa, [inits[col]], kw)
        assert abs(ed1[col, 1] - e1[0, 1]) <= 1e-12 * e0[0, 0], col
