"""Point outputs of the forward sweep (tp_set_probes / tp_get_probes), the
ingredient of Section 6.7's U_C(t): U_h at (point, time) samples, each taken
in the tent that holds it.  Against the oracle's probe_values on the same
tents (binary64 1e-11, mixed 1e-8 relative to the largest value), exact
polynomial solutions reproduced at every sample, several right-hand sides
(split over the cluster too), and the U_C(t) study on a coarse mesh."""
import numpy as np
import pytest

from oracle import energy, pitching
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _probe_run(m, p, T, kappa, inits, pts, times, precision="fp64", rhs_split=0, dirichlet=None):
    import torch
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, nrhs=len(inits), precision=precision, rhs_split=rhs_split)
    s.set_probes(pts, times)
    xq, _ = s.front_points()
    f0 = torch.tensor(np.stack([f(xq) for f in inits]), dtype=torch.float64, device="cuda").contiguous()
    g = None
    if dirichlet is not None and s.n_bnd:
        xt = s.boundary_points()
        g = torch.tensor(np.stack([dirichlet(xt[:, :-1], xt[:, -1])] * len(inits)), dtype=torch.float64,
                         device="cuda").contiguous()
    s.set_state(f0, g)
    s.advance()
    assert s.sync_status() == (0, 0)
    return s.get_probes().cpu().numpy()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-9)])
def test_probes_reproduce_exact_solution(cuda_device, precision, tol):
    mesh = inputs.mesh_square(3, 0.2, seed=5)
    base = inputs.polynomial_solution(2, 1)
    T = 0.25
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.05, 0.95, (12, 2))
    times = np.concatenate([[0.0], np.sort(rng.uniform(0.0, T, 9)), [T]])
    got = _probe_run(mesh, 4, T, inputs.pitch_kappa(mesh), [lambda x: base(x, 0.0)], pts, times, precision,
                     dirichlet=lambda x, t: base(x, t)[:, 1])[0]
    for kt, t in enumerate(times):
        ex = base(pts, np.full(len(pts), t))[:, 0]
        assert np.abs(got[kt] - ex).max() <= tol * max(1.0, np.abs(ex).max()), t


@pytest.mark.parametrize("precision,tol,split,nrhs", [("fp64", 1e-11, 0, 1), ("mixed", 1e-8, 0, 1),
                                                       ("fp64", 1e-11, 1, 3), ("fp64", 1e-11, 2, 32)])
def test_probes_match_oracle_on_interface_tents(cuda_device, precision, tol, split, nrhs):
    w = inputs.workload("inclusion_small")
    m = w.mesh
    rng = np.random.default_rng(8)
    inits = [w.init] + [inputs.gaussian_pulse(rng.uniform(0.3, 0.7, 2), rng.uniform(0.1, 0.2))
                        for _ in range(nrhs - 1)]
    pts = rng.uniform(0.1, 0.9, (9, 2))
    times = np.linspace(0.0, w.T, 11)[:-1] + 0.0007
    got = _probe_run(m, w.p, w.T, w.kappa, inits, pts, times, precision, rhs_split=split)
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    for col in sorted({0, nrhs - 1}):
        ref, owner = energy.probe_values(m.coords, m.elems, m.c, w.p, r, inits[col], pts, times)
        assert np.all(owner >= 0)
        assert np.abs(got[col] - ref).max() <= tol * np.abs(ref).max(), col


def test_point_output_study_coarse(cuda_device):
    """Section 6.7's U_C(t) on a coarse version of the two-speed medium: the
    sweep is clean, U_C vanishes before any wave can reach the box, and it
    has a first arrival no earlier than the fastest path allows."""
    from paper_1907_02367_gb300 import interface_study
    out = interface_study.run(h_left=0.05, h_right=0.1, n_times=41, delta=0.1)
    assert out["status"] == [0, 0]
    t = np.asarray(out["times"])
    uc = np.asarray(out["U_C"])
    assert np.all(np.isfinite(uc)) and uc.max() > 0
    # the pulse (width 0.1 around (1, 1)) is 0.75 away from the box; the fastest
    # route (0.2 at c = 1 to the interface, along it at c = 3, back 0.2) takes > 0.5
    early = t < 0.2
    assert uc[early].max() <= 1e-3 * uc.max()
