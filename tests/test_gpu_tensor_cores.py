"""Tensor-core data moments and outflow of the mixed forward sweep
(tp_params.tensor_cores): with split right-hand sides, single-material tents
contract their float-float operands as five signed 9-bit digit planes on
tcgen05, summed exactly in binary32 tensor memory (Section 4.1's tent system
is unchanged: only the rounding of two sums moves, from the compensated
float-float sums' ~2^-44 to ~2^-42 of their scales).  The sweep must equal
the float-float sweep to that rounding (1e-10 relative L2 per column; four
digits, ~2^-33, were 5e-10 off in 1D) and the oracle to the mixed path's 1e-8, in
1D, 2D and 3D, on chunks of points that are not multiples of the MMA's K
step, on meshes whose interface tents stay on the CUDA cores, for columns
scaled by powers of two over 27 decades and for all-zero columns."""
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


def _sweep(m, p, T, kappa, f0, tensor_cores, rhs_split=0, schedule="dataflow"):
    import torch
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, nrhs=f0.shape[0], precision="mixed",
                   rhs_split=rhs_split, schedule=schedule, tensor_cores=tensor_cores)
    s.set_state(torch.tensor(f0, device="cuda").reshape(s.front_shape()).contiguous())
    s.advance()
    front, tau = s.get_state()
    return s, front.cpu().numpy().reshape(f0.shape), tau.cpu().numpy(), s.sync_status()


def _fronts(m, p, T, kappa, inits):
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, precision="mixed")
    xq, _ = s.front_points()
    C = m.coords.shape[1] + 2
    return np.stack([f(xq).reshape(m.n_elem, -1, C) for f in inits])


@pytest.mark.parametrize("dim,nrhs,split", [(1, 32, 0), (2, 32, 0), (2, 16, 4), (3, 64, 0), (3, 32, 2)])
@pytest.mark.parametrize("schedule", ["dataflow", "levels"])
def test_tensor_cores_match_float_float_and_oracle(cuda_device, dim, nrhs, split, schedule):
    if dim == 1:
        m, p, T = inputs.mesh_interval(9), 4, 0.5
    elif dim == 2:
        m, p, T = inputs.mesh_square(5, 0.2, seed=4), 4, 0.3
    else:
        m, p, T = inputs.mesh_cube(2, 0.1, seed=4), 3, 0.1
    kappa = inputs.pitch_kappa(m)
    inits = _pulses(dim, nrhs, 17 + dim)
    f0 = _fronts(m, p, T, kappa, inits)
    s, got, tau, st = _sweep(m, p, T, kappa, f0, True, split, schedule)
    assert st == (0, 0)
    assert s.tensor_cores_used()
    s2, ref_ff, tau2, st2 = _sweep(m, p, T, kappa, f0, False, split, schedule)
    assert st2 == (0, 0)
    assert not s2.tensor_cores_used()
    assert np.array_equal(tau, tau2)
    for r in range(nrhs):
        assert _rel(got[r], ref_ff[r]) <= 1e-10, r
    r_ = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    for col in (0, nrhs - 1):
        ref, rtau = tdg.sweep(m.coords, m.elems, m.c, p, r_, inits[col], None)
        assert _rel(got[col], ref) <= 1e-8, col
    assert np.array_equal(tau, rtau)


def test_tensor_cores_with_interface_tents(cuda_device):
    """Two materials: the tents that hold both stay on the float-float sums,
    the others take the tensor cores; the sweep equals the float-float one."""
    w = inputs.workload("inclusion_small")
    m = w.mesh
    inits = _pulses(2, 32, 5)
    f0 = _fronts(m, w.p, w.T, w.kappa, inits)
    s, got, _, st = _sweep(m, w.p, w.T, w.kappa, f0, True)
    assert st == (0, 0) and s.tensor_cores_used()
    _, ref_ff, _, st2 = _sweep(m, w.p, w.T, w.kappa, f0, False)
    assert st2 == (0, 0)
    for r in range(32):
        assert _rel(got[r], ref_ff[r]) <= 1e-10, r


def test_tensor_cores_scaled_and_zero_columns(cuda_device):
    """Column r of the data is 2^-(30 (r mod 4)) times column 0, so the rows
    of the contractions span 27 decades (the digit scales are per row and per
    column), and column 31 is zero: each column equals the float-float
    sweep's to 1e-10 and the zero column stays exactly zero."""
    m = inputs.mesh_cube(2, 0.1, seed=3)
    kappa = inputs.pitch_kappa(m)
    base = _fronts(m, 3, 0.1, kappa, _pulses(3, 1, 8))[0]
    f0 = np.stack([base * 2.0 ** (-30 * (r % 4)) for r in range(32)])
    f0[31] = 0.0
    s, got, _, st = _sweep(m, 3, 0.1, kappa, f0, True)
    assert st == (0, 0) and s.tensor_cores_used()
    _, ref_ff, _, st2 = _sweep(m, 3, 0.1, kappa, f0, False)
    assert st2 == (0, 0)
    for r in range(31):
        assert _rel(got[r], ref_ff[r]) <= 1e-10, r
    assert np.all(got[31] == 0.0)
