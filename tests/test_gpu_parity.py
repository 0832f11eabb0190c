"""GPU parity: libtp's CUDA sweep against the FP64 CPU oracle.

Bar (FP64 path): relative L2 of the whole front <= 1e-11; the front times
after the sweep are bit-identical (tau = T, and every intermediate level's
tau equals the pitched t_top); exact polynomial solutions are reproduced to
rounding.  Inputs are the seeded workloads of paper_1907_02367_gb300.inputs.
"""
import math

import numpy as np
import pytest

from oracle import energy as oenergy
from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu_run(mesh, p, T, kappa, init, dirichlet, nrhs_inits=None, alpha=0.5, levels=None,
             layerwise=False, precision="fp64", schedule="dataflow", rhs_split=0):
    import torch
    import paper_1907_02367_gb300 as pkg
    inits = nrhs_inits or [init]
    s = pkg.Solver(mesh.coords, mesh.elems, mesh.c, p, T, kappa, alpha=alpha, nrhs=len(inits),
                   precision=precision, schedule=schedule, rhs_split=rhs_split)
    xq, wq = s.front_points()
    f0 = np.stack([np.asarray(f(xq)) for f in inits])
    front0 = torch.tensor(f0, dtype=torch.float64, device="cuda").contiguous()
    gD = None
    if dirichlet is not None and s.n_bnd:
        xt = s.boundary_points()
        g = np.stack([np.asarray(dirichlet(xt[:, :-1], xt[:, -1])) for _ in inits])
        gD = torch.tensor(g, dtype=torch.float64, device="cuda").contiguous()
    s.set_state(front0, gD)
    L1 = s.n_levels + 1 if levels is None else levels
    if layerwise:
        for L in range(1, L1):
            s.solve_layer(L)
    else:
        s.advance(1, L1)
    front, tau = s.get_state()
    st = s.sync_status()
    return s, front.cpu().numpy(), tau.cpu().numpy(), st


def _oracle(mesh, p, T, kappa, init, dirichlet, alpha=0.5, tent_range=None):
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, kappa, T)
    F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, init, dirichlet, alpha=alpha,
                       tent_range=tent_range)
    return F, tau, r


WORKLOADS = ["plane1d", "small2d", "standing3d_small"]


@pytest.mark.parametrize("name", WORKLOADS)
def test_sweep_matches_oracle(cuda_device, name):
    w = inputs.workload(name)
    m = w.mesh
    s, got, tau, st = _gpu_run(m, w.p, w.T, w.kappa, w.init, w.dirichlet)
    assert st == (0, 0)
    ref, rtau, _ = _oracle(m, w.p, w.T, w.kappa, w.init, w.dirichlet)
    assert np.array_equal(tau, rtau)
    rel = _rel(got.reshape(ref.shape), ref)
    assert rel <= TOL, rel


def test_full_size_2d_standing_wave(cuda_device):
    """The 2+1D p=4 workload at full size (22x22 jittered Delaunay grid,
    968 triangles, T = 1, 20216 tents), in the graph-captured launch
    configuration the benchmark times."""
    w = inputs.workload("standing2d")
    m = w.mesh
    s, got, tau, st = _gpu_run(m, w.p, w.T, w.kappa, w.init, None)
    assert st == (0, 0)
    assert s.tents.n_tents == 20216
    ref, rtau, _ = _oracle(m, w.p, w.T, w.kappa, w.init, None)
    assert np.array_equal(tau, rtau)
    rel = _rel(got.reshape(ref.shape), ref)
    assert rel <= TOL, rel
    # and against the exact solution (discretisation error, Section 6.4 shape)
    lay = tdg.front_layout(m.coords, m.elems, w.p)
    ex = w.solution(lay.xq.reshape(-1, 2), w.T).reshape(ref.shape)
    e = oenergy.error_e(got.reshape(ref.shape), ex, lay.wq, m.c)
    assert e < 1e-4


@pytest.mark.parametrize("dim,p,which,cval", [(1, 3, 1, 1.0), (1, 6, 0, 2.0), (2, 4, 1, 1.0),
                                              (2, 5, 0, 0.5), (3, 3, 1, 1.0), (3, 2, 0, 1.7)])
def test_polynomial_reproduction(cuda_device, dim, p, which, cval):
    mesh = {1: inputs.mesh_interval(6), 2: inputs.mesh_square(3, 0.2, seed=5),
            3: inputs.mesh_cube(1, 0.0, seed=3)}[dim]
    mesh.c[:] = cval
    base = inputs.polynomial_solution(dim, which)

    def sol(x, t):
        out = base(x, cval * np.asarray(t, dtype=np.float64))
        out[:, 1] *= cval
        return out

    T = 0.3 / cval
    s, got, tau, st = _gpu_run(mesh, p, T, inputs.pitch_kappa(mesh), lambda x: sol(x, 0.0),
                               lambda x, t: sol(x, t)[:, 1])
    assert st == (0, 0)
    xq, _ = s.front_points()
    ex = sol(xq, T)
    assert np.abs(got.reshape(ex.shape) - ex).max() <= 1e-11 * max(1.0, np.abs(ex).max())


def test_front_points_match_oracle_layout(cuda_device):
    import paper_1907_02367_gb300 as pkg
    for m, p in [(inputs.mesh_interval(5), 3), (inputs.mesh_square(4, 0.2, seed=1), 4),
                 (inputs.mesh_cube(2, 0.1, seed=2), 3)]:
        s = pkg.Solver(m.coords, m.elems, m.c, p, 0.1, inputs.pitch_kappa(m))
        xq, wq = s.front_points()
        lay = tdg.front_layout(m.coords, m.elems, p)
        assert np.allclose(xq, lay.xq.reshape(-1, m.dim), rtol=0, atol=1e-15)
        assert np.allclose(wq, lay.wq.reshape(-1), rtol=1e-13, atol=0)


def test_layerwise_equals_graph(cuda_device):
    """tp_solve_layer level by level equals the per-level graph bit for bit."""
    w = inputs.workload("small2d")
    m = w.mesh
    _, a, ta, _ = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, schedule="levels")
    _, b, tb, _ = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, layerwise=True)
    assert np.array_equal(a, b) and np.array_equal(ta, tb)


@pytest.mark.parametrize("name,precision", [("small2d", "fp64"), ("standing2d", "fp64"),
                                            ("standing3d_small", "fp64"), ("inclusion_small", "fp64"),
                                            ("standing2d", "mixed")])
def test_dataflow_matches_levels(cuda_device, name, precision):
    """The persistent dataflow sweep (clusters of fixed size pulling tents as
    their inputs complete) gives the per-level result up to rounding (the
    slicing of a tent over its cluster differs), identical front times, and
    repeated sweeps are reproducible."""
    w = inputs.workload(name)
    m = w.mesh
    _, a, ta, sa = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, schedule="levels", precision=precision)
    _, b, tb, sb = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, schedule="dataflow", precision=precision)
    _, c, tc, sc = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, schedule="dataflow", precision=precision)
    assert sa == sb == sc == (0, 0)
    assert np.array_equal(ta, tb) and np.array_equal(tb, tc)
    # the two schedules slice a tent's points differently over its cluster, so
    # the sums are taken in another order: rounding of binary64, or of the
    # compensated float-float sums of the mixed path (~1e-13 relative)
    assert _rel(b, a) <= (1e-13 if precision == "fp64" else 1e-11)
    assert np.array_equal(b, c)


def test_partial_sweep_and_energy_on_curved_front(cuda_device):
    """Stop after some levels (front not flat): fronts, times and the energy
    flux through the front match the oracle run over the same tents."""
    import torch
    w = inputs.workload("small2d")
    m = w.mesh
    L = 7
    s, got, tau, st = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, levels=L)
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    ntent = int(np.sum(r["level"] < L))
    ref, rtau = tdg.sweep(m.coords, m.elems, m.c, w.p, r, w.init, None, tent_range=(0, ntent))
    assert np.array_equal(tau, rtau)
    assert np.any(tau < w.T) and np.any(tau > 0)
    assert _rel(got.reshape(ref.shape), ref) <= TOL
    E = s.energy().cpu().numpy()
    lay = tdg.front_layout(m.coords, m.elems, w.p)
    Eref = oenergy.front_energy(ref, lay.wq, m.c, oenergy.element_gradients(m.coords, m.elems, rtau))
    assert abs(E[0] - Eref) <= 1e-12 * abs(Eref)


def test_energy_flat_front_and_dissipation(cuda_device):
    """Section 6.5 model problem U = sin(pi x) sin(pi t), 5 elements: the GPU
    energy at T matches the oracle's and lies below the initial energy."""
    mesh = inputs.mesh_interval(5)
    pi = math.pi

    def sol(x, t):
        x = np.asarray(x).reshape(-1)
        t = np.broadcast_to(t, x.shape)
        return np.stack([np.sin(pi * x) * np.sin(pi * t), pi * np.sin(pi * x) * np.cos(pi * t),
                         -pi * np.cos(pi * x) * np.sin(pi * t)], axis=1)

    s, got, tau, st = _gpu_run(mesh, 4, 1.0, 0.9, lambda x: sol(x, 0.0), None)
    E = float(s.energy().cpu().numpy()[0])
    ref, _, _ = _oracle(mesh, 4, 1.0, 0.9, lambda x: sol(x, 0.0), None)
    lay = tdg.front_layout(mesh.coords, mesh.elems, 4)
    Eref = oenergy.front_energy(ref, lay.wq, mesh.c)
    E0 = oenergy.front_energy(sol(lay.xq.reshape(-1, 1), 0.0).reshape(ref.shape), lay.wq, mesh.c)
    assert abs(E - Eref) <= 1e-12 * Eref
    assert E < E0


def test_many_rhs_each_equals_single(cuda_device):
    m = inputs.mesh_square(4, 0.2, seed=6)
    kappa = inputs.pitch_kappa(m)
    inits = [inputs.gaussian_pulse((0.4, 0.5), 0.2), inputs.gaussian_pulse((0.6, 0.3), 0.15),
             lambda x: inputs.standing_wave_2d(x, 0.0), inputs.gaussian_pulse((0.5, 0.5), 0.3),
             inputs.gaussian_pulse((0.3, 0.7), 0.25)]
    s, got, tau, st = _gpu_run(m, 3, 0.3, kappa, None, None, nrhs_inits=inits)
    assert st == (0, 0)
    got = got.reshape(len(inits), m.n_elem, -1, 4)
    for r, f in enumerate(inits):
        ref, _, _ = _oracle(m, 3, 0.3, kappa, f, None)
        assert _rel(got[r], ref) <= TOL, r


@pytest.mark.parametrize("case", ["one_element_1d", "two_triangles", "one_level"])
def test_degenerate_meshes(cuda_device, case):
    if case == "one_element_1d":
        m, p, T, kappa = inputs.mesh_interval(1), 3, 0.7, 0.9
        sol = inputs.plane_wave_1d
    elif case == "two_triangles":
        m, p, T = inputs.mesh_square(1, 0.0, seed=1), 4, 0.4
        kappa = inputs.pitch_kappa(m)
        sol = inputs.standing_wave_2d
    else:
        m, p, T, kappa = inputs.mesh_interval(8), 5, 1e-3, 0.9
        sol = inputs.plane_wave_1d
    init = lambda x: sol(x, 0.0)
    dfun = lambda x, t: sol(x, t)[:, 1]
    s, got, tau, st = _gpu_run(m, p, T, kappa, init, dfun)
    assert st == (0, 0)
    ref, rtau, _ = _oracle(m, p, T, kappa, init, dfun)
    assert np.array_equal(tau, rtau)
    assert _rel(got.reshape(ref.shape), ref) <= TOL


def test_non_causal_pitch_is_reported(cuda_device):
    """kappa = 1 in 1D gives characteristic top faces (c|g| = 1, not
    space-like, Section 2.2): the kernel reports TP_ERR_CAUSALITY."""
    m = inputs.mesh_interval(4)
    s, got, tau, st = _gpu_run(m, 3, 0.5, 1.0, lambda x: inputs.plane_wave_1d(x, 0.0), None)
    assert st[0] == 2


# ---------------------------------------------------------------------------
# mixed path: float-float assembly, binary32 factorisation + refinement;
# bar: relative L2 <= 1e-8 against the FP64 oracle
# ---------------------------------------------------------------------------
MIXED_TOL = 1e-8


@pytest.mark.parametrize("name", WORKLOADS)
def test_mixed_sweep_matches_oracle(cuda_device, name):
    w = inputs.workload(name)
    m = w.mesh
    s, got, tau, st = _gpu_run(m, w.p, w.T, w.kappa, w.init, w.dirichlet, precision="mixed")
    assert st == (0, 0)
    ref, rtau, _ = _oracle(m, w.p, w.T, w.kappa, w.init, w.dirichlet)
    assert np.array_equal(tau, rtau)
    rel = _rel(got.reshape(ref.shape), ref)
    assert rel <= MIXED_TOL, rel


def test_mixed_full_size_2d(cuda_device):
    w = inputs.workload("standing2d")
    m = w.mesh
    s, got, tau, st = _gpu_run(m, w.p, w.T, w.kappa, w.init, None, precision="mixed")
    assert st == (0, 0)
    ref, rtau, _ = _oracle(m, w.p, w.T, w.kappa, w.init, None)
    rel = _rel(got.reshape(ref.shape), ref)
    assert rel <= MIXED_TOL, rel


@pytest.mark.parametrize("dim,p,which,cval", [(1, 5, 1, 2.0), (2, 4, 1, 1.0), (2, 5, 0, 0.5),
                                              (3, 3, 1, 1.0)])
def test_mixed_polynomial_reproduction(cuda_device, dim, p, which, cval):
    mesh = {1: inputs.mesh_interval(6), 2: inputs.mesh_square(3, 0.2, seed=5),
            3: inputs.mesh_cube(1, 0.0, seed=3)}[dim]
    mesh.c[:] = cval
    base = inputs.polynomial_solution(dim, which)

    def sol(x, t):
        out = base(x, cval * np.asarray(t, dtype=np.float64))
        out[:, 1] *= cval
        return out

    T = 0.3 / cval
    s, got, tau, st = _gpu_run(mesh, p, T, inputs.pitch_kappa(mesh), lambda x: sol(x, 0.0),
                               lambda x, t: sol(x, t)[:, 1], precision="mixed")
    assert st == (0, 0)
    xq, _ = s.front_points()
    ex = sol(xq, T)
    assert np.abs(got.reshape(ex.shape) - ex).max() <= 1e-9 * max(1.0, np.abs(ex).max())


def test_mixed_many_rhs(cuda_device):
    m = inputs.mesh_square(4, 0.2, seed=6)
    kappa = inputs.pitch_kappa(m)
    inits = [inputs.gaussian_pulse((0.4, 0.5), 0.2), lambda x: inputs.standing_wave_2d(x, 0.0),
             inputs.gaussian_pulse((0.6, 0.3), 0.15)]
    s, got, tau, st = _gpu_run(m, 3, 0.3, kappa, None, None, nrhs_inits=inits, precision="mixed")
    assert st == (0, 0)
    got = got.reshape(len(inits), m.n_elem, -1, 4)
    for r, f in enumerate(inits):
        ref, _, _ = _oracle(m, 3, 0.3, kappa, f, None)
        assert _rel(got[r], ref) <= MIXED_TOL, r


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", MIXED_TOL)])
def test_many_rhs_3d(cuda_device, precision, tol):
    """Thirty-two Gaussian pulses (seeded centres and widths) advanced together
    in 3D at p = 3, sharing every tent's factorisation (the shape of the
    many-right-hand-side target configuration), all in one CTA per slice of
    points (rhs_split = 1; 32 is the most one CTA's shared memory holds at
    p = 3 in 3D); columns against the oracle."""
    m = inputs.mesh_cube(2, 0.1, seed=4)
    kappa = inputs.pitch_kappa(m)
    rng = np.random.default_rng(44)
    inits = [inputs.gaussian_pulse(rng.uniform(0.25, 0.75, 3), rng.uniform(0.15, 0.3)) for _ in range(32)]
    s, got, tau, st = _gpu_run(m, 3, 0.1, kappa, None, None, nrhs_inits=inits, precision=precision,
                               rhs_split=1)
    assert st == (0, 0)
    got = got.reshape(len(inits), m.n_elem, -1, 5)
    for r in (0, 17, 31):
        ref, _, _ = _oracle(m, 3, 0.1, kappa, inits[r], None)
        assert _rel(got[r], ref) <= tol, r


@pytest.mark.parametrize("precision,tol,schedule", [("fp64", TOL, "dataflow"), ("mixed", MIXED_TOL, "dataflow"),
                                                     ("fp64", TOL, "levels")])
def test_many_rhs_3d_in_groups(cuda_device, precision, tol, schedule):
    """Sixty-four Gaussian pulses in 3D at p = 3 kept together in each CTA
    (rhs_split = 1): more right-hand sides than one CTA's shared memory
    holds, so the library sweeps them in two groups of 32 from the same
    front times; columns of both groups against the oracle, and the front
    times after the sweep are the pitched ones.  The default (the 64 split
    over clusters of 4 CTAs of 16, one group) is checked the same way."""
    m = inputs.mesh_cube(2, 0.1, seed=4)
    kappa = inputs.pitch_kappa(m)
    rng = np.random.default_rng(44)
    inits = [inputs.gaussian_pulse(rng.uniform(0.25, 0.75, 3), rng.uniform(0.15, 0.3)) for _ in range(64)]
    for split in (1, 0):
        s, got, tau, st = _gpu_run(m, 3, 0.1, kappa, None, None, nrhs_inits=inits, precision=precision,
                                   schedule=schedule, rhs_split=split)
        assert st == (0, 0)
        got = got.reshape(len(inits), m.n_elem, -1, 5)
        for r in (0, 31, 32, 63):
            ref, tau_ref, _ = _oracle(m, 3, 0.1, kappa, inits[r], None)
            assert _rel(got[r], ref) <= tol, (split, r)
        assert np.array_equal(tau, tau_ref)


def test_autotune_keeps_results(cuda_device):
    """tp_autotune restores the state it found and the schedule it picks
    reproduces the oracle."""
    import torch
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload("small2d")
    m = w.mesh
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa)
    xq, _ = s.front_points()
    f0 = torch.tensor(w.init(xq), device="cuda").reshape(s.front_shape()).contiguous()
    s.set_state(f0)
    chosen, ms = s.autotune()
    assert chosen in (0, 1, 2, 4, 8) and ms > 0
    before, tau0 = s.get_state()
    assert torch.equal(before, f0) and float(tau0.abs().max()) == 0.0
    s.advance()
    got, tau = s.get_state()
    ref, rtau, _ = _oracle(m, w.p, w.T, w.kappa, w.init, None)
    assert np.array_equal(tau.cpu().numpy(), rtau)
    assert _rel(got.cpu().numpy().reshape(ref.shape), ref) <= TOL


def test_more_than_four_materials_is_refused_cleanly(cuda_device):
    """The per-element log-normal medium gives tents with up to 8 speeds;
    tp_create refuses it with TP_ERR_UNSUPPORTED before any device work,
    and the library stays usable for the next context."""
    import paper_1907_02367_gb300 as pkg
    from paper_1907_02367_gb300 import _binding as B
    w = inputs.workload("lognormal2d")
    m = w.mesh
    with pytest.raises(B.TpError) as exc:
        pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa)
    assert exc.value.code == B.TP_ERR_UNSUPPORTED and "materials" in str(exc.value)
    s = inputs.workload("small2d")
    ok = pkg.Solver(s.mesh.coords, s.mesh.elems, s.mesh.c, s.p, s.T, s.kappa)
    assert ok.n_levels > 0


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", MIXED_TOL)])
@pytest.mark.parametrize("name", ["small2d", "inclusion_small"])
def test_penalty_alpha_other_than_half(cuda_device, name, precision, tol):
    """alpha = 1.3 (eq. 2.5) instead of the paper's 0.5, on the Dirichlet
    walls and, for the inclusion, the interface jumps of v; against the
    oracle with the same alpha (alpha moves the oracle's fronts by 1e-4 and
    8e-2 relative on these two workloads)."""
    w = inputs.workload(name)
    m = w.mesh
    dfun = (lambda x, t: w.solution(x, t)[:, 1]) if w.solution is not None else None
    s, got, tau, st = _gpu_run(m, w.p, w.T, w.kappa, w.init, dfun, alpha=1.3, precision=precision)
    assert st == (0, 0)
    ref, tau_ref, _ = _oracle(m, w.p, w.T, w.kappa, w.init, dfun, alpha=1.3)
    assert np.array_equal(tau, tau_ref)
    assert _rel(got.reshape(ref.shape), ref) <= tol
