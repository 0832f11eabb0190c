"""The two large mixed-precision workloads at full size, element by element.

* Graded inclusion (21 054 triangles, 10x finer at the circle, c = 3 / 1,
  p = 5, T = 2; 19.7 million tents in 97 363 levels): the oracle pitches the
  first levels (oracle.pitching with max_level: the first tents of its full
  pitch, in the same order) and sweeps them level by level on all host cores
  (oracle.parallel); the library advances the same levels; every front entry
  the levels touched is compared, in binary64 and in the mixed path.  The
  whole sweep to T = 2 runs too: clean status, every front time at T, the
  energy falls, and the energy balance E(T) = E(0) - D closes on the GPU.
* 3+1D many right-hand sides (48 000 tetrahedra, p = 3, 64 seeded Gaussian
  pulses sharing the tent matrices): levels 1-2 (3076 tents), three columns
  against the oracle element by element, binary64 and mixed.

Bars: binary64 1e-11 relative L2, mixed 1e-8, over the touched entries.
At p = 5 the oracle solves each tent system with extended-precision
refinement (the plain binary64 LU leaves ~1e-11 of its own there)."""
import os

import numpy as np
import pytest

from oracle import parallel, pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu

NPROC = min(16, os.cpu_count() or 1)


def _touched(m, r, L):
    """Elements in the patches of the tents of levels <= L."""
    star = tdg.vertex_star(m.elems, m.n_vert)
    lev = np.asarray(r["level"])
    return np.array(sorted({k for v in np.asarray(r["vert"])[lev <= L] for k in star[int(v)]}))


def _gpu_levels(m, p, T, kappa, inits, L, precision, tents=None, nrhs=None):
    import torch
    import paper_1907_02367_gb300 as pkg
    s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, nrhs=len(inits), precision=precision, tents=tents)
    xq, _ = s.front_points()
    f0 = torch.empty(s.front_shape(), dtype=torch.float64, device="cuda")
    for r, f in enumerate(inits):
        f0[r].copy_(torch.from_numpy(np.ascontiguousarray(f(xq))).reshape(f0.shape[1:]))
    s.set_state(f0)
    s.advance(1, L + 1)
    assert s.sync_status() == (0, 0)
    front, tau = s.get_state()
    return s, front.cpu().numpy(), tau.cpu().numpy()


def _check(got, ref, touched, tol, what):
    g, f = got[touched], ref[touched]
    rel = np.linalg.norm(g - f) / np.linalg.norm(f)
    assert rel <= tol, (what, rel)
    # and no element hides a large local error: per element, relative to the largest element
    per = np.linalg.norm((g - f).reshape(len(touched), -1), axis=1)
    assert per.max() <= tol * np.linalg.norm(f.reshape(len(touched), -1), axis=1).max() * 10.0, what


@pytest.fixture(scope="module")
def graded_oracle():
    w = inputs.workload("inclusion_graded")
    m = w.mesh
    L = 4
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T, max_level=L)
    lay = tdg.front_layout(m.coords, m.elems, w.p)
    f0 = np.asarray(w.init(lay.xq.reshape(-1, 2))).reshape(lay.wq.shape + (4,))
    F, tau, done = parallel.sweep_levels(m.coords, m.elems, m.c, w.p, r, f0, L, nproc=NPROC, refine=True)
    return w, r, L, F, tau, done


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_graded_inclusion_first_levels_elementwise(cuda_device, graded_oracle, precision, tol):
    w, r, L, F, tau_ref, done = graded_oracle
    m = w.mesh
    assert done == len(r["vert"]) > 10000
    s, got, tau = _gpu_levels(m, w.p, w.T, w.kappa, [w.init], L, precision)
    assert int(np.sum(s.tents.export()["level"] <= L)) == done
    assert np.array_equal(tau, tau_ref)
    _check(got[0], F, _touched(m, r, L), tol, precision)


def test_graded_inclusion_whole_sweep(cuda_device):
    import torch
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload("inclusion_graded")
    m = w.mesh
    tents = pkg.Tents(m.coords, m.elems, m.c, w.kappa, w.T)
    assert tents.n_tents == 19661640 and tents.n_levels == 97363
    fronts = {}
    for precision in ("fp64", "mixed"):
        s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, tents=tents, precision=precision,
                       track_dissipation=True)
        xq, _ = s.front_points()
        s.set_state(torch.tensor(w.init(xq)[None], dtype=torch.float64, device="cuda").contiguous())
        E0 = float(s.energy()[0])
        s.advance()
        E1, D = (float(v) for v in s.energy_and_dissipation()[0])
        front, tau = s.get_state()
        assert s.sync_status() == (0, 0)
        assert bool(torch.all(tau == w.T))
        assert 0.0 < E1 < E0
        assert abs(E1 - (E0 - D)) <= 1e-9 * E0, (precision, E0, E1, D)
        fronts[precision] = front.cpu().numpy()
        del s
    rel = np.linalg.norm(fronts["mixed"] - fronts["fp64"]) / np.linalg.norm(fronts["fp64"])
    assert rel <= 1e-8, rel


@pytest.fixture(scope="module")
def many_rhs_oracle():
    w = inputs.workload("many_rhs_3d")
    m = w.mesh
    L = 2
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T, max_level=L)
    lay = tdg.front_layout(m.coords, m.elems, w.p)
    pulses = inputs.gaussian_pulses_3d()
    cols = (0, 37, 63)
    out = {}
    for col in cols:
        f0 = np.asarray(pulses[col](lay.xq.reshape(-1, 3))).reshape(lay.wq.shape + (5,))
        out[col] = parallel.sweep_levels(m.coords, m.elems, m.c, w.p, r, f0, L, nproc=NPROC)
    return w, r, L, pulses, out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_many_rhs_3d_first_levels_elementwise(cuda_device, many_rhs_oracle, precision, tol):
    w, r, L, pulses, ref = many_rhs_oracle
    m = w.mesh
    s, got, tau = _gpu_levels(m, w.p, w.T, w.kappa, pulses, L, precision)
    touched = _touched(m, r, L)
    for col, (F, tau_ref, done) in ref.items():
        assert done == len(r["vert"]) == 3076
        assert np.array_equal(tau, tau_ref)
        _check(got[col], F, touched, tol, (precision, col))
