"""Failure detection and the solver's fallback paths, exercised without any
GPU fault: a dependency wait of the dataflow sweep that runs out (a tent
made to wait, on the host, for completions that never come, with a short
poll limit) must end the sweep with TP_ERR_TIMEOUT naming that tent and
leave the context usable; the direct binary64 LU, which takes every tent
whose refinement does not settle, must meet the same parity bars when
every tent is sent to it; the solve statistics count both paths; and a
sweep resumed from a saved front and its times equals the sweep in one go."""
import numpy as np
import pytest

from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu

TP_ERR_TIMEOUT = 5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solver(w, **kw):
    import torch
    import paper_1907_02367_gb300 as pkg
    m = w.mesh
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, **kw)
    xq, _ = s.front_points()
    f0 = torch.tensor(w.init(xq), dtype=torch.float64, device="cuda").reshape(s.front_shape()).contiguous()
    gD = None
    if w.dirichlet is not None and s.n_bnd:
        xt = s.boundary_points()
        gD = torch.tensor(w.dirichlet(xt[:, :-1], xt[:, -1])[None], dtype=torch.float64, device="cuda").contiguous()
    return s, f0, gD


def test_timeout_is_reported_and_the_context_recovers(cuda_device):
    w = inputs.workload("plane1d")
    s, f0, gD = _solver(w)
    assert s.schedule()["dataflow"]
    lev = s.tents.export()["level"]
    victim = int(np.nonzero(lev == 3)[0][0])
    s.set_limits(max_polls=4096)
    s.inject_wait(victim, 1000)
    s.set_state(f0, gD)
    s.advance()
    st, info = s.sync_status()
    # the first wait to give up is the victim's or that of a tent queued after
    # it and held up by it (with the short limit both run out at about the
    # same time); no tent before the victim waits for anything that never comes
    assert st == TP_ERR_TIMEOUT and info >= victim
    # restore: the next sweep is clean and right
    s.inject_wait(victim, 0)
    s.set_limits()
    s.set_state(f0, gD)
    s.advance()
    assert s.sync_status() == (0, 0)
    got, _ = s.get_state()
    m = w.mesh
    ref, _ = tdg.sweep(m.coords, m.elems, m.c, w.p, pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T),
                       w.init, w.dirichlet)
    assert _rel(got.cpu().numpy().reshape(ref.shape), ref) <= 1e-11


def test_injection_refuses_a_tent_without_dependencies(cuda_device):
    from paper_1907_02367_gb300 import _binding as B
    w = inputs.workload("plane1d")
    s, _, _ = _solver(w)
    with pytest.raises(B.TpError) as exc:
        s.inject_wait(0, 5)                       # a level-1 tent waits for nothing
    assert exc.value.code == B.TP_ERR_ARG


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
@pytest.mark.parametrize("name", ["plane1d", "small2d", "inclusion_small", "standing3d_small"])
def test_every_tent_through_the_direct_lu(cuda_device, name, precision, tol):
    """max_refine = 0: no refinement, every tent solved by the direct binary64
    LU (with partial pivoting on Dirichlet and interface tents)."""
    w = inputs.workload(name)
    m = w.mesh
    s, f0, gD = _solver(w, precision=precision)
    s.set_limits(max_refine=0)
    s.set_state(f0, gD)
    s.advance()
    assert s.sync_status() == (0, 0)
    lu, hist = s.solve_stats()
    assert lu == s.tents.n_tents and hist.sum() == 0
    got, _ = s.get_state()
    ref, _ = tdg.sweep(m.coords, m.elems, m.c, w.p, pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T),
                       w.init, w.dirichlet)
    assert _rel(got.cpu().numpy().reshape(ref.shape), ref) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_statistics_of_the_refinement(cuda_device, precision):
    """Default limits: every tent is counted once, by the refinement (with
    the number of steps it took) or by the direct LU."""
    w = inputs.workload("standing2d")
    s, f0, gD = _solver(w, precision=precision)
    s.set_state(f0, gD)
    s.advance()
    assert s.sync_status() == (0, 0)
    lu, hist = s.solve_stats()
    assert lu + hist.sum() == s.tents.n_tents
    assert lu <= s.tents.n_tents // 100
    assert hist[:2].sum() == 0 and hist.sum() > 0          # at least two steps after the binary32 solution


def test_resume_from_a_saved_front(cuda_device):
    """Levels 1..L, state saved, a new context resumes at level L + 1: the
    final front equals the sweep in one go, bit for bit (each tent's sums run
    in a fixed order whatever the launch)."""
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload("small2d")
    s, f0, gD = _solver(w)
    s.set_state(f0, gD)
    s.advance()
    ref, tref = s.get_state()
    L = s.n_levels // 2
    s.set_state(f0, gD)
    s.advance(1, L + 1)
    mid, tmid = s.get_state()
    mid, tmid = mid.clone(), tmid.clone()
    s2, _, _ = _solver(w)
    s2.set_state(f0, gD)
    s2.set_front(mid, tmid)
    s2.advance(L + 1, s2.n_levels + 1)
    assert s2.sync_status() == (0, 0)
    got, tgot = s2.get_state()
    assert bool((tgot == tref).all())
    assert bool((got == ref).all())
