"""Pins of oracle.energy.probe_values (point outputs U_h(x_j, t_k), the
ingredient of Section 6.7's U_C(t)): an exact polynomial solution in the
Trefftz space is reproduced by every tent, so every sample must equal the
exact U at its point and time whatever tent it falls in; every sample must
be taken by exactly one tent; and the assignment must follow the fronts
(a sample at t = 0 is in a first-level tent, one at T in a tent whose top
reaches T)."""
import numpy as np

from oracle import energy, pitching
from paper_1907_02367_gb300 import inputs


def test_probes_reproduce_an_exact_solution_and_cover_every_sample():
    mesh = inputs.mesh_square(3, 0.2, seed=5)
    base = inputs.polynomial_solution(2, 1)
    T, p = 0.25, 4
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.05, 0.95, (12, 2))
    times = np.concatenate([[0.0], np.sort(rng.uniform(0.0, T, 9)), [T]])
    vals, owner = energy.probe_values(mesh.coords, mesh.elems, mesh.c, p, r, lambda x: base(x, 0.0), pts, times,
                                      dirichlet=lambda x, t: base(x, t)[:, 1])
    assert np.all(owner >= 0)
    for kt, t in enumerate(times):
        ex = base(pts, np.full(len(pts), t))[:, 0]
        assert np.abs(vals[kt] - ex).max() <= 1e-11 * max(1.0, np.abs(ex).max())
    lev = np.asarray(r["level"])
    assert np.all(lev[owner[0]] == 1) or np.all(np.asarray(r["t_bot"])[owner[0]] == 0.0)
    assert np.all(np.asarray(r["t_top"])[owner[-1]] == T)


def test_probe_owner_brackets_the_sample_in_time():
    """A sample's tent starts at or below it and ends above it at the sample's vertex time range."""
    w = inputs.workload("inclusion_small")
    m = w.mesh
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    pts = np.array([[0.31, 0.47], [0.52, 0.5], [0.77, 0.21]])
    times = np.linspace(0.0, w.T, 7)[:-1] + 0.003
    vals, owner = energy.probe_values(m.coords, m.elems, m.c, w.p, r, w.init, pts, times)
    assert np.all(owner >= 0) and np.all(np.isfinite(vals))
    tb, tt = np.asarray(r["t_bot"]), np.asarray(r["t_top"])
    assert np.all(tb[owner] <= times[:, None] + 1e-15)
    assert np.all(tt[owner] > times[:, None] - 1e-15)
