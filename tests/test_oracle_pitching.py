"""Pins for oracle/pitching.py.

* 1D closed form: on a uniform mesh with c = 1 the first round pitches the
  even vertices to delta = kappa*h, every later round pitches the other
  parity to (previous front) + delta, capped at T, and level = round;
* invariants of Section 2.2 on 2D/3D meshes: after every level the front is
  space-like (c_K |grad tau| < 1 on every element), neighbouring front times
  differ by at most the edge limit, tents of one level are independent,
  times increase, and the sweep ends with tau = T everywhere.
"""
import numpy as np
import pytest

from oracle import pitching
from paper_1907_02367_gb300 import inputs


def test_1d_closed_form():
    n_el, kappa, T = 16, 0.9, 1.0
    m = inputs.mesh_interval(n_el)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    h = m.coords[1, 0] - m.coords[0, 0]
    delta = (kappa * np.sqrt(h * h)) / 1.0
    # expected: round r pitches parity (r+1) % 2 ... even first
    tau = np.zeros(n_el + 1)
    exp = []
    rnd = 0
    while np.any(tau < T):
        rnd += 1
        par = (rnd + 1) % 2            # round 1 -> even
        for v in range(par, n_el + 1, 2):
            nb = [w for w in (v - 1, v + 1) if 0 <= w <= n_el]
            tt = min([T] + [tau[w] + delta for w in nb])
            exp.append((rnd, rnd, v, tau[v], tt))
        for (_, _, v, _, tt) in exp[-len(range(par, n_el + 1, 2)):]:
            tau[v] = tt
    exp.sort()
    assert r["n_levels"] == rnd == 19
    assert len(r["vert"]) == len(exp) == 162
    assert np.array_equal(r["level"], [e[0] for e in exp])
    assert np.array_equal(r["vert"], [e[2] for e in exp])
    assert np.array_equal(r["t_bot"], [e[3] for e in exp])       # bit-exact
    assert np.array_equal(r["t_top"], [e[4] for e in exp])


def _replay_and_check(mesh, kappa, T):
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, kappa, T)
    nv = mesh.n_vert
    nbrs = pitching.vertex_neighbours(mesh.elems, nv)
    ce = pitching.mesh_edges(mesh.elems, mesh.c)
    tau = np.zeros(nv)
    lam = np.zeros(nv, dtype=int)
    X = mesh.coords[mesh.elems]
    J = X[:, 1:, :] - X[:, :1, :]
    Jinv = np.linalg.inv(J)
    worst = 0.0
    for L in range(1, r["n_levels"] + 1):
        sel = np.nonzero(r["level"] == L)[0]
        vs = r["vert"][sel]
        # independence: no two tents of a level are neighbours (share an element)
        sv = set(vs.tolist())
        assert len(sv) == len(vs)
        for v in vs:
            assert not (set(nbrs[v]) & sv)
        for i in sel:
            v = r["vert"][i]
            assert r["t_bot"][i] == tau[v]
            assert r["t_top"][i] > r["t_bot"][i]
            assert r["level"][i] == 1 + max([lam[v]] + [lam[w] for w in nbrs[v]])
            tau[v] = r["t_top"][i]
            lam[v] = L
        # front after the level: edge limit and space-like faces
        for (a, b), cc in ce.items():
            d = (kappa * pitching.edge_length(mesh.coords[a], mesh.coords[b])) / cc
            assert abs(tau[a] - tau[b]) <= d * (1 + 1e-14)
        tv = tau[mesh.elems]
        g = np.einsum("eij,ej->ei", Jinv, tv[:, 1:] - tv[:, :1])
        slope = mesh.c * np.linalg.norm(g, axis=1)
        worst = max(worst, float(slope.max()))
        assert np.all(slope < 1.0)
    assert np.all(tau == T)
    return r, worst


@pytest.mark.parametrize("nx,seed", [(4, 1), (7, 3)])
def test_invariants_2d(nx, seed):
    m = inputs.mesh_square(nx, 0.2, seed=seed)
    kappa = inputs.pitch_kappa(m)
    r, worst = _replay_and_check(m, kappa, 0.5)
    assert worst <= 0.9 + 1e-12


def test_invariants_3d():
    m = inputs.mesh_cube(2, 0.1, seed=4)
    kappa = inputs.pitch_kappa(m)
    r, worst = _replay_and_check(m, kappa, 0.3)
    assert worst <= 0.9 + 1e-12


def test_kappa_one_is_not_space_like_in_1d():
    """kappa = 1 in 1D makes the tent faces characteristic (c|g| = 1)."""
    m = inputs.mesh_interval(4)
    r = pitching.pitch(m.coords, m.elems, m.c, 1.0, 0.5)
    h = 0.25
    assert np.isclose(r["t_top"][0], h)       # slope exactly 1 / c


def test_heterogeneous_speed_uses_edge_max():
    m = inputs.mesh_interval(4)
    m.c[:] = [1.0, 3.0, 3.0, 1.0]
    r = pitching.pitch(m.coords, m.elems, m.c, 0.9, 1.0)
    # vertex 0: edge (0,1) touches only element 0 (c = 1): delta = 0.9*0.25
    # vertex 2: edges touch elements 1 and 2 (c = 3): delta = 0.9*0.25/3
    first = {int(v): float(t) for v, t, L in zip(r["vert"], r["t_top"], r["level"]) if L == 1}
    assert first[0] == (0.9 * 0.25) / 1.0
    assert first[2] == (0.9 * 0.25) / 3.0


def test_invariants_2d_heterogeneous():
    """An edge between a slow and a fast element is limited by the fast speed,
    so every front stays space-like on both (c_K |grad tau|_K < 1, Section 2.2).
    In 1D every edge is one element, so only 2D/3D meshes tell max from min."""
    m = inputs.mesh_square(6, 0.2, seed=3)
    cen = m.coords[m.elems].mean(axis=1)
    m.c[:] = np.where(np.linalg.norm(cen - 0.5, axis=1) < 0.3, 3.0, 1.0)
    r, worst = _replay_and_check(m, inputs.pitch_kappa(m), 0.3)
    assert worst <= 0.9 + 1e-12


def test_truncated_pitch_is_a_prefix_of_the_full_pitch():
    """pitch(..., max_level=L) stops early and returns exactly the tents of
    level <= L of the full pitch, in the same order (graded inclusion mesh at
    h_max = 0.05: tents of very different heights, many rounds)."""
    m = inputs.mesh_inclusion_graded(h_max=0.05)
    kappa = inputs.pitch_kappa(m)
    full = pitching.pitch(m.coords, m.elems, m.c, kappa, 0.05)
    for L in (1, 2, 5):
        part = pitching.pitch(m.coords, m.elems, m.c, kappa, 0.05, max_level=L)
        n = int(np.sum(full["level"] <= L))
        assert len(part["vert"]) == n > 0
        for key in ("vert", "t_bot", "t_top", "level", "round"):
            assert np.array_equal(part[key], full[key][:n]), key
        assert part["n_rounds"] <= full["n_rounds"]
        if L == 1:
            assert part["n_rounds"] < full["n_rounds"]
