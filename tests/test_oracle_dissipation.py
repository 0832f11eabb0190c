"""Pins of oracle.energy.tent_dissipation (the jump terms of eq. 2.5 / 4.1
tested with the tent's own solution, Section 6.5): summed over a sweep they
must close the energy balance E(T) = E(0) - sum D exactly (to rounding),
where E is the flux of 1/2 (c^-2 v^2 + |sigma|^2) - v sigma.grad tau through
the final front.  The balance is a theorem of the method (the Trefftz tent
conserves energy in its interior), so a dropped term, a wrong sign or a
wrong penalty in D breaks it; the cases cover every term: the bottom jump
and the recovery term, Dirichlet walls with and without data, Neumann walls
with and without data, interface facets between two speeds, 1D/2D/3D."""
import numpy as np
import pytest

from oracle import energy, pitching, tdg
from paper_1907_02367_gb300 import inputs


def _balance(mesh, p, T, init, kappa=None, **kw):
    kappa = kappa if kappa is not None else inputs.pitch_kappa(mesh)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, kappa, T)
    lay = tdg.front_layout(mesh.coords, mesh.elems, p)
    f0 = np.asarray(init(lay.xq.reshape(-1, mesh.dim))).reshape(lay.wq.shape + (mesh.dim + 2,))
    E0 = energy.front_energy(f0, lay.wq, mesh.c)
    F, tau, D, per = energy.sweep_dissipation(mesh.coords, mesh.elems, mesh.c, p, r, init, **kw)
    E1 = energy.front_energy(F, lay.wq, mesh.c, energy.element_gradients(mesh.coords, mesh.elems, tau))
    return E0, E1, D, per


def _neumann_half(m):
    bnd = np.zeros((m.n_elem, m.dim + 1), np.int8)
    bnd[m.coords[m.elems].mean(axis=1)[:, 0] < 0.5] = 1
    return bnd


def _gN(x, t, n):
    return np.sin(2.0 * x[:, 0] + x[:, 1]) * (1.0 + t) * np.atleast_2d(n)[:, 0]


CASES = {
    "2d_dirichlet": lambda: (inputs.workload("small2d").mesh, 3, 0.2, inputs.workload("small2d").init, {}),
    "1d_dirichlet_data": lambda: (inputs.workload("plane1d").mesh, 3, 0.3, inputs.workload("plane1d").init,
                                  {"kappa": 0.9, "dirichlet": inputs.workload("plane1d").dirichlet}),
    "2d_interface": lambda: (inputs.workload("inclusion_small").mesh, 3, 0.1,
                             inputs.workload("inclusion_small").init, {}),
    "2d_neumann_data": lambda: (inputs.mesh_square(4, 0.2, seed=6), 3, 0.2, inputs.gaussian_pulse((0.4, 0.5), 0.2),
                                {"bnd_type": _neumann_half(inputs.mesh_square(4, 0.2, seed=6)), "neumann": _gN,
                                 "beta": 1.7}),
    "3d_dirichlet": lambda: (inputs.mesh_cube(2, 0.1, seed=4), 2, 0.1, inputs.gaussian_pulse((0.5, 0.45, 0.5), 0.3),
                             {}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_energy_balance_closes(case):
    mesh, p, T, init, kw = CASES[case]()
    E0, E1, D, per = _balance(mesh, p, T, init, **kw)
    assert D > 0.0
    assert abs(E1 - (E0 - D)) <= 1e-12 * E0, (E0, E1, D)


def test_exact_solution_loses_nothing_in_interior_tents():
    """An exact polynomial solution in the Trefftz space is reproduced by every
    tent (Section 3), so in a tent away from the boundary the bottom jump and
    the recovery term vanish: D = 0 to rounding (a D that kept any of the
    data's own energy would not vanish)."""
    mesh = inputs.mesh_square(3, 0.2, seed=5)
    base = inputs.polynomial_solution(2, 1)
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), 0.2)
    bverts = {int(a) for (f, _, _) in tdg.boundary_facets(mesh.coords, mesh.elems) for a in f}
    interior = []

    def rec(it, d):
        if d["v"] not in bverts:
            interior.append(energy.tent_dissipation(mesh.coords, mesh.elems, mesh.c, 4, d))

    tdg.sweep(mesh.coords, mesh.elems, mesh.c, 4, r, lambda x: base(x, 0.0), lambda x, t: base(x, t)[:, 1],
              record=rec)
    assert len(interior) >= 4
    assert max(abs(d) for d in interior) <= 1e-12


@pytest.mark.parametrize("drop", ["alpha", "recovery", "interface_beta"])
def test_balance_fails_when_a_term_is_dropped(drop, monkeypatch):
    """The pin is sharp: dropping one term of D leaves a visible gap."""
    if drop == "interface_beta":
        mesh, p, T, init, kw = CASES["2d_interface"]()
        kw = dict(kw, beta=0.0)                   # D computed without the [[sigma]] term, the sweep with it

        def sweep_diss(*a, **k):
            per = []

            def rec(it, d):
                per.append(energy.tent_dissipation(mesh.coords, mesh.elems, mesh.c, p, d, 0.5, 0.0))

            F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, a[4], a[5], None, record=rec)
            return F, tau, float(np.sum(per)), per

        monkeypatch.setattr(energy, "sweep_dissipation", sweep_diss)
        E0, E1, D, _ = _balance(mesh, p, T, init)
    elif drop == "alpha":
        mesh, p, T, init, kw = CASES["2d_dirichlet"]()
        r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
        lay = tdg.front_layout(mesh.coords, mesh.elems, p)
        per = []
        F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, init, None, record=lambda it, d: per.append(
            energy.tent_dissipation(mesh.coords, mesh.elems, mesh.c, p, d, alpha=0.0)))
        f0 = np.asarray(init(lay.xq.reshape(-1, 2))).reshape(lay.wq.shape + (4,))
        E0 = energy.front_energy(f0, lay.wq, mesh.c)
        E1 = energy.front_energy(F, lay.wq, mesh.c, energy.element_gradients(mesh.coords, mesh.elems, tau))
        D = float(np.sum(per))
    else:
        mesh, p, T, init, kw = CASES["2d_dirichlet"]()
        E0, E1, D, per = _balance(mesh, p, T, init)
        # the recovery part alone, recomputed from the oracle's records, taken out of D
        r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
        lay = tdg.front_layout(mesh.coords, mesh.elems, p)
        rec_sum = [0.0]

        def rec(it, d):
            B, nb = d["basis"], d["basis"].nb
            for k in d["patch"]:
                g = d["groups"][k]
                tb = d["tau_before"][mesh.elems[k]]
                U, _, _ = B.eval_phys(lay.xq[k], lay.bary @ tb, d["xc"], d["tc"], d["h"], d["speeds"][g])
                Uh = U @ d["x"][g * nb:(g + 1) * nb]
                rec_sum[0] += float(np.sum(lay.wq[k] * (Uh - d["front_before"][k][:, 0]) * Uh))

        tdg.sweep(mesh.coords, mesh.elems, mesh.c, p, r, init, None, record=rec)
        D -= rec_sum[0]
    assert abs(E1 - (E0 - D)) > 1e-8 * E0
