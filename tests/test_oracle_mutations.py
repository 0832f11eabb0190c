"""The oracle's pins catch plausible mistakes (CPU, oracle only).

Each case plants one mistake in a copy of an oracle module (the text of the
module with one expression changed, loaded as a separate module), points the
pin tests at the copy, and checks that at least one pin fails.  The planted
mistakes are the kinds the pins are chosen against: a flipped sign, a dropped
term, a dropped wave speed, a wrong index or gradient, a transposed operand,
an off-by-one in the recursion eq. (3.1) or in the quadrature.
"""
from __future__ import annotations

import importlib.util
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, HERE)

import oracle.adjoint  # noqa: E402
import oracle.tdg  # noqa: E402
import test_oracle_adjoint as Az  # noqa: E402
import test_oracle_basis as Bz  # noqa: E402
import test_oracle_basis_variants as Vz  # noqa: E402
import test_oracle_dissipation as Dz  # noqa: E402
import test_oracle_pitching as Pz  # noqa: E402
import test_oracle_quadrature as Qz  # noqa: E402
import test_oracle_tdg as Tz  # noqa: E402


def _mutant(name: str, old: str, new: str):
    # (the basis-variant pins take mutants of oracle/basis.py)
    path = os.path.join(ROOT, "oracle", {"basis_variants": "basis"}.get(name, name) + ".py")
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site not unique in oracle/{name}.py: {old!r}"
    spec = importlib.util.spec_from_loader(f"oracle._mutant_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), f"{path} (mutant)", "exec"), mod.__dict__)
    return mod


TDG_PINS = [
    lambda: Tz.test_polynomial_reproduction(1, 3, 1),
    lambda: Tz.test_polynomial_reproduction(2, 3, 1),
    lambda: Tz.test_polynomial_reproduction_wave_speed(1, 3, 1, 2.5),
    lambda: Tz.test_polynomial_reproduction_wave_speed(2, 3, 1, 0.4),
    lambda: Tz.test_energy_identity_1d_with_dirichlet(2),
    lambda: Tz.test_energy_identity_2d_interior(),
    lambda: Tz.test_interface_reproduction(1, 2, 1.0, 2.5),
    lambda: Tz.test_interface_reproduction(2, 2, 1.0, 3.0),
    lambda: Tz.test_interface_energy_identity_1d(),
    lambda: Tz.test_polynomial_reproduction_with_neumann_faces(2, 3, 1),
    lambda: Tz.test_tent_matrix_symmetric_part_positive_definite(2, 3, True),
    lambda: Tz.test_energy_identity_1d_with_neumann(3, 1.7),
]
BASIS_PINS = [
    lambda: Bz.test_trefftz_property_exact(2, 3),
    lambda: Bz.test_trefftz_property_exact(3, 3),
    lambda: Bz.test_derivative_tables_fd(2, 4),
] + TDG_PINS
VARIANT_PINS = [
    lambda: Vz.test_legendre_and_chebyshev_polynomials_exact(),
    lambda: Vz.test_every_start_gives_trefftz_functions_of_the_same_space("legendre", 2, 4),
    lambda: Vz.test_every_start_gives_trefftz_functions_of_the_same_space("chebyshev", 3, 3),
]
QUAD_PINS = [
    lambda: Qz.test_simplex_moments_exact(2, 3),
    lambda: Qz.test_simplex_moments_exact(3, 3),
]
PITCH_PINS = [
    lambda: Pz.test_1d_closed_form(),
    lambda: Pz.test_invariants_2d(4, 1),
    lambda: Pz.test_heterogeneous_speed_uses_edge_max(),
    lambda: Pz.test_invariants_2d_heterogeneous(),
]
ENERGY_PINS = [
    lambda: Tz.test_energy_through_a_curved_front_is_conserved_for_exact_solutions(2.0),
    lambda: Tz.test_energy_decreases_1d(),
    lambda: Dz.test_energy_balance_closes("1d_dirichlet_data"),
    lambda: Dz.test_energy_balance_closes("2d_interface"),
    lambda: Dz.test_energy_balance_closes("2d_neumann_data"),
]
ADJ_PINS = [
    lambda: Az.test_dot_product_identity(1),
    lambda: Az.test_dot_product_identity(2),
    lambda: Az.test_misfit_gradient_finite_differences(),
    lambda: Az.test_speed_gradient_closed_form(),
    lambda: Az.test_speed_gradient_two_materials_matches_swept_difference(),
    lambda: Az.test_global_space_time_solve_equals_sweep(*Az.GLOBAL_CASES[1]),
    lambda: Az.test_speed_gradient_transposed_system_equals_swept_difference(2),
    lambda: Az.test_multi_material_adjoint_dot_product_and_whole_system("2d_two_materials"),
    lambda: Az.test_multi_material_adjoint_dot_product_and_whole_system("2d_neumann_two_materials"),
    lambda: Az.test_per_material_speed_gradient_two_routes("1d_per_element"),
]

# (id, oracle module, original text, planted text)
MUTATIONS = [
    ("tdg-top-sign", "tdg", "Ak -= (w[:, None] * Sgt).T @ Vt", "Ak += (w[:, None] * Sgt).T @ Vt"),
    ("tdg-drop-recovery-lhs", "tdg", "Ak += (w[:, None] * Ub).T @ Ub", "Ak += 0.0 * (w[:, None] * Ub).T @ Ub"),
    ("tdg-drop-recovery-rhs", "tdg", "bk += (w * Uf) @ Ub", "bk += 0.0 * (w * Uf) @ Ub"),
    ("tdg-dirichlet-penalty-sign", "tdg", "Sn + alpha * Vd)", "Sn - alpha * Vd)"),
    ("tdg-drop-c", "tdg", "c2 = 1.0 / (ck * ck)", "c2 = 1.0"),
    ("tdg-top-gradient-in-bottom-data", "tdg", 'Sgb = np.einsum("qdj,d->qj", Sb, g_b)',
     'Sgb = np.einsum("qdj,d->qj", Sb, g_t)'),
    ("tdg-interface-side-sign", "tdg", "0.5 * st * (", "0.5 * ss * ("),
    ("tdg-interface-beta-sign", "tdg", "+ beta * np.einsum", "- beta * np.einsum"),
    ("tdg-neumann-coupling-sign", "tdg", "wf, Sn, Vd + beta * Sn", "wf, Sn, -Vd + beta * Sn"),
    ("tdg-neumann-penalty-sign", "tdg", "wf, Sn, Vd + beta * Sn", "wf, Sn, Vd - beta * Sn"),
    ("tdg-neumann-data-sign", "tdg", "beta * Sn - Vd)", "beta * Sn + Vd)"),
    ("tdg-neumann-penalty-scale", "tdg", "wf, Sn, Vd + beta * Sn", "wf, Sn, Vd + 2.0 * beta * Sn"),
    ("basis-recursion-denominator", "basis", "c2 / (k * (k - 1)) * s", "c2 / (k * (k + 1)) * s"),
    ("basis-recursion-factor", "basis", "(alpha[m] + 1) * (alpha[m] + 2) * prev",
     "(alpha[m] + 1) * (alpha[m] + 1) * prev"),
    ("basis-derivative-exponent", "basis", "f = float(e[var])", "f = float(e[var] - 1)"),
    ("basis-drop-c-in-map", "basis", "return U, (c / h) * Ut, -(1.0 / h) * G",
     "return U, (1.0 / h) * Ut, -(1.0 / h) * G"),
    ("basis-sigma-sign", "basis", "return U, (c / h) * Ut, -(1.0 / h) * G",
     "return U, (c / h) * Ut, (1.0 / h) * G"),
    ("quad-jacobi-exponent", "quadrature", "gauss_jacobi01(m, n - 1 - d)", "gauss_jacobi01(m, n - d)"),
    ("quad-weight-scale", "quadrature", "w / 2.0 ** (a + 1)", "w / 2.0 ** a"),
    ("quad-collapse-map", "quadrature", "scale *= (1.0 - xi[d])", "scale *= xi[d]"),
    ("pitch-edge-min-speed", "pitching", "ck > ce[key]", "ck < ce[key]"),
    ("pitch-level-ignores-neighbours", "pitching", "level = 1 + max([lam[v]] + [lam[w] for w in nbr[v]])",
     "level = 1 + lam[v]"),
    ("energy-gradient-term-sign", "energy", "dens = dens - 2.0 * v", "dens = dens + 2.0 * v"),
    ("energy-drop-c", "energy", "v * v / (c[:, None] ** 2)", "v * v"),
    ("adjoint-untransposed-solve", "adjoint", "mu = np.linalg.solve(A.T, Em.T @ lt)",
     "mu = np.linalg.solve(A, Em.T @ lt)"),
    ("adjoint-bottom-sign", "adjoint", "(w[:, None] * (c2 * Vb - Sgb)).T", "(w[:, None] * (c2 * Vb + Sgb)).T"),
    ("adjoint-speed-step-not-relative", "adjoint", "(2.0 * rel_step * cm)", "(2.0 * rel_step)"),
    ("adjoint-speed-moves-every-material", "adjoint",
     "cp[c == cm] = cm * (1.0 + sgn * rel_step)\n            F, _ = _tdg.sweep",
     "cp[:] = c * (1.0 + sgn * rel_step)\n            F, _ = _tdg.sweep"),
    ("adjoint-transposed-moves-every-material", "adjoint",
     "cp[c == cm] = cm * (1.0 + j * rel_step)",
     "cp[:] = c * (1.0 + j * rel_step)"),
    ("adjoint-transposed-stencil-weight", "adjoint", "(-sys_[2][i] + 8.0 * sys_[1][i]", "(-sys_[2][i] + 7.0 * sys_[1][i]"),
    ("adjoint-speed-one-sided", "adjoint", "(J[0] - J[1]) / (2.0", "(J[0] - J[1]) / (1.0"),
    ("adjoint-global-coupling-sign", "adjoint", "M[rows, off[tp]:off[tp + 1]] -= Bm[:, cols] @ Ep",
     "M[rows, off[tp]:off[tp + 1]] += Bm[:, cols] @ Ep"),
    ("adjoint-interface-side-sign", "adjoint", "A[blk] += 0.5 * st * (", "A[blk] += 0.5 * ss * ("),
    ("adjoint-neumann-coupling-sign", "adjoint", "wf, Sn, Vd + beta * Sn", "wf, Sn, -Vd + beta * Sn"),
    ("adjoint-top-map-sigma-dropped", "adjoint", "Em[j, :, 2:, blk] = St", "Em[j, :, 2:, blk] = 0.0 * St"),
    ("energy-diss-recovery-dropped", "energy", "(U - fb[:, 0]) * U", "0.0 * U"),
    ("energy-diss-dirichlet-data-sign", "energy", "gd * (alpha * V - sn)", "gd * (alpha * V + sn)"),
    ("energy-diss-neumann-data-sign", "energy", "gn * (beta * sn - V)", "gn * (beta * sn + V)"),
    ("energy-diss-interface-beta-dropped", "energy", "+ beta * dsn * dsn", "+ 0.0 * dsn * dsn"),
    ("energy-diss-bottom-gradient-sign", "energy", "- 2.0 * dv * (ds @ gb)", "+ 2.0 * dv * (ds @ gb)"),
    ("adjoint-global-stale-front", "adjoint", "            last[K] = (it, Em[j * blk:(j + 1) * blk, :])",
     "            last[K] = last[K] or (it, Em[j * blk:(j + 1) * blk, :])"),
    ("adjoint-transposed-gradient-sign", "adjoint", "y @ (dR @ f0 - dM @ x)", "y @ (dR @ f0 + dM @ x)"),
    ("basis-legendre-recursion-sign", "basis_variants",
     "(Fraction(2 * j + 1) * xp[i] - Fraction(j) * prev[i]) / (j + 1)",
     "(Fraction(2 * j + 1) * xp[i] + Fraction(j) * prev[i]) / (j + 1)"),
    ("basis-chebyshev-recursion-factor", "basis_variants",
     "P.append([2 * xp[i] - prev[i] for i in range(j + 2)])", "P.append([xp[i] - prev[i] for i in range(j + 2)])"),
    ("basis-tensor-product-factor-dropped", "basis_variants",
     "new.get(key + (e,), Fraction(0)) + v * cf", "new.get(key + (e,), Fraction(0)) + cf"),
]


def _install(monkeypatch, name, mod):
    if name == "tdg":
        monkeypatch.setattr(Tz, "tdg", mod)
        return TDG_PINS
    if name == "basis":
        monkeypatch.setattr(Bz, "bz", mod)
        monkeypatch.setattr(oracle.tdg, "_basis", mod)
        return BASIS_PINS
    if name == "basis_variants":
        monkeypatch.setattr(Vz, "ob", mod)
        monkeypatch.setattr(oracle.tdg, "_basis", mod)
        return VARIANT_PINS
    if name == "quadrature":
        monkeypatch.setattr(Qz, "q", mod)
        return QUAD_PINS
    if name == "pitching":
        monkeypatch.setattr(Pz, "pitching", mod)
        return PITCH_PINS
    if name == "energy":
        monkeypatch.setattr(Tz, "energy", mod)
        monkeypatch.setattr(Dz, "energy", mod)
        return ENERGY_PINS
    if name == "adjoint":
        monkeypatch.setattr(Az, "adjoint", mod)
        return ADJ_PINS
    raise KeyError(name)


@pytest.mark.parametrize("mid,name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(monkeypatch, mid, name, old, new):
    pins = _install(monkeypatch, name, _mutant(name, old, new))
    caught = []
    for i, pin in enumerate(pins):
        try:
            with np.errstate(all="ignore"):
                pin()
        except (AssertionError, np.linalg.LinAlgError):
            caught.append(i)
            break
    assert caught, f"no pin fails for the planted mistake {mid}"


@pytest.mark.parametrize("name", ["tdg", "basis", "basis_variants", "quadrature", "pitching", "energy", "adjoint"])
def test_unplanted_copy_passes_every_pin(monkeypatch, name):
    """The loader itself changes nothing: an unmodified copy passes the pins."""
    pins = _install(monkeypatch, name, _mutant(name, "from __future__ import annotations",
                                              "from __future__ import annotations"))
    for pin in pins:
        pin()
