"""GPU parity on the L-shaped domain of Section 6.6 (a reentrant corner, the
singular solution cos(10 t) sin(2 phi / 3) J_2/3(10 r) as initial and
Dirichlet data, p = 3, T = 1): the front after the sweep against the
oracle element by element on a graded and a uniform mesh, and the rows of
the Table 1 study (tents, dofs, L2 error at T) against the oracle's."""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

from oracle import pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu

P, T = 3, 1.0


def _sol():
    return inputs.bessel_corner_solution(10.0, 2.0 / 3.0)


def _oracle(mesh):
    sol = _sol()
    r = pitching.pitch(mesh.coords, mesh.elems, mesh.c, inputs.pitch_kappa(mesh), T)
    F, tau = tdg.sweep(mesh.coords, mesh.elems, mesh.c, P, r, lambda x: sol(x, 0.0),
                       lambda x, t: sol(x, t)[:, 1])
    lay = tdg.front_layout(mesh.coords, mesh.elems, P)
    ex = sol(lay.xq.reshape(-1, 2), T)[:, 0]
    err = math.sqrt(float(np.sum(lay.wq.reshape(-1) * (F[..., 0].reshape(-1) - ex) ** 2)))
    return F, tau, err, r


def _gpu(mesh, precision):
    front, tau, status, _, _ = _gpu_full(mesh, precision)
    return front, tau, status


def _gpu_full(mesh, precision):
    import torch
    import paper_1907_02367_gb300 as pkg
    sol = _sol()
    s = pkg.Solver(mesh.coords, mesh.elems, mesh.c, P, T, inputs.pitch_kappa(mesh), precision=precision)
    xq, _ = s.front_points()
    f0 = torch.tensor(sol(xq, 0.0)[None], dtype=torch.float64, device="cuda").contiguous()
    xt = s.boundary_points()
    gD = torch.tensor(sol(xt[:, :-1], xt[:, -1])[:, 1][None], dtype=torch.float64,
                      device="cuda").contiguous()
    s.set_state(f0, gD)
    s.advance()
    front, tau = s.get_state()
    xq, wq = s.front_points()
    return front.cpu().numpy(), tau.cpu().numpy(), s.sync_status(), xq, wq


@pytest.mark.parametrize("h_max,mu,precision,tol", [
    (0.35, 1.0 / 3.0, "fp64", 1e-11),
    (0.35, 1.0 / 3.0, "mixed", 1e-8),
    (0.125, 1.0, "fp64", 1e-11),
    (0.125, 1.0, "mixed", 1e-8),
])
def test_lshape_bessel_matches_oracle(cuda_device, h_max, mu, precision, tol):
    mesh = inputs.mesh_lshape(h_max, mu)
    got, tau, st = _gpu(mesh, precision)
    assert st == (0, 0)
    ref, tau_ref, _, _ = _oracle(mesh)
    assert np.array_equal(tau, tau_ref)
    rel = float(np.linalg.norm(got.reshape(ref.shape) - ref) / np.linalg.norm(ref))
    assert rel <= tol, rel


def test_lshape_study_rows_match_oracle(cuda_device):
    """lshape.study on two uniform meshes and one graded one: tents and
    dofs equal the oracle's pitching, the L2 error equals the oracle's, and
    the error falls from the coarser uniform mesh to the finer one."""
    from paper_1907_02367_gb300 import lshape
    cases = [(0.25, 1.0), (0.125, 1.0), (0.5, 1.0 / 3.0)]
    rows = lshape.study(uniform=(0.25, 0.125), graded=(0.5,), p=P, T=T, repeats=1)
    assert len(rows) == 3
    for row, (h, mu) in zip(rows, cases):
        _, _, err, r = _oracle(inputs.mesh_lshape(h, mu))
        assert row["status"] == [0, 0]
        assert row["n_tents"] == len(r["level"])
        assert row["dofs"] == 16 * len(r["level"])
        assert abs(row["l2_error"] - err) <= 1e-7, (row["l2_error"], err)
    assert rows[1]["l2_error"] < rows[0]["l2_error"] and rows[1]["dof_rate"] > 0
    assert rows[0]["dof_rate"] is None and rows[2]["dof_rate"] is None


GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_maker():
    spec = importlib.util.spec_from_file_location(
        "make_lshape_oracle", os.path.join(GOLDEN_DIR, "make_lshape_oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stored():
    with open(os.path.join(GOLDEN_DIR, "lshape_oracle.json")) as f:
        return json.load(f)["meshes"]


@pytest.mark.parametrize("precision,tol,err_tol", [("fp64", 1e-11, 1e-9), ("mixed", 1e-8, 1e-6)])
@pytest.mark.parametrize("idx", range(len(_stored())))
def test_lshape_table1_sizes_match_stored_oracle(cuda_device, idx, precision, tol, err_tol):
    """At the mesh sizes of the paper's Table 1 (uniform h_max = 0.07, 0.05,
    0.03 and graded 0.12, 0.10, 0.08, 0.06; 13 000 to 520 000 tents) the oracle takes minutes,
    so its results are stored (tests/golden/make_lshape_oracle.py): the
    binary64 and mixed sweeps match them at 256 seeded front entries (the
    relative L2 error over the sample within the parity bound 1e-11 / 1e-8,
    and every sampled entry within the bound times the sample's largest
    entry), in the front's norm and in the L2 error of U at T.  A graded mesh that this platform triangulates
    differently (its point set has mirror symmetry, so Delaunay has ties)
    cannot be compared and is skipped."""
    mk = _golden_maker()
    g = _stored()[idx]
    mesh = inputs.mesh_lshape(g["h_max"], g["mu"])
    if mk.mesh_checksum(mesh) != g["checksum"]:
        assert g["mu"] < 1.0, "the uniform meshes are built without ties and must match"
        pytest.skip("graded mesh triangulated differently from the stored one")
    front, tau, st, xq, wq = _gpu_full(mesh, precision)
    assert st == (0, 0)
    assert np.all(tau == T)
    flat = front.reshape(-1)
    pos = np.asarray(g["sample_pos"])
    ref = np.asarray(g["sample_val"])
    assert np.linalg.norm(flat[pos] - ref) <= tol * np.linalg.norm(ref)
    assert np.max(np.abs(flat[pos] - ref)) <= tol * np.max(np.abs(ref))
    assert abs(float(np.linalg.norm(flat)) - g["front_norm"]) <= tol * g["front_norm"]
    ex = _sol()(xq, T)[:, 0]
    err = math.sqrt(float(np.sum(wq * (front.reshape(len(wq), -1)[:, 0] - ex) ** 2)))
    assert abs(err - g["l2_error"]) <= err_tol, (err, g["l2_error"])
