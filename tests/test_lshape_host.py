"""Host logic of the L-shape benchmark (Section 6.6, Table 1), CPU only:
the rate definition against the rates the paper prints, and the sizes of
the synthetic meshes against the paper's."""
import os

import numpy as np
import pytest

from paper_1907_02367_gb300 import inputs, lshape

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lshape_table1.txt")


def _table():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, h, dofs, err, rate, rt = line.split()
            rows.append((kind, float(h), int(dofs), float(err), None if rate == "-" else float(rate),
                         float(rt)))
    return rows


def test_dof_rate_reproduces_the_printed_rates():
    """The printed rates follow from the printed dofs and errors with the
    rate taken against dofs^(-1/3) (errors printed to 2-3 digits, so within
    3 %); taken against h_max instead they would not (graded: 5.3 vs 5.13)."""
    rows = _table()
    assert len(rows) == 8 and all(d % 16 == 0 for _, _, d, _, _, _ in rows)   # dim U^3 = 16 per tent
    for a, b in zip(rows[:-1], rows[1:]):
        if a[0] != b[0]:
            continue
        got = lshape.dof_rate(a[2], a[3], b[2], b[3])
        assert abs(got - b[4]) <= 0.03 * b[4], (a, b, got)
    g0, g1 = rows[4], rows[5]
    by_h = np.log(g0[3] / g1[3]) / np.log(g0[1] / g1[1])
    assert abs(by_h - g1[4]) > 0.1


def test_synthetic_meshes_match_the_paper_sizes(libtp):
    """The meshes of mesh_lshape at Table 1's h_max: the grading law's
    h_min, 6 n^2 triangles on the uniform ones, and a total number of dofs
    (16 per tent, the library's pitching at kappa = inputs.pitch_kappa)
    within a factor of two of the paper's at every h_max."""
    import paper_1907_02367_gb300 as pkg
    for kind, h, dofs, *_ in _table():
        mu = 1.0 if kind == "uniform" else 1.0 / 3.0
        m = inputs.mesh_lshape(h, mu)
        n = int(np.ceil(1.0 / h - 1e-9))
        assert m.meta["h_min"] == pytest.approx(h ** 3 if mu < 1 else 1.0 / n)
        if kind == "uniform":
            assert m.n_elem == 6 * n * n
        tents = pkg.Tents(m.coords, m.elems, m.c, inputs.pitch_kappa(m), 1.0)
        assert 0.5 <= 16 * tents.n_tents / dofs <= 2.0, (kind, h, 16 * tents.n_tents, dofs)


def test_stored_oracle_values_match_the_meshes_and_the_paper_trend(libtp):
    """tests/golden/lshape_oracle.json (the oracle at Table 1's sizes): the
    uniform meshes rebuild to the stored checksum, the library pitches the
    stored number of tents, and the stored errors fall at a rate near 1
    against dofs^(-1/3) on the uniform meshes, as Table 1 reports (1.26, 1.10;
    the singular solution limits it), with magnitudes within 30 % of the
    paper's (1.78e-2, 1.17e-2, 6.7e-3 at h_max = 0.07, 0.05, 0.03)."""
    import importlib.util
    import json
    import paper_1907_02367_gb300 as pkg
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("mk", os.path.join(here, "make_lshape_oracle.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(here, "lshape_oracle.json")) as f:
        stored = json.load(f)["meshes"]
    paper = {(h, kind): err for kind, h, _, err, _, _ in _table()}
    uni = []
    for g in stored:
        m = inputs.mesh_lshape(g["h_max"], g["mu"])
        if g["mu"] >= 1.0:
            assert mk.mesh_checksum(m) == g["checksum"]
        t = pkg.Tents(m.coords, m.elems, m.c, inputs.pitch_kappa(m), 1.0)
        assert t.n_tents == g["n_tents"]
        assert len(g["sample_pos"]) == len(g["sample_val"]) == mk.N_SAMPLE
        if g["mu"] >= 1.0:
            uni.append((16 * g["n_tents"], g["l2_error"]))
            ref = paper[(g["h_max"], "uniform")]
            assert 0.7 * ref <= g["l2_error"] <= 1.3 * ref, (g["h_max"], g["l2_error"], ref)
    for (d0, e0), (d1, e1) in zip(uni[:-1], uni[1:]):
        assert 0.9 <= lshape.dof_rate(d0, e0, d1, e1) <= 1.5
    # graded meshes: near the optimal rate p + 1 = 4 (Table 1 prints 5.13, 4.70, 4.21)
    gra = sorted(((16 * g["n_tents"], g["l2_error"]) for g in stored if g["mu"] < 1.0))
    assert len(gra) >= 3
    for (d0, e0), (d1, e1) in zip(gra[:-1], gra[1:]):
        assert 3.0 <= lshape.dof_rate(d0, e0, d1, e1) <= 5.5


def test_stored_oracle_values_show_the_graded_mesh_advantage():
    """Section 6.6's point, on the oracle's stored values: the mesh graded
    towards the reentrant corner (h_max = 0.12) reaches a lower L2 error than
    the finest stored uniform mesh (h_max = 0.03) with fewer than half its
    dofs."""
    import json
    with open(os.path.join(os.path.dirname(__file__), "golden", "lshape_oracle.json")) as f:
        stored = json.load(f)["meshes"]
    graded = [g for g in stored if g["mu"] < 1.0][0]
    uniform = min((g for g in stored if g["mu"] >= 1.0), key=lambda g: g["h_max"])
    assert graded["l2_error"] < uniform["l2_error"]
    assert 16 * graded["n_tents"] < 0.5 * 16 * uniform["n_tents"]
