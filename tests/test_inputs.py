"""The seeded input generators (CPU): the graded inclusion mesh of the 2+1D
heterogeneous configuration is a conforming counter-clockwise triangulation
of the unit square, graded about ten times finer at the circle, with the jump
of c along element edges."""
import numpy as np
import pytest

from paper_1907_02367_gb300 import inputs

pytest.importorskip("scipy")


@pytest.fixture(scope="module")
def graded():
    return inputs.mesh_inclusion_graded()


def test_graded_inclusion_mesh_is_a_conforming_triangulation(graded):
    m = graded
    P, T = m.coords, m.elems
    assert 19000 <= m.n_elem <= 23000
    a = (P[T[:, 1], 0] - P[T[:, 0], 0]) * (P[T[:, 2], 1] - P[T[:, 0], 1]) - \
        (P[T[:, 2], 0] - P[T[:, 0], 0]) * (P[T[:, 1], 1] - P[T[:, 0], 1])
    assert np.all(a > 0)                                   # counter-clockwise, none degenerate
    assert abs(0.5 * a.sum() - 1.0) < 1e-12                # covers the unit square
    edges = {}
    for t in T.tolist():
        for k in range(3):
            e = tuple(sorted((t[k], t[(k + 1) % 3])))
            edges[e] = edges.get(e, 0) + 1
    assert set(edges.values()) <= {1, 2}                   # conforming
    for (i, j), cnt in edges.items():
        if cnt == 1:                                       # boundary edges lie on the square's sides
            x = P[[i, j]]
            assert np.any(np.all(np.isclose(x, 0.0), axis=0) | np.all(np.isclose(x, 1.0), axis=0))


def test_graded_inclusion_mesh_grading_and_materials(graded):
    m = graded
    P, T = m.coords, m.elems
    assert set(np.unique(m.c)) == {1.0, 3.0}
    cen = P[T].mean(axis=1)
    r = np.hypot(cen[:, 0] - 0.5, cen[:, 1] - 0.5)
    assert np.all((r < 0.2) == (m.c == 3.0))
    L = np.stack([np.linalg.norm(P[T[:, k]] - P[T[:, (k + 1) % 3]], axis=1) for k in range(3)], 1).max(1)
    near = np.abs(r - 0.2) < 0.005
    far = np.abs(r - 0.2) > 0.15
    assert near.sum() > 100 and far.sum() > 1000
    assert np.median(L[far]) / np.median(L[near]) > 6.0   # about ten times finer at the circle
    assert m.n_elem == inputs.mesh_inclusion_graded().n_elem   # seeded: the same mesh again
