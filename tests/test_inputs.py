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


def _edges(T):
    edges = {}
    for t in T.tolist():
        for k in range(3):
            e = tuple(sorted((t[k], t[(k + 1) % 3])))
            edges[e] = edges.get(e, 0) + 1
    return edges


def _on_lshape_boundary(x):
    """Both end points on one straight side of [-1,1]^2 minus (0,1]x[-1,0)."""
    ax = np.all(np.isclose(x[:, 0], x[0, 0])) and (np.isclose(abs(x[0, 0]), 1.0) or
                                                   (np.isclose(x[0, 0], 0.0) and np.all(x[:, 1] <= 0)))
    ay = np.all(np.isclose(x[:, 1], x[0, 1])) and (np.isclose(abs(x[0, 1]), 1.0) or
                                                   (np.isclose(x[0, 1], 0.0) and np.all(x[:, 0] >= 0)))
    return bool(ax or ay)


@pytest.mark.parametrize("h_max,mu", [(0.25, 1.0), (0.07, 1.0), (0.4, 1.0 / 3.0), (0.12, 1.0 / 3.0)])
def test_lshape_mesh_is_a_conforming_triangulation(h_max, mu):
    """Section 6.6's domain: counter-clockwise triangles covering area 3,
    every edge in one or two triangles, boundary edges on the L's sides,
    every vertex used, the reentrant corner a vertex."""
    m = inputs.mesh_lshape(h_max, mu)
    P, T = m.coords, m.elems
    a = (P[T[:, 1], 0] - P[T[:, 0], 0]) * (P[T[:, 2], 1] - P[T[:, 0], 1]) - \
        (P[T[:, 2], 0] - P[T[:, 0], 0]) * (P[T[:, 1], 1] - P[T[:, 0], 1])
    assert np.all(a > 0)
    assert abs(0.5 * a.sum() - 3.0) < 1e-12
    cen = P[T].mean(axis=1)
    assert not np.any((cen[:, 0] > 0) & (cen[:, 1] < 0))
    edges = _edges(T)
    assert set(edges.values()) <= {1, 2}
    blen = 0.0
    for (i, j), cnt in edges.items():
        if cnt == 1:
            assert _on_lshape_boundary(P[[i, j]]), P[[i, j]]
            blen += float(np.linalg.norm(P[i] - P[j]))
    assert abs(blen - 8.0) < 1e-12                     # perimeter of the L
    assert np.unique(T).size == m.n_vert
    assert np.any(np.all(P == 0.0, axis=1))


def test_lshape_uniform_mesh_size():
    """mu = 1: 6 n^2 congruent right isosceles triangles with legs 1/n."""
    m = inputs.mesh_lshape(0.07, 1.0)
    n = 15
    assert m.n_elem == 6 * n * n
    X = m.coords[m.elems]
    L = np.sort(np.stack([np.linalg.norm(X[:, k] - X[:, (k + 1) % 3], axis=1) for k in range(3)], 1), 1)
    assert np.allclose(L[:, :2], 1.0 / n) and np.allclose(L[:, 2], np.sqrt(2.0) / n)


@pytest.mark.parametrize("h_max", [0.12, 0.06])
def test_lshape_graded_mesh_follows_the_grading_law(h_max):
    """Section 6.6: h_K ~ h_max r^(1 - mu), mu = 1/3, smallest size
    h_min = h_max^3 at the corner: element diameters within a fixed factor
    of that law, the corner's triangles of size ~h_min, and a bounded shape
    (smallest angle above 20 degrees)."""
    mu = 1.0 / 3.0
    m = inputs.mesh_lshape(h_max, mu)
    P, T = m.coords, m.elems
    X = P[T]
    L = np.stack([np.linalg.norm(X[:, k] - X[:, (k + 1) % 3], axis=1) for k in range(3)], 1)
    diam = L.max(axis=1)
    r = np.linalg.norm(X, axis=2).max(axis=1)              # farthest vertex from the corner
    law = np.maximum(h_max * r ** (1.0 - mu), h_max ** (1.0 / mu))
    ratio = diam / law
    assert 0.4 < ratio.min() and ratio.max() < 2.5, (ratio.min(), ratio.max())
    at_corner = np.any(T == int(np.nonzero(np.all(P == 0.0, axis=1))[0][0]), axis=1)
    assert np.all(diam[at_corner] < 3.0 * h_max ** 3)
    cosang = []
    for k in range(3):
        u = X[:, (k + 1) % 3] - X[:, k]
        v = X[:, (k + 2) % 3] - X[:, k]
        cosang.append(np.einsum("ed,ed->e", u, v) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1)))
    assert np.degrees(np.arccos(np.max(cosang))) > 20.0
    assert np.array_equal(inputs.mesh_lshape(h_max, mu).elems, T)   # the same mesh again


def test_bessel_corner_solution_is_a_wave():
    """U = cos(a t) sin(nu phi) J_nu(a r): v = U_t, sigma = -grad U and
    U_tt = Lap U (c = 1) by central differences away from the corner; U and
    v vanish on both cut edges; sigma grows like r^(nu - 1) at the corner."""
    sol = inputs.bessel_corner_solution(10.0, 2.0 / 3.0)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (400, 2))
    x = x[~((x[:, 0] > 0) & (x[:, 1] < 0)) & (np.hypot(x[:, 0], x[:, 1]) > 0.05)]
    t = rng.uniform(0, 1, len(x))
    F = sol(x, t)
    U = lambda y, s: sol(y, s)[:, 0]                       # noqa: E731
    h = 1e-5
    ex, ey = np.array([h, 0.0]), np.array([0.0, h])
    assert np.allclose((U(x, t + h) - U(x, t - h)) / (2 * h), F[:, 1], atol=1e-5)
    assert np.allclose(-(U(x + ex, t) - U(x - ex, t)) / (2 * h), F[:, 2], atol=1e-5)
    assert np.allclose(-(U(x + ey, t) - U(x - ey, t)) / (2 * h), F[:, 3], atol=1e-5)
    h = 1e-3
    ex, ey = np.array([h, 0.0]), np.array([0.0, h])
    utt = (U(x, t + h) - 2 * U(x, t) + U(x, t - h)) / h ** 2
    lap = (U(x + ex, t) + U(x - ex, t) + U(x + ey, t) + U(x - ey, t) - 4 * U(x, t)) / h ** 2
    assert np.abs(utt - lap).max() < 1e-3 * np.abs(utt).max()
    s = np.linspace(0.05, 1.0, 7)
    cut = np.concatenate([np.stack([0 * s, -s], 1), np.stack([s, 0 * s], 1),
                          np.stack([0 * s + 1e-17, -s], 1), np.stack([s, 0 * s - 1e-17], 1)])
    assert np.abs(sol(cut, 0.37)[:, :2]).max() < 1e-14
    g = [np.linalg.norm(sol(np.array([[-rr, rr]]) / np.sqrt(2), 0.0)[0, 2:]) for rr in (1e-4, 1e-6)]
    assert abs(np.log(g[1] / g[0]) / np.log(1e-2) - (2.0 / 3.0 - 1.0)) < 1e-3


def test_sine_product_1d_is_a_wave_with_constant_energy():
    x = np.linspace(0.0, 1.0, 2001)
    h = 1e-5
    for t in (0.0, 0.3, 7.1):
        F = inputs.sine_product_1d(x, t)
        U = lambda y, s: inputs.sine_product_1d(y, s)[:, 0]    # noqa: E731
        assert np.allclose((U(x, t + h) - U(x, t - h)) / (2 * h), F[:, 1], atol=1e-6)
        assert np.allclose(-(U(x + h, t) - U(x - h, t)) / (2 * h), F[:, 2], atol=1e-6)
        dens = 0.5 * (F[:, 1] ** 2 + F[:, 2] ** 2)
        E = float(np.sum(0.5 * (dens[1:] + dens[:-1])) * (x[1] - x[0]))
        assert abs(E - np.pi ** 2 / 4) < 1e-6
        assert abs(F[0, 1]) < 1e-15 and abs(F[-1, 1]) < 1e-12


def test_lognormal_speeds_exceed_four_materials_per_star():
    """The adjoint configuration's medium: c_K = exp(N(-0.045, 0.3^2)) per
    element has mean about 1, and more than 90 % of the vertex stars hold
    more than 4 distinct speeds (the most one tent of the library holds),
    up to 8."""
    w = inputs.workload("lognormal2d")
    m = w.mesh
    assert m.n_elem == 20000 and abs(m.c.mean() - 1.0) < 0.02
    star = [[] for _ in range(m.n_vert)]
    for k, el in enumerate(m.elems.tolist()):
        for v in el:
            star[v].append(k)
    nmat = np.array([len(set(m.c[s].tolist())) for s in star])
    assert np.mean(nmat > 4) > 0.9 and nmat.max() <= 8
