"""Seeded synthetic workloads for the tent-pitched Trefftz-DG solver.

This module only builds inputs: spatial meshes, the wave speed per element,
the pitching parameter kappa, and closed-form solutions of the acoustic wave
equation (first-order fields v = dU/dt, sigma = -grad U, Section 2.1, eq. 2.2)
used as initial and Dirichlet data.  It contains none of the method's own
arithmetic (no quadrature, no Trefftz basis, no pitching, no tent system);
both the CUDA library and the CPU oracle consume what it returns.

Workloads (Section 6 of the paper; sizes as stated in each generator):
  * 1+1D: interval [0,1], uniform elements, plane wave sin(pi(x-t)).
  * 2+1D: unit square, jittered grid made Delaunay by Lawson flips,
    standing wave cos(sqrt2 pi t) sin(pi x) sin(pi y)  (Section 6.4 shape).
  * 3+1D: unit cube, jittered hex grid, six Kuhn tetrahedra per hex,
    Gaussian pulses with v0 = 0.
  * 2+1D L-shape (Section 6.6): uniform and corner-graded meshes of
    [-1,1]^2 minus [0,1]x[-1,0], singular solution cos(10t) sin(2phi/3) J_2/3(10r).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    """A simplicial mesh: coords (n_vert, dim) float64, elems (n_elem, dim+1)
    int32 vertex ids, c (n_elem,) float64 wave speed per element."""
    coords: np.ndarray
    elems: np.ndarray
    c: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    @property
    def n_vert(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.elems.shape[0])


# ----------------------------------------------------------------------------
# 1D
# ----------------------------------------------------------------------------
def mesh_interval(n_el: int, a: float = 0.0, b: float = 1.0, c: float = 1.0) -> Mesh:
    """Uniform partition of [a, b] into n_el elements."""
    x = np.array([a + (b - a) * i / n_el for i in range(n_el + 1)], dtype=np.float64)
    x[-1] = b
    elems = np.stack([np.arange(n_el), np.arange(1, n_el + 1)], axis=1).astype(np.int32)
    return Mesh(x[:, None].copy(), elems, np.full(n_el, c, dtype=np.float64),
                name=f"interval{n_el}")


# ----------------------------------------------------------------------------
# 2D: jittered grid + Lawson flips to a Delaunay triangulation
# ----------------------------------------------------------------------------
def _orient2(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def _incircle(a, b, c, d):
    """> 0 iff d lies strictly inside the circumcircle of CCW triangle abc."""
    m = np.array([[a[0] - d[0], a[1] - d[1], (a[0] - d[0]) ** 2 + (a[1] - d[1]) ** 2],
                  [b[0] - d[0], b[1] - d[1], (b[0] - d[0]) ** 2 + (b[1] - d[1]) ** 2],
                  [c[0] - d[0], c[1] - d[1], (c[0] - d[0]) ** 2 + (c[1] - d[1]) ** 2]])
    return float(np.linalg.det(m))


def lawson_delaunay(coords: np.ndarray, tris: np.ndarray, max_pass: int = 200) -> np.ndarray:
    """Flip interior edges until every edge is locally Delaunay.

    Deterministic: each pass visits edges in sorted order."""
    tris = [list(t) for t in tris]
    for t in tris:
        if _orient2(coords[t[0]], coords[t[1]], coords[t[2]]) < 0:
            t[1], t[2] = t[2], t[1]
    for _ in range(max_pass):
        edge_map: dict = {}
        for ti, t in enumerate(tris):
            for k in range(3):
                a, b = t[k], t[(k + 1) % 3]
                edge_map.setdefault((min(a, b), max(a, b)), []).append(ti)
        flipped = False
        touched = set()
        for e in sorted(edge_map):
            ts = edge_map[e]
            if len(ts) != 2 or ts[0] in touched or ts[1] in touched:
                continue
            t1, t2 = tris[ts[0]], tris[ts[1]]
            # rotate t1 so that it reads (a, b, c) with edge a->b
            for k in range(3):
                if {t1[k], t1[(k + 1) % 3]} == set(e):
                    a, b, c = t1[k], t1[(k + 1) % 3], t1[(k + 2) % 3]
                    break
            d = [x for x in t2 if x != a and x != b][0]
            if _incircle(coords[a], coords[b], coords[c], coords[d]) > 1e-14:
                tris[ts[0]] = [a, d, c]
                tris[ts[1]] = [d, b, c]
                touched.update(ts)
                flipped = True
        if not flipped:
            break
    return np.array(tris, dtype=np.int32)


def mesh_square(nx: int, jitter: float = 0.2, seed: int = 2, c: float = 1.0) -> Mesh:
    """Unit square, (nx+1)^2 grid vertices; interior vertices jittered by
    U(-jitter*h, jitter*h) per coordinate (seeded); two triangles per cell,
    then Lawson flips to a Delaunay mesh.  2*nx^2 triangles."""
    h = 1.0 / nx
    rng = np.random.default_rng(seed)
    g = np.array([[i * h, j * h] for j in range(nx + 1) for i in range(nx + 1)], dtype=np.float64)
    g[g > 1.0] = 1.0
    jit = rng.uniform(-jitter * h, jitter * h, size=g.shape)
    interior = (g[:, 0] > 0) & (g[:, 0] < 1) & (g[:, 1] > 0) & (g[:, 1] < 1)
    g[interior] += jit[interior]
    tris = []
    for j in range(nx):
        for i in range(nx):
            v00 = j * (nx + 1) + i
            v10, v01, v11 = v00 + 1, v00 + nx + 1, v00 + nx + 2
            tris.append([v00, v10, v11])
            tris.append([v00, v11, v01])
    tris = lawson_delaunay(g, np.array(tris))
    return Mesh(g, tris, np.full(len(tris), c, dtype=np.float64), name=f"square{nx}",
                meta={"h": h, "seed": seed, "jitter": jitter})


def mesh_inclusion_graded(h_max: float = 0.015, ratio: float = 10.0, growth: float = 1.25,
                          radius: float = 0.2, center=(0.5, 0.5), seed: int = 3,
                          c_in: float = 3.0, c_out: float = 1.0) -> Mesh:
    """Unit square graded `ratio` times finer around a circular inclusion.

    Points: the circle |x - center| = radius at spacing h_min = h_max / ratio;
    rings inside and outside it whose spacing grows by `growth` per ring up
    to h_max (each ring rotated by a seeded phase); a jittered grid of
    spacing h_max beyond the rings and on the square's boundary.  Their
    Delaunay triangulation (counter-clockwise triangles); c = c_in on the
    triangles whose centroid lies inside the circle, c_out elsewhere, so the
    jump of c follows element edges.  h_max = 0.015 gives about 21 000
    triangles."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    cx, cy = float(center[0]), float(center[1])
    h_min = h_max / ratio
    pts = []

    def ring(rad, sp):
        n = max(3, int(math.ceil(2.0 * math.pi * rad / sp)))
        a = rng.uniform(0.0, 2.0 * math.pi / n) + 2.0 * math.pi * np.arange(n) / n
        return np.stack([cx + rad * np.cos(a), cy + rad * np.sin(a)], axis=1)

    pts.append(ring(radius, h_min))
    sp, rad = h_min, radius
    while sp < h_max:                       # outward rings
        sp = min(h_max, sp * growth)
        rad += sp
        pts.append(ring(rad, sp))
    band = rad - radius
    sp, rad = h_min, radius
    while True:                             # inward rings down to the centre
        sp = min(h_max, sp * growth)
        rad -= sp
        if rad < sp:
            break
        pts.append(ring(rad, sp))
    pts.append(np.array([[cx, cy]]))
    n = int(round(1.0 / h_max))
    h = 1.0 / n
    g = np.array([[i * h, j * h] for j in range(n + 1) for i in range(n + 1)], dtype=np.float64)
    interior = (g[:, 0] > 0) & (g[:, 0] < 1) & (g[:, 1] > 0) & (g[:, 1] < 1)
    g[interior] += rng.uniform(-0.2 * h, 0.2 * h, size=g[interior].shape)
    d = np.hypot(g[:, 0] - cx, g[:, 1] - cy)
    pts.append(g[(d > radius + band + 0.5 * h) | ~interior])
    P = np.ascontiguousarray(np.concatenate(pts), dtype=np.float64)
    tris = Delaunay(P).simplices.astype(np.int32)
    for t in tris:
        if _orient2(P[t[0]], P[t[1]], P[t[2]]) < 0:
            t[1], t[2] = t[2], t[1]
    cen = P[tris].mean(axis=1)
    c = np.where(np.hypot(cen[:, 0] - cx, cen[:, 1] - cy) < radius, c_in, c_out).astype(np.float64)
    return Mesh(P, tris, c, name="inclusion_graded",
                meta={"h_max": h_max, "h_min": h_min, "seed": seed, "radius": radius})


def mesh_two_speeds(h_left: float = 0.01, h_right: float = 0.03, x_if: float = 1.2, length: float = 2.0,
                    c_left: float = 1.0, c_right: float = 3.0, seed: int = 7) -> Mesh:
    """The heterogeneous medium of Section 6.7: the square [0, length]^2 with
    c = c_left for x_1 <= x_if and c_right beyond, spatial mesh size h_left
    on the slow side and h_right on the fast one.  Points: a grid of spacing
    h_left on [0, x_if] x [0, length] (the column x_1 = x_if included) and a
    grid of spacing h_right beyond, interior points jittered by 10 % of
    their spacing (seeded); their Delaunay triangulation (counter-clockwise),
    c by element centroid.  The default sizes give about 52 000 triangles."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)

    def grid(x0, x1, h, skip_first_column):
        nx = int(math.ceil((x1 - x0) / h - 1e-9))
        ny = int(math.ceil(length / h - 1e-9))
        xs = x0 + (x1 - x0) * np.arange(nx + 1) / nx
        ys = length * np.arange(ny + 1) / ny
        if skip_first_column:
            xs = xs[1:]
        P = np.array([[x, y] for y in ys for x in xs], dtype=np.float64)
        inner = (P[:, 0] > 0) & (P[:, 0] < length) & (P[:, 1] > 0) & (P[:, 1] < length) & \
                (np.abs(P[:, 0] - x_if) > 1e-12)
        P[inner] += rng.uniform(-0.1 * h, 0.1 * h, size=P[inner].shape)
        return P

    P = np.ascontiguousarray(np.concatenate([grid(0.0, x_if, h_left, False),
                                             grid(x_if, length, h_right, True)]), dtype=np.float64)
    tris = Delaunay(P).simplices.astype(np.int32)
    for t in tris:
        if _orient2(P[t[0]], P[t[1]], P[t[2]]) < 0:
            t[1], t[2] = t[2], t[1]
    cen = P[tris].mean(axis=1)
    c = np.where(cen[:, 0] <= x_if, c_left, c_right).astype(np.float64)
    return Mesh(P, tris, c, name="two_speeds",
                meta={"h_left": h_left, "h_right": h_right, "x_if": x_if, "seed": seed})


def _ring_polyline(s: float, h: float):
    """The part of the square |x|_inf = s inside the L-shape (Section 6.6):
    four straight pieces from (0,-s) over (-s,-s), (-s,s), (s,s) to (s,0),
    each cut into pieces of length <= h.  Returns a list of four point
    arrays, consecutive pieces sharing their end point."""
    corners = [(0.0, -s), (-s, -s), (-s, s), (s, s), (s, 0.0)]
    out = []
    for (ax, ay), (bx, by) in zip(corners[:-1], corners[1:]):
        m = max(1, int(math.ceil(math.hypot(bx - ax, by - ay) / h - 1e-9)))
        u = np.arange(m + 1) / m
        out.append(np.stack([ax + u * (bx - ax), ay + u * (by - ay)], axis=1))
    return out


def mesh_lshape(h_max: float, mu: float = 1.0 / 3.0, c: float = 1.0) -> Mesh:
    """The L-shaped domain [-1,1]^2 minus [0,1]x[-1,0] of Section 6.6, its
    reentrant corner at the origin, meshed with local size
    h(r) = max(h_max r^(1-mu), h_min), h_min = h_max^(1/mu) (the paper's
    grading law; mu = 1 gives a uniform mesh of size h_max).

    Vertices lie on the squares |x|_inf = s_k around the corner, s_0 = 0
    (the corner itself) < s_1 < ... < s_K = 1 (the outer boundary), with
    s_{k+1} - s_k = h(s_k) (graded) or 1/ceil(1/h_max) (uniform), the whole
    sequence scaled so that s_K = 1; on each square the spacing is at most
    h(s_k).  Uniform: a fan from the corner to the first square, then
    between consecutive squares a strip over each of the four straight
    pieces, zipped by matching the pieces' normalised arc lengths (the
    pieces of two squares are parallel and seen from the corner under the
    same angles, so every strip triangle lies in a convex trapezoid): 6 n^2
    right isosceles triangles.  Graded: the Delaunay triangulation of the
    same points with the triangles inside the cut-out quadrant dropped
    (consecutive points on the two cut edges are Gabriel edges, so the
    triangulation keeps them); it avoids the flat triangles that strips
    leave at the squares' corners where s grows fast near the origin.
    Counter-clockwise triangles; no random numbers."""
    if mu >= 1.0:
        n = int(math.ceil(1.0 / h_max - 1e-9))
        s = np.arange(n + 1) / n
        h_min = 1.0 / n
        sizes = np.full(n + 1, 1.0 / n)
    else:
        h_min = h_max ** (1.0 / mu)
        seq = [0.0, h_min]
        while seq[-1] < 1.0:
            seq.append(seq[-1] + max(h_max * seq[-1] ** (1.0 - mu), h_min))
        s = np.array(seq) / seq[-1]
        sizes = np.maximum(h_max * s ** (1.0 - mu), h_min)
    s[-1] = 1.0
    pts = [np.zeros((1, 2))]
    rings = []                     # per square: four arrays of vertex ids
    nv = 1
    for k in range(1, len(s)):
        pieces = _ring_polyline(float(s[k]), float(sizes[k]))
        ids, flat = [], []
        for j, pc in enumerate(pieces):
            start = nv if j == 0 else ids[-1][-1]
            new = pc if j == 0 else pc[1:]
            idx = np.arange(nv, nv + len(new))
            ids.append(idx if j == 0 else np.concatenate([[start], idx]))
            flat.append(new)
            nv += len(new)
        pts.append(np.concatenate(flat))
        rings.append(ids)
    P = np.ascontiguousarray(np.concatenate(pts), dtype=np.float64)
    P[np.abs(P) < 1e-15] = 0.0
    if mu < 1.0:
        from scipy.spatial import Delaunay
        tris = Delaunay(P).simplices.astype(np.int32)
        cen = P[tris].mean(axis=1)
        tris = np.ascontiguousarray(tris[~((cen[:, 0] > 0.0) & (cen[:, 1] < 0.0))])
        for t in tris:
            if _orient2(P[t[0]], P[t[1]], P[t[2]]) < 0:
                t[1], t[2] = t[2], t[1]
        return Mesh(P, tris, np.full(len(tris), c, dtype=np.float64), name="lshape_graded",
                    meta={"h_max": h_max, "h_min": h_min, "mu": mu, "n_squares": len(s) - 1})
    tris = []
    for piece in rings[0]:
        for a, b in zip(piece[:-1], piece[1:]):
            tris.append([0, int(a), int(b)])
    for inner, outer in zip(rings[:-1], rings[1:]):
        for pi, po in zip(inner, outer):
            mi, mo = len(pi) - 1, len(po) - 1
            i = j = 0
            while i < mi or j < mo:
                if j == mo or (i < mi and (i + 1) * mo <= (j + 1) * mi):
                    tris.append([int(pi[i]), int(pi[i + 1]), int(po[j])])
                    i += 1
                else:
                    tris.append([int(pi[i]), int(po[j + 1]), int(po[j])])
                    j += 1
    tris = np.array(tris, dtype=np.int32)
    for t in tris:
        if _orient2(P[t[0]], P[t[1]], P[t[2]]) < 0:
            t[1], t[2] = t[2], t[1]
    return Mesh(P, tris, np.full(len(tris), c, dtype=np.float64), name="lshape_uniform",
                meta={"h_max": h_max, "h_min": h_min, "mu": mu, "n_squares": len(s) - 1})


# ----------------------------------------------------------------------------
# 3D: jittered hex grid, 6 Kuhn tetrahedra per hex
# ----------------------------------------------------------------------------
def mesh_cube(nx: int, jitter: float = 0.1, seed: int = 4, c: float = 1.0) -> Mesh:
    """Unit cube, (nx+1)^3 vertices, interior jittered by U(-jitter*h, jitter*h)
    per coordinate (seeded), 6 tetrahedra per hex about the main diagonal.
    6*nx^3 tetrahedra."""
    h = 1.0 / nx
    rng = np.random.default_rng(seed)
    n1 = nx + 1
    g = np.array([[i * h, j * h, k * h] for k in range(n1) for j in range(n1) for i in range(n1)],
                 dtype=np.float64)
    g[g > 1.0] = 1.0
    jit = rng.uniform(-jitter * h, jitter * h, size=g.shape)
    interior = np.all((g > 0) & (g < 1), axis=1)
    g[interior] += jit[interior]

    def vid(i, j, k):
        return (k * n1 + j) * n1 + i

    tets = []
    for k in range(nx):
        for j in range(nx):
            for i in range(nx):
                for perm in itertools.permutations(range(3)):
                    cur = [0, 0, 0]
                    tet = [vid(i, j, k)]
                    for ax in perm:
                        cur[ax] += 1
                        tet.append(vid(i + cur[0], j + cur[1], k + cur[2]))
                    tets.append(tet)
    return Mesh(g, np.array(tets, dtype=np.int32), np.full(len(tets), c, dtype=np.float64),
                name=f"cube{nx}", meta={"h": h, "seed": seed, "jitter": jitter})


# ----------------------------------------------------------------------------
# Choice of the pitching parameter kappa
# ----------------------------------------------------------------------------
def element_slope_factor(mesh: Mesh) -> np.ndarray:
    """C_K = max |g| over linear functions on K with |g.(x_i-x_j)| <= |x_i-x_j|
    on every edge of K (vertex enumeration of that polytope).

    If every edge obeys |tau_i - tau_j| <= kappa |x_i - x_j| / c_K, then
    c_K |grad tau| <= kappa C_K, so kappa < 1/C_K keeps the face space-like
    (the causality condition of Section 2.2)."""
    n = mesh.dim
    if n == 1:
        return np.ones(mesh.n_elem)
    X = mesh.coords[mesh.elems]                              # (E, n+1, n)
    pairs = list(itertools.combinations(range(n + 1), 2))
    U = np.stack([X[:, j] - X[:, i] for i, j in pairs], axis=1)   # (E, m, n)
    U = U / np.linalg.norm(U, axis=2, keepdims=True)
    best = np.zeros(mesh.n_elem)
    for rows in itertools.combinations(range(len(pairs)), n):
        M = U[:, list(rows)]                                 # (E, n, n)
        det = np.linalg.det(M)
        ok = np.abs(det) > 1e-12
        if not np.any(ok):
            continue
        for signs in itertools.product([-1.0, 1.0], repeat=n):
            rhs = np.broadcast_to(np.array(signs), (int(ok.sum()), n))
            gg = np.linalg.solve(M[ok], rhs[..., None])[..., 0]   # (E', n)
            feas = np.all(np.abs(np.einsum("emn,en->em", U[ok], gg)) <= 1 + 1e-9, axis=1)
            val = np.where(feas, np.linalg.norm(gg, axis=1), 0.0)
            idx = np.nonzero(ok)[0]
            best[idx] = np.maximum(best[idx], val)
    return best


def boundary_marker(mesh: Mesh, predicate) -> np.ndarray:
    """Per element and local face (the face opposite local vertex o), 1 where
    every vertex of the face satisfies predicate(x) and the face lies on the
    boundary (belongs to one element only), else 0: an (n_elem, dim+1) int8
    array for marking boundary facets (e.g. as Neumann)."""
    E, nv1 = mesh.elems.shape
    count: dict = {}
    for k in range(E):
        el = mesh.elems[k].tolist()
        for o in range(nv1):
            f = tuple(sorted(el[:o] + el[o + 1:]))
            count[f] = count.get(f, 0) + 1
    out = np.zeros((E, nv1), dtype=np.int8)
    for k in range(E):
        el = mesh.elems[k].tolist()
        for o in range(nv1):
            f = tuple(sorted(el[:o] + el[o + 1:]))
            if count[f] == 1 and all(predicate(mesh.coords[a]) for a in f):
                out[k, o] = 1
    return out


def pitch_kappa(mesh: Mesh, safety: float = 0.9) -> float:
    """kappa = safety / max_K C_K (1D: C_K = 1, so kappa = safety)."""
    return float(safety / element_slope_factor(mesh).max())


# ----------------------------------------------------------------------------
# Closed-form solutions.  Every function returns an array (N, n+2) holding
# (U, v, sigma_1..sigma_n) with v = dU/dt and sigma = -grad U.
# ----------------------------------------------------------------------------
def plane_wave_1d(x: np.ndarray, t) -> np.ndarray:
    """U = sin(pi (x - t)), c = 1."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape)
    ph = math.pi * (x - t)
    return np.stack([np.sin(ph), -math.pi * np.cos(ph), -math.pi * np.cos(ph)], axis=1)


def sine_product_1d(x: np.ndarray, t) -> np.ndarray:
    """U = sin(pi x) sin(pi t), c = 1 (Section 6.5): v = 0 at x = 0 and 1, and
    the energy 1/2 int (v^2 + sigma^2) dx = pi^2 / 4 at every t."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape)
    sx, cx = np.sin(math.pi * x), np.cos(math.pi * x)
    st, ct = np.sin(math.pi * t), np.cos(math.pi * t)
    return np.stack([sx * st, math.pi * sx * ct, -math.pi * cx * st], axis=1)


def standing_wave_2d(x: np.ndarray, t) -> np.ndarray:
    """U = cos(sqrt2 pi t) sin(pi x) sin(pi y), c = 1 (v = 0 on the boundary)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 2)
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape[:1])
    w = math.sqrt(2.0) * math.pi
    sx, sy = np.sin(math.pi * x[:, 0]), np.sin(math.pi * x[:, 1])
    cx, cy = np.cos(math.pi * x[:, 0]), np.cos(math.pi * x[:, 1])
    ct, st = np.cos(w * t), np.sin(w * t)
    return np.stack([ct * sx * sy, -w * st * sx * sy,
                     -math.pi * ct * cx * sy, -math.pi * ct * sx * cy], axis=1)


def standing_wave_3d(x: np.ndarray, t) -> np.ndarray:
    """U = cos(sqrt3 pi t) sin(pi x) sin(pi y) sin(pi z), c = 1."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape[:1])
    w = math.sqrt(3.0) * math.pi
    s = np.sin(math.pi * x)
    co = np.cos(math.pi * x)
    ct, st = np.cos(w * t), np.sin(w * t)
    prod = s[:, 0] * s[:, 1] * s[:, 2]
    return np.stack([ct * prod, -w * st * prod,
                     -math.pi * ct * co[:, 0] * s[:, 1] * s[:, 2],
                     -math.pi * ct * s[:, 0] * co[:, 1] * s[:, 2],
                     -math.pi * ct * s[:, 0] * s[:, 1] * co[:, 2]], axis=1)


def corner_angle(x: np.ndarray) -> np.ndarray:
    """Polar angle phi in [-pi/4, 7pi/4) about the L-shape's reentrant
    corner: the cut lies in the middle of the removed quadrant, so the two
    cut edges sit at phi = 0 and phi = 3pi/2 and points that rounding puts
    just outside them stay on the right branch."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 2)
    phi = np.arctan2(x[:, 1], x[:, 0])
    return np.where(phi < -0.25 * math.pi, phi + 2.0 * math.pi, phi)


def bessel_corner_solution(a: float = 10.0, nu: float = 2.0 / 3.0):
    """U(r, phi, t) = cos(a t) sin(nu phi) J_nu(a r), c = 1 (Section 6.6): the
    singular solution on the L-shape; U = 0 on both cut edges for nu = 2/3,
    and grad U ~ r^(nu - 1) at the corner.  Returns sol(x, t) -> (N, 4)
    holding (U, v, sigma_1, sigma_2) with sigma = -(U_r e_r + U_phi / r e_phi).
    At r = 0 sigma is set to 0 (it is unbounded there; no quadrature point
    lies at the corner)."""
    from scipy.special import jv, jvp

    def sol(x: np.ndarray, t) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(-1, 2)
        t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape[:1])
        r = np.hypot(x[:, 0], x[:, 1])
        phi = corner_angle(x)
        J = jv(nu, a * r)
        s, c = np.sin(nu * phi), np.cos(nu * phi)
        ct, st = np.cos(a * t), np.sin(a * t)
        rs = np.where(r > 0.0, r, 1.0)
        f_r = np.where(r > 0.0, a * jvp(nu, a * rs) * s, 0.0)
        f_phi_r = np.where(r > 0.0, nu * J * c / rs, 0.0)
        cp, sp = x[:, 0] / rs, x[:, 1] / rs
        gx = f_r * cp - f_phi_r * sp
        gy = f_r * sp + f_phi_r * cp
        return np.stack([ct * s * J, -a * st * s * J, -ct * gx, -ct * gy], axis=1)
    return sol


def gaussian_pulse(center, delta: float):
    """U0 = exp(-|x-x0|^2/delta^2), v0 = 0, sigma0 = -grad U0 (a t = 0 state)."""
    x0 = np.asarray(center, dtype=np.float64)

    def f(x: np.ndarray, t=0.0) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(-1, x0.size)
        d = x - x0
        u = np.exp(-np.sum(d * d, axis=1) / delta ** 2)
        sig = (2.0 / delta ** 2) * d * u[:, None]
        return np.concatenate([u[:, None], np.zeros((len(u), 1)), sig], axis=1)
    return f


def gaussian_pulses_3d(n: int = 64, seed: int = 64) -> list:
    """n Gaussian pulses in the unit cube (v0 = 0): centres uniform in
    [0.25, 0.75]^3, widths uniform in [0.05, 0.15], seeded; the right-hand
    sides of the 3+1D many-right-hand-side runs."""
    rng = np.random.default_rng(seed)
    cen = rng.uniform(0.25, 0.75, (n, 3))
    wid = rng.uniform(0.05, 0.15, n)
    return [gaussian_pulse(cen[i], float(wid[i])) for i in range(n)]


def polynomial_solution(dim: int, which: int = 0):
    """Polynomial solutions of -Lap U + U_tt = 0 (c = 1), used for the
    reproduction property: U in the discrete Trefftz space is recovered
    exactly by a consistent method.

    dim 1: which 0 -> x^2 + t^2,  which 1 -> x^3 + 3 x t^2
    dim 2: which 0 -> x^2 + y^2 + 2 t^2, which 1 -> x y t + x^3 + 3 x t^2
    dim 3: which 0 -> x^2 + y^2 + z^2 + 3 t^2, which 1 -> x y z + y^3 + 3 y t^2 + x^2 - z^2
    """
    def f(x: np.ndarray, t) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(-1, dim)
        t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape[:1])
        X = x[:, 0]
        if dim == 1:
            if which == 0:
                return np.stack([X**2 + t**2, 2 * t, -2 * X], axis=1)
            return np.stack([X**3 + 3 * X * t**2, 6 * X * t, -(3 * X**2 + 3 * t**2)], axis=1)
        Y = x[:, 1]
        if dim == 2:
            if which == 0:
                return np.stack([X**2 + Y**2 + 2 * t**2, 4 * t, -2 * X, -2 * Y], axis=1)
            U = X * Y * t + X**3 + 3 * X * t**2
            return np.stack([U, X * Y + 6 * X * t, -(Y * t + 3 * X**2 + 3 * t**2),
                             -(X * t)], axis=1)
        Z = x[:, 2]
        if which == 0:
            return np.stack([X**2 + Y**2 + Z**2 + 3 * t**2, 6 * t, -2 * X, -2 * Y, -2 * Z], axis=1)
        U = X * Y * Z + Y**3 + 3 * Y * t**2 + X**2 - Z**2
        return np.stack([U, 6 * Y * t,
                         -(Y * Z + 2 * X), -(X * Z + 3 * Y**2 + 3 * t**2),
                         -(X * Y - 2 * Z)], axis=1)
    return f


# ----------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped runs)
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mesh: Mesh
    p: int
    T: float
    kappa: float
    solution: object          # callable(x, t) -> (N, n+2); None if only initial data
    init: object              # callable(x) -> (N, n+2) at t = 0
    dirichlet: object         # callable(x, t) -> (N,) values of v on the boundary, or None (= 0)
    alpha: float = 0.5
    beta: float = 0.5


def _vfield(sol):
    return lambda x, t: sol(x, t)[:, 1]


def workload(name: str) -> Workload:
    """Named workloads.

    plane1d      : [0,1], 16 elements, p=3, T=1, plane wave, Dirichlet both ends.
    standing2d   : unit square, 22x22 jittered Delaunay grid (968 triangles),
                   p=4, T=1, standing wave (v = 0 on the boundary).
    small2d      : unit square, 6x6 jittered grid (72 triangles), p=4, T=0.25.
    standing3d_small : unit cube 3^3 hexes (162 tets), p=3, T=0.2.
    inclusion_small : unit square 8x8 jittered grid (128 triangles), c = 3 in the
                   disc |x - (0.5,0.5)| < 0.2 (by element centroid), c = 1 outside,
                   p=3, T=0.15, Gaussian pulse (Section 6.7 shape, small).
    inclusion_graded: the same inclusion on about 21 000 triangles graded 10x
                   finer around the circle (mesh_inclusion_graded), p=5, T=2,
                   Gaussian pulse of width 0.05 at a seeded centre.
    many_rhs_3d  : unit cube 20^3 hexes (48 000 tets, jitter 0.1, seed 4), p=3,
                   T=1; init is the first of the 64 pulses of gaussian_pulses_3d().
    lognormal2d  : unit square 100x100 jittered grid (20 000 triangles, seed 5),
                   c_K = exp(N(-0.045, 0.3^2)) per element (seed 5, mean about 1),
                   p=4, T=1; init is the first of 16 pulses of width 0.05
                   (centres uniform in [0.2, 0.8]^2, seed 55): the adjoint
                   configuration's forward problem.
    """
    if name == "plane1d":
        m = mesh_interval(16)
        return Workload(name, m, 3, 1.0, 0.9, plane_wave_1d,
                        lambda x: plane_wave_1d(x, 0.0), _vfield(plane_wave_1d))
    if name == "standing2d":
        m = mesh_square(22, 0.2, seed=2)
        return Workload(name, m, 4, 1.0, pitch_kappa(m), standing_wave_2d,
                        lambda x: standing_wave_2d(x, 0.0), None)
    if name == "small2d":
        m = mesh_square(6, 0.2, seed=7)
        return Workload(name, m, 4, 0.25, pitch_kappa(m), standing_wave_2d,
                        lambda x: standing_wave_2d(x, 0.0), None)
    if name == "standing3d_small":
        m = mesh_cube(3, 0.1, seed=4)
        return Workload(name, m, 3, 0.2, pitch_kappa(m), standing_wave_3d,
                        lambda x: standing_wave_3d(x, 0.0), None)
    if name == "inclusion_small":
        m = mesh_square(8, 0.2, seed=13)
        cen = m.coords[m.elems].mean(axis=1)
        m.c[:] = np.where(np.linalg.norm(cen - 0.5, axis=1) < 0.2, 3.0, 1.0)
        pulse = gaussian_pulse((0.42, 0.55), 0.15)
        return Workload(name, m, 3, 0.15, pitch_kappa(m), None, pulse, None)
    if name == "inclusion_graded":
        m = mesh_inclusion_graded()
        rng = np.random.default_rng(17)
        pulse = gaussian_pulse(rng.uniform(0.3, 0.7, 2), 0.05)
        return Workload(name, m, 5, 2.0, pitch_kappa(m), None, pulse, None)
    if name == "lognormal2d":
        m = mesh_square(100, 0.2, seed=5)
        m.c[:] = np.exp(np.random.default_rng(5).normal(-0.045, 0.3, m.n_elem))
        cen = np.random.default_rng(55).uniform(0.2, 0.8, (16, 2))
        return Workload(name, m, 4, 1.0, pitch_kappa(m), None, gaussian_pulse(cen[0], 0.05), None)
    if name == "many_rhs_3d":
        m = mesh_cube(20, 0.1, seed=4)
        return Workload(name, m, 3, 1.0, pitch_kappa(m), None, gaussian_pulses_3d()[0], None)
    raise KeyError(name)


def interface_solution(dim: int, a: float, c1: float, c2: float):
    """Exact piecewise-quadratic solution across the interface x_1 = a between
    speeds c1 (x_1 < a) and c2 (x_1 > a):
        U_i = alpha_i x^2 + beta t^2 + gamma_i x + e_i + 0.4 y  (x = x_1, y = x_2 in 2D)
    with alpha_1 = c2^2, alpha_2 = c1^2, beta = c1^2 c2^2, so that each piece
    solves -Lap U + c_i^-2 U_tt = 0, and gamma_2, e_2 chosen so that U and
    dU/dx_1 (hence v and sigma.n) are continuous at x_1 = a.
    Returns (sol(x, t) -> (N, n+2), speed(x) -> c)."""
    al1, al2 = c2 * c2, c1 * c1
    be = c1 * c1 * c2 * c2
    g1, e1 = 0.3, 0.1
    g2 = g1 + 2.0 * (al1 - al2) * a
    e2 = e1 + (al1 - al2) * a * a + (g1 - g2) * a

    def sol(x, t):
        x = np.asarray(x, dtype=np.float64).reshape(-1, dim)
        t = np.broadcast_to(np.asarray(t, dtype=np.float64), x.shape[:1])
        X = x[:, 0]
        left = X < a
        al = np.where(left, al1, al2)
        g = np.where(left, g1, g2)
        e = np.where(left, e1, e2)
        U = al * X * X + be * t * t + g * X + e
        cols = [U, 2.0 * be * t, -(2.0 * al * X + g)]
        if dim == 2:
            U = U + 0.4 * x[:, 1]
            cols[0] = U
            cols.append(np.full_like(X, -0.4))
        return np.stack(cols, axis=1)

    def speed(xc):
        xc = np.asarray(xc, dtype=np.float64).reshape(-1, dim)
        return np.where(xc[:, 0] < a, c1, c2)
    return sol, speed
