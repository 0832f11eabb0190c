"""Tent pitching, oracle version (TEST INFRASTRUCTURE; see oracle/__init__.py).

Section 2.2 defines a tent-pitched mesh (every face space-like,
c|n_x| < n_t) and says that tents are stacked by progressively advancing the
front in time with a local causality limit; the Section 6 setup says the tent
height is limited by the slope of the edges, not of the faces.  The paper
only cites the algorithm, so this module implements one exact rule, written
out here so that a second implementation can reproduce it bit for bit:

  * edges e = (v, w) of the spatial mesh; length
        l_e = sqrt(((dx0*dx0) + dx1*dx1) + dx2*dx2)   (coordinate order);
    speed c_e = max c_K over the elements K containing e;
    slope limit  delta_e = (kappa * l_e) / c_e.
  * front times tau_v = 0, last level lam_v = 0 for every vertex.
  * repeat while some tau_v < T:
      R0 = { v : tau_v < T and tau_v <= tau_w for every neighbour w }
      R  = greedy independent subset of R0, scanning v in increasing order
           and keeping v when no neighbour of v is already kept;
      for v in R:  t_top = min(T, min_w (tau_w + delta_vw))
                   level = 1 + max(lam_v, max_w lam_w)
                   tent (v, t_bot = tau_v, t_top, level, round)
                   tau_v = t_top, lam_v = level
  * tents are listed sorted by (level, round, v); the layers are the levels.

Tents of one level never share a vertex patch, so they are independent
(Section 2.2: "independent tents can be computed in parallel").
All arithmetic is IEEE binary64 without fused multiply-add.
"""
from __future__ import annotations

import math

import numpy as np


def mesh_edges(elems: np.ndarray, c: np.ndarray):
    """Unique edges (v < w) and their speed c_e = max over adjacent elements."""
    ce: dict = {}
    for k, el in enumerate(elems.tolist()):
        for i in range(len(el)):
            for j in range(i + 1, len(el)):
                a, b = el[i], el[j]
                key = (a, b) if a < b else (b, a)
                ck = float(c[k])
                if key not in ce or ck > ce[key]:
                    ce[key] = ck
    return ce


def edge_length(xa, xb) -> float:
    """sqrt(((dx0*dx0) + dx1*dx1) + dx2*dx2), summed in coordinate order."""
    s = 0.0
    for d in range(len(xa)):
        dx = float(xb[d]) - float(xa[d])
        s = s + dx * dx
    return math.sqrt(s)


def pitch(coords: np.ndarray, elems: np.ndarray, c: np.ndarray, kappa: float, T: float,
          max_level: int | None = None):
    """Return dict of arrays sorted by (level, round, v):
    vert, t_bot, t_top, level, round; and n_levels, n_rounds.

    max_level: stop the rounds once every vertex's last level is at least
    max_level and keep the tents of level <= max_level.  A later tent at v
    has level >= 1 + lam_v, and lam never decreases, so no later round adds
    a tent of level <= max_level: the result is the first tents of the full
    pitch, in the same order (n_levels = max_level then)."""
    nv = coords.shape[0]
    ce = mesh_edges(elems, c)
    nbr = [[] for _ in range(nv)]
    delta: dict = {}
    for (a, b), cc in ce.items():
        d = (kappa * edge_length(coords[a], coords[b])) / cc
        delta[(a, b)] = d
        delta[(b, a)] = d
        nbr[a].append(b)
        nbr[b].append(a)
    for v in range(nv):
        nbr[v].sort()

    tau = [0.0] * nv
    lam = [0] * nv
    tents = []            # (level, round, v, t_bot, t_top)
    rnd = 0
    while any(t < T for t in tau):
        if max_level is not None and min(lam) >= max_level:
            break
        rnd += 1
        r0 = [v for v in range(nv)
              if tau[v] < T and all(tau[v] <= tau[w] for w in nbr[v])]
        kept = set()
        for v in r0:
            if not any(w in kept for w in nbr[v]):
                kept.add(v)
        new = []
        for v in sorted(kept):
            t_top = T
            for w in nbr[v]:
                cand = tau[w] + delta[(v, w)]
                if cand < t_top:
                    t_top = cand
            level = 1 + max([lam[v]] + [lam[w] for w in nbr[v]])
            new.append((level, rnd, v, tau[v], t_top))
        for (level, r, v, tb, tt) in new:
            tau[v] = tt
            lam[v] = level
        tents.extend(new)

    if max_level is not None:
        tents = [e for e in tents if e[0] <= max_level]
    tents.sort(key=lambda e: (e[0], e[1], e[2]))
    arr = np.array(tents, dtype=object) if tents else np.zeros((0, 5), dtype=object)
    out = {
        "level": np.array([e[0] for e in tents], dtype=np.int32),
        "round": np.array([e[1] for e in tents], dtype=np.int32),
        "vert": np.array([e[2] for e in tents], dtype=np.int32),
        "t_bot": np.array([e[3] for e in tents], dtype=np.float64),
        "t_top": np.array([e[4] for e in tents], dtype=np.float64),
    }
    del arr
    out["n_levels"] = int(out["level"].max()) if len(tents) else 0
    out["n_rounds"] = rnd
    return out


def vertex_neighbours(elems: np.ndarray, nv: int):
    nb = [set() for _ in range(nv)]
    for el in elems.tolist():
        for a in el:
            for b in el:
                if a != b:
                    nb[a].add(b)
    return [sorted(s) for s in nb]
