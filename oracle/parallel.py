"""The oracle's tent sweep over the independent tents of a level on several
host cores (TEST INFRASTRUCTURE; see oracle/__init__.py).

Tents of one level never share an element (Section 2.2: a level is a set of
causally independent tents), so the level can be split into chunks that run
oracle.tdg.sweep on their own tents from the same front and front times, and
the chunks' results merged: each tent writes only its own patch.  This is
the paper's own parallel loop (tents of a layer on threads, Section 6), here
on processes started with `spawn`.  Nothing here changes the oracle's
arithmetic: every tent is computed by oracle.tdg.sweep as it stands.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from . import tdg as _tdg

_W = {}


def _init(coords, elems, c, p, tents, kw):
    _W.update(coords=coords, elems=elems, c=c, p=p, tents=tents, kw=kw,
              star=_tdg.vertex_star(np.asarray(elems), coords.shape[0]))


def _chunk(args):
    front, tau, t0, t1 = args
    W = _W
    F, tau1 = _tdg.sweep(W["coords"], W["elems"], W["c"], W["p"], W["tents"], None, front0=front,
                         tau0=tau, tent_range=(t0, t1), **W["kw"])
    ks = sorted({k for it in range(t0, t1) for k in W["star"][int(W["tents"]["vert"][it])]})
    vs = [int(W["tents"]["vert"][it]) for it in range(t0, t1)]
    return np.asarray(ks, dtype=np.int64), F[ks], np.asarray(vs, dtype=np.int64), tau1[vs]


def sweep_levels(coords, elems, c, p, tents, front0, levels, nproc=None, **sweep_kw):
    """Front and front times after levels 1 .. `levels` of the pitched sweep,
    starting from front0 (E, Q, n+2) at t = 0.  Each level's tents are split
    into about 4 nproc contiguous chunks run in a pool of nproc processes.
    Returns (front, tau, n_tents_done)."""
    coords = np.asarray(coords, dtype=np.float64)
    elems = np.asarray(elems)
    c = np.asarray(c, dtype=np.float64)
    nproc = nproc or os.cpu_count() or 1
    lev = np.asarray(tents["level"])
    front = np.array(front0, dtype=np.float64)
    tau = np.zeros(coords.shape[0])
    done = 0
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc, initializer=_init, initargs=(coords, elems, c, p, tents, sweep_kw)) as pool:
        for L in range(1, levels + 1):
            idx = np.nonzero(lev == L)[0]
            if len(idx) == 0:
                continue
            a, b = int(idx[0]), int(idx[-1]) + 1
            assert b - a == len(idx)          # the tents are sorted by level
            nch = max(1, min(len(idx), 4 * nproc))
            cuts = np.linspace(a, b, nch + 1).astype(int)
            jobs = [(front, tau, int(cuts[i]), int(cuts[i + 1])) for i in range(nch) if cuts[i + 1] > cuts[i]]
            for ks, vals, vs, tv in pool.map(_chunk, jobs):
                front[ks] = vals
                tau[vs] = tv
            done = b
    return front, tau, done
