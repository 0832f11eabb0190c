"""Writes tests/golden/inclusion_graded_oracle.json: the oracle's sweep over
the first two levels of the full-size graded inclusion workload
(inputs.workload("inclusion_graded"): 21 054 triangles graded 10x finer at
the circle, c = 3 inside, 1 outside, p = 5, T = 2, 19.7 million tents), for
the GPU test that runs the library at that size.

Stored: a checksum of the mesh arrays (the mesh comes from a Delaunay
triangulation, so a test can tell whether its platform rebuilt the same
mesh), the number of tents in levels 1-2, the norm of the front after them,
and the front at 256 seeded positions of its flattened (element, point,
component) array among the entries above 1e-3 of the largest.  Calls only
oracle/ and the shared input generators; the oracle's pitching of the whole
mesh takes tens of minutes.

    python tests/golden/make_inclusion_graded_oracle.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pitching, tdg  # noqa: E402
from paper_1907_02367_gb300 import inputs  # noqa: E402

LEVELS = 2
N_SAMPLE = 256


def mesh_checksum(mesh) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(mesh.elems, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(mesh.coords, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(mesh.c, dtype=np.float64).tobytes())
    return h.hexdigest()


def sample_positions(flat: np.ndarray, seed: int = 88) -> np.ndarray:
    big = np.nonzero(np.abs(flat) > 1e-3 * np.abs(flat).max())[0]
    return np.sort(np.random.default_rng(seed).choice(big, size=N_SAMPLE, replace=False))


def main():
    w = inputs.workload("inclusion_graded")
    m = w.mesh
    t0 = time.time()
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    print(f"pitched {len(r['level'])} tents in {r['n_levels']} levels, {time.time() - t0:.0f}s", flush=True)
    ntent = int(np.sum(r["level"] <= LEVELS))
    t0 = time.time()
    F, _ = tdg.sweep(m.coords, m.elems, m.c, w.p, r, w.init, None, tent_range=(0, ntent))
    print(f"swept {ntent} tents, {time.time() - t0:.0f}s", flush=True)
    flat = F.reshape(-1)
    pos = sample_positions(flat)
    out = {"source": "oracle.tdg.sweep over levels 1-2 of inclusion_graded "
                     "(tests/golden/make_inclusion_graded_oracle.py)",
           "checksum": mesh_checksum(m), "n_tents_total": int(len(r["level"])),
           "levels": LEVELS, "n_tents": ntent, "front_norm": float(np.linalg.norm(flat)),
           "sample_pos": pos.tolist(), "sample_val": flat[pos].tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "inclusion_graded_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
