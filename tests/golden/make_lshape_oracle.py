"""Writes tests/golden/lshape_oracle.json: the oracle's sweep on L-shape meshes
of Section 6.6 at the sizes of the paper's Table 1, for the GPU test that
checks the library at sizes the oracle takes minutes for.

Per mesh: the mesh's size and a checksum of its arrays (so a test can tell
whether it rebuilt the same mesh), the number of tents, the L2 error of U at
T = 1 against the closed form, and the final front at 256 seeded positions of
its flattened (element, point, component) array.  Calls only oracle/ and the
shared input generators.

    python tests/golden/make_lshape_oracle.py
"""
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pitching, tdg  # noqa: E402
from paper_1907_02367_gb300 import inputs  # noqa: E402

P, T = 3, 1.0
MESHES = [(0.07, 1.0), (0.05, 1.0), (0.03, 1.0), (0.12, 1.0 / 3.0), (0.10, 1.0 / 3.0), (0.08, 1.0 / 3.0),
          (0.06, 1.0 / 3.0)]
N_SAMPLE = 256


def mesh_checksum(mesh) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(mesh.elems, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(mesh.coords, dtype=np.float64).tobytes())
    return h.hexdigest()


def sample_positions(n_total: int, seed: int = 66) -> np.ndarray:
    return np.sort(np.random.default_rng(seed).choice(n_total, size=N_SAMPLE, replace=False))


def main():
    sol = inputs.bessel_corner_solution()
    out = []
    for h, mu in MESHES:
        t0 = time.time()
        m = inputs.mesh_lshape(h, mu)
        r = pitching.pitch(m.coords, m.elems, m.c, inputs.pitch_kappa(m), T)
        F, tau = tdg.sweep(m.coords, m.elems, m.c, P, r, lambda x: sol(x, 0.0),
                           lambda x, t: sol(x, t)[:, 1])
        lay = tdg.front_layout(m.coords, m.elems, P)
        ex = sol(lay.xq.reshape(-1, 2), T)[:, 0]
        err = math.sqrt(float(np.sum(lay.wq.reshape(-1) * (F[..., 0].reshape(-1) - ex) ** 2)))
        flat = F.reshape(-1)
        pos = sample_positions(flat.size)
        out.append({"h_max": h, "mu": mu, "n_elem": m.n_elem, "checksum": mesh_checksum(m),
                    "n_tents": int(len(r["level"])), "n_levels": int(r["n_levels"]),
                    "l2_error": err, "front_norm": float(np.linalg.norm(flat)),
                    "sample_pos": pos.tolist(), "sample_val": flat[pos].tolist()})
        print(f"h={h} mu={mu:.3f} tents={len(r['level'])} err={err:.4e} {time.time() - t0:.0f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lshape_oracle.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.tdg.sweep, p = 3, T = 1, Section 6.6 corner solution "
                             "(tests/golden/make_lshape_oracle.py)", "meshes": out}, f, indent=1)


if __name__ == "__main__":
    main()
