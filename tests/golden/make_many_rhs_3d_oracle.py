"""Writes tests/golden/many_rhs_3d_oracle.json: the oracle's sweep over the
first two levels of the full-size 3+1D many-right-hand-side workload
(inputs.workload("many_rhs_3d"): 48 000 tetrahedra, p = 3, T = 1, 3076 tents
in levels 1-2) for two of its 64 pulses (columns 0 and 63), for the GPU test
that runs the library at that size with all 64 right-hand sides.

Per column: the norm of the front after those tents and the front at 256
seeded positions of its flattened (element, point, component) array, taken
among the entries above 1e-3 of the largest; the number of tents.  Calls only oracle/ and the shared input generators.

    python tests/golden/make_many_rhs_3d_oracle.py
"""
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
COLUMNS = (0, 63)
N_SAMPLE = 256


def sample_positions(flat: np.ndarray, seed: int = 77) -> np.ndarray:
    """N_SAMPLE seeded positions among the entries above 1e-3 of the largest
    (the pulses are narrow: most of the front is near zero)."""
    big = np.nonzero(np.abs(flat) > 1e-3 * np.abs(flat).max())[0]
    return np.sort(np.random.default_rng(seed).choice(big, size=N_SAMPLE, replace=False))


def main():
    w = inputs.workload("many_rhs_3d")
    m = w.mesh
    pulses = inputs.gaussian_pulses_3d()
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    ntent = int(np.sum(r["level"] <= LEVELS))
    cols = []
    for col in COLUMNS:
        t0 = time.time()
        F, _ = tdg.sweep(m.coords, m.elems, m.c, w.p, r, pulses[col], None, tent_range=(0, ntent))
        flat = F.reshape(-1)
        pos = sample_positions(flat)
        cols.append({"column": col, "front_norm": float(np.linalg.norm(flat)),
                     "sample_pos": pos.tolist(), "sample_val": flat[pos].tolist()})
        print(f"column {col}: {ntent} tents {time.time() - t0:.0f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "many_rhs_3d_oracle.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.tdg.sweep over levels 1-2 of many_rhs_3d "
                             "(tests/golden/make_many_rhs_3d_oracle.py)",
                   "levels": LEVELS, "n_tents": ntent, "columns": cols}, f, indent=1)


if __name__ == "__main__":
    main()
