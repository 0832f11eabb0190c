"""Writes tests/golden/energy_oracle.json: the oracle's energy of the final
front for the long-time study of Section 6.5 (U = sin(pi x) sin(pi t) on 5
uniform elements of [0, 1], kappa = 0.9, homogeneous Dirichlet data) at the
paper's final times T = 100, 1000, 10000 for p = 2 ... 8, for the GPU test
that runs the library at those times.  Calls only oracle/ and the shared
input generators; T = 10000 takes about a minute per degree.

    python tests/golden/make_energy_oracle.py
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import energy, pitching, tdg  # noqa: E402
from paper_1907_02367_gb300 import inputs  # noqa: E402

N_ELEM, KAPPA = 5, 0.9
PS = (2, 3, 4, 5, 6, 7, 8)
TS = (100.0, 1000.0, 10000.0)


def main():
    m = inputs.mesh_interval(N_ELEM)
    rows = []
    for T in TS:
        r = pitching.pitch(m.coords, m.elems, m.c, KAPPA, T)
        for p in PS:
            t0 = time.time()
            F, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, lambda x: inputs.sine_product_1d(x, 0.0), None)
            lay = tdg.front_layout(m.coords, m.elems, p)
            E = energy.front_energy(F, lay.wq, m.c)
            rows.append({"p": p, "T": T, "n_tents": int(len(r["level"])), "energy": E,
                         "rel_energy_error": (math.pi ** 2 / 4 - E) / (math.pi ** 2 / 4)})
            print(f"T={T} p={p} E={E:.15e} {time.time() - t0:.0f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "energy_oracle.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.tdg.sweep + oracle.energy.front_energy "
                             "(tests/golden/make_energy_oracle.py)", "rows": rows}, f, indent=1)


if __name__ == "__main__":
    main()
