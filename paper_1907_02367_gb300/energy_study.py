"""Long-time energy of the tent sweep (Section 6.5): U = sin(pi x) sin(pi t)
on [0, 1] with 5 uniform elements, c = 1, homogeneous Dirichlet data, swept
to T = 100, 1000, 10000 for p = 2 ... 8.  The exact energy
E = 1/2 int (v^2 + sigma^2) dx is pi^2 / 4 at every t; the method is
dissipative, so the relative error (E - E_h) / E of the numerical energy
E_h at t = T grows with T (the paper observes linearly) and falls with p
(exponentially).  E_h is the library's energy of the flat final front.

    python -m paper_1907_02367_gb300.energy_study               # the paper's grid
    python -m paper_1907_02367_gb300.energy_study --p 4,6 --T 100

One JSON line per (p, T) on stdout.
"""
from __future__ import annotations

import argparse
import json
import math

from . import inputs

P_LIST = (2, 3, 4, 5, 6, 7, 8)
T_LIST = (100.0, 1000.0, 10000.0)
N_ELEM = 5
KAPPA = 0.9
EXACT_ENERGY = math.pi ** 2 / 4.0


def run(p: int, T: float, n_elem: int = N_ELEM, precision: str = "fp64") -> dict:
    """One sweep on the GPU from the closed form's data at t = 0."""
    import torch
    from . import Solver

    m = inputs.mesh_interval(n_elem)
    s = Solver(m.coords, m.elems, m.c, p, T, KAPPA, precision=precision)
    xq, _ = s.front_points()
    front0 = torch.tensor(inputs.sine_product_1d(xq, 0.0)[None], dtype=torch.float64,
                          device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    s.set_state(front0)
    s.advance()                                   # warm-up (graph capture, first launch)
    s.set_state(front0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance()
    e1.record(stream)
    e1.synchronize()
    E = float(s.energy()[0])
    status = s.sync_status()
    return {"p": p, "T": T, "n_elem": n_elem, "n_tents": s.tents.n_tents, "n_levels": s.n_levels,
            "energy": E, "exact_energy": EXACT_ENERGY,
            "rel_energy_error": (EXACT_ENERGY - E) / EXACT_ENERGY,
            "sweep_ms": e0.elapsed_time(e1), "precision": precision, "status": list(status)}


def study(ps=P_LIST, Ts=T_LIST, precision: str = "fp64", emit=None) -> list:
    rows = []
    for p in ps:
        for T in Ts:
            row = run(p, T, precision=precision)
            rows.append(row)
            if emit is not None:
                emit(row)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--p", default=",".join(str(p) for p in P_LIST))
    ap.add_argument("--T", default=",".join(str(t) for t in T_LIST))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    args = ap.parse_args(argv)
    study([int(v) for v in args.p.split(",")], [float(v) for v in args.T.split(",")],
          args.precision, emit=lambda r: print(json.dumps(r), flush=True))


if __name__ == "__main__":
    main()
