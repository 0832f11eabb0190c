"""Run one sweep (or a range of levels) of a seeded workload and print its
time and status: the driver for profiling a kernel on a chosen size.

    python -m paper_1907_02367_gb300.sweep_case --case cube --n 8 --nrhs 64 --precision mixed \\
        --schedule levels --levels 1 6

Cases: cube (mesh_cube(n), p = 3, the 3+1D many-pulse workload at n^3 x 6
tetrahedra, the first nrhs of gaussian_pulses_3d), square (mesh_square(n),
p = 4, standing wave), graded (mesh_inclusion_graded(h_max = 1/n), p = 5,
Gaussian pulse).  One JSON line on stdout.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--case", default="cube", choices=["cube", "square", "graded"])
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--schedule", default="dataflow", choices=["dataflow", "levels"])
    ap.add_argument("--rhs-split", type=int, default=0)
    ap.add_argument("--T", type=float, default=1.0)
    ap.add_argument("--levels", type=int, nargs=2, default=None, metavar=("BEGIN", "END"))
    ap.add_argument("--no-tensor-cores", action="store_true",
                    help="keep the float-float sums on the CUDA cores (tp_params.tensor_cores = -1)")
    args = ap.parse_args(argv)
    import torch
    from . import Solver
    if args.case == "cube":
        m, p = inputs.mesh_cube(args.n, 0.1, seed=4), 3
        pulses = inputs.gaussian_pulses_3d()
        inits = [pulses[r % len(pulses)] for r in range(args.nrhs)]
    elif args.case == "square":
        m, p = inputs.mesh_square(args.n, 0.2, seed=2), 4
        inits = [lambda x: inputs.standing_wave_2d(x, 0.0)] * args.nrhs
    else:
        m, p = inputs.mesh_inclusion_graded(h_max=1.0 / args.n), 5
        inits = [inputs.gaussian_pulse((0.45, 0.58), 0.08)] * args.nrhs
    s = Solver(m.coords, m.elems, m.c, p, args.T, inputs.pitch_kappa(m), nrhs=args.nrhs,
               precision=args.precision, schedule=args.schedule, rhs_split=args.rhs_split,
               tensor_cores=not args.no_tensor_cores)
    xq, _ = s.front_points()
    f0 = torch.empty(s.front_shape(), dtype=torch.float64, device="cuda")
    for r, f in enumerate(inits):
        f0[r].copy_(torch.from_numpy(np.ascontiguousarray(f(xq))).reshape(f0.shape[1:]))
    s.set_state(f0)
    L0, L1 = (1, s.n_levels + 1) if args.levels is None else tuple(args.levels)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.advance(L0, L1)
    e1.record()
    e1.synchronize()
    print(json.dumps({"case": args.case, "n": args.n, "n_elem": m.n_elem, "n_tents": s.tents.n_tents,
                      "levels": [L0, L1], "nrhs": args.nrhs, "precision": args.precision,
                      "schedule": s.schedule(), "tensor_cores": s.tensor_cores_used(),
                      "ms": e0.elapsed_time(e1), "status": list(s.sync_status())}))


if __name__ == "__main__":
    main()
