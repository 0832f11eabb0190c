"""The L-shape benchmark of Section 6.6 (Table 1): the singular solution
U = cos(10 t) sin(2 phi / 3) J_2/3(10 r) on [-1,1]^2 minus [0,1]x[-1,0],
p = 3, T = 1, on uniform meshes and on meshes graded towards the reentrant
corner (h_K = h_max r^(1 - mu), mu = 1/3).  For each mesh: elements,
tents, total dofs (sum over tents of dim U^3 = 16), the L2 error of U at
t = T against the closed form (the recovered U of Section 5 at the front's
quadrature points), the rate against (total dofs)^(-1/3) as the paper
plots it, and the sweep's device time.

    python -m paper_1907_02367_gb300.lshape                     # Table 1's meshes
    python -m paper_1907_02367_gb300.lshape --uniform 0.25,0.125 --graded 0.35

One JSON line per mesh on stdout.  Meshes, initial and Dirichlet data are
synthetic (the paper's meshes are not published): see inputs.mesh_lshape.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import inputs

UNIFORM_H = (0.07, 0.05, 0.03, 0.01)      # Table 1, uniform meshes
GRADED_H = (0.12, 0.10, 0.08, 0.06)       # Table 1, graded meshes


def dof_rate(dofs0: float, err0: float, dofs1: float, err1: float) -> float:
    """Convergence rate against (total dofs)^(-1/3), the abscissa of the
    paper's convergence plot: log(err0 / err1) / log((dofs1 / dofs0)^(1/3))."""
    return math.log(err0 / err1) / (math.log(dofs1 / dofs0) / 3.0)


def run_mesh(mesh, p: int = 3, T: float = 1.0, precision: str = "fp64", repeats: int = 1,
             a: float = 10.0, nu: float = 2.0 / 3.0) -> dict:
    """One row: sweep the mesh on the GPU with the corner solution's initial
    and Dirichlet data, return the error of U at T and the sweep time."""
    import torch
    from . import Solver

    sol = inputs.bessel_corner_solution(a, nu)
    s = Solver(mesh.coords, mesh.elems, mesh.c, p, T, inputs.pitch_kappa(mesh), precision=precision)
    xq, wq = s.front_points()
    front0 = torch.tensor(sol(xq, 0.0)[None], dtype=torch.float64, device="cuda").contiguous()
    xt = s.boundary_points()
    gD = torch.tensor(sol(xt[:, :-1], xt[:, -1])[:, 1][None], dtype=torch.float64,
                      device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    s.set_state(front0, gD)
    s.advance()                                   # warm-up (graph capture, first launch)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(1, repeats)):
        s.set_state(front0, gD)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.advance()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    status = s.sync_status()
    front, tau = s.get_state()
    U = front.cpu().numpy().reshape(len(wq), -1)[:, 0]
    ex = sol(xq, T)[:, 0]
    err = math.sqrt(float(np.sum(wq * (U - ex) ** 2)))
    dofs = s.dofs_per_sweep()
    sweep_ms = float(np.median(ms))
    return {"mesh": mesh.name, "h_max": mesh.meta.get("h_max"), "mu": mesh.meta.get("mu"),
            "n_elem": mesh.n_elem, "n_tents": s.tents.n_tents, "n_levels": s.n_levels,
            "dofs": dofs, "l2_error": err, "sweep_ms": sweep_ms,
            "dofs_per_s": dofs / (sweep_ms * 1e-3), "precision": precision,
            "status": list(status), "tau_min": float(tau.min())}


def study(uniform=UNIFORM_H, graded=GRADED_H, p: int = 3, T: float = 1.0,
          precision: str = "fp64", repeats: int = 3, emit=None) -> list:
    """Rows for the uniform meshes, then the graded ones, each family with the
    rate from its previous row (None for the first)."""
    rows = []
    for hs, mu in ((uniform, 1.0), (graded, 1.0 / 3.0)):
        prev = None
        for h in hs:
            row = run_mesh(inputs.mesh_lshape(h, mu), p, T, precision, repeats)
            row["dof_rate"] = None if prev is None else dof_rate(prev["dofs"], prev["l2_error"],
                                                                  row["dofs"], row["l2_error"])
            prev = row
            rows.append(row)
            if emit is not None:
                emit(row)
    return rows


def _floats(s: str):
    return tuple(float(v) for v in s.split(",") if v.strip())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--uniform", type=_floats, default=UNIFORM_H)
    ap.add_argument("--graded", type=_floats, default=GRADED_H)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--T", type=float, default=1.0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--repeats", type=int, default=3)
    args = ap.parse_args(argv)
    study(args.uniform, args.graded, args.p, args.T, args.precision, args.repeats,
          emit=lambda r: print(json.dumps(r), flush=True))


if __name__ == "__main__":
    main()
