"""The heterogeneous-medium example of Section 6.7: a Gaussian pulse
U_0 = exp(-|x - x_0|^2 / delta^2), v_0 = 0, x_0 = (1, 1), delta = 0.01, in
[0, 2]^2 with c = 1 for x_1 <= 1.2 and c = 3 beyond, homogeneous Dirichlet
data, p = 4, T = 1, spatial mesh size 0.01 on the slow side and 0.03 on the
fast one (inputs.mesh_two_speeds).  The output is the point functional
    U_C(t) = || U_h(., t) ||_L1(Omega_C),  Omega_C = [1 - e, 1 + e] x [0.25 - e, 0.25 + e],  e = 2^-7,
on a grid of times, from the library's point outputs (tp_set_probes): U_h
at a tensor Gauss-Legendre grid of Omega_C at every time, summed with the
rule's weights.  The paper reads three arrivals off this curve: the weak
Huygens wave that ran along the interface in the fast medium, the initial
wave, and the wave reflected at the interface.

    python -m paper_1907_02367_gb300.interface_study [--h-left 0.01 --h-right 0.03 --times 201]

One JSON line with the curve, its local maxima and the sweep's time.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import inputs


def box_rule(center=(1.0, 0.25), eps: float = 2.0 ** -7, m: int = 8):
    """Tensor Gauss-Legendre points and weights of [cx - eps, cx + eps] x [cy - eps, cy + eps]."""
    g, w = np.polynomial.legendre.leggauss(m)
    x = center[0] + eps * g
    y = center[1] + eps * g
    X, Y = np.meshgrid(x, y, indexing="ij")
    W = np.outer(w, w) * eps * eps
    return np.stack([X.ravel(), Y.ravel()], axis=1), W.ravel()


def local_maxima(t, f, min_rel: float = 1e-3):
    """Times of the interior local maxima of f above min_rel * max f."""
    out = []
    for i in range(1, len(f) - 1):
        if f[i] > f[i - 1] and f[i] >= f[i + 1] and f[i] > min_rel * np.max(f):
            out.append(float(t[i]))
    return out


def run(h_left: float = 0.01, h_right: float = 0.03, n_times: int = 201, p: int = 4, T: float = 1.0,
        precision: str = "fp64", delta: float = 0.01, quad: int = 8) -> dict:
    import torch
    from . import Solver
    m = inputs.mesh_two_speeds(h_left, h_right)
    kappa = inputs.pitch_kappa(m)
    s = Solver(m.coords, m.elems, m.c, p, T, kappa, precision=precision)
    pts, wts = box_rule(m=quad)
    times = np.linspace(0.0, T, n_times)
    s.set_probes(pts, times)
    xq, _ = s.front_points()
    pulse = inputs.gaussian_pulse((1.0, 1.0), delta)
    s.set_state(torch.tensor(pulse(xq)[None], dtype=torch.float64, device="cuda").contiguous())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.advance()
    e1.record()
    e1.synchronize()
    status = s.sync_status()
    U = s.get_probes()[0].cpu().numpy()                 # (n_times, n_points)
    uc = np.abs(U) @ wts
    return {"study": "Section 6.7 point output U_C(t)", "n_elem": m.n_elem, "n_tents": s.tents.n_tents,
            "n_levels": s.n_levels, "p": p, "precision": precision, "status": list(status),
            "sweep_ms": e0.elapsed_time(e1), "times": times.tolist(), "U_C": uc.tolist(),
            "local_maxima_t": local_maxima(times, uc)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--h-left", type=float, default=0.01)
    ap.add_argument("--h-right", type=float, default=0.03)
    ap.add_argument("--times", type=int, default=201)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    args = ap.parse_args(argv)
    print(json.dumps(run(args.h_left, args.h_right, args.times, precision=args.precision)), flush=True)


if __name__ == "__main__":
    main()
