"""Benchmark: Trefftz dofs advanced per second for the tent-pitched Trefftz-DG sweep.

Workload (N = 1): the 2+1D FP64 batched case -- unit square, 22x22 jittered
grid made Delaunay (968 triangles, h ~ 0.045), c = 1, p = 4 (dim U^4 = 25
unknowns per tent), standing wave cos(sqrt2 pi t) sin(pi x) sin(pi y), T = 1,
all tents of a level in one launch, the level sweep replayed as a CUDA graph.
One step = reset the front to the initial data + the full sweep (20216 tents,
320 levels) with the schedule the library's autotuner picks before timing.
dofs advanced per step = sum over tents of dim U^p x nrhs.

--impl reference times the CPU oracle (plain numpy, FP64) on a bounded
sample of the same workload (the first tents of the sweep).
Under torchrun each rank runs an independent replica (no data exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

# the CPU baseline reports the cores it uses: keep numpy's BLAS on one thread
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_var] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Trefftz dofs advanced/s, mixed vs FP64 at rel err ≤1e-8; % of roofline"
UNIT = "dofs/s"
WORKLOAD = "standing2d"
CONFIG = {"workload": "2+1D plain FP64 batched: unit square, 968-triangle seeded jittered-grid "
                      "Delaunay mesh (h~0.045), c=1, p=4 (25 dofs/tent), standing wave, T=1, "
                      "layer-parallel tents",
          "n_elem": 968, "p": 4, "T": 1.0, "nrhs": 1, "precision": "fp64",
          "l2": "flushed between timed steps (256 MiB write); working set ~1 MB < L2"}
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 rate (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)
# DRAM read + write bytes of one binary64 sweep launch of this workload, from the
# ncu capture summarised in profiles/k_layer_dataflow_standing2d.md, and the
# kernel source it was taken on
SWEEP_DRAM_BYTES = 5.153536e6 + 0.393984e6
SWEEP_DRAM_SOURCE = "ncu capture of k_layer<2,0,0,1,0> at commit d48bde1"


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest x over all ranks (the slowest rank's time); x itself at world 1."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units processed by all ranks per second, over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def algorithmic_flops(solver, tents_export, mesh) -> float:
    """FP64 flops (2 per FMA) of one sweep, counted from the method's operations
    per tent (patch of P elements, Q front points each, nb = dim U^p):
      * basis at the P*Q bottom and P*Q top points, and again at the top points
        for the outflow: monomial chain (nmono - 1) + U-values (nnz of the U
        coefficient table); first derivatives from U-values ((n+1) nb products);
      * symmetric Gram of (n+2) rows per point: (n+2) nb (nb+1)/2;
      * right-hand sides (n+2) nb nrhs per point; outflow (n+2) nb nrhs per point;
      * LU nb^3/3 and the triangular solves nb^2 nrhs;
      * Dirichlet faces: basis + nb^2 + 3 nb per face point."""
    n, nb, Q, nrhs = solver.dim, solver.basis.nb, solver.Q, solver.nrhs
    C = n + 2
    exps, coef = solver.basis.export()
    nnz_U = int(np.count_nonzero(coef))
    nmono = solver.basis.nmono
    basis = (nmono - 1) + nnz_U
    deriv = (n + 1) * nb
    star = np.bincount(mesh.elems.reshape(-1), minlength=mesh.n_vert)
    P = star[tents_export["vert"]].astype(np.float64)
    pts = P * Q
    per_point = (2 * (basis + deriv)                       # assembly: bottom + top
                 + C * nb * (nb + 1) / 2                    # Gram, symmetric
                 + C * nb * nrhs                            # RHS
                 + basis + C * nb * nrhs)                   # outflow
    fma = pts * per_point + nb ** 3 / 3.0 + nb * nb * nrhs
    fma_sum = float(fma.sum()) + solver.n_bnd * (basis + deriv + nb * nb + 3 * nb)
    return 2.0 * fma_sum


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import paper_1907_02367_gb300 as pkg
    from paper_1907_02367_gb300 import inputs

    torch.cuda.set_device(local)
    w = inputs.workload(WORKLOAD)
    m = w.mesh
    solver = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa)
    xq, _ = solver.front_points()
    front0_host = torch.tensor(w.init(xq), dtype=torch.float64).reshape(solver.front_shape())
    front0_host = front0_host.contiguous().pin_memory()
    front0 = front0_host.to("cuda")
    out_host = torch.empty(solver.front_shape(), dtype=torch.float64).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    dofs = solver.dofs_per_sweep()
    te = solver.tents.export()
    # schedule chosen by the library's autotuner (outside the timed region)
    solver.set_state(front0)
    chosen, tune_ms = (4, 0.0) if args.no_autotune else solver.autotune()
    # kernels per step: dataflow = sweep set-up + one persistent sweep kernel;
    # per-level schedule = one launch per level
    n_launch = 2 if chosen > 0 else solver.n_levels

    def step():
        solver.set_state(front0)
        solver.advance()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st, info = solver.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} at tent {info}")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    total_ms = 0.0
    sweep_ms = 0.0                          # the sweep kernel(s) alone, for the roofline
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        em = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.set_state(front0)
        em.record(stream)
        solver.advance()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        sweep_ms += em.elapsed_time(e1)
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, world)
    sweep_ms = max_over_ranks(sweep_ms, world)
    ms_step = total_ms / args.steps
    ms_sweep = sweep_ms / args.steps

    # end to end through the public API with host buffers: H2D of the initial
    # front from pinned memory, sweep, D2H of the final front, every step
    front_dev = torch.empty_like(front0)
    barrier()
    e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        front_dev.copy_(front0_host, non_blocking=True)
        solver.set_state(front_dev)
        solver.advance()
        out, _ = solver.get_state()
        out_host.copy_(out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e_ms += e0.elapsed_time(e1)
    barrier()
    e_ms = max_over_ranks(e_ms, world)
    e_step = e_ms / args.steps
    nbytes = front0.numel() * 8

    flops = algorithmic_flops(solver, te, m)
    achieved = flops / (ms_sweep * 1e-3) / 1e12
    # the mixed-precision path on the same workload (float-float assembly,
    # binary32 factorisation + refinement): dofs/s and its error against this
    # run's binary64 front (which the tests hold within 1e-11 of the oracle)
    mixed = None
    if not args.no_mixed:
        ref_front, _ = solver.get_state()
        ref_front = ref_front.clone()
        ms_solver = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, precision="mixed")
        ms_solver.set_state(front0)
        if not args.no_autotune:
            ms_solver.autotune()
        for _ in range(args.warmup):
            ms_solver.set_state(front0)
            ms_solver.advance()
        torch.cuda.synchronize()
        mx_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ms_solver.set_state(front0)
            ms_solver.advance()
            e1.record(stream)
            e1.synchronize()
            mx_ms += e0.elapsed_time(e1)
        mst = ms_solver.sync_status()
        mfront, _ = ms_solver.get_state()
        rel = float(torch.linalg.norm(mfront - ref_front) / torch.linalg.norm(ref_front))
        mixed = {"value": whole_job_rate(dofs, world, mx_ms / args.steps), "unit": UNIT,
                 "ms_per_step": mx_ms / args.steps, "rel_err_vs_fp64": rel, "status": mst[0]}
    result = {
        "metric": METRIC, "value": whole_job_rate(dofs, world, ms_step), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded mesh, closed-form standing wave)",
        "config": dict(CONFIG, parallelism=f"replicas{world}", n_tents=solver.tents.n_tents,
                       n_levels=solver.n_levels, dofs_per_step=dofs,
                       schedule=("dataflow, clusters of %d CTAs" % chosen) if chosen > 0 else "one launch per level"),
        "e2e": {"value": whole_job_rate(dofs, world, e_step), "unit": UNIT,
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": n_launch * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": SWEEP_DRAM_BYTES,
                     "traffic_source": SWEEP_DRAM_SOURCE,
                     "kernel": "k_layer<dim 2, binary64> (tp_kernel.cuh)",
                     "sweep_ms": ms_sweep,
                     "note": "algorithmic FP64 flops of one sweep / mean duration of the sweep "
                             "(events around tp_advance on its stream: the sweep kernel and its "
                             "set-up kernel); peak = GB300 FP64, 152 SMs x 2 DFMA/clk x 2 flop "
                             "x 2.07 GHz"},
        "clocks": clk,
        "mixed": mixed,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.cpu_tents)
    return result


def cpu_baseline(n_tents: int):
    """The oracle, as it stands, on the host cores: the first n_tents of the
    same sweep (bounded sample)."""
    from paper_1907_02367_gb300 import inputs
    from oracle import pitching, tdg
    w = inputs.workload(WORKLOAD)
    m = w.mesh
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    n = min(n_tents, len(r["vert"]))
    t0 = time.perf_counter()
    tdg.sweep(m.coords, m.elems, m.c, w.p, r, w.init, None, tent_range=(0, n))
    dt = time.perf_counter() - t0
    nb = (w.p + 1) ** 2
    return {"value": n * nb / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {len(r['vert'])} tents of the same sweep ({dt:.1f} s, numpy FP64, 1 thread)"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(max(50, args.cpu_tents // 20))
    samples = []
    for _ in range(args.steps):
        cb = cpu_baseline(args.cpu_tents)
        vals.append(cb["value"])
        samples.append(cb)
    v = statistics.median(vals)
    cb = dict(samples[0], value=v)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mesh, closed-form standing wave)",
            "config": dict(CONFIG, parallelism="cpu-oracle"),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-tents", type=int, default=8000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default schedule (dataflow sweep) instead of tuning it")
    ap.add_argument("--no-mixed", action="store_true")
    args = ap.parse_args()
    rank, world, local = _dist()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
