"""Benchmark: Trefftz dofs advanced per second for the tent-pitched Trefftz-DG sweep.

Workload (N = 1): the 3+1D many-right-hand-side configuration -- unit cube,
20^3 jittered hexahedra split into 48 000 tetrahedra (seed 4), c = 1, p = 3
(dim U^3 = 30 unknowns per tent), 64 seeded Gaussian pulses advanced
together and sharing every tent's matrix, T = 1 (468 243 tents in 1099
levels).  One step = reset the front to the 64 initial fields + the full
sweep (one CUDA graph holding the persistent dataflow sweep kernel).
dofs advanced per step = sum over tents of dim U^p x 64.

`value` is the mixed path (float-float assembly on the binary32 pipes,
binary32 inverse of the equilibrated tent matrix, refinement to float-float
accuracy); the binary64 path runs the same workload beside it (`fp64`).
Each has its roofline against the measured peak of the ALU pipe it runs on.
The mixed error is given against the binary64 sweep (whole front, all 64
columns) and against the CPU oracle after the first level (every touched
front entry of one column).

--impl reference times the CPU oracle (plain numpy, FP64) on the host cores,
on the tents of the first level (independent tents, split over processes).
Under torchrun each rank runs an independent replica (no data exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

# the oracle's processes each run numpy on one core
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_var] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Trefftz dofs advanced/s, mixed vs FP64 at rel err ≤1e-8; % of roofline"
UNIT = "dofs/s"
WORKLOAD = "many_rhs_3d"
NRHS = 64
CONFIG = {"workload": "3+1D many-RHS mixed precision: unit cube, 20^3 seeded jittered hexes x 6 tets "
                      "= 48000 tets, c=1, p=3 (30 dofs/tent), 64 seeded Gaussian pulses sharing the tent "
                      "matrices, T=1, dataflow sweep in one CUDA graph",
          "n_elem": 48000, "p": 3, "T": 1.0, "nrhs": NRHS, "precision": "mixed",
          "l2": "inputs larger than L2: the 64-column front is 7.9 GB against a 129 MB L2"}
# instructions of one compensated float-float multiply-add of the mixed path
# (product and its error by fmaf: 4, TwoSum of the running sum: 6, error sum: 2)
FF_INSTR_PER_FMA = 12


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
    """Flops (2 per multiply-add) of one sweep, counted from the method's
    operations per tent (patch of P elements, Q front points each,
    nb = dim U^p, nrhs right-hand sides sharing the tent matrix):
      * basis at the P*Q bottom and P*Q top points, and again at the top points
        for the outflow: monomial chain (nmono - 1) + U-values (nnz of the U
        coefficient table); first derivatives from U-values ((n+1) nb products);
      * symmetric Gram of (n+2) rows per point: (n+2) nb (nb+1)/2 (once per tent);
      * right-hand sides (n+2) nb nrhs per point; outflow (n+2) nb nrhs per point;
      * LU nb^3/3 (once per tent) and the triangular solves nb^2 nrhs;
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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return platform.processor() or platform.machine()


def oracle_level1(nproc: int, single_tents: int):
    """The oracle as it stands on the first level of the workload's sweep
    (column 0): the level's tents are independent, so they run split over
    nproc processes (oracle.parallel); and one process alone on the first
    single_tents tents.  Returns (all-core record, single-thread record,
    oracle front after level 1, the level-1 tent list)."""
    from paper_1907_02367_gb300 import inputs
    from oracle import parallel, pitching, tdg
    w = inputs.workload(WORKLOAD)
    m = w.mesh
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T, max_level=1)
    lay = tdg.front_layout(m.coords, m.elems, w.p)
    pulse = inputs.gaussian_pulses_3d()[0]
    f0 = np.asarray(pulse(lay.xq.reshape(-1, 3))).reshape(lay.wq.shape + (5,))
    nt = len(r["vert"])
    nb = 30
    t0 = time.perf_counter()
    F, tau, done = parallel.sweep_levels(m.coords, m.elems, m.c, w.p, r, f0, 1, nproc=nproc)
    dt_all = time.perf_counter() - t0
    n1 = min(single_tents, nt)
    t0 = time.perf_counter()
    tdg.sweep(m.coords, m.elems, m.c, w.p, r, None, front0=f0, tent_range=(0, n1))
    dt_one = time.perf_counter() - t0
    model = _cpu_model()
    all_core = {"value": done * nb / dt_all, "unit": UNIT, "cores": nproc, "kind": "oracle",
                "sample": f"the {done} independent tents of level 1 of column 0, split over {nproc} "
                          f"processes ({dt_all:.1f} s wall, numpy FP64, one thread each; {model})"}
    single = {"value": n1 * nb / dt_one, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"the first {n1} tents of level 1 of column 0 in one process ({dt_one:.1f} s, "
                        f"numpy FP64, one thread; {model})"}
    return all_core, single, F, r


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import paper_1907_02367_gb300 as pkg
    from paper_1907_02367_gb300 import inputs

    # the CPU legs first: the oracle's process pool starts before any GPU use
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nproc = os.cpu_count() or 1
        cpu = oracle_level1(nproc, args.cpu_tents)

    torch.cuda.set_device(local)
    w = inputs.workload(WORKLOAD)
    m = w.mesh
    pulses = inputs.gaussian_pulses_3d()
    fp64_peak, fp32_peak = pkg.measure_alu_peaks()
    ff_peak = fp32_peak / FF_INSTR_PER_FMA        # float-float multiply-adds at the binary32 pipe's rate
    tents = pkg.Tents(m.coords, m.elems, m.c, w.kappa, w.T)
    te = tents.export()
    stream = torch.cuda.current_stream()

    def make(precision):
        return pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, nrhs=NRHS, precision=precision,
                          tents=tents, rhs_split=args.rhs_split)

    solver = make("mixed")
    xq, _ = solver.front_points()
    front0_host = torch.empty(solver.front_shape(), dtype=torch.float64).pin_memory()
    for r in range(NRHS):
        front0_host[r].copy_(torch.from_numpy(np.ascontiguousarray(pulses[r](xq))).reshape(front0_host.shape[1:]))
    front0 = front0_host.to("cuda")
    dofs = solver.dofs_per_sweep()
    flops = algorithmic_flops(solver, te, m)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_sweeps(s, steps, warmup):
        for _ in range(warmup):
            s.set_state(front0)
            s.advance()
        torch.cuda.synchronize()
        st = s.sync_status()
        if st[0] != 0:
            raise RuntimeError(f"device status {st[0]} at tent {st[1]}")
        barrier()
        total = sweep = 0.0
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            em = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.set_state(front0)
            em.record(stream)
            s.advance()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            sweep += em.elapsed_time(e1)
        barrier()
        return max_over_ranks(total, world) / steps, max_over_ranks(sweep, world) / steps

    clocks = ClockSampler(local)
    clocks.start()
    ms_step, ms_sweep = timed_sweeps(solver, args.steps, args.warmup)
    clk = clocks.stop()
    mixed_front, _ = solver.get_state()
    st_mixed = solver.sync_status()

    # end to end through the public API with host buffers: H2D of the 64
    # initial fields from pinned memory, the sweep, D2H of the final front
    out_host = torch.empty(solver.front_shape(), dtype=torch.float64).pin_memory()
    front_dev = torch.empty_like(front0)
    e2e_steps = min(args.steps, args.e2e_steps)
    barrier()
    e_ms = 0.0
    for _ in range(e2e_steps):
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
    e_step = max_over_ranks(e_ms, world) / e2e_steps
    nbytes = front0.numel() * 8
    del out, front_dev

    # the binary64 path on the same workload, and the mixed error against it
    fp64 = None
    if not args.no_fp64:
        s64 = make("fp64")
        ms64_step, ms64_sweep = timed_sweeps(s64, args.fp64_steps, 1)
        f64_front, _ = s64.get_state()
        rel_vs_fp64 = float(torch.linalg.norm(mixed_front - f64_front) / torch.linalg.norm(f64_front))
        ach64 = flops / (ms64_sweep * 1e-3) / 1e12
        fp64 = {"value": whole_job_rate(dofs, world, ms64_step), "unit": UNIT, "ms_per_step": ms64_step,
                "steps": args.fp64_steps, "warmup": 1, "status": s64.sync_status()[0],
                "roofline": {"bound": "alu", "achieved": ach64, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": ach64 / fp64_peak, "traffic": None,
                             "kernel": "k_layer<3, binary64, dataflow> (tp_kernel.cuh)",
                             "note": "algorithmic flops / mean sweep duration; peak = binary64 "
                                     "multiply-add rate measured by tp_measure_alu_peaks on this GPU"}}
        mixed_front_rel = rel_vs_fp64
        del s64, f64_front
    else:
        mixed_front_rel = None

    # mixed and binary64 against the CPU oracle after level 1 (column 0, every touched entry)
    vs_oracle = None
    if cpu is not None:
        F_ref, r1 = cpu[2], cpu[3]
        from oracle import tdg as otdg
        star = otdg.vertex_star(m.elems, m.n_vert)
        touched = np.array(sorted({k for v in r1["vert"] for k in star[int(v)]}))
        vs_oracle = {"levels": 1, "column": 0, "touched_elements": int(len(touched))}
        for precision in ("mixed", "fp64"):
            s1 = make(precision)
            s1.set_state(front0)
            s1.advance(1, 2)
            g, _ = s1.get_state()
            g0 = g[0].cpu().numpy()[touched]
            vs_oracle[precision] = float(np.linalg.norm(g0 - F_ref[touched]) / np.linalg.norm(F_ref[touched]))
            del s1, g

    ach = flops / (ms_sweep * 1e-3) / 1e12
    result = {
        "metric": METRIC, "value": whole_job_rate(dofs, world, ms_step), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32x2 (float-float)",
        "data": "synthetic (seeded mesh, 64 seeded Gaussian pulses)",
        "config": dict(CONFIG, parallelism=f"replicas{world}", n_tents=tents.n_tents,
                       n_levels=tents.n_levels, dofs_per_step=dofs,
                       schedule=solver.schedule(), tensor_cores=solver.tensor_cores_used()),
        "e2e": {"value": whole_job_rate(dofs, world, e_step), "unit": UNIT,
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": e2e_steps},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": ach, "peak": ff_peak, "unit": "TFLOP/s",
                     "frac": ach / ff_peak, "traffic": None,
                     "kernel": "k_layer<3, float-float, dataflow> (tp_kernel.cuh); data moments and "
                               "outflow as exact bf16 digit products on tcgen05 (tp_tc.cuh)",
                     "sweep_ms": ms_sweep,
                     "note": "algorithmic flops of one sweep / mean duration of the sweep (events "
                             "around tp_advance on its stream: the sweep kernel and its set-up "
                             "kernel); peak = the float-float multiply-add rate, the binary32 "
                             f"multiply-add peak measured by tp_measure_alu_peaks ({fp32_peak:.1f} "
                             f"TFLOP/s) / {FF_INSTR_PER_FMA} binary32 instructions per compensated "
                             "multiply-add (the rate of the float-float path this kernel replaces; "
                             "the two contractions that carry most of the flops run on the tensor "
                             "cores, whose bf16 rate is not the bound: their products take ~2% of "
                             "the sweep)"},
        "clocks": clk,
        "mixed_status": st_mixed[0],
        "mixed_rel_err_vs_fp64": mixed_front_rel,
        "rel_err_vs_oracle": vs_oracle,
        "fp64": fp64,
        "measured_alu_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
    }
    if cpu is not None:
        result["cpu_baseline"] = cpu[0]
        result["cpu_baseline_single_thread"] = cpu[1]
    return result


def run_reference(args, rank, world):
    if rank != 0:
        return None
    nproc = os.cpu_count() or 1
    vals = []
    cb = None
    for i in range(args.warmup + args.steps):
        all_core, single, _, _ = oracle_level1(nproc, max(8, args.cpu_tents // 4))
        if i >= args.warmup:
            vals.append(all_core["value"])
            cb = all_core
    v = statistics.median(vals) if vals else None
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mesh, 64 seeded Gaussian pulses)",
            "config": dict(CONFIG, parallelism="cpu-oracle"),
            "cpu_baseline": dict(cb, value=v) if cb else None,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-tents", type=int, default=200,
                    help="tents of the single-thread oracle sample")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--rhs-split", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
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
