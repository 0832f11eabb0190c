"""GB300-native tent-pitched space-time Trefftz-DG solver for the acoustic
wave equation (Perugia, Schoberl, Stocker, Wintersteiger).

The numerics run in libtp (C ABI, include/tp.h): host C++ for pitching and
tables, hand-written sm_103a CUDA kernels for the layer-by-layer tent solve.
This package is the thin Python layer over it: `Tents`, `Basis` and `Solver`
mirror tp_pitch_mesh / tp_build_basis / tp_create ... tp_energy; `TentSweep` and
`Solver.speed_gradient` differentiate the sweep (tp_adjoint).  `inputs` builds the seeded
workloads; `lshape` and `energy_study` run the studies of Section 6.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _binding as B

__all__ = ["Tents", "Basis", "Solver", "TentSweep", "pitch_mesh", "build_basis", "load_library",
           "measure_alu_peaks"]


def load_library():
    return B.load()


def measure_alu_peaks(stream=None):
    """tp_measure_alu_peaks: measured (binary64, binary32) fused multiply-add
    peaks of the current GPU in TFLOP/s."""
    f64, f32 = ct.c_double(), ct.c_double()
    B.check(B.load().tp_measure_alu_peaks(ct.byref(f64), ct.byref(f32), B.stream_ptr(stream)))
    return float(f64.value), float(f32.value)


class Tents:
    """Result of tp_pitch_mesh (Section 2.2 tent pitching)."""

    def __init__(self, coords, elems, c, kappa: float, T: float):
        lib = B.load()
        self._mesh = B._MeshArrays(coords, elems, c)
        prm = B.make_params(1, T, kappa)
        h = ct.c_void_p()
        B.check(lib.tp_pitch_mesh(ct.byref(self._mesh.desc), ct.byref(prm), ct.byref(h)))
        self.handle = h
        self.kappa, self.T = float(kappa), float(T)
        n = ct.c_int64()
        L = ct.c_int32()
        B.check(lib.tp_tents_info(h, ct.byref(n), ct.byref(L)))
        self.n_tents, self.n_levels = int(n.value), int(L.value)

    def export(self) -> dict:
        n = self.n_tents
        vert = np.zeros(n, np.int32)
        tb = np.zeros(n)
        tt = np.zeros(n)
        lev = np.zeros(n, np.int32)
        B.check(B.load().tp_tents_export(self.handle, vert.ctypes.data, tb.ctypes.data,
                                         tt.ctypes.data, lev.ctypes.data))
        return {"vert": vert, "t_bot": tb, "t_top": tt, "level": lev, "n_levels": self.n_levels}

    def __del__(self):
        if getattr(self, "handle", None) and B._lib is not None:
            B._lib.tp_destroy_tents(self.handle)
            self.handle = None


def pitch_mesh(coords, elems, c, kappa, T) -> Tents:
    return Tents(coords, elems, c, kappa, T)


class Basis:
    """Result of tp_build_basis (Section 3, eq. 3.1)."""

    def __init__(self, dim: int, p: int):
        lib = B.load()
        h = ct.c_void_p()
        B.check(lib.tp_build_basis(int(dim), int(p), ct.byref(h)))
        self.handle = h
        self.dim, self.p = int(dim), int(p)
        nb = ct.c_int32()
        nm = ct.c_int32()
        B.check(lib.tp_basis_info(h, ct.byref(nb), ct.byref(nm)))
        self.nb, self.nmono = int(nb.value), int(nm.value)

    def export(self):
        exps = np.zeros((self.nmono, self.dim + 1), np.int32)
        coef = np.zeros((self.nb, self.nmono))
        B.check(B.load().tp_basis_export(self.handle, exps.ctypes.data, coef.ctypes.data))
        return exps, coef

    def __del__(self):
        if getattr(self, "handle", None) and B._lib is not None:
            B._lib.tp_destroy_basis(self.handle)
            self.handle = None


def build_basis(dim, p) -> Basis:
    return Basis(dim, p)


class Solver:
    """A tp_ctx: device-resident mesh, tents, tables and front state.

    precision "fp64": assembly, residual and outflow in binary64.  "mixed":
    the same in float-float on the binary32 pipes.  Both invert the
    equilibrated local matrix in binary32 and refine the solution in their
    own precision (a direct binary64 LU where the refinement does not settle).
    alpha, beta: the penalties of eq. (2.5) (Dirichlet, interface and Neumann
    facets).  bnd_type: optional (n_elem, dim+1) array, 1 marks the boundary
    facet opposite local vertex o of element k as Neumann (sigma.n = g_N),
    else Dirichlet; boundary_kinds() tells which data each boundary point
    takes.  nrhs right-hand sides share the tents and their matrices (in
    groups when one CTA cannot hold all of them); rhs_split: 0 picks how a
    tent's right-hand sides are shared out over the CTAs of its cluster, 1
    keeps them together, 2/4/8 gives each CTA that fraction of them
    (tp_params.rhs_split).  track_dissipation: every tent adds the energy it
    loses (the jump terms of eq. 2.5) to a sum that energy_and_dissipation()
    reports.  ckpt_stride: levels between the forward checkpoints of the
    wave-speed gradient (adjoint(..., dJ_dc=...)); 0 = no gradient with
    respect to c.  tensor_cores: True lets the mixed forward sweep with split
    right-hand sides run its data moments and outflow as exact digit
    products on the tensor cores where the plan allows it
    (tp_params.tensor_cores; tensor_cores_used() tells); False keeps the
    float-float sums.  tents: a Tents object to
    sweep over instead of pitching the mesh with c (the wave speeds always
    come from c; see speed_gradient).  All device memory handed to libtp is
    torch CUDA float64 memory; the current torch stream is passed to every
    call."""

    def __init__(self, coords, elems, c, p: int, T: float, kappa: float, alpha: float = 0.5,
                 nrhs: int = 1, tents: Tents | None = None, precision: str = "fp64",
                 schedule: str = "dataflow", bnd_type=None, beta: float = 0.5, rhs_split: int = 0,
                 track_dissipation: bool = False, ckpt_stride: int = 0, tensor_cores: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libtp Solver needs a CUDA device")
        lib = B.load()
        self._mesh = B._MeshArrays(coords, elems, c, bnd_type)
        self.tents = tents if tents is not None else Tents(coords, elems, c, kappa, T)
        self.basis = Basis(self._mesh.coords.shape[1], p)
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        self.precision = precision
        if schedule not in ("dataflow", "levels"):
            raise ValueError("schedule must be 'dataflow' or 'levels'")
        self.params = B.make_params(p, T, kappa, alpha=alpha, beta=beta, nrhs=nrhs,
                                    precision=B.TP_FP64 if precision == "fp64" else B.TP_MIXED,
                                    schedule=B.TP_SCHED_DATAFLOW if schedule == "dataflow"
                                    else B.TP_SCHED_LEVELS, rhs_split=rhs_split,
                                    dissipation=1 if track_dissipation else 0, ckpt_stride=ckpt_stride,
                                    tensor_cores=0 if tensor_cores else -1)
        h = ct.c_void_p()
        B.check(lib.tp_create(ct.byref(self._mesh.desc), self.tents.handle, self.basis.handle,
                              ct.byref(self.params), ct.byref(h)))
        self.handle = h
        nf, ncomp, nbnd, nlev = ct.c_int64(), ct.c_int32(), ct.c_int64(), ct.c_int32()
        B.check(lib.tp_ctx_info(h, ct.byref(nf), ct.byref(ncomp), ct.byref(nbnd), ct.byref(nlev)))
        self.n_front, self.n_comp = int(nf.value), int(ncomp.value)
        self.n_bnd, self.n_levels = int(nbnd.value), int(nlev.value)
        self.dim = self._mesh.coords.shape[1]
        self.n_elem = self._mesh.elems.shape[0]
        self.Q = self.n_front // self.n_elem
        self.nrhs = int(nrhs)
        self.p = int(p)

    # -- host-side geometry ------------------------------------------------
    def front_points(self):
        xq = np.zeros((self.n_front, self.dim))
        wq = np.zeros(self.n_front)
        B.check(B.load().tp_front_points(self.handle, xq.ctypes.data, wq.ctypes.data))
        return xq, wq

    def boundary_points(self):
        xt = np.zeros((max(self.n_bnd, 0), self.dim + 1))
        if self.n_bnd:
            B.check(B.load().tp_boundary_points(self.handle, xt.ctypes.data))
        return xt

    def boundary_kinds(self):
        """Per boundary point: the facet's outward unit normal (n_bnd, dim) and
        kind (n_bnd,), 0 = Dirichlet (data g_D), 1 = Neumann (data g_N)."""
        nrm = np.zeros((max(self.n_bnd, 0), self.dim))
        kind = np.zeros(max(self.n_bnd, 0), np.int8)
        if self.n_bnd:
            B.check(B.load().tp_boundary_kinds(self.handle, nrm.ctypes.data, kind.ctypes.data))
        return nrm, kind

    # -- device state ------------------------------------------------------
    def front_shape(self):
        return (self.nrhs, self.n_elem, self.Q, self.n_comp)

    def set_state(self, front, gD=None, stream=None):
        import torch
        assert front.is_cuda and front.dtype == torch.float64 and front.is_contiguous()
        assert front.numel() == self.nrhs * self.n_front * self.n_comp
        gptr = None
        if gD is not None:
            assert gD.is_cuda and gD.dtype == torch.float64 and gD.is_contiguous()
            assert gD.numel() == self.nrhs * self.n_bnd
            gptr = B.tensor_ptr(gD)
        B.check(B.load().tp_set_state(self.handle, B.tensor_ptr(front), gptr, B.stream_ptr(stream)))

    def set_probes(self, points, times):
        """tp_set_probes: U_h at every (point, time) sample during the next
        forward sweeps (points (n, dim) inside the mesh, increasing times)."""
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, self.dim)
        ts = np.ascontiguousarray(times, dtype=np.float64).reshape(-1)
        B.check(B.load().tp_set_probes(self.handle, int(len(pts)), pts.ctypes.data, int(len(ts)), ts.ctypes.data))
        self._probe_shape = (self.nrhs, len(ts), len(pts))

    def get_probes(self, stream=None):
        """tp_get_probes: CUDA float64 tensor (nrhs, n_times, n_points) of U_h."""
        import torch
        out = torch.empty(self._probe_shape, dtype=torch.float64, device="cuda")
        B.check(B.load().tp_get_probes(self.handle, B.tensor_ptr(out), B.stream_ptr(stream)))
        return out

    def set_front(self, front, tau, stream=None):
        """tp_set_front: resume from a front and its vertex times (e.g. what
        get_state returned after some levels)."""
        import torch
        assert front.is_cuda and front.dtype == torch.float64 and front.is_contiguous()
        assert front.numel() == self.nrhs * self.n_front * self.n_comp
        assert tau.is_cuda and tau.dtype == torch.float64 and tau.is_contiguous()
        assert tau.numel() == self._mesh.coords.shape[0]
        B.check(B.load().tp_set_front(self.handle, B.tensor_ptr(front), B.tensor_ptr(tau), B.stream_ptr(stream)))

    def set_limits(self, max_polls: int = 0, max_refine: int = -1):
        """tp_set_limits: dependency-wait polls and refinement steps (defaults for 0 / -1)."""
        B.check(B.load().tp_set_limits(self.handle, int(max_polls), int(max_refine)))

    def inject_wait(self, tent: int, extra: int):
        """tp_inject_wait: make tent `tent` wait for completions that never come (testing)."""
        B.check(B.load().tp_inject_wait(self.handle, int(tent), int(extra)))

    def solve_stats(self, nhist: int = 41):
        """tp_solve_stats: (tents solved by the direct LU, histogram of refinement steps)."""
        lu = ct.c_int64()
        hist = np.zeros(nhist, np.int64)
        B.check(B.load().tp_solve_stats(self.handle, ct.byref(lu), hist.ctypes.data, int(nhist)))
        return int(lu.value), hist

    def solve_layer(self, level: int, stream=None):
        B.check(B.load().tp_solve_layer(self.handle, int(level), B.stream_ptr(stream)))

    def advance(self, level_begin: int = 1, level_end: int | None = None, stream=None):
        if level_end is None:
            level_end = self.n_levels + 1
        B.check(B.load().tp_advance(self.handle, int(level_begin), int(level_end), B.stream_ptr(stream)))

    def adjoint(self, lam_T, out=None, dJ_dc=None, stream=None):
        """Gradient with respect to the initial front of a functional whose
        gradient with respect to the final front is lam_T (tp_adjoint).
        dJ_dc: optional CUDA float64 tensor of n_elem entries that receives
        the gradient with respect to the wave speed (per element; summed over
        a material's elements it is dJ/dc of the material), computed in the
        same reverse sweep from the initial state of the last set_state (the
        solver must be created with ckpt_stride > 0)."""
        import torch
        assert lam_T.is_cuda and lam_T.dtype == torch.float64 and lam_T.is_contiguous()
        assert lam_T.numel() == self.nrhs * self.n_front * self.n_comp
        if out is None:
            out = torch.empty(self.front_shape(), dtype=torch.float64, device="cuda")
        gptr = None
        if dJ_dc is not None:
            assert dJ_dc.is_cuda and dJ_dc.dtype == torch.float64 and dJ_dc.is_contiguous()
            assert dJ_dc.numel() == self.n_elem
            gptr = B.tensor_ptr(dJ_dc)
        B.check(B.load().tp_adjoint(self.handle, B.tensor_ptr(lam_T), gptr, B.tensor_ptr(out),
                                    B.stream_ptr(stream)))
        return out

    def speed_gradient(self, lam_T, stream=None):
        """dJ/dc per element (CUDA float64, n_elem) of J = <lam_T, front(T)>
        from the initial state of the last set_state (tp_adjoint)."""
        import torch
        g = torch.empty(self.n_elem, dtype=torch.float64, device="cuda")
        self.adjoint(lam_T, dJ_dc=g, stream=stream)
        return g

    def autotune(self, stream=None):
        """tp_autotune: pick the sweep schedule (one launch per level, or the
        dataflow sweep with clusters of 1/2/4/8 CTAs) by timing full sweeps.
        Returns (chosen, ms): chosen = 0 for per-level launches, else the
        cluster size."""
        c, ms = ct.c_int32(), ct.c_double()
        B.check(B.load().tp_autotune(self.handle, B.stream_ptr(stream), ct.byref(c), ct.byref(ms)))
        return int(c.value), float(ms.value)

    def energy(self, stream=None):
        """Energy flux through the current front per right-hand side (nrhs,)."""
        return self.energy_and_dissipation(stream=stream)[:, 0]

    def energy_and_dissipation(self, out=None, stream=None):
        """tp_energy: (nrhs, 2) CUDA tensor, column 0 the energy flux through
        the current front, column 1 the energy the swept tents lost since
        set_state (zero unless the solver tracks it, track_dissipation=True)."""
        import torch
        if out is None:
            out = torch.empty((self.nrhs, 2), dtype=torch.float64, device="cuda")
        B.check(B.load().tp_energy(self.handle, B.tensor_ptr(out), B.stream_ptr(stream)))
        return out

    def get_state(self, front=None, tau=None, stream=None):
        import torch
        if front is None:
            front = torch.empty(self.front_shape(), dtype=torch.float64, device="cuda")
        if tau is None:
            tau = torch.empty(self._mesh.coords.shape[0], dtype=torch.float64, device="cuda")
        B.check(B.load().tp_get_state(self.handle, B.tensor_ptr(front), B.tensor_ptr(tau),
                                      B.stream_ptr(stream)))
        return front, tau

    def sync_status(self):
        s, i = ct.c_int32(), ct.c_int64()
        B.check(B.load().tp_sync_status(self.handle, ct.byref(s), ct.byref(i)))
        return int(s.value), int(i.value)

    def schedule(self) -> dict:
        """tp_ctx_schedule: dataflow (bool), cluster (CTAs per tent),
        rhs_split (CTAs the right-hand sides are split over), rhs_groups."""
        v = [ct.c_int32() for _ in range(4)]
        B.check(B.load().tp_ctx_schedule(self.handle, *[ct.byref(x) for x in v]))
        return {"dataflow": bool(v[0].value), "cluster": int(v[1].value), "rhs_split": int(v[2].value),
                "rhs_groups": int(v[3].value)}

    def tensor_cores_used(self) -> bool:
        """tp_ctx_tensor_cores: whether the forward sweep runs the data moments
        and the outflow of single-material tents on the tensor cores."""
        v = ct.c_int32()
        B.check(B.load().tp_ctx_tensor_cores(self.handle, ct.byref(v)))
        return bool(v.value)

    def dofs_per_sweep(self) -> int:
        """Trefftz dofs advanced by one full sweep: sum over tents of (materials
        of the tent) x dim U^p, times nrhs (Section 4.2: one polynomial per
        material of the tent's patch)."""
        el = self._mesh.elems
        pairs = np.stack([el.reshape(-1).astype(np.float64), np.repeat(self._mesh.c, el.shape[1])], axis=1)
        uv = np.unique(pairs, axis=0)
        ng = np.bincount(uv[:, 0].astype(np.int64), minlength=self._mesh.coords.shape[0])
        vert = self.tents.export()["vert"]
        return int(ng[vert].sum()) * self.basis.nb * self.nrhs

    def __del__(self):
        if getattr(self, "handle", None) and B._lib is not None:
            B._lib.tp_destroy_ctx(self.handle)
            self.handle = None


def _make_tent_sweep():
    import torch

    class TentSweep(torch.autograd.Function):
        """front(T) = F(front(0); c) through libtp, differentiable: the
        backward pass is the reverse tent sweep (tp_adjoint), which returns
        the gradient with respect to the initial front and, when a tensor c
        of the element speeds is passed, with respect to c (the solver must
        then be created with ckpt_stride > 0; c must hold the speeds the
        solver was created with, the gradient is taken there with the tents
        held fixed)."""

        @staticmethod
        def forward(ctx, front0, solver, c=None):
            solver.set_state(front0.contiguous())
            solver.advance()
            out, _ = solver.get_state()
            ctx.solver = solver
            ctx.with_c = c is not None
            return out

        @staticmethod
        def backward(ctx, grad_out):
            g = grad_out.contiguous()
            if ctx.with_c:
                dc = torch.empty(ctx.solver.n_elem, dtype=torch.float64, device="cuda")
                return ctx.solver.adjoint(g, dJ_dc=dc), None, dc
            return ctx.solver.adjoint(g), None, None

    return TentSweep


class _LazyTentSweep:
    _cls = None

    def apply(self, front0, solver, c=None):
        if _LazyTentSweep._cls is None:
            _LazyTentSweep._cls = _make_tent_sweep()
        return _LazyTentSweep._cls.apply(front0, solver, c)


TentSweep = _LazyTentSweep()
