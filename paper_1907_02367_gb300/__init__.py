"""GB300-native tent-pitched space-time Trefftz-DG solver for the acoustic
wave equation (Perugia, Schoberl, Stocker, Wintersteiger).

The numerics run in libtp (C ABI, include/tp.h): host C++ for pitching and
tables, hand-written sm_103a CUDA kernels for the layer-by-layer tent solve.
This package is the thin Python layer over it: `Tents`, `Basis` and `Solver`
mirror tp_pitch_mesh / tp_build_basis / tp_create ... tp_energy; `TentSweep`
and `speed_gradient` differentiate the sweep.  `inputs` builds the seeded
workloads; `lshape` and `energy_study` run the studies of Section 6.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _binding as B

__all__ = ["Tents", "Basis", "Solver", "TentSweep", "speed_gradient", "pitch_mesh", "build_basis",
           "load_library"]


def load_library():
    return B.load()


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
    groups when one CTA cannot hold all of them).  tents: a Tents object to
    sweep over instead of pitching the mesh with c (the wave speeds always
    come from c; see speed_gradient).  All device memory handed to libtp is
    torch CUDA float64 memory; the current torch stream is passed to every
    call."""

    def __init__(self, coords, elems, c, p: int, T: float, kappa: float, alpha: float = 0.5,
                 nrhs: int = 1, tents: Tents | None = None, precision: str = "fp64",
                 schedule: str = "dataflow", bnd_type=None, beta: float = 0.5):
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
                                    else B.TP_SCHED_LEVELS)
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

    def solve_layer(self, level: int, stream=None):
        B.check(B.load().tp_solve_layer(self.handle, int(level), B.stream_ptr(stream)))

    def advance(self, level_begin: int = 1, level_end: int | None = None, stream=None):
        if level_end is None:
            level_end = self.n_levels + 1
        B.check(B.load().tp_advance(self.handle, int(level_begin), int(level_end), B.stream_ptr(stream)))

    def adjoint(self, lam_T, out=None, stream=None):
        """Gradient with respect to the initial front of a functional whose
        gradient with respect to the final front is lam_T (tp_adjoint)."""
        import torch
        assert lam_T.is_cuda and lam_T.dtype == torch.float64 and lam_T.is_contiguous()
        assert lam_T.numel() == self.nrhs * self.n_front * self.n_comp
        if out is None:
            out = torch.empty(self.front_shape(), dtype=torch.float64, device="cuda")
        B.check(B.load().tp_adjoint(self.handle, B.tensor_ptr(lam_T), B.tensor_ptr(out), B.stream_ptr(stream)))
        return out

    def autotune(self, stream=None):
        """tp_autotune: pick the sweep schedule (one launch per level, or the
        dataflow sweep with clusters of 1/2/4/8 CTAs) by timing full sweeps.
        Returns (chosen, ms): chosen = 0 for per-level launches, else the
        cluster size."""
        c, ms = ct.c_int32(), ct.c_double()
        B.check(B.load().tp_autotune(self.handle, B.stream_ptr(stream), ct.byref(c), ct.byref(ms)))
        return int(c.value), float(ms.value)

    def energy(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.nrhs, dtype=torch.float64, device="cuda")
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

    def dofs_per_sweep(self) -> int:
        """Trefftz dofs advanced by one full sweep: sum over tents of dim U^p, times nrhs."""
        return self.tents.n_tents * self.basis.nb * self.nrhs

    def __del__(self):
        if getattr(self, "handle", None) and B._lib is not None:
            B._lib.tp_destroy_ctx(self.handle)
            self.handle = None


def _make_tent_sweep():
    import torch

    class TentSweep(torch.autograd.Function):
        """front(T) = F(front(0)) through libtp, differentiable: the backward
        pass is the reverse tent sweep (tp_adjoint).  g_D must be zero (the
        map is then linear)."""

        @staticmethod
        def forward(ctx, front0, solver):
            solver.set_state(front0.contiguous())
            solver.advance()
            out, _ = solver.get_state()
            ctx.solver = solver
            return out

        @staticmethod
        def backward(ctx, grad_out):
            return ctx.solver.adjoint(grad_out.contiguous()), None

    return TentSweep


class _LazyTentSweep:
    _cls = None

    def apply(self, front0, solver):
        if _LazyTentSweep._cls is None:
            _LazyTentSweep._cls = _make_tent_sweep()
        return _LazyTentSweep._cls.apply(front0, solver)


TentSweep = _LazyTentSweep()


def speed_gradient(coords, elems, c, p: int, T: float, kappa: float, front0, lam_T, gD=None,
                   rel_step: float = 1e-6, **solver_kw):
    """Gradient of J(c) = <lam_T, front_T(c)> with respect to the wave speed of
    each material (the distinct values of c, all elements of a material
    moving together), the tents pitched once with c and held fixed.

    Central differences of two GPU sweeps per material,
    dJ/dc_m ~ (J(c_m (1 + s)) - J(c_m (1 - s))) / (2 s c_m), s = rel_step:
    each sweep runs in a context created with the perturbed speeds over the
    same Tents (tp_create reads the speeds from the mesh and the tent times
    from the pitched tents).  front0, lam_T: CUDA float64 tensors of
    front_shape(); gD: boundary data as for Solver.set_state (independent of
    c: the boundary points depend only on the mesh and the tents).
    solver_kw goes to Solver (precision, bnd_type, alpha, beta, schedule).
    Returns (speeds (M,) float64, dJ/dc (M,) float64) as numpy arrays."""
    import torch
    c = np.ascontiguousarray(c, dtype=np.float64)
    tents = Tents(coords, elems, c, kappa, T)
    speeds = np.unique(c)
    grad = np.zeros(len(speeds))
    for m, cm in enumerate(speeds):
        J = []
        for sgn in (1.0, -1.0):
            cp = c.copy()
            cp[c == cm] = cm * (1.0 + sgn * rel_step)
            s = Solver(coords, elems, cp, p, T, kappa, tents=tents, **solver_kw)
            s.set_state(front0, gD)
            s.advance()
            F, _ = s.get_state()
            st = s.sync_status()
            if st[0] != 0:
                raise RuntimeError(f"speed_gradient: device status {st[0]} at tent {st[1]}")
            J.append(float(torch.sum(lam_T * F)))
        grad[m] = (J[0] - J[1]) / (2.0 * rel_step * cm)
    return speeds, grad
