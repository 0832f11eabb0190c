"""ctypes binding of libtp (include/tp.h): argument marshalling only.

Every step of the solve runs inside libtp's CUDA kernels; PyTorch supplies
device memory and the current stream.  There is no fallback: if libtp.so is
missing or the device is absent the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtp.so")

TP_OK, TP_ERR_ARG, TP_ERR_CAUSALITY, TP_ERR_SINGULAR, TP_ERR_NOCONV = 0, 1, 2, 3, 4
TP_ERR_TIMEOUT, TP_ERR_CUDA, TP_ERR_OOM, TP_ERR_UNSUPPORTED = 5, 6, 7, 8
TP_FP64, TP_MIXED = 0, 1
TP_SCHED_DATAFLOW, TP_SCHED_LEVELS = 0, 1

EXPORTED = [
    "tp_last_error", "tp_pitch_mesh", "tp_tents_info", "tp_tents_export", "tp_destroy_tents",
    "tp_build_basis", "tp_basis_info", "tp_basis_export", "tp_destroy_basis", "tp_create",
    "tp_ctx_info", "tp_ctx_schedule", "tp_ctx_tensor_cores", "tp_set_probes", "tp_get_probes", "tp_set_front", "tp_set_limits", "tp_inject_wait", "tp_solve_stats",
    "tp_front_points", "tp_boundary_points", "tp_boundary_kinds", "tp_set_state", "tp_solve_layer",
    "tp_advance", "tp_adjoint", "tp_autotune", "tp_energy", "tp_get_state", "tp_sync_status", "tp_destroy_ctx",
    "tp_front_energy_noalloc", "tp_measure_alu_peaks",
]


class TpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtp error {code}: {msg}")
        self.code = code


class MeshDesc(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("n_vert", ct.c_int64), ("coords", ct.c_void_p),
                ("n_elem", ct.c_int64), ("elems", ct.c_void_p), ("c", ct.c_void_p),
                ("bnd_type", ct.c_void_p)]


class Params(ct.Structure):
    _fields_ = [("p", ct.c_int32), ("alpha", ct.c_double), ("beta", ct.c_double),
                ("kappa", ct.c_double), ("T", ct.c_double), ("precision", ct.c_int32),
                ("nrhs", ct.c_int32), ("schedule", ct.c_int32), ("rhs_split", ct.c_int32),
                ("dissipation", ct.c_int32), ("ckpt_stride", ct.c_int32), ("tensor_cores", ct.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libtp.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libtp.so not built at {path}; run __graft_entry__.build()")
    lib = ct.CDLL(path)
    vp, i32, i64, d = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
    P = ct.POINTER
    sig = {
        "tp_last_error": (ct.c_char_p, []),
        "tp_pitch_mesh": (ct.c_int, [P(MeshDesc), P(Params), P(vp)]),
        "tp_tents_info": (ct.c_int, [vp, P(i64), P(i32)]),
        "tp_tents_export": (ct.c_int, [vp, vp, vp, vp, vp]),
        "tp_destroy_tents": (None, [vp]),
        "tp_build_basis": (ct.c_int, [i32, i32, P(vp)]),
        "tp_basis_info": (ct.c_int, [vp, P(i32), P(i32)]),
        "tp_basis_export": (ct.c_int, [vp, vp, vp]),
        "tp_destroy_basis": (None, [vp]),
        "tp_create": (ct.c_int, [P(MeshDesc), vp, vp, P(Params), P(vp)]),
        "tp_ctx_info": (ct.c_int, [vp, P(i64), P(i32), P(i64), P(i32)]),
        "tp_ctx_schedule": (ct.c_int, [vp, P(i32), P(i32), P(i32), P(i32)]),
        "tp_ctx_tensor_cores": (ct.c_int, [vp, P(i32)]),
        "tp_set_probes": (ct.c_int, [vp, i32, vp, i32, vp]),
        "tp_get_probes": (ct.c_int, [vp, vp, vp]),
        "tp_set_front": (ct.c_int, [vp, vp, vp, vp]),
        "tp_set_limits": (ct.c_int, [vp, i64, i32]),
        "tp_inject_wait": (ct.c_int, [vp, i64, i32]),
        "tp_solve_stats": (ct.c_int, [vp, P(i64), vp, i32]),
        "tp_front_points": (ct.c_int, [vp, vp, vp]),
        "tp_boundary_points": (ct.c_int, [vp, vp]),
        "tp_boundary_kinds": (ct.c_int, [vp, vp, vp]),
        "tp_set_state": (ct.c_int, [vp, vp, vp, vp]),
        "tp_solve_layer": (ct.c_int, [vp, i32, vp]),
        "tp_advance": (ct.c_int, [vp, i32, i32, vp]),
        "tp_energy": (ct.c_int, [vp, vp, vp]),
        "tp_adjoint": (ct.c_int, [vp, vp, vp, vp, vp]),
        "tp_autotune": (ct.c_int, [vp, vp, P(i32), P(d)]),
        "tp_get_state": (ct.c_int, [vp, vp, vp, vp]),
        "tp_sync_status": (ct.c_int, [vp, P(i32), P(i64)]),
        "tp_destroy_ctx": (None, [vp]),
        "tp_front_energy_noalloc": (ct.c_int, [i32, i64, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "tp_measure_alu_peaks": (ct.c_int, [P(d), P(d), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != TP_OK:
        msg = load().tp_last_error()
        raise TpError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _MeshArrays:
    """Keeps contiguous copies alive while a MeshDesc points at them."""

    def __init__(self, coords, elems, c, bnd_type=None):
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        if self.coords.ndim == 1:
            self.coords = self.coords[:, None].copy()
        self.elems = np.ascontiguousarray(elems, dtype=np.int32)
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        self.bnd_type = None
        if bnd_type is not None:
            self.bnd_type = np.ascontiguousarray(bnd_type, dtype=np.int8)
            if self.bnd_type.shape != self.elems.shape:
                raise ValueError("bnd_type must have the shape of elems (n_elem, dim+1)")
        self.desc = MeshDesc(self.coords.shape[1], self.coords.shape[0], _ptr(self.coords),
                             self.elems.shape[0], _ptr(self.elems), _ptr(self.c),
                             _ptr(self.bnd_type) if self.bnd_type is not None else None)


def make_params(p, T, kappa, alpha=0.5, beta=0.5, precision=TP_FP64, nrhs=1,
                schedule=TP_SCHED_DATAFLOW, rhs_split=0, dissipation=0, ckpt_stride=0, tensor_cores=0) -> Params:
    return Params(int(p), float(alpha), float(beta), float(kappa), float(T), int(precision), int(nrhs),
                  int(schedule), int(rhs_split), int(dissipation), int(ckpt_stride), int(tensor_cores))


def stream_ptr(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def tensor_ptr(t) -> int:
    return int(t.data_ptr())
