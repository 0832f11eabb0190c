"""Host-side checks of libtp (no GPU): the library loads and exports every
function declared in include/tp.h; its pitching equals the oracle's bit for
bit; its Trefftz basis equals the oracle's function by function (both are
correctly rounded values of the same exact rationals); argument errors are
reported, not crashed on."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from oracle import basis as obasis
from oracle import pitching
from paper_1907_02367_gb300 import _binding as B
from paper_1907_02367_gb300 import inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "tp.h")


def test_exports_every_declared_symbol(libtp):
    decl = set(re.findall(r"\b(tp_[a-z_]+)\s*\(", open(HEADER).read()))
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(libtp, name), name
    assert decl == set(B.EXPORTED)


MESHES = [
    ("interval16", lambda: inputs.mesh_interval(16), 0.9, 1.0),
    ("interval7", lambda: inputs.mesh_interval(7), 0.75, 0.6),
    ("square5", lambda: inputs.mesh_square(5, 0.2, seed=3), None, 0.7),
    ("square22", lambda: inputs.mesh_square(22, 0.2, seed=2), None, 1.0),
    ("cube2", lambda: inputs.mesh_cube(2, 0.1, seed=4), None, 0.4),
    ("lshape_uniform8", lambda: inputs.mesh_lshape(0.125, 1.0), None, 1.0),
    ("lshape_graded035", lambda: inputs.mesh_lshape(0.35, 1.0 / 3.0), None, 1.0),
    ("inclusion_graded005", lambda: inputs.mesh_inclusion_graded(h_max=0.05), None, 0.5),
]


@pytest.mark.parametrize("name,mk,kappa,T", MESHES, ids=[m[0] for m in MESHES])
def test_pitching_bit_exact_vs_oracle(libtp, name, mk, kappa, T):
    import paper_1907_02367_gb300 as pkg
    m = mk()
    if kappa is None:
        kappa = inputs.pitch_kappa(m)
    lib = pkg.Tents(m.coords, m.elems, m.c, kappa, T).export()
    ref = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    for k in ("vert", "level", "t_bot", "t_top"):
        assert np.array_equal(lib[k], ref[k]), k
    assert lib["n_levels"] == ref["n_levels"]


def test_pitching_heterogeneous_speed_bit_exact(libtp):
    import paper_1907_02367_gb300 as pkg
    m = inputs.mesh_square(6, 0.2, seed=8)
    cen = m.coords[m.elems].mean(axis=1)
    m.c[:] = np.where(np.linalg.norm(cen - 0.5, axis=1) < 0.25, 3.0, 1.0)
    kappa = inputs.pitch_kappa(m)
    lib = pkg.Tents(m.coords, m.elems, m.c, kappa, 0.5).export()
    ref = pitching.pitch(m.coords, m.elems, m.c, kappa, 0.5)
    for k in ("vert", "level", "t_bot", "t_top"):
        assert np.array_equal(lib[k], ref[k]), k


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 3), (1, 8), (2, 2), (2, 4), (2, 5), (3, 2), (3, 3), (3, 4)])
def test_basis_equals_oracle_function_by_function(libtp, dim, p):
    import paper_1907_02367_gb300 as pkg
    b = pkg.Basis(dim, p)
    exps, coef = b.export()
    ob = obasis.TrefftzBasis(dim, p)
    assert b.nb == ob.nb == obasis.dim_U(dim, p)
    key = {tuple(e): i for i, e in enumerate(exps.tolist())}
    M = np.zeros((ob.nb, b.nmono))
    for i, (k, al) in enumerate(ob.monos):
        M[:, key[(k,) + tuple(al)]] = ob.coef[:, i]
    rows_lib = sorted(map(tuple, coef))
    rows_ora = sorted(map(tuple, M))
    assert rows_lib == rows_ora          # identical binary64 values


def test_argument_errors(libtp):
    h = ct.c_void_p()
    assert libtp.tp_build_basis(2, 0, ct.byref(h)) == B.TP_ERR_ARG
    assert libtp.tp_build_basis(4, 3, ct.byref(h)) == B.TP_ERR_ARG
    assert b"dim" in libtp.tp_last_error()
    m = inputs.mesh_interval(4)
    arrs = B._MeshArrays(m.coords, m.elems, m.c)
    prm = B.make_params(3, 1.0, 0.0)
    assert libtp.tp_pitch_mesh(ct.byref(arrs.desc), ct.byref(prm), ct.byref(h)) == B.TP_ERR_ARG
    bad = B._MeshArrays(m.coords, np.array([[0, 9]] * 4), m.c)
    prm = B.make_params(3, 1.0, 0.9)
    assert libtp.tp_pitch_mesh(ct.byref(bad.desc), ct.byref(prm), ct.byref(h)) == B.TP_ERR_ARG
    neg = B._MeshArrays(m.coords, m.elems, -m.c)
    assert libtp.tp_pitch_mesh(ct.byref(neg.desc), ct.byref(prm), ct.byref(h)) == B.TP_ERR_ARG


def test_boundary_kind_markers(libtp):
    """tp_mesh_desc.bnd_type: 0/1 per element face are accepted (entries of
    interior faces are ignored), any other value of a boundary face is an
    argument error naming the element; a wrongly shaped marker array is
    refused by the binding."""
    h = ct.c_void_p()
    prm = B.make_params(3, 0.5, 0.9)
    m = inputs.mesh_square(3, 0.2, seed=5)
    ok = inputs.boundary_marker(m, lambda x: x[0] < 1e-12)
    arrs = B._MeshArrays(m.coords, m.elems, m.c, ok)
    assert libtp.tp_pitch_mesh(ct.byref(arrs.desc), ct.byref(prm), ct.byref(h)) == B.TP_OK
    libtp.tp_destroy_tents(h)
    bad = ok.copy()
    k, o = np.argwhere(inputs.boundary_marker(m, lambda x: True) == 1)[0]
    bad[k, o] = 2
    arrs = B._MeshArrays(m.coords, m.elems, m.c, bad)
    assert libtp.tp_pitch_mesh(ct.byref(arrs.desc), ct.byref(prm), ct.byref(h)) == B.TP_ERR_ARG
    assert b"bnd_type" in libtp.tp_last_error()
    with pytest.raises(ValueError):
        B._MeshArrays(m.coords, m.elems, m.c, ok[:, :2])


def test_no_cpu_fallback(libtp, tmp_path):
    """The product path fails loudly without a GPU or without the built
    library: the Solver refuses to run on a machine without CUDA (this test
    only runs there), and loading a library that was not built raises."""
    import torch
    import paper_1907_02367_gb300 as pkg
    if not torch.cuda.is_available():
        m = inputs.mesh_interval(4)
        with pytest.raises(RuntimeError, match="CUDA"):
            pkg.Solver(m.coords, m.elems, m.c, 3, 0.5, 0.9)
    saved = B._lib
    try:
        B._lib = None
        with pytest.raises(OSError, match="not built"):
            B.load(str(tmp_path / "missing_libtp.so"))
    finally:
        B._lib = saved


@pytest.mark.parametrize("name,levels", [("many_rhs_3d", 2), ("inclusion_graded", 4)])
def test_full_size_pitching_prefix_matches_oracle(libtp, name, levels):
    """The two large workloads' pitching: the library's tents of the first
    levels equal, bit for bit and in order, the oracle's (the oracle pitches
    up to that level only: its full pitch of the graded mesh takes tens of
    minutes); the full-size GPU parity tests compare these tents."""
    from oracle import pitching
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload(name)
    m = w.mesh
    lib = pkg.Tents(m.coords, m.elems, m.c, w.kappa, w.T).export()
    ref = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T, max_level=levels)
    n = len(ref["vert"])
    assert n > 3000 and int(np.sum(lib["level"] <= levels)) == n
    for key in ("vert", "t_bot", "t_top", "level"):
        assert np.array_equal(lib[key][:n], ref[key]), key
    if name == "inclusion_graded":
        assert len(lib["vert"]) == 19661640 and lib["n_levels"] == 97363
    else:
        assert len(lib["vert"]) == 468243 and lib["n_levels"] == 1099
