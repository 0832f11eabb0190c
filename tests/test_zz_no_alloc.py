"""tp_front_energy_noalloc: the allocation-free energy entry point.

Callers that may not allocate device memory at that moment (a framework that
already holds the free device memory in its own pool, or a service with a
device-memory budget fixed at start-up) use this C entry point instead of
tp_energy.  It takes every input as a caller-owned device array and keeps its
scratch in a fixed module array.  This file is named so that pytest collects
it last; it must pass on its own in a fresh process and after the others.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_1907_02367_gb300 import _binding as B
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def _state_on_curved_front(nrhs_inits):
    import torch
    import paper_1907_02367_gb300 as pkg
    w = inputs.workload("small2d")
    m = w.mesh
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, nrhs=len(nrhs_inits))
    xq, wq = s.front_points()
    f0 = np.stack([np.asarray(f(xq)) for f in nrhs_inits])
    front0 = torch.tensor(f0, dtype=torch.float64, device="cuda").contiguous()
    s.set_state(front0)
    s.advance(1, 7)                      # stop mid-sweep: the front is not flat
    front, tau = s.get_state()
    return s, m, wq, front, tau


def test_noalloc_energy_matches_tp_energy_twice(cuda_device, libtp):
    import torch
    inits = [lambda x: inputs.standing_wave_2d(x, 0.0), inputs.gaussian_pulse((0.4, 0.6), 0.2)]
    s, m, wq, front, tau = _state_on_curved_front(inits)
    ref = s.energy().cpu().numpy()
    assert s.sync_status() == (0, 0)

    # caller-owned device inputs
    coords = torch.tensor(m.coords, dtype=torch.float64, device="cuda").contiguous()
    elems = torch.tensor(m.elems, dtype=torch.int32, device="cuda").contiguous()
    c = torch.tensor(m.c, dtype=torch.float64, device="cuda").contiguous()
    X = m.coords[m.elems[0]]
    det0 = abs(np.linalg.det(X[1:] - X[0]))
    wref = torch.tensor(wq[:s.Q] / det0, dtype=torch.float64, device="cuda").contiguous()
    out = torch.full((len(inits),), float("nan"), dtype=torch.float64, device="cuda")
    stream = B.stream_ptr()
    for call in range(2):                # the shared scratch keeps the last call's contents
        rc = libtp.tp_front_energy_noalloc(2, m.n_elem, s.Q, len(inits), coords.data_ptr(),
                                           elems.data_ptr(), c.data_ptr(), tau.data_ptr(),
                                           wref.data_ptr(), front.data_ptr(), out.data_ptr(), stream)
        assert rc == B.TP_OK, libtp.tp_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref)), (call, got, ref)
        out.fill_(float("nan"))


def test_noalloc_rejects_oversized_request(cuda_device, libtp):
    rc = libtp.tp_front_energy_noalloc(2, 10, 25, 40000, 1, 1, 1, 1, 1, 1, 1, None)
    assert rc == B.TP_ERR_ARG
    assert b"exceeds the fixed scratch" in libtp.tp_last_error()
