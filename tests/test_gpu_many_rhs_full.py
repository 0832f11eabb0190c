"""The 3+1D many-right-hand-side workload at full size (48 000 tetrahedra,
p = 3, 64 seeded Gaussian pulses, swept as two groups of 32 right-hand
sides): the library advances all 64 columns over the first two levels
(3076 tents), and columns 0 and 63 match the oracle's values for the same
tents, stored by tests/golden/make_many_rhs_3d_oracle.py because the oracle
takes minutes per column at this size: at 256 seeded front entries within
the parity bound times the front's norm, and in the front's norm."""
import json
import os

import numpy as np
import pytest

from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "many_rhs_3d_oracle.json")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-8)])
def test_many_rhs_3d_full_size_first_levels(cuda_device, precision, tol):
    import torch
    import paper_1907_02367_gb300 as pkg
    with open(GOLDEN) as f:
        g = json.load(f)
    w = inputs.workload("many_rhs_3d")
    m = w.mesh
    pulses = inputs.gaussian_pulses_3d()
    s = pkg.Solver(m.coords, m.elems, m.c, w.p, w.T, w.kappa, nrhs=len(pulses), precision=precision)
    lev = s.tents.export()["level"]
    assert int(np.sum(lev <= g["levels"])) == g["n_tents"]
    xq, _ = s.front_points()
    f0 = torch.empty(s.front_shape(), dtype=torch.float64, device="cuda")
    for r, pulse in enumerate(pulses):          # one column at a time through host memory
        f0[r].copy_(torch.from_numpy(np.ascontiguousarray(pulse(xq))).reshape(f0.shape[1:]))
    s.set_state(f0)
    s.advance(1, g["levels"] + 1)
    assert s.sync_status() == (0, 0)
    front, _ = s.get_state()
    for col in g["columns"]:
        flat = front[col["column"]].reshape(-1).cpu().numpy()
        pos = np.asarray(col["sample_pos"])
        ref = np.asarray(col["sample_val"])
        assert np.max(np.abs(flat[pos] - ref)) <= tol * col["front_norm"], col["column"]
        assert abs(float(np.linalg.norm(flat)) - col["front_norm"]) <= tol * col["front_norm"]
