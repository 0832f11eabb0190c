"""The graded inclusion mesh (c = 3 inside the circle |x - (0.5, 0.5)| = 0.2,
c = 1 outside, elements 10x finer at the circle) at a size the oracle cannot
sweep at p = 5: h_max = 0.05 (4450 triangles), T = 0.5, about 350 000 tents
whose pitching the CPU tests hold bit-exact against the oracle.  Checked here: the
sweep finishes with a clean device status, the energy of the flat final
front is below the initial one (the method is dissipative with g_D = 0 and
interface penalties, Section 6.5 and eq. 2.5), and the mixed path agrees
with binary64 within 1e-8."""
import numpy as np
import pytest

from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_graded_inclusion_p5_dissipative_and_mixed_agrees(cuda_device):
    import torch
    import paper_1907_02367_gb300 as pkg
    m = inputs.mesh_inclusion_graded(h_max=0.05)
    p, T = 5, 0.5
    kappa = inputs.pitch_kappa(m)
    tents = pkg.Tents(m.coords, m.elems, m.c, kappa, T)
    assert tents.n_tents > 300000
    pulse = inputs.gaussian_pulse((0.45, 0.58), 0.08)
    fronts = {}
    for precision in ("fp64", "mixed"):
        s = pkg.Solver(m.coords, m.elems, m.c, p, T, kappa, tents=tents, precision=precision)
        xq, _ = s.front_points()
        f0 = torch.tensor(pulse(xq)[None], dtype=torch.float64, device="cuda").contiguous()
        s.set_state(f0)
        e0 = float(s.energy()[0])
        s.advance()
        e1 = float(s.energy()[0])
        front, tau = s.get_state()
        assert s.sync_status() == (0, 0)
        assert bool(torch.all(tau == T))
        assert 0.0 < e1 < e0, (precision, e0, e1)
        fronts[precision] = front.cpu().numpy()
    rel = np.linalg.norm(fronts["mixed"] - fronts["fp64"]) / np.linalg.norm(fronts["fp64"])
    assert rel <= 1e-8, rel
