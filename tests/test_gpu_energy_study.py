"""GPU parity of the long-time energy study (Section 6.5): U = sin(pi x)
sin(pi t) on 5 elements swept to T = 100 (1671 tents); the library's
energy of the final front against the oracle's, and the dissipation sign."""
import numpy as np
import pytest

from oracle import energy, pitching, tdg
from paper_1907_02367_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [2, 4, 6])
def test_energy_study_matches_oracle(cuda_device, p):
    from paper_1907_02367_gb300 import energy_study
    T = 100.0
    row = energy_study.run(p, T)
    assert row["status"] == [0, 0]
    m = inputs.mesh_interval(energy_study.N_ELEM)
    r = pitching.pitch(m.coords, m.elems, m.c, energy_study.KAPPA, T)
    F, tau = tdg.sweep(m.coords, m.elems, m.c, p, r, lambda x: inputs.sine_product_1d(x, 0.0), None)
    assert np.all(tau == T)
    lay = tdg.front_layout(m.coords, m.elems, p)
    E = energy.front_energy(F, lay.wq, m.c)
    assert row["n_tents"] == len(r["level"])
    assert abs(row["energy"] - E) <= 1e-11 * E, (row["energy"], E)
    assert row["rel_energy_error"] > 0
