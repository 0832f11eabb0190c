"""oracle.parallel.sweep_levels (the tents of a level split over processes)
must reproduce the serial oracle sweep over the same levels bit for bit:
tents of one level share no element (Section 2.2), so the chunks' results
merge without any arithmetic."""
import numpy as np

from oracle import parallel, pitching, tdg
from paper_1907_02367_gb300 import inputs


def test_level_parallel_sweep_equals_serial():
    w = inputs.workload("inclusion_small")
    m = w.mesh
    r = pitching.pitch(m.coords, m.elems, m.c, w.kappa, w.T)
    lay = tdg.front_layout(m.coords, m.elems, w.p)
    f0 = np.asarray(w.init(lay.xq.reshape(-1, 2))).reshape(lay.wq.shape + (4,))
    L = 3
    Fp, taup, done = parallel.sweep_levels(m.coords, m.elems, m.c, w.p, r, f0, L, nproc=3)
    nt = int(np.sum(np.asarray(r["level"]) <= L))
    assert done == nt and nt > 20
    Fs, taus = tdg.sweep(m.coords, m.elems, m.c, w.p, r, None, front0=f0, tent_range=(0, nt))
    assert np.array_equal(Fp, Fs)
    assert np.array_equal(taup, taus)
