"""Pins for oracle/adjoint.py.

* dot-product identity with the forward oracle: for the linear sweep F
  (g_D = 0, fixed tents), <lambda, F f> = <F^* lambda, f> for random f, lambda;
* finite differences of the L2 misfit J(f0) = 1/2 ||U_h(T) - U_obs||^2.
"""
import numpy as np
import pytest

from oracle import adjoint, pitching, tdg
from paper_1907_02367_gb300 import inputs


def _setup(dim):
    if dim == 1:
        m, p, T = inputs.mesh_interval(5), 3, 0.4
    elif dim == 2:
        m, p, T = inputs.mesh_square(3, 0.2, seed=4), 3, 0.25
    else:
        m, p, T = inputs.mesh_cube(1, 0.0, seed=3), 2, 0.15
    kappa = inputs.pitch_kappa(m)
    r = pitching.pitch(m.coords, m.elems, m.c, kappa, T)
    return m, p, r


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_dot_product_identity(dim):
    m, p, r = _setup(dim)
    lay = tdg.front_layout(m.coords, m.elems, p)
    shape = lay.wq.shape + (dim + 2,)
    rng = np.random.default_rng(dim)
    f = rng.standard_normal(shape)
    lam = rng.standard_normal(shape)
    Ff, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None, front0=f)
    Fl = adjoint.adjoint_sweep(m.coords, m.elems, m.c, p, r, lam)
    lhs = float(np.sum(lam * Ff))
    rhs = float(np.sum(Fl * f))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), np.linalg.norm(lam) * np.linalg.norm(Ff))


def test_misfit_gradient_finite_differences():
    m, p, r = _setup(2)
    lay = tdg.front_layout(m.coords, m.elems, p)
    x = lay.xq.reshape(-1, 2)
    f0 = inputs.gaussian_pulse((0.5, 0.5), 0.3)(x).reshape(lay.wq.shape + (4,))
    obs, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None,
                       front0=inputs.gaussian_pulse((0.45, 0.55), 0.3)(x).reshape(f0.shape))

    def J(f):
        F, _ = tdg.sweep(m.coords, m.elems, m.c, p, r, None, None, front0=f)
        return adjoint.misfit_gradient(F, obs, lay.wq)

    j0, gT = J(f0)
    g0 = adjoint.adjoint_sweep(m.coords, m.elems, m.c, p, r, gT)
    rng = np.random.default_rng(7)
    d = rng.standard_normal(f0.shape)
    eps = 1e-5
    fd = (J(f0 + eps * d)[0] - J(f0 - eps * d)[0]) / (2 * eps)
    an = float(np.sum(g0 * d))
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12)
