"""Pins of the zero-Dirichlet wall (odd ghost mirror) in the oracle.

- The prediction (Eq. 4) reproduces cell averages of a linear function that
  vanishes on a Dirichlet wall exactly, also in the cells next to the wall:
  the odd mirror extends it linearly (an even mirror would bend it).
- 1D Burgers from sin(2 pi x) (odd about both walls) with Dirichlet walls is
  the periodic run.
- 2D Burgers with Dirichlet walls and eps = 0 equals an independent numpy
  finite-volume solver whose ghost cells are odd mirrors (Butcher RK)."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I
from tests import fv_reference as R

DIR = 2


@pytest.mark.parametrize("bc,exact", [(DIR, True), (I.BC_NEUMANN, False)])
def test_prediction_exact_for_linear_data_at_walls(bc, exact):
    """f(x) = x on [0, 1] vanishes on the left wall: with the odd mirror the
    prediction of level L from coarse leaves on level L-1 reproduces its cell
    averages exactly in the left half, wall cells included"""
    L = 6
    n = 1 << L
    p = I.Problem(dim=1, equation=I.EQ_BURGERS, max_level=L, min_level=L - 1, eps=0.0,
                  bc=(bc, bc, bc), adapt_mode=I.ADAPT_NEVER)
    q = ((np.arange(n) + 0.5) / n)[None, :]  # cell averages of f(x) = x
    o = oracle.Oracle(p, q)
    o.set_tree(np.full(n, L - 1, dtype=np.uint8))  # coarse leaves everywhere
    u = o.uniform()[0]  # level L rebuilt by prediction from level L-1 and its ghosts
    err = np.abs(u - q[0])[: n // 2].max()
    if exact:
        assert err <= 1e-15
    else:
        assert err > 1e-4  # an even mirror bends the extension at the wall


def test_odd_data_dirichlet_equals_periodic_1d():
    p, q = I.burgers_1d(L=9, eps=1e-3)
    out = []
    for bc in (I.BC_PERIODIC, DIR):
        o = oracle.Oracle(p.replace(bc=(bc,) * 3), q)
        o.step(0.3)  # through shock formation
        out.append(o.uniform()[0])
    scale = np.abs(out[0]).max()
    assert np.abs(out[0] - out[1]).max() <= 1e-12 * scale


@pytest.mark.parametrize("rk", [2, 3])
def test_dirichlet_2d_eps0_equals_fv(rk):
    L = 6
    n = 1 << L
    p, q = I.burgers_2d(L=L, eps=0.0, min_level=3, rk_order=rk, time_mode=I.TIME_GTS)
    p = p.replace(bc=(DIR, DIR, DIR))
    o = oracle.Oracle(p, q)
    dt = 0.4 / n
    o.iterate(dt, 20)
    u = o.uniform()[0]
    fv = R.rk_solve(q[0].copy(), lambda v: R.burgers_rhs_nd(v, 1.0 / n, (DIR, DIR)), dt, 20, rk)
    assert np.abs(u - fv).max() <= 1e-12 * np.abs(fv).max()
    # and it differs from the periodic run: the walls matter in 2D
    fvp = R.rk_solve(q[0].copy(), lambda v: R.burgers_rhs_nd(v, 1.0 / n, (0, 0)), dt, 20, rk)
    assert np.abs(fvp - fv).max() > 1e-6


def test_dirichlet_3d_eps0_equals_fv():
    """corner ghosts take the product of the per-direction signs"""
    L = 4
    n = 1 << L
    p, q = I.burgers_3d(L=L, eps=0.0, min_level=2, time_mode=I.TIME_GTS, bc=DIR)
    o = oracle.Oracle(p, q)
    dt = 0.3 / n
    o.iterate(dt, 8)
    u = o.uniform()[0]
    fv = R.rk_solve(q[0].copy(), lambda v: R.burgers_rhs_nd(v, 1.0 / n, (DIR, DIR, DIR)), dt, 8, 3)
    assert np.abs(u - fv).max() <= 1e-12 * np.abs(fv).max()
