"""Dimensional embedding pins of the oracle: a 2D or 3D run whose data vary
along one axis only must reproduce the 1D run on every line along that axis,
with the momentum component of that axis in the 1D momentum's place and the
others zero.  Fluxes across the other axes are equal on both sides of every
cell and cancel exactly.  A transposed index, a wrong normal velocity or a
momentum component swapped between directions fails this."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I

G = 1.4


def _run(p, q, dt, n):
    o = oracle.Oracle(p, q)
    o.iterate(dt, n)
    return o.uniform()


def _sod_1d(L):
    p, q = I.euler_1d_sod(L=L, eps=0.0, min_level=2, rk_order=3, time_mode=I.TIME_GTS)
    return p.replace(adapt_mode=I.ADAPT_NEVER), q


def _embed(q1, d, axis):
    """1D Euler data (rho, m, E) [3, n] -> d-dim data varying along `axis`
    (0 = x, 1 = y, 2 = z), arrays indexed [v][z][y][x]"""
    n = q1.shape[1]
    out = np.zeros((d + 2,) + (n,) * d)
    shape = [1] * d
    shape[d - 1 - axis] = n
    for v, src in ((0, q1[0]), (1 + axis, q1[1]), (d + 1, q1[2])):
        out[v] = np.broadcast_to(src.reshape(shape), (n,) * d)
    return out


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("d,axis", [(2, 0), (2, 1), (3, 0), (3, 2)])
def test_euler_along_one_axis_reproduces_1d(d, axis, flux):
    L = 6 if d == 2 else 4
    p1, q1 = _sod_1d(L)
    p1 = p1.replace(flux=flux)
    # a moving shock tube: add a uniform velocity so that both signs of u occur
    q1 = q1.copy()
    q1[2] += 0.5 * 0.3 ** 2 * q1[0]
    q1[1] = 0.3 * q1[0]
    dt, n = 0.2 / (1 << L), 12
    u1 = _run(p1, q1, dt, n)
    pd = p1.replace(dim=d, bc=(I.BC_NEUMANN,) * 3)
    ud = _run(pd, _embed(q1, d, axis), dt, n)
    want = _embed(u1, d, axis)
    assert np.abs(ud - want).max() <= 1e-13 * np.abs(want).max()
    others = [1 + k for k in range(d) if k != axis]
    assert np.all(ud[others] == 0.0)


@pytest.mark.parametrize("d,axis", [(2, 0), (2, 1), (3, 1)])
def test_burgers_along_one_axis_reproduces_1d(d, axis):
    L = 6 if d == 2 else 4
    p1, q1 = I.burgers_1d(L=L, eps=0.0, min_level=2, rk_order=2, time_mode=I.TIME_GTS)
    p1 = p1.replace(adapt_mode=I.ADAPT_NEVER)
    dt, n = 0.4 / (1 << L), 10
    u1 = _run(p1, q1, dt, n)[0]
    nn = 1 << L
    shape = [1] * d
    shape[d - 1 - axis] = nn
    qd = np.broadcast_to(q1[0].reshape(shape), (nn,) * d)[None].copy()
    ud = _run(p1.replace(dim=d), qd, dt, n)[0]
    want = np.broadcast_to(u1.reshape(shape), (nn,) * d)
    assert np.abs(ud - want).max() <= 1e-14


@pytest.mark.parametrize("rk,mode,flux", [(3, I.TIME_LT, 0), (2, I.TIME_LT, 1), (3, I.TIME_GTS, 0)])
def test_adaptive_2d_solve_is_transpose_invariant(rk, mode, flux):
    """Swapping x and y in the data (and rho u with rho v) swaps them in the
    whole adaptive solve: the same tree transposed, the same values to
    round-off (the x and y flux differences are summed in the other order).
    This ties together the tensor-product prediction, the detail norm, the
    grading closure and both flux directions in a genuinely 2D flow."""
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, min_level=2, rk_order=rk, time_mode=mode)
    p = p.replace(flux=flux)
    qt = q.transpose(0, 2, 1)[[0, 2, 1, 3]].copy()
    a, b = oracle.Oracle(p, q), oracle.Oracle(p, qt)
    a.step(0.05)
    b.step(0.05)
    ka, kb = a.leaves()[0], b.leaves()[0]
    assert {tuple(r) for r in ka[:, :3].tolist()} == {(l, j, i) for l, i, j in kb[:, :3].tolist()}
    assert a.stats()["iters"] == b.stats()["iters"]
    ua, ub = a.uniform(), b.uniform().transpose(0, 2, 1)[[0, 2, 1, 3]]
    assert np.abs(ua - ub).max() <= 1e-13 * np.abs(ua).max()


@pytest.mark.parametrize("flux", [0, 1])
def test_adaptive_3d_blast_keeps_the_cube_symmetry(flux):
    """The 3D blast (a ball at the centre of the unit cube, Neumann walls) is
    symmetric under every swap of two axes, so the adaptive LT solve must be:
    the leaf set maps onto itself and the fields onto themselves with the
    momentum components swapped (z-direction handling included)."""
    p, q = I.euler_3d_blast(L=5, eps=1e-2, min_level=2, precision=I.PREC_FP64)
    o = oracle.Oracle(p.replace(flux=flux), q)
    o.step(0.02)
    u = o.uniform()  # [v][z][y][x]
    keys = {tuple(r) for r in o.leaves()[0].tolist()}  # (level, i, j, k) = (level, x, y, z)
    for axes, comps, swap in (((1, 3, 2), [0, 2, 1, 3, 4], (1, 0, 2)),
                              ((3, 2, 1), [0, 3, 2, 1, 4], (2, 1, 0)),
                              ((2, 1, 3), [0, 1, 3, 2, 4], (0, 2, 1))):
        up = u.transpose((0,) + axes)[comps]
        assert np.abs(u - up).max() <= 1e-13 * np.abs(u).max()
        assert {(r[0],) + tuple(r[1 + s] for s in swap) for r in keys} == keys
