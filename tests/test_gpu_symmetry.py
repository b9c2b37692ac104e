"""Symmetries of the CUDA path itself, checked without the oracle: swapping
two axes of the data swaps them in the whole adaptive solve (tree and
fields, momentum components swapped).  The GPU sums the directional flux
differences in a fixed order, so the values agree to round-off."""
import numpy as np
import pytest

from paper_1905_08717_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_08717_gb300 import build
    build.build()


@pytest.mark.parametrize("rk,mode,flux", [(3, I.TIME_LT, 0), (2, I.TIME_LT, 1)])
def test_adaptive_2d_solve_is_transpose_invariant(rk, mode, flux):
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, min_level=3, rk_order=rk, time_mode=mode)
    p = p.replace(flux=flux)
    qt = q.transpose(0, 2, 1)[[0, 2, 1, 3]].copy()
    a, b = pkg.Solver(p, q), pkg.Solver(p, qt)
    a.step(0.05)
    b.step(0.05)
    ka, kb = a.leaves()[0], b.leaves()[0]
    assert {tuple(r) for r in ka[:, :3].tolist()} == {(l, j, i) for l, i, j in kb[:, :3].tolist()}
    ua, ub = a.uniform(), b.uniform().transpose(0, 2, 1)[[0, 2, 1, 3]]
    assert np.abs(ua - ub).max() <= 1e-13 * np.abs(ua).max()
    a.close()
    b.close()


def test_adaptive_3d_blast_keeps_the_cube_symmetry():
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_3d_blast(L=6, eps=1e-2, min_level=2, precision=I.PREC_FP64)
    s = pkg.Solver(p, q)
    s.step(0.02)
    u = s.uniform()  # [v][z][y][x]
    keys = {tuple(r) for r in s.leaves()[0].tolist()}
    for axes, comps, swap in (((1, 3, 2), [0, 2, 1, 3, 4], (1, 0, 2)),
                              ((3, 2, 1), [0, 3, 2, 1, 4], (2, 1, 0)),
                              ((2, 1, 3), [0, 1, 3, 2, 4], (0, 2, 1))):
        up = u.transpose((0,) + axes)[comps]
        assert np.abs(u - up).max() <= 1e-13 * np.abs(u).max()
        assert {(r[0],) + tuple(r[1 + k] for k in swap) for r in keys} == keys
    s.close()
