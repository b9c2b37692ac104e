"""The seeded input recipes against what they stand for: the paper's printed
initial states (golden fixture), exact cell averages checked by independent
Gauss-Legendre quadrature, and the textbook Sod states.  The generators hold
none of the method's arithmetic; these tests fix that the workloads are the
paper's."""
import os

import numpy as np
import pytest

from paper_1905_08717_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "euler2d_laxliu6_initial_states.txt")


def _golden_states():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    return {int(r[0]): tuple(float(x) for x in r[1:]) for r in rows}


def test_quadrant_problem_is_the_papers_table():
    st = _golden_states()
    assert sorted(st) == [1, 2, 3, 4]
    p, q = I.euler_2d_quadrants(L=4, seed=0)
    g = p.phys[0]
    assert g == 1.4 and p.cfl == 0.5 and p.t_end == 0.25
    assert p.bc[:2] == (I.BC_NEUMANN, I.BC_NEUMANN)
    n = 16
    xc = (np.arange(n) + 0.5) / n
    for j in range(n):          # y (rows)
        for i in range(n):      # x (x-fastest)
            right, top = xc[i] > 0.5, xc[j] > 0.5
            quad = 1 if (right and top) else 2 if top else 3 if not right else 4
            rho, pr, vx, vy = st[quad]
            expect = [rho, rho * vx, rho * vy, pr / (g - 1) + 0.5 * rho * (vx * vx + vy * vy)]
            assert np.allclose(q[:, j, i], expect, rtol=0, atol=1e-15), (i, j, quad)


def _gl_average(f, lo, hi, npts=12):
    """cell average of f over [lo, hi] by Gauss-Legendre quadrature"""
    x, w = np.polynomial.legendre.leggauss(npts)
    xs = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
    return 0.5 * np.sum(w * f(xs))


def test_sine_initial_data_are_exact_cell_averages():
    _, u1 = I.burgers_1d(L=5)
    n = 32
    for i in (0, 3, 17, 31):
        ref = _gl_average(lambda x: np.sin(2 * np.pi * x), i / n, (i + 1) / n)
        assert abs(u1[0, i] - ref) < 1e-14
    p2, u2 = I.burgers_2d_paper(L=4)
    assert p2.bc[:2] == (I.BC_DIRICHLET0, I.BC_DIRICHLET0) and p2.t_end == 0.9
    m = 16
    for (j, i) in ((0, 0), (5, 9), (15, 2)):
        ax = _gl_average(lambda x: np.sin(2 * np.pi * x), i / m, (i + 1) / m)
        ay = _gl_average(lambda y: np.sin(2 * np.pi * y), j / m, (j + 1) / m)
        assert abs(u2[0, j, i] - ax * ay) < 1e-14


def test_sod_states():
    p, q = I.euler_1d_sod(L=5)
    g = p.phys[0]
    n = 32
    xc = (np.arange(n) + 0.5) / n
    left = xc < 0.5
    assert np.all(q[0][left] == 1.0) and np.all(q[0][~left] == 0.125)
    assert np.all(q[1] == 0.0)
    assert np.allclose(q[2][left], 1.0 / (g - 1)) and np.allclose(q[2][~left], 0.1 / (g - 1))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_quadrant_states_follow_their_recipe(seed):
    st = I.quadrant_states(seed)
    assert st.shape == (4, 4)
    assert np.all((st[:, 0] >= 0.5) & (st[:, 0] <= 3.0))
    assert np.all((st[:, 1] >= 0.5) & (st[:, 1] <= 2.0))
    assert np.all(np.abs(st[:, 2:]) <= 0.75)
    assert np.array_equal(st, I.quadrant_states(seed))  # seeded
