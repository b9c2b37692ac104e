"""Pins of the oracle's time integration (Secs. 3-4; Algs. 3-9) against what
the mathematics and the paper fix: FV equivalence at eps = 0, the Butcher
form and NERK order conditions, conservation, convergence of LT to the global
step, the paper's time-order table, and the pre-shock Burgers solution."""
import os

import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I
from tests import fv_reference as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_convergence_orders.txt")


@pytest.mark.parametrize("rk", [2, 3])
def test_eps0_is_uniform_fv(rk):
    """With threshold 0 every leaf is on level L and MR-GTS, MRLT and the
    uniform FV scheme (Eq. 2 with RK in Butcher form, independent numpy code)
    give the same solution."""
    L, lb = 7, 3
    p, q = I.burgers_1d(L=L, eps=0.0, min_level=lb, rk_order=rk)
    dt = 0.5 / (1 << L)
    n = 2 * (1 << (L - lb))
    sols = []
    for mode in (I.TIME_GTS, I.TIME_LT):
        o = oracle.Oracle(p.replace(time_mode=mode), q)
        assert o.stats()["leaves_per_level"][L] == 1 << L
        o.iterate(dt, n)
        sols.append(o.uniform()[0])
    fv = R.rk_solve(q[0], lambda u: R.burgers_rhs(u, 1.0 / (1 << L)), dt, n, rk)
    assert np.array_equal(sols[0], sols[1])
    assert np.abs(sols[0] - fv).max() < 1e-13


def _ode_only(rk):
    """uniform field + D = 0: every leaf integrates u' = k u (1-u)(u-a)"""
    p, q = I.rd_bumps_2d(L=4, eps=1e-3, rk_order=rk, min_level=2)
    p = p.replace(dim=1, phys=(0.0, 100.0, 0.3) + (0.0,) * 5, bc=(I.BC_PERIODIC,) * 3)
    q = np.full((1, 16), 0.6)
    return p, q


def _f(u):
    return 100.0 * u * (1 - u) * (u - 0.3)


@pytest.mark.parametrize("rk", [2, 3])
def test_compact_rk_is_butcher_form(rk):
    """The compact stages (Sec. 3) reproduce Eqs. 8-9 with the Sec. 3 tableau."""
    p, q = _ode_only(rk)
    o = oracle.Oracle(p, q)
    o.iterate(2e-3, 1)
    keys, _ = o.leaves()
    dt = 2e-3 * 2 ** (p.max_level - keys[0, 0])  # Eq. 13: the leaf's own step
    F = o.fields()[0, :, 0]  # q^n q* q** q^{n+1} NERK1/2 NERK1/4 NERK3/4 Eq14
    A, b = R.BUTCHER[rk]
    u0 = F[0]
    K = []
    for i in range(len(b)):
        K.append(dt * _f(u0 + sum(A[i, j] * K[j] for j in range(i))))
    want = u0 + sum(bi * ki for bi, ki in zip(b, K))
    assert abs(F[3] - want) < 1e-15
    assert abs(F[1] - (u0 + K[0])) < 1e-16
    assert abs(F[7] - (F[1] + dt * _f(F[1]))) < 1e-16  # Eq. 14: q* + dt f(q*)


def _nerk2_beta(theta):
    """beta_i of the two-stage natural continuous extension from its defining
    conditions (Sec. 3): beta_1 + beta_2 = theta (order 1) and
    beta_2 c_2 = theta^2 / 2 (order 2) with c_2 = 1."""
    M = np.array([[1.0, 1.0], [0.0, 1.0]])
    return np.linalg.solve(M, np.array([theta, theta ** 2 / 2]))


def test_nerk2_beta_conditions():
    """The order conditions make NERK2 exact for q' = a + b t at any theta."""
    a, b, tn, h = 0.7, -1.3, 0.4, 0.05
    for th in (0.25, 0.5, 0.75, 1.0):
        b1, b2 = _nerk2_beta(th)
        k1 = h * (a + b * tn)
        k2 = h * (a + b * (tn + h))
        exact = a * th * h + b * (tn * th * h + (th * h) ** 2 / 2)
        assert abs(b1 * k1 + b2 * k2 - exact) < 1e-15
    # at theta = 1 the extension returns the RK2 weights b = (1/2, 1/2)
    assert np.allclose(_nerk2_beta(1.0), [0.5, 0.5])


@pytest.mark.parametrize("rk", [2, 3])
def test_stored_nerk_values(rk):
    """The oracle's stored theta = 1/2 (RK2) and 1/4, 3/4 (RK3) values are the
    NERK2 continuous extension with the betas fixed by the order conditions."""
    p, q = _ode_only(rk)
    o = oracle.Oracle(p, q)
    o.iterate(3e-3, 1)
    F = o.fields()[0, :, 0]
    k1 = F[1] - F[0]
    k2 = F[7] - F[1]
    thetas = [(0.5, 4)] if rk == 2 else [(0.25, 5), (0.75, 6)]
    for th, col in thetas:
        b1, b2 = _nerk2_beta(th)
        assert abs(F[col] - (F[0] + b1 * k1 + b2 * k2)) < 1e-15


def _offset_burgers(L, rk, reflux, eps=1e-3):
    p, q = I.burgers_1d(L=L, eps=eps, rk_order=rk)
    return p.replace(reflux=reflux), q + 0.5


@pytest.mark.parametrize("rk", [2, 3])
def test_mass_conservation_1d(rk):
    """Flux registers keep the LT scheme conservative across levels (mass to
    round-off after the shock forms); without them mass drifts."""
    drift = {}
    for reflux in (1, 0):
        p, q = _offset_burgers(8, rk, reflux)
        o = oracle.Oracle(p, q)
        m0 = o.stats()["mass"][0]
        o.step(0.4)
        s = o.stats()
        assert (s["leaves_per_level"] > 0).sum() >= 3
        drift[reflux] = abs(s["mass"][0] - m0)
    assert drift[1] < 1e-13
    assert drift[0] > 1e-8


def test_mass_conservation_2d_euler():
    """Periodic 2D Euler (all four conserved variables) with registers."""
    p, q = I.euler_2d_quadrants(L=6, eps=1e-2, seed=0)
    p = p.replace(bc=(I.BC_PERIODIC,) * 3)
    drift = {}
    for reflux in (1, 0):
        o = oracle.Oracle(p.replace(reflux=reflux), q)
        m0 = o.stats()["mass"]
        o.step(0.05)
        s = o.stats()
        assert (s["leaves_per_level"] > 0).sum() >= 3
        drift[reflux] = np.abs((s["mass"] - m0) / m0).max()
    assert drift[1] < 1e-13
    assert drift[0] > 1e-8


def test_mass_conservation_2d_burgers_rk2():
    p, q = I.burgers_2d(L=6, eps=1e-2, rk_order=2)
    q = q + 0.25
    o = oracle.Oracle(p, q)
    m0 = o.stats()["mass"][0]
    o.step(0.15)
    assert abs(o.stats()["mass"][0] - m0) < 1e-13


def _nested_map(L):
    """graded four-level fixed tree: L inside L-1 inside L-2, L-3 elsewhere"""
    lev = np.full(1 << L, L - 3, np.uint8)
    lev[32:160] = L - 2
    lev[56:128] = L - 1
    lev[72:104] = L
    return lev


def _three_level_map(L):
    lev = np.full(1 << L, L - 1, np.uint8)
    lev[40:140] = L
    lev[200:] = L - 2
    return lev


@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("tree", ["three", "nested"])
def test_lt_converges_to_gts(rk, tree):
    """At a fixed tree the LT and global-step solutions converge to each other
    at least at second order in dt (LT/NERK is second order, Sec. 4.4): the gap
    shrinks by 4x to 8x per halving of dt."""
    L = 8
    p, q = I.burgers_1d(L=L, eps=0.0, min_level=L - 3, rk_order=rk)
    p = p.replace(adapt_mode=I.ADAPT_NEVER)
    lev = _three_level_map(L) if tree == "three" else _nested_map(L)
    gaps = []
    for dt in (2e-3, 1e-3, 5e-4):
        n = int(round(0.096 / dt))
        out = []
        for mode in (I.TIME_GTS, I.TIME_LT):
            o = oracle.Oracle(p.replace(time_mode=mode), q)
            o.set_tree(lev)
            o.iterate(dt, n)
            out.append(o.uniform()[0])
        gaps.append(np.abs(out[0] - out[1]).sum() / (1 << L))
    r1, r2 = gaps[0] / gaps[1], gaps[1] / gaps[2]
    assert 3.5 < r1 < 8.5 and 3.5 < r2 < 8.5, (gaps, r1, r2)


def _orders(L, dts, rk, mode, two_level):
    sols = []
    for dt in dts:
        p, q = I.advection_gaussian_1d(L=L, rk_order=rk, time_mode=mode)
        p = p.replace(min_level=L - 1)
        o = oracle.Oracle(p, q)
        if two_level:
            o.set_tree(I.two_level_map_1d(L))
        o.iterate(dt, int(round(1.0 / dt)))
        sols.append(o.uniform()[0])
    return [np.log2(np.linalg.norm(sols[i] - sols[i + 1]) / np.linalg.norm(sols[i + 1] - sols[i + 2]))
            for i in range(len(dts) - 2)]


def _golden():
    rows = [list(map(float, ln.split())) for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    return np.array(rows)


COLUMNS = {"FV/RK2": (1, 2, 0, False), "MR/RK2": (2, 2, 0, True), "MRLT/NERK2": (4, 2, 1, True),
           "FV/RK3": (5, 3, 0, False), "MR/RK3": (6, 3, 0, True), "MRLT/NERK3": (7, 3, 1, True)}


def _check_orders(got, col, name, gold):
    if name == "MRLT/NERK3":
        # paper: 1.79, 1.92 at these steps, tending to 2; the oracle tends to 2
        # from above (its asymptote is pinned by test_nerk3_lt_asymptotic_order)
        assert all(1.9 < g < 2.9 for g in got), got
        assert got[1] < got[0]
    else:
        tol = 0.05
        for g, w in zip(got, gold[:, col]):
            assert abs(g - w) < tol, (name, got, gold[:, col])


@pytest.mark.parametrize("name", list(COLUMNS))
def test_time_order_table_reduced(name):
    """Table 1 at a quarter of the resolution (same Courant numbers)."""
    col, rk, mode, two = COLUMNS[name]
    got = _orders(7, [6.25e-4, 3.125e-4, 1.5625e-4, 7.8125e-5], rk, mode, two)
    _check_orders(got, col, name, _golden())


def test_nerk3_lt_asymptotic_order():
    """Sec. 4.5: MRLT/NERK3 loses third order on the two-level grid; its time
    order tends to 2 as dt -> 0 (Table 1: 1.79, 1.92).  On the reduced grid,
    continued to dt = 1.95e-5, the observed order decreases at every halving
    and ends within 2 +- 0.1: a scheme that kept order 3 (no LT perturbation)
    or fell to first order (a first-order coarse half-step value, as in the
    classic MRLT/RK2 column) fails.  NERK2 on the same steps stays at 2."""
    dts = [6.25e-4, 3.125e-4, 1.5625e-4, 7.8125e-5, 3.90625e-5, 1.953125e-5]
    got = _orders(7, dts, 3, 1, True)
    assert all(b < a for a, b in zip(got, got[1:])), got
    assert abs(got[-1] - 2.0) < 0.1, got
    got2 = _orders(7, dts[-3:], 2, 1, True)
    assert abs(got2[-1] - 2.0) < 0.01, got2


def _linear_profile_run(rk):
    """Linear advection q_t + q_x = 0 of q0 = x + 2 (cell averages = centre
    values) on a fixed four-level nested tree, one LT iteration at n = 0 (every
    level active).  Returns the internal nodes away from the periodic wrap."""
    L, lb = 7, 3
    lev = np.full(1 << L, L - 3, np.uint8)
    lev[40:88] = L - 2
    lev[48:80] = L - 1
    lev[56:72] = L
    x = (np.arange(1 << L) + 0.5) / (1 << L)
    p = I.Problem(dim=1, equation=I.EQ_ADVECTION, max_level=L, min_level=lb, eps=0.0, rk_order=rk,
                  adapt_mode=I.ADAPT_NEVER, phys=(1.0,) + (0.0,) * 7)
    o = oracle.Oracle(p, (x + 2.0)[None, :])
    o.set_tree(lev)
    dt = 0.25 / (1 << L)
    o.iterate(dt, 1)
    keys, f = o.nodes()
    xc = (keys[:, 1] + 0.5) / 2.0 ** keys[:, 0]
    dtl = dt * 2.0 ** (L - keys[:, 0])
    keep = (xc > 0.25) & (xc < 0.75)
    return keys[keep], f[keep, :, 0], xc[keep], dtl[keep]


@pytest.mark.parametrize("rk", [2, 3])
def test_internal_nodes_exact_for_linear_in_time_solution(rk):
    """The exact solution q = (x - t) + 2 is linear in space and time: the
    centred flux and the prediction (Eq. 4) are exact on it, the right-hand
    side is constant, so every RK stage, NERK value (Sec. 3) and tree refresh
    (Eqs. 14-18, 20-21) must reproduce the exact value at its own instant.
    This observes the internal-node values no leaf reads on a graded tree,
    including the internal-child branches of Alg. 4 (Eq. 15) and Alg. 6:
    q* = q(t^n + dt_l) after the stage-2 projection, half-step value (Eq. 17)
    = q(t^n + dt_l/2); RK3 also q** = q(t^n + dt_l/2), end value q(t^n + dt_l),
    theta = 1/4 and 3/4 values q(t^n + dt_l/4), q(t^n + 3 dt_l/4)."""
    keys, f, xc, dtl = _linear_profile_run(rk)
    # nodes with an internal child exist on three levels of the check region
    assert len(set(keys[:, 0])) >= 3 and len(keys) >= 12
    ex = lambda th: xc - th * dtl + 2.0
    want = {0: ex(0.0), 1: ex(1.0), 4: ex(0.5)}
    if rk == 3:
        want.update({2: ex(0.5), 3: ex(1.0), 5: ex(0.25), 6: ex(0.75)})
    for col, w in want.items():
        err = np.abs(f[:, col] - w).max()
        assert err < 1e-13, (col, err)


@pytest.mark.slow
@pytest.mark.parametrize("name", list(COLUMNS))
def test_time_order_table_paper_size(name):
    """Table 1 at the paper's grid and time steps."""
    col, rk, mode, two = COLUMNS[name]
    got = _orders(9, [1.6e-4, 0.8e-4, 0.4e-4, 0.2e-4], rk, mode, two)
    _check_orders(got, col, name, _golden())


def test_burgers_preshock_matches_characteristics():
    """Before the shock (t < 1/(2 pi)) the solution is u = sin(2 pi (x - u t));
    at eps = 0 the scheme converges to its cell averages at ~2nd order, and the
    adaptive MRLT solution stays within a threshold-controlled distance."""
    T = 0.1
    errs = []
    for L in (8, 9, 10):
        p, q = I.burgers_1d(L=L, eps=0.0)
        o = oracle.Oracle(p, q)
        o.step(T)
        ex = R.cell_average_1d(lambda x: R.burgers_exact_sine(x, T), 1 << L)
        errs.append(np.abs(o.uniform()[0] - ex).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 1.8).all(), (errs, orders)
    p, q = I.burgers_1d(L=10, eps=1e-4)
    o = oracle.Oracle(p, q)
    o.step(T)
    ex = R.cell_average_1d(lambda x: R.burgers_exact_sine(x, T), 1 << 10)
    err = np.abs(o.uniform()[0] - ex).mean()
    assert err < 5e-4
    assert o.stats()["leaves"] < 600


def test_euler_lax_liu_positivity():
    """Table 8 quadrant states, LT/NERK3: density and pressure stay positive."""
    p, q = I.euler_2d_quadrants(L=6, eps=1e-2, seed=0)
    o = oracle.Oracle(p, q)
    o.step(0.25)
    u = o.uniform()
    rho = u[0]
    pr = 0.4 * (u[3] - 0.5 * (u[1] ** 2 + u[2] ** 2) / rho)
    assert rho.min() > 0.3 and pr.min() > 0.1
    assert o.stats()["leaves"] < 64 * 64


def test_rd_bumps_bounded():
    """2D bistable reaction-diffusion, LT/NERK2: the solution stays in [0, 1]
    up to small overshoot."""
    p, q = I.rd_bumps_2d(L=6, eps=1e-3, seed=1)
    o = oracle.Oracle(p, q)
    o.step(0.05)
    u = o.uniform()[0]
    assert -0.02 < u.min() and u.max() < 1.02
