"""Pins of the oracle's numerical fluxes for the Euler equations: HLL (the
default) and AUSM+ (Liou 1996, the flux the paper uses, Sec. 5).  Each pin
fixes a property of the exact flux that a plausible mistake breaks: equal
states give the physical flux (a wrong splitting sum, a dropped pressure
term); supersonic states give the upwind physical flux (a wrong sign or
branch of the Mach splitting); mirror symmetry (a wrong sign on one side);
the Sod shock tube converges to the exact Riemann solution (anything that
makes the scheme inconsistent); and AUSM+ resolves contacts exactly (split
halves that do not sum to M or to 1)."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I

from tests.fv_reference import exact_riemann

G = 1.4


def _problem(d, flux):
    if d == 1:
        p, _ = I.euler_1d_sod(L=4)
    else:
        p = I.Problem(dim=d, equation=I.EQ_EULER, max_level=3, min_level=1, eps=0.0,
                      bc=(I.BC_NEUMANN,) * 3, phys=(G,) + (0.0,) * 7)
    return p.replace(flux=flux)


def _cons(rho, vel, p):
    vel = np.asarray(vel, float)
    return np.concatenate([[rho], rho * vel, [p / (G - 1.0) + 0.5 * rho * vel @ vel]])


def _phys_flux(U, k):
    d = len(U) - 2
    rho, vel = U[0], U[1:d + 1] / U[0]
    p = (G - 1.0) * (U[d + 1] - 0.5 * rho * vel @ vel)
    F = U * vel[k]
    F[1 + k] += p
    F[d + 1] += p * vel[k]
    return F


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_equal_states_give_physical_flux(flux, d):
    rng = np.random.default_rng(10 * d + flux)
    p = _problem(d, flux)
    for _ in range(20):
        U = _cons(rng.uniform(0.2, 3.0), rng.uniform(-2.0, 2.0, d), rng.uniform(0.1, 5.0))
        for k in range(d):
            F = oracle.num_flux(p, k, np.tile(U, (4, 1)))
            assert np.allclose(F, _phys_flux(U, k), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_supersonic_states_are_upwinded(flux, d):
    rng = np.random.default_rng(7 + d + 3 * flux)
    p = _problem(d, flux)
    for _ in range(20):
        k = int(rng.integers(0, d))
        sgn = 1.0 if rng.uniform() < 0.5 else -1.0
        def state():
            rho, pr = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
            vel = rng.uniform(-0.3, 0.3, d)
            vel[k] = sgn * rng.uniform(4.0, 6.0) * np.sqrt(G * pr / rho)
            return _cons(rho, vel, pr)
        UL, UR = state(), state()
        # piecewise-constant stencil: the limited reconstruction returns UL, UR
        F = oracle.num_flux(p, k, np.array([UL, UL, UR, UR]))
        up = UL if sgn > 0 else UR
        assert np.allclose(F, _phys_flux(up, k), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("flux", [0, 1])
def test_mirror_symmetry(flux):
    rng = np.random.default_rng(5 + flux)
    p = _problem(2, flux)
    for _ in range(30):
        W = np.array([_cons(rng.uniform(0.3, 2.0), rng.uniform(-1.5, 1.5, 2), rng.uniform(0.2, 3.0))
                      for _ in range(4)])
        F = oracle.num_flux(p, 0, W)
        Mw = W[::-1].copy()
        Mw[:, 1] *= -1.0  # reflect x: reverse the stencil, flip the normal momentum
        Fm = oracle.num_flux(p, 0, Mw)
        assert np.allclose(Fm, F * np.array([-1.0, 1.0, -1.0, -1.0]), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("flux", [0, 1])
def test_sod_converges_to_exact_riemann_solution(flux):
    t = 0.15
    errs = []
    for L in (7, 8, 9):
        p, q = I.euler_1d_sod(L=L, eps=0.0, min_level=L - 2, time_mode=I.TIME_GTS)
        o = oracle.Oracle(p.replace(flux=flux), q)
        o.step(t)
        u = o.uniform()
        n = 1 << L
        x = (np.arange(n) + 0.5) / n
        rho, _, _ = exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G, (x - 0.5) / t)
        errs.append(np.abs(u[0] - rho).mean())
    assert errs[2] < errs[1] < errs[0], errs
    assert errs[2] < 6e-3, errs


def test_ausm_pressure_split_is_twice_differentiable_at_sonic_point():
    """AUSM+'s pressure splitting P+(M) joins its supersonic value 1 at M = 1
    with matching first and second derivatives (this is what its constant
    alpha = 3/16 achieves).  With equal normal velocities u on both sides the
    interface Mach number is the same for both, so the momentum flux is
    rho_L u^2 + p_R + P+(M) (p_L - p_R) for u > 0, and P+ can be read off the
    flux as a function of u.  Below the sonic point 1 - P+ must then vanish
    faster than the square of the distance to it."""
    p = _problem(1, 1)

    def P_of(u):
        L, R = _cons(1.0, [u], 1.0), _cons(0.5, [u], 0.4)
        F = oracle.num_flux(p, 0, np.array([L, L, R, R]))
        return (F[1] - 1.0 * u * u - 0.4) / (1.0 - 0.4)

    us = np.linspace(0.3, 2.5, 4401)
    P = np.array([P_of(u) for u in us])
    i = int(np.argmax(P >= 1.0 - 1e-14))  # first sample at the supersonic value
    assert 0 < i < len(us) - 1
    lo, hi = us[i - 1], us[i]
    for _ in range(60):  # bisect the sonic point
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if P_of(mid) < 1.0 - 1e-14 else (lo, mid)
    us_star = hi
    r = [(1.0 - P_of(us_star - h)) / h ** 2 for h in (4e-3, 2e-3, 1e-3)]
    # cubic behaviour: the ratio halves with h (a quadratic term would keep it)
    assert r[2] < 0.6 * r[0] + 1e-6, r


@pytest.mark.parametrize("d", [1, 2, 3])
def test_ausm_plus_resolves_contacts_exactly(d):
    """Liou's splittings satisfy M+(M) + M-(M) = M and P+(M) + P-(M) = 1 for
    every Mach number, so across a contact (equal velocity and pressure, any
    density jump) AUSM+ returns the upwind physical flux exactly, and zero
    mass flux for a contact at rest.  A splitting whose halves do not sum to
    M or to 1 (a wrong sign or coefficient in one half) fails this.  HLL
    smears a contact at rest (mass flux -c (rho_R - rho_L) / 2 for equal
    sound speeds' bound), which shows that the check discriminates."""
    rng = np.random.default_rng(40 + d)
    pa, ph = _problem(d, 1), _problem(d, 0)
    for _ in range(20):
        rhoL = rng.uniform(0.2, 1.5)
        rhoR = rhoL * rng.uniform(1.5, 3.0)
        pr = rng.uniform(0.1, 5.0)
        for k in range(d):
            vel = rng.uniform(-2.5, 2.5, d)  # sub- and supersonic normal speeds
            for un in (0.0, vel[k], -vel[k]):
                v = vel.copy()
                v[k] = un
                UL, UR = _cons(rhoL, v, pr), _cons(rhoR, v, pr)
                F = oracle.num_flux(pa, k, np.array([UL, UL, UR, UR]))
                expect = _phys_flux(UL if un >= 0.0 else UR, k)
                assert np.allclose(F, expect, rtol=1e-13, atol=1e-13 * (1.0 + np.abs(expect).max()))
                if un == 0.0:
                    assert abs(F[0]) < 1e-14
        rest = np.zeros(d)
        W = np.array([_cons(rhoL, rest, pr)] * 2 + [_cons(rhoR, rest, pr)] * 2)
        assert abs(oracle.num_flux(ph, 0, W)[0]) > 0.05 * (rhoR - rhoL)
