"""Pins of the oracle's reaction-diffusion operator u_t = D lap u + k u (1 - u) (u - a)
(the bistable case of Sec. 2), each from mathematics the oracle does not share:

- diffusion alone: a Fourier mode is an eigenvector of the finite-volume
  operator with the two-point flux, so n steps of RK2/RK3 multiply it by the
  stability polynomial R(z)^n exactly (a wrong sign, factor, face width or
  stage weight fails);
- reaction alone: a spatially uniform state follows the ODE u' = k u (1 - u)
  (u - a); the error against a high-accuracy ODE solution must shrink at the
  RK order (a wrong sign, or k and a swapped, fails)."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I


def _problem(d, L, rk, D, k, a):
    return I.Problem(dim=d, equation=I.EQ_REACTION_DIFFUSION, max_level=L, min_level=2, eps=0.0,
                     rk_order=rk, time_mode=I.TIME_GTS, adapt_mode=I.ADAPT_NEVER,
                     bc=(I.BC_PERIODIC,) * 3, phys=(D, k, a) + (0.0,) * 5)


def _sine_averages(n):
    """cell averages of sin(2 pi x) on n cells of [0, 1]"""
    h = 1.0 / n
    x = np.arange(n) * h
    return (np.cos(2 * np.pi * x) - np.cos(2 * np.pi * (x + h))) / (2 * np.pi * h)


@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_diffusion_mode_decays_by_the_stability_polynomial(rk, d):
    L, D, steps = 4, 0.01, 25
    n, h = 1 << L, 1.0 / (1 << L)
    s = _sine_averages(n)
    q0 = s
    for _ in range(d - 1):
        q0 = np.multiply.outer(q0, s)
    q0 = q0.T.copy()  # cell ids are x-fastest: the array is indexed [z][y][x]
    o = oracle.Oracle(_problem(d, L, rk, D, 0.0, 0.3), q0[None])
    dt = 0.4 * h * h / (2 * d * D)
    o.iterate(dt, steps)
    u = o.uniform()[0]
    z = dt * d * (-4.0 * D * np.sin(np.pi * h) ** 2 / (h * h))  # each factor contributes one 1D rate
    R = 1 + z + z * z / 2 + (z ** 3 / 6 if rk == 3 else 0.0)
    assert np.abs(u - q0 * R ** steps).max() < 1e-13
    assert 0.0 < R ** steps < 0.9  # the mode has decayed visibly


@pytest.mark.parametrize("rk", [2, 3])
def test_uniform_state_follows_the_reaction_ode(rk):
    from scipy.integrate import solve_ivp
    k, a, u0, T = 5.0, 0.25, 0.4, 1.0
    ref = solve_ivp(lambda t, u: k * u * (1 - u) * (u - a), (0.0, T), [u0], method="DOP853",
                    rtol=1e-13, atol=1e-15).y[0, -1]
    errs = []
    for steps in (40, 80, 160):
        o = oracle.Oracle(_problem(1, 3, rk, 0.0, k, a), np.full((1, 8), u0))
        o.iterate(T / steps, steps)
        u = o.uniform()[0]
        assert np.ptp(u) == 0.0  # stays uniform
        errs.append(abs(u[0] - ref))
    assert errs[-1] < 1e-4
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - rk) < 0.1), orders
