"""Mixed-precision mode (state, exposures, MUSCL reconstruction, numerical
fluxes and the RK stage updates in FP32; flux registers and the detail-norm
threshold test in FP64) against the FP64 oracle.

The mixed path cannot match the oracle to 1e-12.  The bar is a bound derived
for it from two sources of error, with u32 = 2^-24 the FP32 unit roundoff:

- fluxes: a flux evaluation of the MUSCL + HLL chain (about 60 dependent
  operations, cancellations included) is taken to lose at most C = 64 units of
  u32.  Through an update dt_l / dx_l (F_{-} - F_{+}) with Courant number sigma
  that is a relative state error of at most 2 C u32 sigma per stage, and
  6 C u32 sigma per RK3 step;
- storage and stage arithmetic: every stored value is rounded to FP32 (u32);
  an RK stage and the NERK exposures it reads (at most 4 q** - 3 q^n, a factor
  7 on |q|) take a few FP32 operations each.  That is bounded by C_S = 32 units
  of u32 of the state per fine iteration, plus one u32 for the initial data.

Over n fine iterations the error of the uniform reconstruction, in L1 relative
to the oracle's L1 norm, is therefore bounded by

    tol = n (6 C u32 sigma + C_S u32) + u32

(linear accumulation, no cancellation assumed).  Thresholding decisions near
eps can flip between the two runs.  A flipped node changes its cells by a
detail of order eps * s_v, where s_v is the variable's scale, so flips add
eps * (flipped fraction) to the bound.  The leaf-count check below limits that
fraction, and the tests add eps * 1e-2.

The tests also check that the mixed result differs from the GPU's own FP64
result by more than FP64 round-off, so that the FP32 path really ran, and that
mass is conserved to FP32 round-off: every face flux enters both sides of the
face and the registers are FP64, so the total changes only by the rounding of
the stored values, at most 6 u32 of the total absolute mass per iteration."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
C_FLUX = 64
C_STATE = 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_08717_gb300 import build
    build.build()


def _solver(p, q):
    import paper_1905_08717_gb300 as pkg
    return pkg.Solver(p, q)


def _rel_l1(a, b):
    """per-variable L1 difference relative to the L1 norm of b"""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.abs(a - b).sum(axis=1) / np.maximum(np.abs(b).sum(axis=1), 1e-300)


def _check(p, q, t):
    """run mixed GPU, FP64 GPU and the FP64 oracle to t; return the errors"""
    pm = p.replace(precision=I.PREC_MIXED)
    p64 = p.replace(precision=I.PREC_FP64)
    gm, g64, ref = _solver(pm, q), _solver(p64, q), oracle.Oracle(p64, q)
    gm.step(t)
    g64.step(t)
    ref.step(t)
    sm, so = gm.stats(), ref.stats()
    n = so["iters"]
    assert sm["iters"] == n
    tol = n * (6 * C_FLUX * U32 * p.cfl + C_STATE * U32) + U32 + p.eps * 1e-2
    uo = ref.uniform()
    e_mixed = _rel_l1(gm.uniform(), uo)
    e_fp64 = _rel_l1(g64.uniform(), uo)
    assert e_fp64.max() <= 1e-12, f"FP64 GPU path off the oracle: {e_fp64}"
    assert e_mixed.max() <= tol, f"mixed L1 error {e_mixed} above the bound {tol:.3e}"
    assert e_mixed.max() > 1e-12, "mixed result equals the FP64 one: FP32 flux path not taken"
    # thresholding flips stay rare
    assert abs(sm["leaves"] - so["leaves"]) <= 0.02 * so["leaves"] + 8
    return e_mixed, tol


def _check_leafwise(p, q, dt, n):
    """n fine iterations from the same state: identical leaf sets, and every
    leaf within (n (6 C u32 sigma + C_S u32) + u32) (|q| + s_v) of the FP64
    oracle -- the per-step bound of the module docstring applied leaf by leaf,
    which a wrong FP32 flux or update formula (an O(1) relative error in the
    cells it touches) fails"""
    pm = p.replace(precision=I.PREC_MIXED)
    gm, ref = _solver(pm, q), oracle.Oracle(p.replace(precision=I.PREC_FP64), q)
    gm.iterate(dt, n)
    ref.iterate(dt, n)
    kg, vg = gm.leaves()
    ko, vo = ref.leaves()
    assert np.array_equal(kg, ko), "leaf sets differ"
    scale = np.abs(vo).max(axis=0)
    err = np.abs(vg - vo) / (np.abs(vo) + scale + 1e-300)
    sigma_eff = dt * _max_speed(p, q) * (1 << p.max_level)
    tol = n * (6 * C_FLUX * U32 * max(sigma_eff, 1e-3) + C_STATE * U32) + U32
    assert err.max() <= tol, f"max leaf error {err.max():.3e} above {tol:.3e}"
    assert err.max() > 1e-13, "FP32 flux path not taken"
    return err.max(), tol


def _max_speed(p, q):
    """largest characteristic speed of the initial data (for the Courant number
    dt s / dx_L of a fixed dt)"""
    if p.equation == I.EQ_EULER:
        g = p.phys[0]
        m = q.shape[0]
        rho = q[0]
        mom = q[1:m - 1]
        ke = 0.5 * (mom ** 2).sum(axis=0) / rho
        pr = (g - 1.0) * (q[m - 1] - ke)
        return float((np.sqrt((mom ** 2).sum(axis=0)) / rho + np.sqrt(g * pr / rho)).max())
    if p.equation == I.EQ_BURGERS:
        return float(np.abs(q).max())
    if p.equation == I.EQ_REACTION_DIFFUSION:  # diffusion number D dt / dx^2, scaled to dx
        return p.phys[0] * (1 << p.max_level) + p.phys[1] / (1 << p.max_level)
    return float(np.abs(p.phys[:3]).max())


@pytest.mark.parametrize("case", ["burgers1d", "euler2d", "rd2d", "euler3d"])
def test_mixed_first_iterations_leafwise(case):
    if case == "burgers1d":
        p, q = I.burgers_1d(L=10, eps=1e-3)
        dt = 0.5 / 1024
    elif case == "euler2d":
        p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=0)
        dt = 0.5 / 128 / 3.7
    elif case == "rd2d":
        p, q = I.rd_bumps_2d(L=7, eps=1e-3, seed=1)
        dt = 0.2 * (1.0 / 128) ** 2 / 1e-3
    else:
        p, q = I.euler_3d_blast(L=5, eps=1e-2, min_level=2)
        dt = 0.5 / 32 / 4.0
    _check_leafwise(p, q, dt, 1)
    _check_leafwise(p, q, dt, 3)


def test_mixed_ausm_plus_leafwise():
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=0)
    p = p.replace(flux=I.FLUX_AUSM_PLUS)
    dt = 0.5 / 128 / 3.7
    _check_leafwise(p, q, dt, 1)
    _check_leafwise(p, q, dt, 3)


def test_mixed_full_size_first_iterations_leafwise():
    """the 2D Euler L=10 workload: four fine iterations (lmin = 3, 10, 9, 10)"""
    p, q = I.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    _check_leafwise(p, q, 0.5 / 1024 / 3.7, 4)


@pytest.mark.slow
def test_mixed_blast_3d_full_size():
    """the 3D blast precision workload at its full size (L = 8, 256^3 finest),
    Courant number about 0.3 summed over the three directions: four fine
    iterations leaf by leaf against the FP64 oracle, then one whole macro step
    (32 fine iterations, every lmin) by the L1 distance of the finest-grid
    reconstructions, where threshold decisions may flip"""
    p, q = I.euler_3d_blast(L=8, eps=1e-3, min_level=3)
    dt = 1.0e-4
    err, tol = _check_leafwise(p, q, dt, 4)
    pm = p.replace(precision=I.PREC_MIXED)
    gm, ref = _solver(pm, q), oracle.Oracle(p.replace(precision=I.PREC_FP64), q)
    gm.iterate(dt, 32)
    ref.iterate(dt, 32)
    e = _rel_l1(gm.uniform(), ref.uniform())
    tol32 = 32 * (6 * C_FLUX * U32 * 0.3 + C_STATE * U32) + U32 + p.eps * 1e-2
    print(f"3D blast L=8 mixed: 4 iterations max leaf error {err:.2e} (bound {tol:.2e}); "
          f"32 iterations relative L1 {e.max():.2e} (bound {tol32:.2e})")
    assert e.max() <= tol32, (e, tol32)
    assert e.max() > 1e-12


def test_mixed_burgers_1d():
    p, q = I.burgers_1d(L=10, eps=1e-3)
    _check(p, q, 0.3)


def test_mixed_euler_2d_quadrants():
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=0)
    _check(p, q, 0.1)


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_euler_2d_quadrants_random_states(seed):
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, seed=seed)
    _check(p, q, 0.1)


def test_mixed_rd_2d_rk2():
    p, q = I.rd_bumps_2d(L=7, eps=1e-3, seed=1)
    _check(p, q, 0.05)


def test_mixed_euler_3d_blast():
    p, q = I.euler_3d_blast(L=5, eps=1e-2, min_level=2)
    _check(p, q, 0.02)


def test_mixed_conserves_mass():
    """periodic 2D Euler: FP64 flux registers and fluxes that enter both sides
    of a face keep the FP32-state run conservative to FP32 round-off (a lost
    register correction or a one-sided flux changes the total by the flux
    itself, orders of magnitude more)"""
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=0)
    p = p.replace(bc=(I.BC_PERIODIC,) * 3, precision=I.PREC_MIXED)
    g = _solver(p, q)
    m0 = np.array(g.stats()["mass"])
    g.step(0.05)
    st = g.stats()
    m1 = np.array(st["mass"])
    absmass = np.abs(q.reshape(q.shape[0], -1)).sum(axis=1) / q[0].size
    bound = st["iters"] * 6 * U32 * absmass
    assert np.all(np.abs(m1 - m0)[: len(absmass)] <= bound), (m1 - m0, bound)


def test_mixed_gts_mode():
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, seed=0, time_mode=I.TIME_GTS)
    _check(p, q, 0.1)
