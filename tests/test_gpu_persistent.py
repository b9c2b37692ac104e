"""The persistent macro-step kernel (MR_LAUNCH_PERSISTENT) against the
kernel-per-phase path (MR_LAUNCH_GRAPH, the default): the
same device bodies in the same order, for every time mode, order, equation,
dimension, wall type, precision, stop inside a macro step and grid size.  The
bodies are inlined into different kernels, where the compiler may contract a
different set of multiply-adds into FMAs, so the two agree to FP64 round-off
(identical leaf sets, |difference| <= 1e-14 (|q| + s_v)) rather than bit for
bit; within one launch mode every grid size gives bitwise the same result.
The bounded grid barrier gives up with MR_E_TIMEOUT when CTAs are missing,
and the device stays usable."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_08717_gb300 import build
    build.build()


def _pair(p, q, cap=0):
    import paper_1905_08717_gb300 as pkg
    a, b = pkg.Solver(p, q), pkg.Solver(p, q)
    a.set_launch_mode(pkg.MR_LAUNCH_PERSISTENT)
    b.set_launch_mode(pkg.MR_LAUNCH_GRAPH)
    if cap:
        a.set_grid_cap(cap)
    return a, b


def _same(a, b, what="", exact=False):
    if a.p.precision == I.PREC_MIXED and not exact:
        # FP32 state: the two kernels may round differently, so near-threshold
        # decisions may differ too; the reconstructions agree to FP32 round-off
        ua, ub = a.uniform(), b.uniform()
        ua, ub = ua.reshape(ua.shape[0], -1), ub.reshape(ub.shape[0], -1)
        e = np.abs(ua - ub).sum(axis=1) / np.abs(ub).sum(axis=1)
        assert e.max() <= 1e-5, f"{what}: mixed runs differ by {e.max():.3e} (L1)"
        return
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb), f"{what}: leaf sets differ"
    if exact:
        assert np.array_equal(va, vb), f"{what}: values differ (max {np.abs(va - vb).max():.3e})"
    else:
        err = np.abs(va - vb) / (np.abs(vb) + np.abs(vb).max(axis=0) + 1e-300)
        assert err.max() <= 1e-14, f"{what}: values differ by {err.max():.3e} relative"
    sa, sb = a.stats(), b.stats()
    for k in ("iters", "macros", "pos", "near", "updates"):
        assert sa[k] == sb[k], (what, k, sa[k], sb[k])
    assert abs(sa["t"] - sb["t"]) <= 1e-14 * abs(sb["t"]), (what, sa["t"], sb["t"])


CASES = {
    "burgers1d_lt_rk3": (lambda: I.burgers_1d(L=10, eps=1e-3), 0.3),
    "burgers1d_lt_rk2": (lambda: I.burgers_1d(L=10, eps=1e-3, rk_order=2), 0.3),
    "burgers1d_gts_rk3": (lambda: I.burgers_1d(L=9, eps=1e-3, time_mode=I.TIME_GTS), 0.3),
    "euler2d_walls": (lambda: I.euler_2d_quadrants(L=7, eps=1e-3, seed=2), 0.05),
    "euler2d_ausm_rk2": (lambda: I.euler_2d_quadrants(L=7, eps=1e-3, seed=0, rk_order=2), 0.05),
    "rd2d_rk2": (lambda: I.rd_bumps_2d(L=7, eps=1e-3, seed=3), 0.02),
    "burgers2d_dirichlet": (lambda: I.burgers_2d_paper(L=7, eps=1e-2), 0.1),
    "euler3d_blast": (lambda: I.euler_3d_blast(L=5, eps=1e-2, min_level=2, precision=I.PREC_FP64), 0.02),
    "euler3d_blast_mixed": (lambda: I.euler_3d_blast(L=5, eps=1e-2, min_level=2), 0.02),
}


@pytest.mark.parametrize("name", list(CASES))
def test_persistent_equals_kernel_per_phase(name):
    mk, t = CASES[name]
    p, q = mk()
    if name == "euler2d_ausm_rk2":
        p = p.replace(flux=I.FLUX_AUSM_PLUS)
    a, b = _pair(p, q)
    a.step(t / 2)
    b.step(t / 2)
    _same(a, b, f"{name} t/2")
    a.step(t)
    b.step(t)
    _same(a, b, f"{name} t")
    assert a.launch_count() < b.launch_count()


@pytest.mark.parametrize("prec", [I.PREC_FP64, I.PREC_MIXED])
@pytest.mark.parametrize("cap", [0, 1, 7, 152])
def test_persistent_stops_inside_macro_step_and_grid_caps(prec, cap):
    """stops after 1, 3, 7, 17 fine iterations (every l_min pattern), then
    whole macro steps; grid caps of 1, 7, 152 CTAs or the resident capacity"""
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=1, min_level=2)
    p = p.replace(precision=prec)
    a, b = _pair(p, q, cap)
    dt = 0.5 / 128 / 3.5
    for n in (1, 3, 7, 17, 4):  # 32 = one macro step of 2^(7-2) iterations
        a.iterate(dt, n)
        b.iterate(dt, n)
        _same(a, b, f"n={n}")
    a.step(0.03)
    b.step(0.03)
    _same(a, b, "t=0.03")
    if cap:  # persistent mode at the resident capacity: bitwise the same as with the cap
        import paper_1905_08717_gb300 as pkg
        c = pkg.Solver(p, q)
        c.set_launch_mode(pkg.MR_LAUNCH_PERSISTENT)
        for n in (1, 3, 7, 17, 4):
            c.iterate(dt, n)
        c.step(0.03)
        _same(a, c, "cap vs resident capacity", exact=True)


def test_persistent_matches_oracle_and_profiles():
    """the persistent path against the oracle, with the phase profile on:
    stage phases are timed and counted"""
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=8, eps=1e-3, seed=0)
    g, ref = pkg.Solver(p, q), oracle.Oracle(p, q)
    g.set_launch_mode(pkg.MR_LAUNCH_PERSISTENT)
    g.profile(True)
    g.step(0.02)
    ref.step(0.02)
    prof = g.profile_read()
    g.profile(False)
    kg, vg = g.leaves()
    ko, vo = ref.leaves()
    assert np.array_equal(kg, ko)
    err = np.abs(vg - vo) / (np.abs(vo) + np.abs(vo).max(axis=0))
    assert err.max() <= 1e-12
    assert prof["stage_launches"] > 0 and prof["stage_ms"] > 0.0
    assert sum(prof["leaf_stages"]) > 0


def test_grid_barrier_gives_up_and_device_stays_usable():
    import paper_1905_08717_gb300 as pkg
    assert pkg.selftest_grid_wait(8, 0, 1.0) == 0
    assert pkg.selftest_grid_wait(8, 1, 0.2) == 4  # MR_E_TIMEOUT
    assert pkg.selftest_grid_wait(1, 3, 0.2) == 4
    p, q = I.burgers_1d(L=8, eps=1e-3, min_level=3)
    g, ref = pkg.Solver(p, q), oracle.Oracle(p, q)
    g.step(0.1)
    ref.step(0.1)
    kg, vg = g.leaves()
    ko, vo = ref.leaves()
    assert np.array_equal(kg, ko)
    assert np.abs(vg - vo).max() <= 1e-12 * (np.abs(vo).max() + 1.0)
