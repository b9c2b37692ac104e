"""GPU (CUDA C-ABI) versus the FP64 oracle, leaf by leaf.

Bar: identical adaptive leaf sets (keys), and every leaf value within
1e-12 relative, measured as |gpu - oracle| <= 1e-12 (|oracle| + s_v) with
s_v = max |q_v| over the oracle's leaves (the variable's scale).  Cases span
several levels, ragged level populations, walls and periodic boxes, both time
modes, RK2 and RK3, and stops inside a macro step."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def assert_parity(gpu, ref, what=""):
    kg, vg = gpu.leaves()
    ko, vo = ref.leaves()
    sg, so = gpu.stats(), ref.stats()
    assert kg.shape == ko.shape and np.array_equal(kg, ko), (
        f"{what}: leaf sets differ ({len(kg)} vs {len(ko)}), near-threshold "
        f"gpu {sg['near']} oracle {so['near']}")
    scale = np.abs(vo).max(axis=0)
    err = np.abs(vg - vo) / (np.abs(vo) + scale + 1e-300)
    assert err.max() <= TOL, f"{what}: max relative error {err.max():.3e}"
    assert sg["iters"] == so["iters"] and sg["pos"] == so["pos"]
    return err.max()


def _run_both(p, q, t=None, dt=None, n=None, tree=None):
    gpu, ref = _solver(p, q), oracle.Oracle(p, q)
    if tree is not None:
        gpu.set_tree(tree)
        ref.set_tree(tree)
    assert_parity(gpu, ref, "initial")
    if t is not None:
        gpu.step(t)
        ref.step(t)
    if n is not None:
        gpu.iterate(dt, n)
        ref.iterate(dt, n)
    return gpu, ref


@pytest.mark.parametrize("rk,mode", [(3, I.TIME_LT), (2, I.TIME_LT), (3, I.TIME_GTS), (2, I.TIME_GTS)])
def test_burgers_1d_full_size(rk, mode):
    """1D Burgers L=10, level-scaled eps=1e-3 to t_end=0.5 (through the shock)."""
    p, q = I.burgers_1d(L=10, eps=1e-3, rk_order=rk, time_mode=mode)
    gpu, ref = _run_both(p, q, t=0.5)
    assert_parity(gpu, ref, "t_end")
    assert (ref.stats()["leaves_per_level"] > 0).sum() >= 3
    u_g, u_o = gpu.uniform(), ref.uniform()
    assert np.abs(u_g - u_o).max() <= TOL * (np.abs(u_o).max() + 1)


@pytest.mark.parametrize("n", [1, 3, 7, 17, 64])
def test_burgers_1d_inside_macro_step(n):
    """Stop after n fine iterations: every lmin pattern of Alg. 3 occurs."""
    p, q = I.burgers_1d(L=9, eps=1e-3, min_level=3)
    gpu, ref = _run_both(p, q + 0.3, dt=4e-4, n=n)
    assert_parity(gpu, ref, f"n={n}")


def test_burgers_1d_conservation_on_gpu():
    p, q = I.burgers_1d(L=9, eps=1e-3)
    gpu = _solver(p, q + 0.5)
    m0 = gpu.stats()["mass"][0]
    gpu.step(0.4)
    assert abs(gpu.stats()["mass"][0] - m0) < 1e-13


@pytest.mark.parametrize("seed,rk,mode", [(0, 3, I.TIME_LT), (3, 3, I.TIME_LT), (0, 2, I.TIME_LT),
                                          (0, 3, I.TIME_GTS)])
def test_euler_2d_quadrants(seed, rk, mode):
    """2D Euler four-quadrant problem (Table 8 states for seed 0), walls."""
    p, q = I.euler_2d_quadrants(L=6, eps=1e-2, seed=seed, rk_order=rk, time_mode=mode, min_level=3)
    gpu, ref = _run_both(p, q, t=0.05)
    assert_parity(gpu, ref, "t=0.05")
    assert (ref.stats()["leaves_per_level"] > 0).sum() >= 3


def test_euler_2d_periodic_conservation_and_parity():
    p, q = I.euler_2d_quadrants(L=6, eps=1e-2, seed=1)
    p = p.replace(bc=(I.BC_PERIODIC,) * 3)
    gpu, ref = _run_both(p, q, t=0.04)
    assert_parity(gpu, ref)
    m_g, m_o = gpu.stats()["mass"], ref.stats()["mass"]
    assert np.abs((m_g - m_o) / m_o).max() < 1e-13


def test_burgers_2d_periodic():
    p, q = I.burgers_2d(L=6, eps=1e-2)
    gpu, ref = _run_both(p, q + 0.2, t=0.1)
    assert_parity(gpu, ref)


def test_rd_2d_rk2():
    p, q = I.rd_bumps_2d(L=6, eps=1e-3, seed=2)
    gpu, ref = _run_both(p, q, t=0.02)
    assert_parity(gpu, ref)


def test_euler_1d_sod_walls():
    p, q = I.euler_1d_sod(L=8, eps=1e-3)
    gpu, ref = _run_both(p, q, t=0.1)
    assert_parity(gpu, ref)


def test_euler_3d_small():
    """3D Euler blast on a small grid (tensor-product prediction in 3D)."""
    L = 5
    n = 1 << L
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    pr = np.where((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2 < 0.2 ** 2, 10.0, 1.0)
    q = np.zeros((5, n, n, n))
    q[0] = 1.0
    q[4] = pr / 0.4
    p = I.Problem(dim=3, equation=I.EQ_EULER, max_level=L, min_level=2, eps=1e-2,
                  bc=(I.BC_NEUMANN,) * 3, phys=(1.4,) + (0.0,) * 7)
    gpu, ref = _run_both(p, q, t=0.01)
    assert_parity(gpu, ref)


def test_fixed_two_level_advection():
    """The Sec. 4.5 fixed two-level grid (set_tree) with the centred flux."""
    L = 8
    p, q = I.advection_gaussian_1d(L=L, rk_order=3)
    p = p.replace(min_level=L - 1)
    gpu, ref = _run_both(p, q, dt=1e-3, n=150, tree=I.two_level_map_1d(L))
    assert_parity(gpu, ref)


def test_eps_zero_uniform():
    p, q = I.burgers_1d(L=8, eps=0.0)
    gpu, ref = _run_both(p, q, t=0.3)
    assert_parity(gpu, ref)
    assert gpu.stats()["leaves"] == 256


@pytest.mark.parametrize("L,lb", [(2, 2), (3, 0), (6, 6)])
def test_degenerate_levels(L, lb):
    """single-level trees and the coarsest possible base level"""
    p, q = I.burgers_1d(L=L, eps=1e-3, min_level=lb)
    gpu, ref = _run_both(p, q + 0.1, t=0.05)
    assert_parity(gpu, ref)


def test_reset_reproduces_create():
    p, q = I.burgers_1d(L=9, eps=1e-3)
    gpu = _solver(p, q)
    k0, v0 = gpu.leaves()
    gpu.step(0.1)
    gpu.reset(q)
    k1, v1 = gpu.leaves()
    assert np.array_equal(k0, k1) and np.array_equal(v0, v1)
    assert gpu.stats()["iters"] == 0


def test_euler_2d_full_size_macro_step():
    """2D Euler L=10 (1024^2 finest), eps=1e-3, LT/NERK3 -- the benchmark
    workload: the first four fine iterations (lmin = 3, 10, 9, 10), then the
    rest of the first macro step (128 iterations, every lmin, adaptation at
    every iteration, registers applied at the macro-step end), leaf by leaf."""
    p, q = I.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    gpu, ref = _run_both(p, q)
    dt = 0.5 / 1024 / 3.7
    gpu.iterate(dt, 4)
    ref.iterate(dt, 4)
    assert_parity(gpu, ref, "L=10 after 4 iterations")
    gpu.iterate(dt, 124)
    ref.iterate(dt, 124)
    assert_parity(gpu, ref, "L=10 after one macro step")
    assert gpu.stats()["macros"] == 1


@pytest.mark.slow
def test_benchmark_solve_against_oracle():
    """The benchmark solve itself (2D Euler quadrants, L=10, eps=1e-3, LT/NERK3,
    CFL macro steps) run side by side with the oracle through all of its 1920
    fine iterations (t = 0.25; the oracle needs about two minutes), compared
    leaf by leaf every 0.05 time units.  The leaf sets must stay identical
    through every remesh; near-threshold decisions (a detail norm within 1e-10
    of eps or 8 eps) are counted on both sides and printed."""
    p, q = I.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    gpu, ref = _run_both(p, q)
    for t in (0.05, 0.1, 0.15, 0.2, 0.25):
        gpu.step(t)
        ref.step(t)
        err = assert_parity(gpu, ref, f"t = {t}")
        sg, so = gpu.stats(), ref.stats()
        print(f"t={t}: {sg['leaves']} leaves, {sg['iters']} iterations, max rel err {err:.2e}, "
              f"near-threshold decisions gpu {sg['near']} oracle {so['near']}")
    assert gpu.stats()["iters"] == 1920


@pytest.mark.parametrize("mode,rk", [(I.TIME_LT, 3), (I.TIME_LT, 2), (I.TIME_GTS, 2)])
def test_euler_2d_ausm_plus(mode, rk):
    """the paper's Euler flux (AUSM+, Sec. 5) on the quadrant problem"""
    p, q = I.euler_2d_quadrants(L=8, eps=1e-3, seed=0, rk_order=rk, time_mode=mode)
    gpu, ref = _run_both(p.replace(flux=I.FLUX_AUSM_PLUS), q, t=0.05)
    assert_parity(gpu, ref)


def test_euler_1d_sod_ausm_plus():
    p, q = I.euler_1d_sod(L=9, eps=1e-3)
    gpu, ref = _run_both(p.replace(flux=I.FLUX_AUSM_PLUS), q, t=0.12)
    assert_parity(gpu, ref)


def test_euler_3d_ausm_plus():
    p, q = I.euler_3d_blast(L=5, eps=1e-2, min_level=2, precision=I.PREC_FP64)
    gpu, ref = _run_both(p.replace(flux=I.FLUX_AUSM_PLUS), q, t=0.01)
    assert_parity(gpu, ref)


def test_largest_1d_grid():
    """the finest 1D grid the layout allows (L = 16, 65536 cells), LT/NERK3"""
    p, q = I.burgers_1d(L=16, eps=1e-3, min_level=10)
    gpu, ref = _run_both(p, q)
    dt = 0.5 / (1 << 16)
    gpu.iterate(dt, 8)
    ref.iterate(dt, 8)
    assert_parity(gpu, ref)


def test_oversize_problem_reports_nomem():
    """a 3D Euler problem at L = 10 needs about 1 TB: creation fails with
    MR_E_NOMEM before anything is allocated or read (a one-element buffer
    stands in for the finest data), and the device stays usable"""
    import ctypes
    import paper_1905_08717_gb300 as pkg
    p = I.Problem(dim=3, equation=I.EQ_EULER, max_level=10, min_level=9, eps=1e-3,
                  bc=(I.BC_NEUMANN,) * 3, phys=(1.4,) + (0.0,) * 7)
    lib = pkg.library()
    cfg = pkg.make_config(p)
    tiny = np.zeros(1)
    h = ctypes.c_void_p()
    r = lib.mr_create(ctypes.byref(cfg), tiny.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                      ctypes.byref(h))
    assert r == 2 and not h.value  # MR_E_NOMEM, no handle
    p2, q2 = I.burgers_1d(L=8, eps=1e-3)
    gpu, ref = _run_both(p2, q2, t=0.05)  # the device still works
    assert_parity(gpu, ref)


@pytest.mark.parametrize("mode,rk", [(I.TIME_LT, 2), (I.TIME_LT, 3), (I.TIME_GTS, 2)])
def test_burgers_2d_paper_case_dirichlet(mode, rk):
    """the paper's 2D Burgers case (Sec. 5.1, u = 0 on the walls), reduced size"""
    p, q = I.burgers_2d_paper(L=7, eps=1e-3, min_level=3, rk_order=rk, time_mode=mode)
    gpu, ref = _run_both(p, q, t=0.25)
    assert_parity(gpu, ref)


def test_burgers_1d_dirichlet():
    p, q = I.burgers_1d(L=10, eps=1e-3)
    gpu, ref = _run_both(p.replace(bc=(I.BC_DIRICHLET0,) * 3), q, t=0.3)
    assert_parity(gpu, ref)


def test_rd_2d_dirichlet():
    p, q = I.rd_bumps_2d(L=7, eps=1e-3, seed=4)
    gpu, ref = _run_both(p.replace(bc=(I.BC_DIRICHLET0,) * 3), q, t=0.03)
    assert_parity(gpu, ref)


@pytest.mark.parametrize("bc", [I.BC_PERIODIC, I.BC_NEUMANN, I.BC_DIRICHLET0])
def test_burgers_3d_walls(bc):
    """3D scalar problem: prediction and stencils across walls and corners"""
    p, q = I.burgers_3d(L=5, eps=1e-2, min_level=2, bc=bc)
    gpu, ref = _run_both(p, q, t=0.04)
    assert_parity(gpu, ref)


def test_release_cached_memory_returns_device_memory():
    """destroyed solvers' memory stays cached in the library's pool until
    released back to the device"""
    import torch
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=10, eps=1e-3)
    s = pkg.Solver(p, q)
    s.close()
    torch.cuda.synchronize()
    free_cached, _ = torch.cuda.mem_get_info()
    pkg.release_cached_memory()
    torch.cuda.synchronize()
    free_released, _ = torch.cuda.mem_get_info()
    assert free_released - free_cached > 200 << 20  # the solver holds about 0.8 GB


_MOVING = {
    # name: (problem and data, fine iterations, fine step below the CFL limit)
    "sod": (lambda: I.euler_1d_sod(L=8, eps=1e-3, min_level=2), 48, 0.25 / 256),
    "quadrants2d": (lambda: I.euler_2d_quadrants(L=6, eps=1e-3, min_level=2), 32, 0.125 / 64),
    "burgers2d": (lambda: I.burgers_2d(L=6, eps=1e-3, min_level=2), 32, 0.25 / 64),
}


@pytest.mark.parametrize("case", sorted(_MOVING))
def test_every_lt_iteration_matches_oracle(case):
    """Leaf sets and values agree with the oracle after every single fine
    iteration of an LT run whose tree moves (restricted remesh at every
    iteration, stops at every position inside the macro step)."""
    make, steps, dt = _MOVING[case]
    p, q = make()
    p = p.replace(adapt_mode=I.ADAPT_EVERY)
    gpu, ref = _solver(p, q), oracle.Oracle(p, q)
    moved = 0
    prev = ref.leaves()[0]
    for n in range(steps):
        gpu.iterate(dt, 1)
        ref.iterate(dt, 1)
        assert_parity(gpu, ref, f"{case}, iteration {n}")
        k = ref.leaves()[0]
        moved += not np.array_equal(k, prev)
        prev = k
    assert moved >= 2
    gpu.close()
