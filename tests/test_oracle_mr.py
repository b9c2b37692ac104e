"""Pins of the oracle's multiresolution part (Sec. 2; Algs. 1-2) against facts
fixed by the mathematics: exactness of the quadratic prediction, the
projection/prediction consistency, the thresholding error bound, and a
brute-force construction of the graded tree on tiny inputs."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I
from tests import fv_reference as R
from tests import mr_reference as M


def _problem(dim, L, lb, eq=I.EQ_BURGERS, bc=I.BC_NEUMANN, **kw):
    base = dict(dim=dim, equation=eq, max_level=L, min_level=lb, eps=0.0,
                adapt_mode=I.ADAPT_NEVER, bc=(bc,) * 3)
    base.update(kw)
    return I.Problem(**base)


def _poly_avgs_1d(coeffs, L):
    n = 1 << L
    e = np.arange(n + 1) / n
    return R.poly_cell_average(coeffs, e[:-1], e[1:])


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("coarsen", [1, 2])
def test_prediction_exact_on_quadratics(dim, coarsen):
    """Eq. 4 (and its tensor product) reproduces cell averages of polynomials of
    degree <= 2 per direction exactly away from the walls (Harten's 3rd order)."""
    L = {1: 8, 2: 6, 3: 5}[dim]
    px = [0.3, -1.7, 2.5]          # 0.3 - 1.7 x + 2.5 x^2
    py = [1.1, 0.4, -3.0]
    pz = [-0.5, 2.0, 1.25]
    ax = _poly_avgs_1d(px, L)
    ay = _poly_avgs_1d(py, L)
    az = _poly_avgs_1d(pz, L)
    if dim == 1:
        q = ax[None]
    elif dim == 2:
        q = (ay[:, None] * ax[None, :] + 0.7 * ax[None, :])[None]
    else:
        q = (az[:, None, None] * ay[None, :, None] * ax[None, None, :])[None]
    p = _problem(dim, L, L - coarsen)
    o = oracle.Oracle(p, q)
    o.set_tree(np.full((1 << L,) * dim, L - coarsen, np.uint8))
    keys, _ = o.leaves()
    assert set(keys[:, 0]) == {L - coarsen}
    u = o.uniform()
    # interior: away from the walls by the prediction stencil of every level
    m = 2 * (1 << coarsen) + 2
    sl = (slice(None),) + (slice(m, (1 << L) - m),) * dim
    err = np.abs(u[sl] - q[sl]).max()
    assert err < 1e-12, err


@pytest.mark.parametrize("dim", [1, 2])
def test_projection_prediction_consistency(dim):
    """P_{l+1->l} o P_{l->l+1} = Identity (Sec. 2): projecting the inverse-MR
    reconstruction back to the leaves returns the leaf values."""
    L = 7 if dim == 1 else 5
    rng = np.random.default_rng(3)
    n = 1 << L
    q = rng.normal(size=(1,) + (n,) * dim)
    p = _problem(dim, L, 2, bc=I.BC_PERIODIC)
    o = oracle.Oracle(p, q)
    # a graded two-region map: level L on the first quarter, L-1 elsewhere
    lev = np.full((n,) * dim, L - 1, np.uint8)
    lev[(slice(0, n // 4),) * dim] = L
    o.set_tree(lev)
    keys, vals = o.leaves()
    u = o.uniform()[0]
    lv = M.project_levels(u[None], 2)
    for (l, i, j, k), v in zip(keys, vals):
        idx = (i, j, k)[:dim][::-1]
        assert abs(lv[l][(0,) + idx] - v[0]) <= 1e-13 * (1 + abs(v[0]))
    # leaf values are the projections of the finest data (Eq. 3)
    lq = M.project_levels(q, 2)
    for (l, i, j, k), v in zip(keys, vals):
        idx = (i, j, k)[:dim][::-1]
        assert abs(lq[l][(0,) + idx] - v[0]) <= 1e-13 * (1 + abs(v[0]))


def test_full_tree_roundtrip():
    """eps = 0 keeps every node: the leaves are the finest data (MR transform
    of Eq. 6 is invertible) and the reconstruction returns q0 exactly."""
    p, q = I.euler_2d_quadrants(L=5, eps=0.0, seed=7, min_level=2)
    o = oracle.Oracle(p, q)
    s = o.stats()
    assert s["leaves"] == 32 * 32
    assert np.array_equal(o.uniform(), q)


@pytest.mark.parametrize("L", [8, 10])
def test_threshold_error_bound(L):
    """The thresholded representation stays within O(eps) of the data
    (Harten's error control by the threshold, Sec. 2 and Alg. 2)."""
    eps = 1e-3
    p, q = I.burgers_1d(L=L, eps=eps)
    o = oracle.Oracle(p, q)
    err = np.abs(o.uniform() - q).max()
    assert err < 2 * eps, err
    # compression is real: far fewer leaves than finest cells
    assert o.stats()["leaves"] < (1 << L) // 4
    # a smaller threshold keeps more leaves and a smaller error
    p2 = p.replace(eps=eps / 10)
    o2 = oracle.Oracle(p2, q)
    assert o2.stats()["leaves"] > o.stats()["leaves"]
    assert np.abs(o2.uniform() - q).max() < err


def _step_field(dim, L, seed):
    n = 1 << L
    rng = np.random.default_rng(seed)
    c = (np.arange(n) + 0.5) / n
    if seed >= 10:  # a spike two finest cells wide: only the finest levels see it
        x0 = rng.uniform(0.3, 0.7)
        if dim == 1:
            return np.exp(-((c - x0) * n / 2.0) ** 2)[None]
        X, Y = np.meshgrid(c, c)
        return np.exp(-((X - x0) ** 2 + (Y - 0.5) ** 2) * (n / 2.0) ** 2)[None]
    if dim == 1:
        f = np.tanh((c - rng.uniform(0.3, 0.7)) * 60) + 0.3 * np.sin(2 * np.pi * c)
        return f[None]
    X, Y = np.meshgrid(c, c)
    r = np.hypot(X - rng.uniform(0.3, 0.7), Y - rng.uniform(0.3, 0.7))
    return (np.tanh((r - 0.2) * 40) + 0.2 * np.cos(2 * np.pi * X))[None]


@pytest.mark.parametrize("dim,L,seed,bc,eps_mode", [
    (1, 7, 0, I.BC_PERIODIC, 0), (1, 7, 1, I.BC_NEUMANN, 1), (1, 6, 2, I.BC_NEUMANN, 0),
    (2, 5, 0, I.BC_PERIODIC, 0), (2, 5, 1, I.BC_NEUMANN, 0), (2, 6, 2, I.BC_NEUMANN, 1),
    (1, 8, 10, I.BC_PERIODIC, 0), (1, 8, 11, I.BC_NEUMANN, 1), (2, 6, 12, I.BC_NEUMANN, 0),
    (2, 6, 13, I.BC_PERIODIC, 1)])
def test_tree_matches_brute_force(dim, L, seed, bc, eps_mode):
    """The adapted leaf set equals the one built by brute force: details from
    an independent numpy MR transform, then the grading rule iterated to a
    global fix-point."""
    q = _step_field(dim, L, seed)
    eps = 2e-3
    p = _problem(dim, L, 2, bc=bc, eps=eps, eps_mode=eps_mode, adapt_mode=I.ADAPT_EVERY)
    o = oracle.Oracle(p, q)
    keys, _ = o.leaves()
    got = M.keys_to_set(keys, dim)
    want = M.brute_force_tree(q, 2, eps, eps_mode, bc == I.BC_PERIODIC)
    assert got == want
    # leaves partition the domain
    vol = sum(2.0 ** (-dim * l) for l, _ in got)
    assert abs(vol - 1.0) < 1e-12
    # a second full adaptation at the same data changes nothing (idempotent)
    o.adapt()
    k2, _ = o.leaves()
    assert np.array_equal(k2, keys)


@pytest.mark.parametrize("dim,L,seed", [(1, 8, 5), (2, 6, 5), (1, 9, 14), (2, 6, 15)])
def test_leaf_stencils_are_graded(dim, L, seed):
    """Every leaf's radius-2 same-level stencil is stored or predictable from
    stored parent-level nodes, i.e. neighbouring leaves differ by <= 1 level."""
    q = _step_field(dim, L, seed)
    p = _problem(dim, L, 2, bc=I.BC_NEUMANN, eps=1e-3, adapt_mode=I.ADAPT_EVERY)
    o = oracle.Oracle(p, q)
    keys, _ = o.leaves()
    leaves = M.keys_to_set(keys, dim)
    # level of the leaf covering each finest cell
    n = 1 << L
    cover = np.zeros((n,) * dim, int)
    for l, idx in leaves:
        s = 1 << (L - l)
        cover[tuple(slice(a * s, (a + 1) * s) for a in idx)] = l
    assert cover.min() >= 2
    assert cover.max() - cover.min() >= 2  # the case really spans several levels
    for ax in range(dim):
        dif = np.abs(np.diff(cover, axis=ax))
        assert dif.max() <= 1
    # radius 2 at the parent level: a level-l leaf lies at least two level-(l-1)
    # cells away from any leaf of level l-2 or coarser
    for l, idx in leaves:
        if l < 4:
            continue
        s = 1 << (L - l + 1)
        lo = [max((a >> 1) * s - 2 * s, 0) for a in idx]
        hi = [min((a >> 1) * s + 3 * s, n) for a in idx]
        blk = cover[tuple(slice(a, b) for a, b in zip(lo, hi))]
        assert blk.min() >= l - 1


def _cover(keys, dim, L):
    """level of the leaf covering each finest cell; -1 where no leaf does
    (asserting that no cell is covered twice)"""
    n = 1 << L
    cover = np.full((n,) * dim, -1, int)
    for row in keys:
        l, idx = int(row[0]), [int(a) for a in row[1:1 + dim]]
        s = 1 << (L - l)
        blk = tuple(slice(a * s, (a + 1) * s) for a in reversed(idx))  # arrays are [z][y][x]
        assert np.all(cover[blk] == -1), "overlapping leaves"
        cover[blk] = l
    return cover


_LT_CASES = {
    # name: (problem and data, fine iterations, fine step below the CFL limit)
    "burgers1d": (lambda: I.burgers_1d(L=8, eps=1e-3, min_level=3), 96, 0.5 / 256),
    "burgers2d": (lambda: I.burgers_2d(L=6, eps=1e-3, min_level=2), 48, 0.25 / 64),
    "sod": (lambda: I.euler_1d_sod(L=8, eps=1e-3, min_level=2), 120, 0.25 / 256),
    "quadrants2d": (lambda: I.euler_2d_quadrants(L=6, eps=1e-3, min_level=2), 64, 0.125 / 64),
    "advection": (lambda: (lambda pq: (pq[0].replace(eps=1e-4, min_level=2), pq[1]))(
        I.advection_gaussian_1d(L=8)), 128, 0.5 / 256),
}


@pytest.mark.parametrize("case", sorted(_LT_CASES))
def test_lt_adaptation_keeps_invariants_every_iteration(case):
    """Adaptation inside the LT loop (Sec. 4, restricted remesh): after every
    fine iteration n the leaves still partition the box, neighbouring leaves
    differ by at most one level (across a periodic wrap too), no leaf below
    l_min(n) = the coarsest level whose step ends at n has split, merged or
    appeared, and every prediction source the iteration needs exists (the
    oracle reports a missing one as an error).  Fronts move through the
    tree, so it really changes; planted mistakes in the admissibility mask,
    in the grading closure, or an unrestricted remesh each fail a case."""
    make, steps, dt = _LT_CASES[case]
    p, q = make()
    dim = p.dim
    p = p.replace(adapt_mode=I.ADAPT_EVERY)
    L, lb = p.max_level, p.min_level
    nit = 1 << (L - lb)
    o = oracle.Oracle(p, q)
    prev = _cover(o.leaves()[0], dim, L)
    changed_total = changed_above_base = 0
    for n in range(steps):
        pos = n % nit
        lmin = next(l for l in range(lb, L + 1) if pos % (1 << (L - l)) == 0)
        o.iterate(dt, 1)
        cur = _cover(o.leaves()[0], dim, L)
        assert cur.min() >= lb, "a hole in the partition or a leaf below the base level"
        for ax in range(dim):
            assert np.abs(np.diff(cur, axis=ax)).max() <= 1
            if p.bc[dim - 1 - ax] == I.BC_PERIODIC:  # neighbours across the wrap ([z][y][x] arrays)
                assert np.abs(cur - np.roll(cur, 1, axis=ax)).max() <= 1
        low = (np.minimum(prev, cur) < lmin)
        assert np.array_equal(prev[low], cur[low]), f"iteration {n}: a level below l_min = {lmin} changed"
        if not np.array_equal(prev, cur):
            changed_total += 1
            changed_above_base += lmin > lb
        prev = cur
    assert changed_total >= 3 and changed_above_base >= 1
