"""mr_leaf_mass_noalloc -- the entry point for callers that cannot allocate
device memory (their GPU memory is held by another allocator, or they run in
a loop that must not pay for cudaMalloc).  It must give the same per-variable
totals as MR_READ_STATS, call after call, although its only scratch is a fixed
array inside the library that every call reuses, and it must leave the
device's free memory untouched.  Collected last on purpose."""
import numpy as np
import pytest

from paper_1905_08717_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the tolerance of the GPU parity tests


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_08717_gb300 import build
    build.build()
    return t


def _state(torch, p, solver):
    """leaf keys and values on the device, the STATS totals, and their scale"""
    keys, vals = solver.leaves()
    want = solver.stats()["mass"]
    vol = np.prod([(p.hi[k] - p.lo[k]) for k in range(p.dim)]) * 2.0 ** (-p.dim * keys[:, 0])
    scale = (np.abs(vals) * vol[:, None]).sum(axis=0)
    kd = torch.from_numpy(np.ascontiguousarray(keys)).cuda()
    vd = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    return kd, vd, len(keys), want, scale


def _call(torch, pkg, p, st, out):
    kd, vd, n, want, scale = st
    pkg.leaf_mass_noalloc(p.dim, p.lo, p.hi, kd.data_ptr(), vd.data_ptr(), n, p.nvars(), out.data_ptr())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.abs(got - want) <= TOL * scale), (got, want)
    return got


@pytest.mark.parametrize("case", ["euler2d", "burgers1d"])
def test_leaf_mass_noalloc_matches_stats_on_consecutive_calls(torch, case):
    import paper_1905_08717_gb300 as pkg
    if case == "euler2d":
        p, q = I.euler_2d_quadrants(L=6, eps=1e-2, seed=1)
        times = (0.02, 0.05)
    else:
        p, q = I.burgers_1d(L=9, eps=1e-3)
        q = q + 0.5
        times = (0.1, 0.3)
    solver = pkg.Solver(p, q)
    states = []
    for t in times:
        solver.step(t)
        states.append(_state(torch, p, solver))
    out = torch.full((p.nvars(),), float("nan"), dtype=torch.float64, device="cuda")
    _call(torch, pkg, p, states[0], out)  # first call on the device: address look-up
    free0, res0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    # two calls in a row on different states share the scratch, then the first again
    got = [_call(torch, pkg, p, st, out) for st in (states[0], states[1], states[0])]
    assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed"
    assert torch.cuda.memory_reserved() == res0
    assert np.array_equal(got[0], got[2])
    if case == "euler2d":
        assert not np.array_equal(got[0], got[1])
    else:  # periodic Burgers with flux registers conserves the initial total exactly
        m0 = q.sum() / q.size
        for g in got:
            assert abs(g[0] - m0) <= TOL * np.abs(q).sum() / q.size, (g, m0)
    solver.close()


def test_leaf_mass_noalloc_rejects_sizes_beyond_its_scratch(torch):
    import paper_1905_08717_gb300 as pkg
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    keys = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    vals = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MRError, match="at most 5"):
        pkg.leaf_mass_noalloc(2, (0, 0, 0), (1, 1, 1), keys.data_ptr(), vals.data_ptr(), 4, 6,
                              out.data_ptr())
