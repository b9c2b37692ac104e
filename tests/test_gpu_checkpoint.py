"""Checkpoint / resume at a macro-step boundary: a solver created from the
saved leaves, time and iteration count continues exactly as the original
one (bit for bit on the same GPU); invalid states are rejected."""
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


def _cases():
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=0)
    yield p, q, 0.04, 0.09
    p, q = I.burgers_1d(L=10, eps=1e-3)
    yield p.replace(rk_order=2), q, 0.1, 0.3
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, seed=2, time_mode=I.TIME_GTS)
    yield p, q, 0.03, 0.06
    p, q = I.euler_3d_blast(L=5, eps=1e-2, min_level=2)
    yield p, q, 0.01, 0.02
    p, q = I.burgers_2d_paper(L=6, eps=1e-3, min_level=3)
    yield p, q, 0.1, 0.2


@pytest.mark.parametrize("case", range(5))
def test_resume_continues_bit_for_bit(case):
    import paper_1905_08717_gb300 as pkg
    p, q, t1, t2 = list(_cases())[case]
    a = pkg.Solver(p, q)
    a.step(t1)
    keys, vals, t, iters = a.state()
    assert t == t1 and iters % (1 << (p.max_level - p.min_level)) == 0
    b = pkg.Solver.from_state(p, keys, vals, t, iters)
    kb, vb = b.leaves()
    assert np.array_equal(kb, keys) and np.array_equal(vb, vals)
    a.step(t2)
    b.step(t2)
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    sa, sb = a.stats(), b.stats()
    assert sa["t"] == sb["t"] and sa["iters"] == sb["iters"] and sa["macros"] == sb["macros"]


def test_invalid_states_are_rejected():
    import paper_1905_08717_gb300 as pkg
    p, q = I.burgers_1d(L=8, eps=1e-3)
    a = pkg.Solver(p, q)
    a.step(0.05)
    keys, vals, t, iters = a.state()
    with pytest.raises(pkg.MRError) as e:  # not a macro-step boundary
        pkg.Solver.from_state(p, keys, vals, t, iters + 1)
    assert e.value.status == 5
    with pytest.raises(pkg.MRError) as e:  # a hole in the partition
        pkg.Solver.from_state(p, keys[1:], vals[1:], t, iters)
    assert e.value.status == 1
    dup = np.concatenate([keys, keys[:1]])
    with pytest.raises(pkg.MRError) as e:  # overlapping leaves
        pkg.Solver.from_state(p, dup, np.concatenate([vals, vals[:1]]), t, iters)
    assert e.value.status == 1


def test_async_calls_give_the_same_result():
    """mr_set_async: step/iterate return once enqueued; mr_sync reports errors"""
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3, seed=1)
    a, b = pkg.Solver(p, q), pkg.Solver(p, q)
    b.set_async(True)
    dt = 0.5 / 128 / 3.7
    for s in (a, b):
        s.iterate(dt, 16)   # one whole macro step (graph) ...
        s.iterate(dt, 5)    # ... and single iterations
        s.iterate(dt, 11)
        s.step(0.08)
    b.sync()
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    b.set_async(False)
