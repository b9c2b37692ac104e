"""Batched instances (C-ABI `mr_batch`): every instance of a batch must give
exactly what the same problem gives when solved alone, and match the FP64
oracle like a single solve does.  The batch runs the same kernels in the
same order per instance (only the interleaving between instances differs),
so the comparison with the standalone solve is bitwise."""
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


def _mixed_problems():
    probs, qs = I.rd_batch(n=4, seed=3, levels=(5, 7), t_end=0.05)
    p, q = I.burgers_1d(L=8, eps=1e-3)
    probs.append(p); qs.append(q)
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, seed=1)
    probs.append(p); qs.append(q)
    p, q = I.euler_1d_sod(L=7, eps=1e-3, rk_order=2)
    probs.append(p); qs.append(q)
    p, q = I.euler_3d_blast(L=4, eps=1e-2, min_level=2, precision=I.PREC_FP64)
    probs.append(p); qs.append(q)
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, seed=2, time_mode=I.TIME_GTS)
    probs.append(p); qs.append(q)
    return probs, qs


def test_batch_equals_standalone_bitwise():
    import paper_1905_08717_gb300 as pkg
    probs, qs = _mixed_problems()
    b = pkg.Batch(probs, qs)
    for t in (0.02, 0.04):
        b.step(t)
    for i, (p, q) in enumerate(zip(probs, qs)):
        s = pkg.Solver(p, q)
        s.step(0.02)
        s.step(0.04)
        kb, vb = b.instances[i].leaves()
        ks, vs = s.leaves()
        assert np.array_equal(kb, ks), f"instance {i} ({p.name}): leaf sets differ"
        assert np.array_equal(vb, vs), f"instance {i} ({p.name}): values differ"
        sb, ss = b.instances[i].stats(), s.stats()
        assert sb["iters"] == ss["iters"] and sb["t"] == ss["t"] == 0.04
        s.close()
    b.close()


def test_batch_matches_oracle():
    import paper_1905_08717_gb300 as pkg
    probs, qs = I.rd_batch(n=3, seed=11, levels=(5, 6), t_end=0.03)
    p, q = I.burgers_1d(L=9, eps=1e-3)
    probs.append(p); qs.append(q)
    b = pkg.Batch(probs, qs)
    b.step(0.03)
    for i, (p, q) in enumerate(zip(probs, qs)):
        ref = oracle.Oracle(p, q)
        ref.step(0.03)
        kg, vg = b.instances[i].leaves()
        ko, vo = ref.leaves()
        assert np.array_equal(kg, ko), f"instance {i}: leaf sets differ"
        scale = np.abs(vo).max(axis=0)
        err = np.abs(vg - vo) / (np.abs(vo) + scale + 1e-300)
        assert err.max() <= TOL, f"instance {i}: {err.max():.3e}"
    b.close()


def test_batch_uneven_levels_reach_target():
    import paper_1905_08717_gb300 as pkg
    probs, qs = I.rd_batch(n=12, seed=5, levels=(5, 8), t_end=0.02)
    b = pkg.Batch(probs, qs)
    n = b.step(0.02)
    its = [v.stats()["iters"] for v in b.instances]
    assert n == sum(its)
    for v, p in zip(b.instances, probs):
        st = v.stats()
        assert st["t"] == 0.02 and st["pos"] == 0
        assert st["iters"] % (1 << (p.max_level - p.min_level)) == 0
    # finer instances need more fine iterations
    Ls = [p.max_level for p in probs]
    assert its[int(np.argmax(Ls))] >= its[int(np.argmin(Ls))]
    b.close()


def test_batch_rejects_bad_instance():
    import paper_1905_08717_gb300 as pkg
    probs, qs = I.rd_batch(n=3, seed=1, levels=(5, 5), t_end=0.02)
    probs[1] = probs[1].replace(rk_order=4)
    with pytest.raises(pkg.MRError, match="instance 1"):
        pkg.Batch(probs, qs)
