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
        s.set_launch_mode(pkg.MR_LAUNCH_GRAPH)  # the batch instances' launch path
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


def test_grid_cap_does_not_change_results():
    """A stage launch of 1, 7 or 152 thread blocks (or the resident capacity)
    computes bitwise the same leaves, also when the cap changes between macro
    steps (the captured macro-step graph is replaced)."""
    import paper_1905_08717_gb300 as pkg
    probs, qs = _mixed_problems()
    for i in (4, 5, 6, 7):
        p, q = probs[i], qs[i]
        ref = pkg.Solver(p, q)
        ref.step(0.02)
        ref.step(0.04)
        kr, vr = ref.leaves()
        for caps in ((1, 1), (7, 7), (152, 152), (0, 3), (5, 0)):
            s = pkg.Solver(p, q)
            s.set_grid_cap(caps[0])
            s.step(0.02)
            s.set_grid_cap(caps[1])
            s.step(0.04)
            k, v = s.leaves()
            assert np.array_equal(k, kr), f"{p.name}, caps {caps}: leaf sets differ"
            assert np.array_equal(v, vr), f"{p.name}, caps {caps}: values differ"
            s.close()
        with pytest.raises(pkg.MRError):
            ref.set_grid_cap(-1)
        ref.close()


def test_autotuned_batch_equals_default():
    """The package's tuner picks a cap by timing; whichever it picks, the
    batch gives bitwise the default batch's results."""
    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import autotune
    probs, qs = _mixed_problems()
    tune = autotune.tune_batch(probs, qs, 0.01, 0.01, caps=[0, 16, 4])
    assert tune["best"] in (0, 16, 4) and set(tune["seconds"]) == {0, 16, 4}
    assert all(v > 0 for v in tune["seconds"].values())
    b0 = pkg.Batch(probs, qs)
    bt = pkg.Batch(probs, qs, grid_cap=4)
    for b in (b0, bt):
        b.step(0.02)
    for i in range(len(probs)):
        k0, v0 = b0.instances[i].leaves()
        kt, vt = bt.instances[i].leaves()
        assert np.array_equal(k0, kt) and np.array_equal(v0, vt), f"instance {i}"
    b0.close()
    bt.close()
