"""Leaf-proportional storage: node values live in slot arrays sized by the
tree, not by the dense grids.  The footprint of the benchmark solve is a
fraction of the dense layout's, the 3D blast at L = 8 fits in 2 GB, the
arrays are compacted once the tree grows slowly, and neither the capacity
nor the slot numbering changes a result (bit for bit)."""
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


def _dense_bytes(p):
    """bytes of a layout that stores every field and both registers for every
    cell of every level (the values alone, 8 fields + 2 x 2d registers)"""
    cells = sum(1 << (p.dim * l) for l in range(p.min_level, p.max_level + 1))
    esz = 4 if p.precision == I.PREC_MIXED else 8
    return cells * p.nvars() * (8 * esz + 2 * 2 * p.dim * 8)


def test_benchmark_footprint_and_growth():
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    s = pkg.Solver(p, q)
    st0 = s.stats()
    assert st0["node_slots"] >= st0["nodes"]
    s.step(0.05)  # the tree grows about 2.5x, then slowly: compacted
    st = s.stats()
    assert st["node_slots"] >= st["nodes"] > st0["nodes"]
    assert st["node_slots"] < st0["node_slots"]
    dense = _dense_bytes(p)
    print(f"nodes {st['nodes']}, slots {st['node_slots']}, halts {st['halts']}, "
          f"{st['device_bytes'] / 2**20:.1f} MiB against {dense / 2**20:.1f} MiB for dense values "
          f"({dense / st['device_bytes']:.1f}x)")
    assert st["device_bytes"] * 8 < dense, (st["device_bytes"], dense)
    s.close()


def test_capacity_and_slot_numbering_do_not_change_results():
    """the same solve with node arrays reserved far larger (no growth, other
    slot numbers) and with the default rule (several compacting growths)"""
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=9, eps=1e-3, seed=2)
    a, b = pkg.Solver(p, q), pkg.Solver(p, q)
    b.reserve_nodes(250000)
    assert b.stats()["node_slots"] >= 250000
    for t in (0.02, 0.06):
        a.step(t)
        b.step(t)
        ka, va = a.leaves()
        kb, vb = b.leaves()
        assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    assert a.stats()["node_slots"] <= b.stats()["node_slots"]
    print(f"default rule: {a.stats()['node_slots']} slots, {a.stats()['halts']} halts; "
          f"reserved: {b.stats()['node_slots']} slots, {b.stats()['halts']} halts")


def test_blast_3d_L8_mixed_fits_in_2GB():
    """the 3D precision workload (256^3 finest) to t = 0.1: about 1.9 M
    leaves, held in less than 2 GB of device memory"""
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_3d_blast(L=8, eps=1e-3, min_level=3)
    s = pkg.Solver(p, q)
    s.step(0.1)
    st = s.stats()
    assert st["leaves"] > 1_000_000
    assert st["device_bytes"] < 2 * 2**30, st["device_bytes"]
    print(f"3D L=8 mixed: {st['leaves']} leaves, {st['node_slots']} slots, "
          f"{st['device_bytes'] / 2**30:.2f} GiB")
    s.close()


def test_batch_instances_recover_from_halts_bitwise():
    """batch instances read the halt record at their next boundary instead of
    every 16 fine iterations: a fast-growing tree (2D Euler quadrants, L = 9,
    the opening phase) halts and resumes, with results bitwise those of the
    standalone solver"""
    import paper_1905_08717_gb300 as pkg
    probs = [I.euler_2d_quadrants(L=9, eps=1e-3, seed=s) for s in (2, 3)]
    b = pkg.Batch([p for p, _ in probs], [q for _, q in probs])
    b.step(0.06)
    halts = 0
    for (p, q), inst in zip(probs, b.instances):
        s = pkg.Solver(p, q)
        s.set_launch_mode(pkg.MR_LAUNCH_GRAPH)
        s.step(0.06)
        ka, va = inst.leaves()
        kb, vb = s.leaves()
        assert np.array_equal(ka, kb) and np.array_equal(va, vb)
        st = inst.stats()
        assert st["node_slots"] >= st["nodes"] and st["pos"] == 0
        halts += st["halts"]
        s.close()
    print(f"batch of 2: {halts} halts")
    b.close()


def test_single_iterations_equal_whole_macro_steps_bitwise():
    """one fine iteration per call (direct launches, a check point at the end
    of every call) against whole macro steps in one call (graphs, check points
    at macro-step ends): the same bits, with the default capacity rule and its
    resizes, over twelve macro steps of a growing tree (2D Euler quadrants,
    L = 9)"""
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=9, eps=1e-3, seed=3)
    a, b = pkg.Solver(p, q), pkg.Solver(p, q)
    dt = 3.0e-5
    nit = 1 << (p.max_level - p.min_level)
    n = 12 * nit + 5
    for _ in range(n):
        a.iterate(dt, 1)
    b.iterate(dt, n)
    ka, va = a.leaves()
    kb, vb = b.leaves()
    assert np.array_equal(ka, kb) and np.array_equal(va, vb)
    sa, sb = a.stats(), b.stats()
    assert sa["iters"] == sb["iters"] == n and sa["pos"] == sb["pos"] == 5
    print(f"single iterations: {sa['halts']} halts; whole macro steps: {sb['halts']} halts")
    a.close()
    b.close()


def test_persistent_mode_keeps_room_for_every_cell():
    """switching to the persistent kernel (which installs trees without a host
    check) gives the node arrays a slot for every cell; switching back
    compacts them again at the next boundary, and the result matches a solve
    that never switched to FP64 round-off"""
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=9, eps=1e-3, seed=2)
    cells = sum(1 << (2 * l) for l in range(p.min_level, p.max_level + 1))
    s, ref = pkg.Solver(p, q), pkg.Solver(p, q)
    s.step(0.01)
    ref.step(0.01)
    assert s.stats()["node_slots"] < cells
    s.set_launch_mode(pkg.MR_LAUNCH_PERSISTENT)
    assert s.stats()["node_slots"] == cells
    s.step(0.02)
    ref.step(0.02)
    s.set_launch_mode(pkg.MR_LAUNCH_GRAPH)
    s.step(0.03)
    ref.step(0.03)
    assert s.stats()["node_slots"] < cells
    ka, va = s.leaves()
    kb, vb = ref.leaves()
    assert np.array_equal(ka, kb)
    scale = np.abs(vb).max(axis=0)
    assert np.all(np.abs(va - vb) <= 1e-13 * (np.abs(vb) + scale))
    s.close()
    ref.close()
