"""The N > 1 path of bench.py on CPU: two gloo ranks stand in for two GPUs.
Replicas share no data; the bench only combines their timings (max over
ranks) and counts every rank's units.  The reference arm runs on rank 0
alone."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    total = [2.0, 3.0][rank]
    e2e = [2.5, 2.2][rank]
    out = bench.replica_aggregate(dist, ws, total, e2e, updates=600, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_replica_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        tmax, e2e, value, e2e_value = res[r]
        assert tmax == 3.0 and e2e == 2.5           # slowest rank on both clocks
        assert value == 2 * 600 / 3.0                 # units of both replicas
        assert e2e_value == 2 * 600 / 2.5


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_aggregate(None, 1, 2.0, 4.0, 100) == (2.0, 4.0, 50.0, 25.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env["RANK"], env["LOCAL_RANK"] = "0", "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_traffic_figure_comes_from_the_committed_dram_summary():
    """roofline.traffic is the committed per-leaf-stage DRAM figure times the
    leaf-stages of one launch, and only while the summary's kernel_sha16 line
    names the stage-kernel sources built here (null otherwise); the figure
    parses to a positive number below the algorithmic bytes of a leaf-stage
    (the state is L2-resident)."""
    sys.path.insert(0, ROOT)
    import bench
    val, sha = None, None
    for ln in open(os.path.join(ROOT, "profiles", "stage_kernel_dram_euler2d_L10.md")):
        if ln.startswith("dram_bytes_per_leaf_stage:"):
            val = float(ln.split(":")[1].split()[0])
        elif ln.startswith("kernel_sha16:"):
            sha = ln.split(":")[1].strip()
    assert val is not None and 0.0 < val < max(bench.BYTES_PER_LEAF_STAGE.values())
    tpl = bench._traffic_per_leaf_stage()
    if sha == bench.stage_kernel_hash():
        assert tpl == val
    else:
        assert tpl is None
