"""Request server (C-ABI `mr_server`): problems submitted over time, admitted
at round boundaries under a device-memory budget, finished at their own end
times.  Each result must equal the same problem solved alone, bit for bit
(the server runs the same kernels in the same order per problem)."""
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


def _requests():
    probs, qs = I.rd_batch(n=3, seed=21, levels=(5, 7), t_end=0.0)
    ends = [0.02, 0.035, 0.01]
    p, q = I.burgers_1d(L=9, eps=1e-3)
    probs.append(p); qs.append(q); ends.append(0.15)
    p, q = I.euler_2d_quadrants(L=6, eps=1e-3, seed=3)
    probs.append(p); qs.append(q); ends.append(0.05)
    p, q = I.euler_3d_blast(L=4, eps=1e-2, min_level=2)
    probs.append(p); qs.append(q); ends.append(0.01)
    return probs, qs, ends


def _drain(srv, done, seconds=300.0):
    import time
    t_stop = time.monotonic() + seconds
    while time.monotonic() < t_stop:
        a, qd = srv.advance()
        got = srv.poll()
        done.extend(got)
        if a == 0 and qd == 0:
            return
        if not got:
            time.sleep(1e-4)
    raise AssertionError("server did not drain")


@pytest.mark.parametrize("caps", [(0, 0), (5, 152)])
def test_serve_results_equal_standalone(caps):
    """caps: stage-launch block caps for the first and the later requests
    (0: the default launch shape); the results must not depend on them"""
    import paper_1905_08717_gb300 as pkg
    probs, qs, ends = _requests()
    srv = pkg.Server(mem_budget_bytes=8 << 30, max_active=16)
    srv.set_grid_cap(caps[0])
    ids, done = [], []
    for p, q, t in zip(probs[:3], qs[:3], ends[:3]):
        ids.append(srv.submit(p, q, t))
    for _ in range(50):  # later requests join a running set
        srv.advance()
        done.extend(srv.poll())
    srv.set_grid_cap(caps[1])
    for p, q, t in zip(probs[3:], qs[3:], ends[3:]):
        ids.append(srv.submit(p, q, t))
    _drain(srv, done)
    assert sorted(done) == sorted(ids)
    for rid, p, q, t in zip(ids, probs, qs, ends):
        assert srv.status(rid) == 0
        r = srv.result(rid)
        s = pkg.Solver(p, q)
        s.step(t)
        kr, vr = r.leaves()
        ks, vs = s.leaves()
        assert np.array_equal(kr, ks) and np.array_equal(vr, vs), p.name
        assert r.stats()["t"] == t
        s.close()
        srv.release(rid)
    assert srv.memory() == 0
    srv.close()


def test_serve_memory_budget_limits_admission():
    import paper_1905_08717_gb300 as pkg
    probs, qs = I.rd_batch(n=6, seed=2, levels=(6, 6), t_end=0.0)
    one = pkg.Server(mem_budget_bytes=8 << 30, max_active=1)
    rid = one.submit(probs[0], qs[0], 0.01)
    _drain(one, [])
    need = one.memory()  # footprint of one such problem (result still held)
    one.release(rid)
    one.close()
    assert need > 0
    srv = pkg.Server(mem_budget_bytes=2 * need + need // 2, max_active=8)
    ids = [srv.submit(p, q, 0.01) for p, q in zip(probs, qs)]
    import time
    done, peak = [], 0
    t_stop = time.monotonic() + 300.0
    while time.monotonic() < t_stop:
        a, qd = srv.advance()
        peak = max(peak, srv.memory())
        assert srv.memory() <= 2 * need + need // 2
        got = srv.poll()
        for rid in got:
            done.append(rid)
            srv.release(rid)  # frees room for the queue
        if a == 0 and qd == 0:
            break
        if not got:
            time.sleep(1e-4)
    assert sorted(done) == sorted(ids)
    assert peak == 2 * need  # two problems in flight at most
    srv.close()


def test_serve_rejects_oversize_and_invalid():
    import paper_1905_08717_gb300 as pkg
    p, q = I.euler_2d_quadrants(L=7, eps=1e-3)
    srv = pkg.Server(mem_budget_bytes=1 << 20, max_active=4)
    with pytest.raises(pkg.MRError, match="budget"):
        srv.submit(p, q, 0.01)
    with pytest.raises(pkg.MRError):
        srv.submit(p.replace(rk_order=5), q, 0.01)
    srv.close()
