"""Request server (C-ABI `mr_server`): problems submitted over time, admitted
at round boundaries under a device-memory budget, finished at their own end
times.  Each result must equal the same problem solved alone, bit for bit
(the server runs the same kernels in the same order per problem), and the
FP64 oracle: leaf by leaf within 1e-12 in FP64, and within the mixed-precision
L1 bound (derived in test_gpu_mixed) in the mixed mode."""
import numpy as np
import pytest

import oracle
from paper_1905_08717_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12
U32 = 2.0 ** -24
C_FLUX = 64
C_STATE = 32


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


def _vs_oracle(r, p, q, t):
    """a served result against the FP64 oracle run of the same request"""
    ref = oracle.Oracle(p.replace(precision=I.PREC_FP64), q)
    ref.step(t)
    if p.precision == I.PREC_FP64:
        kr, vr = r.leaves()
        ko, vo = ref.leaves()
        assert np.array_equal(kr, ko), (p.name, len(kr), len(ko))
        err = np.abs(vr - vo) / (np.abs(vo) + np.abs(vo).max(axis=0) + 1e-300)
        assert err.max() <= TOL, (p.name, err.max())
    else:
        n = ref.stats()["iters"]
        tol = n * (6 * C_FLUX * U32 * p.cfl + C_STATE * U32) + U32 + p.eps * 1e-2
        a, b = r.uniform(), ref.uniform()
        a = a.reshape(a.shape[0], -1)
        b = b.reshape(b.shape[0], -1)
        e = np.abs(a - b).sum(axis=1) / np.maximum(np.abs(b).sum(axis=1), 1e-300)
        assert e.max() <= tol, (p.name, e, tol)
    ref.close()


@pytest.mark.parametrize("caps,prec", [((0, 0), I.PREC_FP64), ((5, 152), I.PREC_FP64),
                                       ((0, 0), I.PREC_MIXED)])
def test_serve_results_equal_standalone(caps, prec):
    """caps: stage-launch block caps for the first and the later requests
    (0: the default launch shape); the results must not depend on them.
    Every served result also matches the FP64 oracle (see the module note)."""
    import paper_1905_08717_gb300 as pkg
    probs, qs, ends = _requests()
    probs = [p.replace(precision=prec) for p in probs]
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
        s.set_launch_mode(pkg.MR_LAUNCH_GRAPH)  # the served requests' launch path
        s.step(t)
        kr, vr = r.leaves()
        ks, vs = s.leaves()
        assert np.array_equal(kr, ks) and np.array_equal(vr, vs), p.name
        assert r.stats()["t"] == t
        _vs_oracle(r, p, q, t)
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
