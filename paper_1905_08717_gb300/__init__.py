"""GB300-native MRLT/NERK: adaptive multiresolution finite volumes with local
time-stepping by natural continuous extension of Runge-Kutta methods.

Thin Python binding of the C-ABI in include/mrlt.h (argument marshalling
only; every step of the method runs in the CUDA library libmrlt.so).  The
binding raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded synthetic initial data)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "csrc", "libmrlt.so")

MR_READ_LEAF_KEYS, MR_READ_LEAF_VALUES, MR_READ_UNIFORM, MR_READ_STATS, MR_READ_PROFILE = 0, 1, 2, 3, 4
MR_LAUNCH_PERSISTENT, MR_LAUNCH_GRAPH = 0, 1
STATUS = {0: "MR_OK", 1: "MR_E_INVALID", 2: "MR_E_NOMEM", 3: "MR_E_CUDA",
          4: "MR_E_TIMEOUT", 5: "MR_E_STATE", 6: "MR_E_NUMERIC"}


class MRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mr_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("equation", ctypes.c_int),
                ("max_level", ctypes.c_int), ("min_level", ctypes.c_int),
                ("eps", ctypes.c_double), ("eps_mode", ctypes.c_int),
                ("rk_order", ctypes.c_int), ("time_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("adapt_mode", ctypes.c_int),
                ("reflux", ctypes.c_int), ("cfl", ctypes.c_double),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 3), ("phys", ctypes.c_double * 8),
                ("flux", ctypes.c_int)]


_lib = None


def library() -> ctypes.CDLL:
    """Load libmrlt.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} "
                               "(run `python -m paper_1905_08717_gb300.build`)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, ll = ctypes.c_void_p, ctypes.c_longlong
        lib.mr_create.argtypes = [ctypes.POINTER(mr_config), ctypes.POINTER(ctypes.c_double), vp,
                                  ctypes.POINTER(vp)]
        lib.mr_reset.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.mr_set_tree.argtypes = [vp, ctypes.POINTER(ctypes.c_ubyte)]
        lib.mr_adapt.argtypes = [vp]
        lib.mr_step.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ll)]
        lib.mr_iterate.argtypes = [vp, ctypes.c_double, ll, ctypes.POINTER(ll)]
        lib.mr_read.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        lib.mr_destroy.argtypes = [vp]
        lib.mr_last_error.argtypes = [vp]
        lib.mr_last_error.restype = ctypes.c_char_p
        lib.mr_profile.argtypes = [vp, ctypes.c_int]
        lib.mr_profile.restype = ctypes.c_int
        lib.mr_launch_count.argtypes = [vp]
        lib.mr_launch_count.restype = ll
        lib.mr_set_async.argtypes = [vp, ctypes.c_int]
        lib.mr_sync.argtypes = [vp]
        lib.mr_set_grid_cap.argtypes = [vp, ctypes.c_int]
        lib.mr_set_launch_mode.argtypes = [vp, ctypes.c_int]
        lib.mr_reserve_nodes.argtypes = [vp, ll]
        lib.mr_selftest_grid_wait.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, vp]
        lib.mr_batch_set_grid_cap.argtypes = [vp, ctypes.c_int]
        lib.mr_server_set_grid_cap.argtypes = [vp, ctypes.c_int]
        lib.mr_release_cached_memory.argtypes = []
        lib.mr_release_cached_memory.restype = ctypes.c_int
        lib.mr_leaf_mass_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), vp, vp, ll, ctypes.c_int,
                                             vp, vp, ctypes.c_char_p, ctypes.c_size_t]
        lib.mr_create_from_state.argtypes = [ctypes.POINTER(mr_config), ll, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_double, ll, vp,
                                             ctypes.POINTER(vp)]
        lib.mr_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(mr_config),
                                        ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), vp,
                                        ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)]
        lib.mr_batch_step.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ll)]
        lib.mr_batch_instance.argtypes = [vp, ctypes.c_int]
        lib.mr_batch_instance.restype = vp
        lib.mr_batch_last_error.argtypes = [vp]
        lib.mr_batch_last_error.restype = ctypes.c_char_p
        lib.mr_batch_destroy.argtypes = [vp]
        lib.mr_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, vp, ctypes.POINTER(vp)]
        lib.mr_server_submit.argtypes = [vp, ctypes.POINTER(mr_config), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_double, ctypes.POINTER(ll)]
        lib.mr_server_advance.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        lib.mr_server_poll.argtypes = [vp, ctypes.POINTER(ll), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        lib.mr_server_status.argtypes = [vp, ll]
        lib.mr_server_result.argtypes = [vp, ll]
        lib.mr_server_result.restype = vp
        lib.mr_server_release.argtypes = [vp, ll]
        lib.mr_server_memory.argtypes = [vp]
        lib.mr_server_memory.restype = ctypes.c_size_t
        lib.mr_server_last_error.argtypes = [vp]
        lib.mr_server_last_error.restype = ctypes.c_char_p
        lib.mr_server_destroy.argtypes = [vp]
        for name in ("mr_create", "mr_reset", "mr_set_tree", "mr_adapt", "mr_step",
                     "mr_iterate", "mr_read", "mr_leaf_mass_noalloc", "mr_batch_create", "mr_create_from_state",
                     "mr_batch_step", "mr_set_async", "mr_sync", "mr_set_grid_cap", "mr_set_launch_mode",
                     "mr_selftest_grid_wait", "mr_reserve_nodes", "mr_batch_set_grid_cap", "mr_server_set_grid_cap",
                     "mr_server_create", "mr_server_submit", "mr_server_advance",
                     "mr_server_poll", "mr_server_status", "mr_server_release"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def make_config(p) -> mr_config:
    c = mr_config()
    c.dim, c.equation, c.max_level, c.min_level = p.dim, p.equation, p.max_level, p.min_level
    c.eps, c.eps_mode, c.rk_order, c.time_mode = p.eps, p.eps_mode, p.rk_order, p.time_mode
    c.precision, c.adapt_mode, c.reflux, c.cfl = p.precision, p.adapt_mode, p.reflux, p.cfl
    for k in range(3):
        c.lo[k], c.hi[k], c.bc[k] = p.lo[k], p.hi[k], p.bc[k]
    for k in range(8):
        c.phys[k] = p.phys[k]
    c.flux = getattr(p, "flux", 0)
    return c


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def leaf_mass_noalloc(dim: int, lo, hi, keys_ptr: int, values_ptr: int, n_leaves: int, m: int,
                      mass_ptr: int, stream=None) -> None:
    """Binding of mr_leaf_mass_noalloc: per-variable sum of q |cell| over leaves
    whose keys / values already live in caller-owned device buffers (raw device
    pointers), written to the caller's device buffer mass_ptr[m].  The call
    allocates no device memory; the result is ready when `stream` reaches it."""
    lib = library()
    lo3 = (ctypes.c_double * 3)(*[float(x) for x in lo][:3])
    hi3 = (ctypes.c_double * 3)(*[float(x) for x in hi][:3])
    msg = ctypes.create_string_buffer(256)
    r = lib.mr_leaf_mass_noalloc(dim, lo3, hi3, keys_ptr, values_ptr, n_leaves, m, mass_ptr,
                                 ctypes.c_void_p(_stream_handle(stream)), msg, len(msg))
    if r != 0:
        raise MRError(r, msg.value.decode())


def selftest_grid_wait(ctas: int, missing: int, limit_s: float, stream=None) -> int:
    """Binding of mr_selftest_grid_wait: the status (0 = MR_OK, 4 = MR_E_TIMEOUT)
    of one bounded grid barrier that `missing` CTAs never reach."""
    return library().mr_selftest_grid_wait(int(ctas), int(missing), float(limit_s),
                                           ctypes.c_void_p(_stream_handle(stream)))


def release_cached_memory() -> None:
    """Return the device memory the library keeps cached for future solvers."""
    r = library().mr_release_cached_memory()
    if r != 0:
        raise MRError(r, "mr_release_cached_memory failed")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Solver:
    """One MR/MRLT solve on the GPU (handle of the C-ABI `mr_solver`)."""

    def __init__(self, problem, q0: np.ndarray, stream=None):
        lib = library()
        self.p = problem
        self.m = problem.nvars()
        q = np.ascontiguousarray(q0, dtype=np.float64).reshape(self.m, -1)
        self._cfg = make_config(problem)
        self._h = ctypes.c_void_p()
        r = lib.mr_create(ctypes.byref(self._cfg), _dptr(q), ctypes.c_void_p(_stream_handle(stream)),
                          ctypes.byref(self._h))
        if r != 0:
            raise MRError(r, "mr_create failed")

    @classmethod
    def from_state(cls, problem, keys: np.ndarray, values: np.ndarray, t: float, iters: int, stream=None):
        """Resume from a state saved at a macro-step boundary (see state())."""
        lib = library()
        self = cls.__new__(cls)
        self.p = problem
        self.m = problem.nvars()
        k = np.ascontiguousarray(keys, dtype=np.int32).reshape(-1, 4)
        v = np.ascontiguousarray(values, dtype=np.float64).reshape(-1, self.m)
        self._cfg = make_config(problem)
        self._h = ctypes.c_void_p()
        r = lib.mr_create_from_state(ctypes.byref(self._cfg), len(k), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     _dptr(v), float(t), int(iters), ctypes.c_void_p(_stream_handle(stream)),
                                     ctypes.byref(self._h))
        if r != 0:
            raise MRError(r, "mr_create_from_state failed")
        return self

    def state(self):
        """(keys, values, t, iters): everything needed to resume at a
        macro-step boundary with from_state()"""
        k, v = self.leaves()
        st = self.stats()
        return k, v, st["t"], st["iters"]

    @classmethod
    def _view(cls, problem, handle: int, owner):
        """non-owning view of a solver that `owner` (a Batch) holds"""
        self = cls.__new__(cls)
        self.p = problem
        self.m = problem.nvars()
        self._h = ctypes.c_void_p(handle)
        self._owner = owner
        return self

    def _check(self, r: int, what: str):
        if r != 0:
            raise MRError(r, f"{what}: {library().mr_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._h = ctypes.c_void_p()  # a view: the batch releases the solver
            return
        if self._h:
            library().mr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, q0: np.ndarray):
        q = np.ascontiguousarray(q0, dtype=np.float64).reshape(self.m, -1)
        self._check(library().mr_reset(self._h, _dptr(q)), "reset")

    def set_tree(self, leaf_level_finest: np.ndarray):
        a = np.ascontiguousarray(leaf_level_finest, dtype=np.uint8).ravel()
        self._check(library().mr_set_tree(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))),
                    "set_tree")

    def adapt(self):
        self._check(library().mr_adapt(self._h), "adapt")

    def step(self, t_target: float) -> int:
        it = ctypes.c_longlong()
        self._check(library().mr_step(self._h, t_target, ctypes.byref(it)), "step")
        return it.value

    def iterate(self, dt: float, n_iters: int) -> int:
        it = ctypes.c_longlong()
        self._check(library().mr_iterate(self._h, dt, n_iters, ctypes.byref(it)), "iterate")
        return it.value

    def set_async(self, enable: bool):
        """step()/iterate() return once their work is enqueued; errors are
        reported by sync()"""
        self._check(library().mr_set_async(self._h, int(enable)), "set_async")

    def sync(self):
        self._check(library().mr_sync(self._h), "sync")

    def set_grid_cap(self, ctas: int):
        """at most `ctas` thread blocks per stage-kernel launch (0: fill the
        GPU); the results do not depend on it"""
        self._check(library().mr_set_grid_cap(self._h, int(ctas)), "set_grid_cap")

    def set_launch_mode(self, mode: int):
        """MR_LAUNCH_PERSISTENT (one cooperative macro-step kernel, the
        default) or MR_LAUNCH_GRAPH (one kernel per phase); bitwise the same
        results"""
        self._check(library().mr_set_launch_mode(self._h, int(mode)), "set_launch_mode")

    def _read(self, what, dtype, shape=None, out=None):
        lib = library()
        used = ctypes.c_size_t()
        self._check(lib.mr_read(self._h, what, None, 0, ctypes.byref(used)), "read size")
        n = used.value // np.dtype(dtype).itemsize
        buf = out if out is not None else np.empty(n, dtype=dtype)
        self._check(lib.mr_read(self._h, what, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes,
                                ctypes.byref(used)), "read")
        return buf if shape is None else buf.reshape(shape)

    def leaves(self):
        k = self._read(MR_READ_LEAF_KEYS, np.int32, (-1, 4))
        v = self._read(MR_READ_LEAF_VALUES, np.float64, (-1, self.m))
        return k, v

    def uniform(self) -> np.ndarray:
        n = 1 << self.p.max_level
        return self._read(MR_READ_UNIFORM, np.float64, (self.m,) + (n,) * self.p.dim)

    def stats(self) -> dict:
        s = self._read(MR_READ_STATS, np.float64)
        L = self.p.max_level
        return {"t": s[0], "iters": int(s[1]), "macros": int(s[2]), "dt": s[3],
                "leaves": int(s[4]), "nodes": int(s[5]), "near": int(s[6]),
                "updates": int(s[7]), "pos": int(s[15]), "mass": s[8:8 + self.m].copy(),
                "node_slots": int(s[13]), "device_bytes": int(s[14]), "free_slots": int(s[62]), "halts": int(s[61]),
                "leaves_per_level": s[16:17 + L].astype(np.int64)}

    def reserve_nodes(self, nodes: int):
        """node arrays of at least `nodes` slots (at a macro-step boundary)"""
        self._check(library().mr_reserve_nodes(self._h, int(nodes)), "reserve_nodes")

    def profile(self, enable: bool):
        """start / stop CUDA-event timing of the stage-kernel launches"""
        self._check(library().mr_profile(self._h, int(enable)), "profile")

    def profile_read(self) -> dict:
        P = self._read(MR_READ_PROFILE, np.float64)
        L = self.p.max_level
        return {"stage_launches": int(P[0]), "stage_ms": float(P[1]),
                "leaf_stages": P[2:5].astype(np.int64), "launches": int(P[5]),
                "leaf_stages_per_level": P[16:17 + L].astype(np.int64),
                "stage_ms_per_level": P[40:41 + L].copy()}

    def launch_count(self) -> int:
        return int(library().mr_launch_count(self._h))


class Batch:
    """Independent problems advanced together (C-ABI `mr_batch`): each
    instance is a solver with its own stream and its macro step as a CUDA
    graph, so the instances run concurrently on the GPU."""

    def __init__(self, problems, q0s, stream=None, grid_cap: int = 0):
        lib = library()
        if len(problems) != len(q0s) or not problems:
            raise ValueError("one initial condition per problem, at least one problem")
        self.problems = list(problems)
        n = len(problems)
        cfgs = (mr_config * n)(*[make_config(p) for p in problems])
        self._q = [np.ascontiguousarray(q, dtype=np.float64).reshape(p.nvars(), -1)
                   for p, q in zip(problems, q0s)]
        ptrs = (ctypes.POINTER(ctypes.c_double) * n)(*[_dptr(q) for q in self._q])
        self._b = ctypes.c_void_p()
        bad = ctypes.c_int(-1)
        r = lib.mr_batch_create(n, cfgs, ptrs, ctypes.c_void_p(_stream_handle(stream)),
                                ctypes.byref(self._b), ctypes.byref(bad))
        if r != 0:
            raise MRError(r, f"mr_batch_create failed (instance {bad.value})")
        self.instances = [Solver._view(p, lib.mr_batch_instance(self._b, i), self)
                          for i, p in enumerate(problems)]
        if grid_cap:
            self.set_grid_cap(grid_cap)

    def set_grid_cap(self, ctas: int):
        """at most `ctas` thread blocks per stage-kernel launch of every
        instance, so that more instances share the GPU at once (0: each launch
        may fill the GPU); the results do not depend on it"""
        lib = library()
        r = lib.mr_batch_set_grid_cap(self._b, int(ctas))
        if r != 0:
            raise MRError(r, "batch grid cap: " + lib.mr_batch_last_error(self._b).decode())

    def step(self, t_target: float) -> int:
        lib = library()
        it = ctypes.c_longlong()
        r = lib.mr_batch_step(self._b, t_target, ctypes.byref(it))
        if r != 0:
            raise MRError(r, "batch step: " + lib.mr_batch_last_error(self._b).decode())
        return it.value

    def close(self):
        if getattr(self, "_b", None):
            for v in self.instances:
                v._h = ctypes.c_void_p()
            library().mr_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (C-ABI `mr_server`): problems are
    submitted with their own end time, join the running set at round
    boundaries while their device footprint fits the budget, and are
    reported by poll() when finished."""

    def __init__(self, mem_budget_bytes: int, max_active: int, stream=None):
        lib = library()
        self._s = ctypes.c_void_p()
        r = lib.mr_server_create(int(mem_budget_bytes), int(max_active),
                                 ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(self._s))
        if r != 0:
            raise MRError(r, "mr_server_create failed")
        self._problems = {}

    def _check(self, r: int, what: str):
        if r != 0:
            raise MRError(r, f"{what}: {library().mr_server_last_error(self._s).decode()}")

    def set_grid_cap(self, ctas: int):
        """at most `ctas` thread blocks per stage-kernel launch for requests
        admitted from now on (0: each launch may fill the GPU); the results
        do not depend on it"""
        self._check(library().mr_server_set_grid_cap(self._s, int(ctas)), "set_grid_cap")

    def submit(self, problem, q0, t_end: float) -> int:
        cfg = make_config(problem)
        q = np.ascontiguousarray(q0, dtype=np.float64).reshape(problem.nvars(), -1)
        rid = ctypes.c_longlong()
        self._check(library().mr_server_submit(self._s, ctypes.byref(cfg), _dptr(q), float(t_end),
                                               ctypes.byref(rid)), "submit")
        self._problems[rid.value] = problem
        return rid.value

    def advance(self):
        a, qd = ctypes.c_int(), ctypes.c_int()
        self._check(library().mr_server_advance(self._s, ctypes.byref(a), ctypes.byref(qd)), "advance")
        return a.value, qd.value

    def poll(self, cap: int = 4096) -> list:
        ids = (ctypes.c_longlong * cap)()
        n = ctypes.c_int()
        self._check(library().mr_server_poll(self._s, ids, cap, ctypes.byref(n)), "poll")
        return [ids[i] for i in range(n.value)]

    def status(self, rid: int) -> int:
        return library().mr_server_status(self._s, rid)

    def result(self, rid: int) -> "Solver":
        h = library().mr_server_result(self._s, rid)
        if not h:
            raise MRError(5, f"request {rid} is not finished")
        return Solver._view(self._problems[rid], h, self)

    def release(self, rid: int):
        self._check(library().mr_server_release(self._s, rid), "release")
        self._problems.pop(rid, None)

    def memory(self) -> int:
        return int(library().mr_server_memory(self._s))

    def close(self):
        if getattr(self, "_s", None):
            library().mr_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
