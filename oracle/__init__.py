"""ctypes wrapper of the plain FP64 C oracle (test infrastructure only).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mr_oracle.c")
_LIB = os.path.join(_HERE, "libmr_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with FMA contraction off (same bits on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mr_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
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


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        _lib.or_create.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(vp)]
        _lib.or_set_tree.argtypes = [vp, ctypes.POINTER(ctypes.c_ubyte)]
        _lib.or_adapt.argtypes = [vp]
        _lib.or_step.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)]
        _lib.or_iterate.argtypes = [vp, ctypes.c_double, ctypes.c_longlong,
                                    ctypes.POINTER(ctypes.c_longlong)]
        _lib.or_read.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t,
                                 ctypes.POINTER(ctypes.c_size_t)]
        _lib.or_destroy.argtypes = [vp]
        _lib.or_last_error.argtypes = [vp]
        _lib.or_last_error.restype = ctypes.c_char_p
        _lib.or_num_flux.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    return _lib


def _cfg(p) -> _Cfg:
    c = _Cfg()
    c.dim, c.equation, c.max_level, c.min_level = p.dim, p.equation, p.max_level, p.min_level
    c.eps, c.eps_mode, c.rk_order, c.time_mode = p.eps, p.eps_mode, p.rk_order, p.time_mode
    c.precision, c.adapt_mode, c.reflux, c.cfl = p.precision, p.adapt_mode, p.reflux, p.cfl
    for k in range(3):
        c.lo[k], c.hi[k], c.bc[k] = p.lo[k], p.hi[k], p.bc[k]
    for k in range(8):
        c.phys[k] = p.phys[k]
    c.flux = getattr(p, "flux", 0)
    return c


def num_flux(problem, k: int, W: np.ndarray, dxf: float = 1.0) -> np.ndarray:
    """The oracle's numerical flux across the face between cells 1 and 2 of
    the 4-cell stencil W[4][m] (conservative values), direction k."""
    m = problem.nvars()
    w = np.ascontiguousarray(W, dtype=np.float64).reshape(4, m)
    F = np.zeros(m)
    cfg = _cfg(problem)
    r = _load().or_num_flux(ctypes.byref(cfg), k, dxf, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if r != 0:
        raise OracleError(f"or_num_flux: status {r}")
    return F


class OracleError(RuntimeError):
    pass


class Oracle:
    """One MR/MRLT solve on the host (same calls as the CUDA library)."""

    READ_LEAF_KEYS, READ_LEAF_VALUES, READ_UNIFORM, READ_STATS, READ_FIELDS, READ_NODES = 0, 1, 2, 3, 4, 5

    def __init__(self, problem, q0: np.ndarray):
        lib = _load()
        self.p = problem
        self.m = problem.nvars()
        q = np.ascontiguousarray(q0, dtype=np.float64).reshape(self.m, -1)
        self._h = ctypes.c_void_p()
        cfg = _cfg(problem)
        r = lib.or_create(ctypes.byref(cfg), q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          ctypes.byref(self._h))
        if r != 0:
            raise OracleError(f"or_create failed with status {r}")

    def _check(self, r, what):
        if r != 0:
            msg = _load().or_last_error(self._h).decode()
            raise OracleError(f"{what}: status {r}: {msg}")

    def close(self):
        if self._h:
            _load().or_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tree(self, leaf_level_finest: np.ndarray):
        a = np.ascontiguousarray(leaf_level_finest, dtype=np.uint8).ravel()
        self._check(_load().or_set_tree(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))),
                    "set_tree")

    def adapt(self):
        self._check(_load().or_adapt(self._h), "adapt")

    def step(self, t_target: float) -> int:
        it = ctypes.c_longlong()
        self._check(_load().or_step(self._h, t_target, ctypes.byref(it)), "step")
        return it.value

    def iterate(self, dt: float, n_iters: int) -> int:
        """n fine iterations with step dt (may stop inside a macro step)."""
        it = ctypes.c_longlong()
        self._check(_load().or_iterate(self._h, dt, n_iters, ctypes.byref(it)), "iterate")
        return it.value

    def _read(self, what, dtype, shape=None):
        used = ctypes.c_size_t()
        self._check(_load().or_read(self._h, what, None, 0, ctypes.byref(used)), "read size")
        n = used.value // np.dtype(dtype).itemsize
        buf = np.empty(n, dtype=dtype)
        self._check(_load().or_read(self._h, what, buf.ctypes.data_as(ctypes.c_void_p),
                                    used.value, ctypes.byref(used)), "read")
        return buf if shape is None else buf.reshape(shape)

    def leaves(self):
        """(keys int32 [n,4] = level,i,j,k ; values float64 [n,m])"""
        k = self._read(self.READ_LEAF_KEYS, np.int32, (-1, 4))
        v = self._read(self.READ_LEAF_VALUES, np.float64, (-1, self.m))
        return k, v

    def fields(self) -> np.ndarray:
        """stored per-leaf values [n, 8, m]: q^n, q*, q**, q^{n+1},
        NERK theta=1/2, 1/4, 3/4 and the Eq. 14 extrapolation"""
        return self._read(self.READ_FIELDS, np.float64, (-1, 8, self.m))

    def nodes(self):
        """internal nodes as stored by the latest iteration: (keys int [n,4] =
        level,i,j,k ; fields float64 [n,7,m] = q^n, q*, q**, q^{n+1}, half-step
        value, theta=1/4 and theta=3/4 values)"""
        rows = self._read(self.READ_NODES, np.float64, (-1, 4 + 7 * self.m))
        return rows[:, :4].astype(np.int64), rows[:, 4:].reshape(-1, 7, self.m)

    def uniform(self) -> np.ndarray:
        n = 1 << self.p.max_level
        shape = (self.m,) + (n,) * self.p.dim
        return self._read(self.READ_UNIFORM, np.float64, shape)

    def stats(self) -> dict:
        s = self._read(self.READ_STATS, np.float64)
        L = self.p.max_level
        return {"t": s[0], "iters": int(s[1]), "macros": int(s[2]), "dt": s[3],
                "leaves": int(s[4]), "nodes": int(s[5]), "near": int(s[6]),
                "updates": int(s[7]), "pos": int(s[15]), "mass": s[8:8 + self.m].copy(),
                "leaves_per_level": s[16:17 + L].astype(np.int64)}
