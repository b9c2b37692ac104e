"""Brute-force multiresolution tree construction on tiny inputs, used to pin
the oracle's single-pass adaptation.  Dense numpy arrays per level; the
graded closure is computed by a naive global fix-point iteration (repeat the
grading rule over all levels until nothing changes) instead of the oracle's
one fine-to-coarse pass."""
from __future__ import annotations

import itertools

import numpy as np


def project_levels(qL: np.ndarray, lb: int):
    """qL: (m, n, ...) finest averages -> dict level -> (m, n_l, ...) means (Eq. 3)."""
    d = qL.ndim - 1
    L = int(np.log2(qL.shape[1]))
    out = {L: qL}
    q = qL
    for l in range(L - 1, lb - 1, -1):
        s = q
        for ax in range(1, d + 1):
            sh = list(s.shape)
            sh[ax] //= 2
            sh.insert(ax + 1, 2)
            s = s.reshape(sh).mean(axis=ax + 1)
        out[l] = s
        q = s
    return out


def _ghost_index(i, n, periodic):
    if periodic:
        return i % n
    while i < 0 or i >= n:
        if i < 0:
            i = -1 - i
        if i >= n:
            i = 2 * n - 1 - i
    return i


def predict_children(qp: np.ndarray, periodic: bool) -> np.ndarray:
    """Tensor-product quadratic prediction (Eq. 4) of level l+1 from level l,
    for every cell: axis by axis, child a=0 gets c - (q+ - q-)/8, a=1 c + (...)/8.
    Array layout [var, ... spatial axes with x last] (numpy [var, z, y, x])."""
    d = qp.ndim - 1
    q = qp
    for ax in range(1, d + 1):
        n = q.shape[ax]
        idx_m = [_ghost_index(i - 1, n, periodic) for i in range(n)]
        idx_p = [_ghost_index(i + 1, n, periodic) for i in range(n)]
        qm = np.take(q, idx_m, axis=ax)
        qpl = np.take(q, idx_p, axis=ax)
        c0 = q - (qpl - qm) / 8.0
        c1 = q + (qpl - qm) / 8.0
        st = np.stack([c0, c1], axis=ax + 1)
        sh = list(q.shape)
        sh[ax] *= 2
        q = st.reshape(sh)
    return q


def brute_force_tree(qL, lb, eps, eps_mode, periodic):
    """Leaf set {(level, idx tuple in numpy axis order)} of the adapted tree."""
    d = qL.ndim - 1
    L = int(np.log2(qL.shape[1]))
    lv = project_levels(qL, lb)
    scale = np.maximum(np.abs(qL).reshape(qL.shape[0], -1).max(axis=1), 1e-14)
    R = {l: np.zeros((1 << l,) * d, bool) for l in range(lb, L)}

    def epsl(l):
        return eps * 2.0 ** (d * (l - L)) if eps_mode == 1 else eps

    sig, big = {}, {}
    for l in range(lb, L):
        pred = predict_children(lv[l], periodic)
        det = np.abs(lv[l + 1] - pred) / scale.reshape((-1,) + (1,) * d)
        det = det.max(axis=0)
        # max over the 2^d children of each node
        for ax in range(d):
            sh = list(det.shape)
            sh[ax] //= 2
            sh.insert(ax + 1, 2)
            det = det.reshape(sh).max(axis=ax + 1)
        sig[l] = det > epsl(l + 1)
        big[l] = det > 8 * epsl(l + 1)
    offs = list(itertools.product((-1, 0, 1), repeat=d))

    def neigh(l, idx):
        n = 1 << l
        for o in offs:
            j = []
            ok = True
            for a, b in zip(idx, o):
                t = a + b
                if periodic:
                    t %= n
                elif t < 0 or t >= n:
                    ok = False
                    break
                j.append(t)
            if ok:
                yield tuple(j)

    for l in range(lb, L):
        for idx in zip(*np.nonzero(sig[l])):
            for j in neigh(l, idx):
                R[l][j] = True
            if big[l][idx] and l + 1 < L:
                for t in itertools.product((0, 1), repeat=d):
                    R[l + 1][tuple(2 * a + b for a, b in zip(idx, t))] = True
    changed = True
    while changed:  # naive global fix-point of the grading rule
        changed = False
        for l in range(lb + 1, L):
            for idx in zip(*np.nonzero(R[l])):
                par = tuple(a >> 1 for a in idx)
                for j in neigh(l - 1, par):
                    if not R[l - 1][j]:
                        R[l - 1][j] = True
                        changed = True
    leaves = set()
    for l in range(lb, L + 1):
        n = 1 << l
        for idx in itertools.product(range(n), repeat=d):
            exists = l == lb or R[l - 1][tuple(a >> 1 for a in idx)]
            refined = l < L and R[l][idx]
            if exists and not refined:
                leaves.add((l, idx))
    return leaves


def keys_to_set(keys: np.ndarray, d: int):
    """oracle/CUDA leaf keys (level, i, j, k with i = x) -> set in numpy axis order."""
    out = set()
    for l, i, j, k in keys:
        c = (i, j, k)[:d]
        out.add((int(l), tuple(int(x) for x in reversed(c))))
    return out
