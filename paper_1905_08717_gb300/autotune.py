"""Launch-shape tuning for batches of solvers.

The stage kernel's tile shapes are compile-time constants: they fix its shared
memory layout and its per-level tile lists.  What depends on the workload is
how many thread blocks one stage launch may occupy (`mr_set_grid_cap`).  A lone
large problem wants every SM for each launch.  A batch of many small problems
does better when each instance's launches take a share of the GPU, so that
launches of different instances run side by side.

`tune_batch` times a short span of the batch itself under each candidate cap
and returns the fastest.  Each cell is updated by one thread whatever the grid,
so a tuned batch computes bit for bit what the default one does.  The timings
are host wall clock around the synchronous `mr_batch_step`.
"""

from __future__ import annotations

import time


def candidate_caps(sms: int) -> list[int]:
    """Caps tried by default: 0 (the kernel's resident capacity, every SM
    for each launch), then two, one, a half and a quarter block per SM."""
    sms = max(int(sms), 1)
    caps = [0, 2 * sms, sms, sms // 2, sms // 4]
    out = []
    for c in caps:
        if (c == 0 or c >= 1) and c not in out:
            out.append(c)
    return out


def choose(seconds: dict) -> int:
    """The cap with the smallest time; on a tie the default (0) or else the
    larger cap, which needs no more of the GPU than the other instances leave."""
    if not seconds:
        raise ValueError("no timings")
    return min(seconds, key=lambda c: (seconds[c], 0 if c == 0 else 1, -c))


def tune_batch(problems, q0s, t_warm: float, t_span: float, caps=None, sms: int | None = None,
               stream=None, batch_cls=None, clock=time.perf_counter) -> dict:
    """Time the batch from t_warm to t_warm + t_span under each cap.

    A fresh batch is built for every cap and first advanced to t_warm, which
    captures its macro-step graphs and warms the caches.  Returns
    {"best": cap, "seconds": {cap: s}, "caps": [...]}.  `sms` defaults to the
    current device's multiprocessor count.  `batch_cls` and `clock` exist so
    that the selection logic can be exercised without a GPU.
    """
    if t_span <= 0.0:
        raise ValueError("t_span must be positive")
    if batch_cls is None:
        from . import Batch as batch_cls
    if caps is None:
        if sms is None:
            import torch
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        caps = candidate_caps(sms)
    seconds = {}
    for cap in caps:
        b = batch_cls(problems, q0s, stream=stream, grid_cap=cap)
        try:
            b.step(t_warm)
            t0 = clock()
            b.step(t_warm + t_span)
            seconds[cap] = clock() - t0
        finally:
            b.close()
    return {"best": choose(seconds), "seconds": seconds, "caps": list(caps)}
