"""Pick the spreading tile shape (brick_log2) for a workload by timing candidates.

The transfer step's cost depends on the tile shape through the spreading
kernel (markers per tile, accumulator size, halo overlap) and the sort (bin
count).  For a given grid and a device-resident marker set, each candidate
context runs build + interpolate + spread a few times; the fastest median
wins.  Results are cached per (grid shape, periodicity, marker count bucket,
device name, method) for the life of the process.
"""

import statistics

import torch

from . import api

CANDIDATES = [(3, 3, 3), (4, 3, 3), (4, 4, 3), (4, 4, 2), (5, 3, 3), (3, 3, 2)]
_CACHE = {}


def _key(faces, periodic, M, method, field):
    n = tuple(len(f) - 1 for f in faces)
    bucket = 1 << max(0, int(M).bit_length() - 1)
    return (n, tuple(bool(p) for p in periodic), bucket, torch.cuda.get_device_name(), method, field)


def tune(faces, periodic, x, area, u, F, method="exact", real="f32", field=None, reps=5, candidates=CANDIDATES):
    """Return (best brick_log2, {candidate: median ms}) for build + interp + spread of these markers."""
    field = field or real
    k = _key(faces, periodic, x.shape[1], method, field)
    if k in _CACHE:
        return _CACHE[k]
    M = x.shape[1]
    f = torch.zeros_like(u)
    U = torch.empty((3, M), dtype=x.dtype, device=x.device)
    times = {}
    for b in candidates:
        try:
            ctx = api.Context(faces, periodic, real=real, field=field, brick_log2=b)
        except Exception:
            continue
        T = ctx.transfer(M)
        ms = []
        for r in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.build_transfer(T, x, area, method)
            ctx.interpolate(T, u, U)
            ctx.spread(T, F, f)
            e1.record()
            torch.cuda.synchronize()
            if r >= 2:
                ms.append(e0.elapsed_time(e1))
        times[b] = statistics.median(ms)
        T.close()
        ctx.close()
    best = min(times, key=times.get)
    _CACHE[k] = (best, times)
    return best, times
