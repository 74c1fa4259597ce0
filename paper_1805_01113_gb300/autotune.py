"""Pick the spreading tile shape (brick_log2) for a workload by timing candidates.

The transfer step's cost depends on the tile shape through the spreading
kernel (markers per tile, accumulator size, halo overlap) and the sort (bin
count).  For a given grid and a device-resident marker set, each candidate
context runs build + interpolate + spread a few times; the fastest median
wins.  Results are cached per (grid shape, a hash of the face coordinates,
periodicity, marker count bucket, device name, compute capability, method,
arithmetic type, field type, basis size) for the life of the process and,
when the environment variable MLS_AUTOTUNE_CACHE names a JSON file, across
processes in that file.
"""

import hashlib
import json
import os
import statistics
import tempfile

import torch

from . import api

CANDIDATES = [(3, 3, 3), (4, 3, 3), (4, 4, 3), (4, 4, 2), (5, 3, 3), (3, 3, 2)]
CACHE_ENV = "MLS_AUTOTUNE_CACHE"
_CACHE = {}


def _device():
    return torch.cuda.get_device_name(), tuple(torch.cuda.get_device_capability())


def _faces_hash(faces):
    """16 hex digits of sha256 over the face coordinates (float64, little-endian), axis by axis."""
    import numpy as np
    d = hashlib.sha256()
    for f in faces:
        d.update(np.ascontiguousarray(np.asarray(f, dtype="<f8")).tobytes())
        d.update(b"|")
    return d.hexdigest()[:16]


def _key(faces, periodic, M, method, field, real="f32", basis=4):
    n = tuple(len(f) - 1 for f in faces)
    bucket = 1 << max(0, int(M).bit_length() - 1)
    name, cap = _device()
    return (n, _faces_hash(faces), tuple(bool(p) for p in periodic), bucket, name, cap, method, real, field,
            int(basis))


def _disk_key(k):
    return json.dumps(k)


def disk_load(path, k):
    """(best, times) stored for key k in the JSON cache file, or None."""
    try:
        with open(path) as fh:
            entry = json.load(fh).get(_disk_key(k))
    except (OSError, ValueError):
        return None
    if not entry:
        return None
    times = {tuple(int(v) for v in c.split(",")): float(ms) for c, ms in entry["times"].items()}
    return tuple(entry["best"]), times


def disk_store(path, k, best, times):
    """Add key k to the JSON cache file (read, update, write to a temporary file, rename)."""
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {}
    data[_disk_key(k)] = {"best": list(best), "times": {",".join(map(str, c)): ms for c, ms in times.items()}}
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune")
    with os.fdopen(fd, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(faces, periodic, x, area, u, F, method="exact", real="f32", field=None, reps=5, candidates=CANDIDATES,
         basis=4):
    """Return (best brick_log2, {candidate: median ms}) for build + interp + spread of these markers."""
    field = field or real
    k = _key(faces, periodic, x.shape[1], method, field, real, basis)
    if k in _CACHE:
        return _CACHE[k]
    path = os.environ.get(CACHE_ENV)
    if path:
        hit = disk_load(path, k)
        if hit is not None:
            _CACHE[k] = hit
            return hit
    M = x.shape[1]
    f = torch.zeros_like(u)
    U = torch.empty((3, M), dtype=x.dtype, device=x.device)
    times = {}
    failures = {}
    for b in candidates:
        try:
            ctx = api.Context(faces, periodic, real=real, field=field, brick_log2=b, basis=basis)
        except Exception as exc:  # a shape this grid or device cannot take; the others still compete
            failures[b] = exc
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
    if not times:
        detail = "; ".join(f"{c}: {e}" for c, e in failures.items()) or "no candidates given"
        raise RuntimeError(f"autotune: no candidate tile shape could be set up ({detail})")
    best = min(times, key=times.get)
    _CACHE[k] = (best, times)
    if path:
        disk_store(path, k, best, times)
    return best, times
