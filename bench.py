"""Benchmark: markers/s of one MLS transfer step (marker prep + build + interpolate + spread).

Default workload: 2000 ellipsoids of 1280 markers each (2.56 M markers) in a
uniform periodic 512^3 grid, single precision, exact-MLS (the fast-MLS step
is timed alongside and reported under "fast").  Inputs are synthetic and
resident in HBM before timing; L2 is flushed (256 MiB write) between timed
steps, outside the timed events.  Each step is replayed from a CUDA graph
captured once (--no-graph: plain stream-ordered calls; both are reported).
One JSON line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c2|c3|c1] [--method exact|fast]

With N > 1 (torchrun) every rank runs its own copy of the workload on its
GPU (independent bodies, no data-path collective: weak scaling); value is
the markers of all ranks over the slowest rank's time.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "markers/s (build+interp+spread) and HBM roofline fraction at stated err vs FP64"
WORKLOAD_TEXT = {
    "c1": "1 level-4 icosphere (5120 markers), R=0.25, periodic 64^3 grid, float64",
    "c2": "2000 ellipsoids x 1280 markers (2.56M), periodic uniform 512^3 grid, float32",
    "c3": "10^4 deformed icospheres (50/50 1280/5120 markers, 32M), 1024^3 grid tanh-stretched in z, float32",
}

# Algorithmic bytes per marker of each kernel (float32 path; u_cells = distinct
# touched cells per marker, measured): the bytes the method must move at least,
# counted as in the hot-path scope table: the marker's position and area, its
# 27 shape-function values, its home-cell index and c_l, its force or
# velocity, and the touched field cells.  The tile-order permutation (4 bytes
# per marker that the build, interpolation and spreading also read) is this
# implementation's layout, not the method's, and is not counted.
def algorithmic_bytes(kernel, rs, u_cells, verts_per_marker):
    return {
        "marker_prep": 12 + 3 * rs * verts_per_marker + 4 * rs,
        # the preparation with the locate pass fused in: the markers are formed,
        # stored and located without being read back; tile key and rank written
        "prep_locate": 12 + 3 * rs * verts_per_marker + 4 * rs + 8,
        "locate": 3 * rs + 8,
        "scatter": 12,
        "build_exact": 4 * rs + 27 * rs + rs + 4,
        "build_fast": 4 * rs + 27 * rs + rs + 4,
        "build_surrogate": 4 * rs + 27 * rs + rs + 4,
        "interp": 27 * rs + 4 + 3 * rs * u_cells + 3 * rs,
        # the build's bytes plus the touched u read and U written (phi is not read back)
        "build_exact_interp": 4 * rs + 27 * rs + rs + 4 + 3 * rs * u_cells + 3 * rs,
        "spread": 27 * rs + rs + 4 + 3 * rs + 6 * rs * u_cells,
        # phi, c, home, V_b in, F and U out, touched u read, touched f read-modify-write
        "direct_forcing": 27 * rs + rs + 4 + 3 * rs + 3 * rs + 3 * rs + 3 * rs * u_cells + 6 * rs * u_cells,
    }.get(kernel)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c3", choices=["c1", "c2", "c3"])
    p.add_argument("--method", default="exact", choices=["exact", "fast"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--sample-bodies", type=int, default=160, help="bodies in the CPU oracle sample")
    p.add_argument("--grid", type=int, default=None, help="cells per axis (smaller profiling cases)")
    p.add_argument("--bodies", type=int, default=None, help="number of bodies (smaller profiling cases)")
    p.add_argument("--graph", action="store_true", help="replay each step from a captured CUDA graph (the default)")
    p.add_argument("--no-graph", action="store_true", help="issue every step as plain stream-ordered calls")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--tiles", default=None, help="spreading tile log2 sizes, e.g. 3,3,2 (skips the autotuner)")
    p.add_argument("--no-surrogate", action="store_true")
    p.add_argument("--surrogate-epochs", type=int, default=128,
                   help="training epochs of 2^20 samples (128, the default schedule; fewer for profiling runs)")
    p.add_argument("--residual-max", type=float, default=1e-4,
                   help="the surrogate's gate threshold for the timed surrogate step")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world, device):
    """The largest `value` over all ranks (every rank gets it); identity for one rank."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(markers_per_rank, world, steps, slowest_ms):
    """Whole-job markers/s: the markers all ranks processed over the slowest rank's time."""
    return world * markers_per_rank * steps / (slowest_ms / 1e3)


def workload(name, grid=None, bodies=None):
    from workloads import make_workload
    kw = {}
    if grid is not None:
        kw["n"] = grid
    if bodies is not None and name != "c1":
        kw["n_bodies"] = bodies
    return make_workload(name, **kw)


# ---------------------------------------------------------------- CPU oracle leg
ORACLE_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, os.environ["MLS_ROOT"])
import numpy as np
import oracle
from workloads import make_workload
from workloads.fields import field_at_cells_np
args = json.loads(sys.argv[1])
w = make_workload(args["workload"], **args["kw"])
g = oracle.Grid(w.faces, w.periodic)
b0, b1 = args["bodies"]
f0, f1 = int(w.body_faces[b0]), int(w.body_faces[b1])
tri = w.tri[f0:f1]
real = w.real
V = w.vertices.astype(np.float32 if real == "f32" else np.float64)
F = w.forces()[:, f0:f1].astype(V.dtype)
times = []
for rep in range(args["reps"]):
    t0 = time.perf_counter()
    x, area = oracle.marker_prep(V, tri, real)
    tr = oracle.shape_exact(g, x, 1.0) if args["method"] == "exact" else oracle.shape_fast(g, x, 1.0, 9)
    c = oracle.forcing_scale(tr, area)
    ix, iy, iz = tr.sup.idx
    usup = field_at_cells_np(w.modes, w.faces, ix.ravel(), iy.ravel(), iz.ravel()).reshape((3,) + ix.shape)
    U = np.einsum("mk,cmk->cm", tr.phi, usup)
    sp = oracle.spread(tr, c, F, g.n)
    times.append(time.perf_counter() - t0)
out = {"phi": tr.phi, "U": U, "c": c, "fk": sp.keys, "fv": sp.values}
if args.get("grad"):
    # velocity gradient at the markers (exact-MLS shape-function derivatives)
    dphi = oracle.shape_exact_gradient(g, x, 1.0)
    out["G"] = np.einsum("mdk,cmk->cdm", dphi, usup)
if args.get("dt"):
    # direct forcing with V_b = 0 (bodies at rest): F = (V_b - U)/dt, spread on the same support
    F_df = (0.0 - U) / args["dt"]
    out["F_df"] = F_df
    out["fv_df"] = oracle.spread(tr, c, F_df, g.n).values
if args.get("fast_too") and args["method"] == "exact":
    out["phi_fast"] = oracle.shape_fast(g, x, 1.0, 9).phi
np.savez(args["out"], **out)
print(json.dumps({"markers": int(f1 - f0), "times": times}))
"""


def run_oracle_sample(name, method, bodies, reps, out, kw=None, fast_too=False, dt=None, grad=False):
    env = dict(os.environ)
    env["MLS_ROOT"] = ROOT
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    args = json.dumps({"workload": name, "method": method, "bodies": bodies, "reps": reps, "out": out,
                       "kw": kw or {}, "fast_too": fast_too, "dt": dt, "grad": grad})
    r = subprocess.run([sys.executable, "-c", ORACLE_CHILD, args], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle leg failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_all_cores(name, method, bodies_each, kw=None, return_sample=False):
    """The same oracle, unchanged, in one process per host core at once, each on
    its own bodies_each-body sample of the workload (distinct ranges, wrapping
    around the workload): aggregate markers over the slowest process's compute
    time.  Returns (markers/s, processes) or None when the workload has fewer
    bodies than one sample."""
    from workloads import make_workload
    n_bodies = len(make_workload(name, **(kw or {})).body_faces) - 1
    if n_bodies < bodies_each:
        return None
    procs = max(1, os.cpu_count() or 1)
    env = dict(os.environ)
    env["MLS_ROOT"] = ROOT
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    with tempfile.TemporaryDirectory() as td:
        children = []
        for q in range(procs):
            b0 = (q * bodies_each) % (n_bodies - bodies_each + 1)
            args = json.dumps({"workload": name, "method": method, "bodies": [b0, b0 + bodies_each], "reps": 1,
                               "out": os.path.join(td, f"p{q}.npz"), "kw": kw or {}})
            children.append(subprocess.Popen([sys.executable, "-c", ORACLE_CHILD, args], stdout=subprocess.PIPE,
                                             stderr=subprocess.PIPE, text=True, env=env))
        results = []
        for ch in children:
            out, err = ch.communicate()
            if ch.returncode != 0:
                raise RuntimeError("oracle leg failed: " + err[-2000:])
            results.append(json.loads(out.strip().splitlines()[-1]))
    markers = sum(r["markers"] for r in results)
    slowest = max(r["times"][0] for r in results)
    if return_sample:
        return markers / slowest, procs, markers, slowest
    return markers / slowest, procs


def _errs(got, ref):
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(float(np.max(np.abs(ref))), 1e-300)
    return {"max_rel": float(np.max(np.abs(got - ref)) / scale),
            "rms_rel": float(np.sqrt(np.mean((got - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [v.strip() for v in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel on this
    workload (default sizes), if the kernel's sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(p))
    except Exception:
        return None
    ent = data.get(kernel, {}).get(workload)
    if not ent:
        return None
    h = source_sha(ent["source"])
    return ent["bytes_per_launch"] if h is not None and h == ent["source_sha"] else None


def source_sha(files):
    """sha256 (16 hex digits) of the named csrc files, concatenated in the order given."""
    if isinstance(files, str):
        files = [files]
    d = hashlib.sha256()
    try:
        for name in files:
            d.update(open(os.path.join(ROOT, "paper_1805_01113_gb300", "csrc", name), "rb").read())
    except OSError:
        return None
    return d.hexdigest()[:16]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- our arm
def run_ours(a, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1805_01113_gb300 import build_ext
    build_ext.build()
    from paper_1805_01113_gb300 import api, autotune
    from workloads.fields import field_full_torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(a.workload, a.grid, a.bodies)
    real = w.real
    tdt = torch.float32 if real == "f32" else torch.float64
    ndt = np.float32 if real == "f32" else np.float64
    rs = 4 if real == "f32" else 8
    M = w.n_markers
    V_host = torch.as_tensor(w.vertices.astype(ndt)).pin_memory()
    F_host = torch.as_tensor(w.forces().astype(ndt)).pin_memory()
    V = V_host.to(dev)
    tri = torch.as_tensor(w.tri, device=dev)
    F = F_host.to(dev)
    u = field_full_torch(w.modes, w.faces, tdt, dev)
    f = torch.zeros_like(u)
    x = torch.empty((3, M), dtype=tdt, device=dev)
    area = torch.empty((M,), dtype=tdt, device=dev)
    U = torch.empty((3, M), dtype=tdt, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # Spreading tile shape: autotuned on this workload (exact-MLS step), else 8x8x8.
    tiles, tune_ms = (3, 3, 3), None
    api.Context(w.faces, w.periodic, real=real).marker_prep(V, tri, x, area)
    if a.tiles:
        tiles = tuple(int(t) for t in a.tiles.split(","))
    elif not a.no_autotune:
        tiles, tune_ms = autotune.tune(w.faces, w.periodic, x, area, u, F, "exact", real)
    ctx = api.Context(w.faces, w.periodic, real=real, brick_log2=tiles, residual_max=a.residual_max)
    T = ctx.transfer(M)
    ctx.fast_table()
    methods = ["exact", "fast"]
    train = None
    if real == "f32" and not a.no_surrogate:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = ctx.train_surrogate(epochs=a.surrogate_epochs)
        train = {"seconds": time.perf_counter() - t0, "final_loss": loss}
        methods.append("surrogate")

    # Direct forcing (interp -> F = (V_b - U)/dt -> spread, fused): bodies at rest, V_b = 0.
    DT = 1e-3
    Vb0 = torch.zeros((3, M), dtype=tdt, device=dev)
    F_df = torch.empty((3, M), dtype=tdt, device=dev)

    def step(method):
        ctx.marker_prep(V, tri, x, area)
        if method == "direct_forcing":
            ctx.build_transfer(T, x, area, "exact")
            ctx.direct_forcing(T, u, Vb0, DT, f, F=F_df, U=U)
            return
        if method == "build_direct_forcing":
            ctx.build_direct_forcing(T, x, area, u, Vb0, DT, f, F=F_df, U=U, method="exact")
            return
        if method == "exact":
            # the exact step through the build call with the interpolation fused in
            ctx.build_interpolate(T, x, area, u, U, method="exact")
            ctx.spread(T, F, f)
            return
        if method == "exact_separate":
            ctx.build_transfer(T, x, area, "exact")
            ctx.interpolate(T, u, U)
        else:
            # exact: the interpolation inside the build kernel; fast-MLS and the surrogate: the two calls in turn
            ctx.build_interpolate(T, x, area, u, U, method=method)
        ctx.spread(T, F, f)

    # distinct touched cells per marker (u_cells) from one spread into a zero field
    step(a.method)
    st = ctx.status(T)
    if st["dropped"]:
        raise RuntimeError(f"{st['dropped']} markers dropped")
    f.zero_()
    ctx.spread(T, F, f)
    touched = int(torch.count_nonzero(f[0]).item())
    u_cells = touched / M

    # A step is replayed from a CUDA graph captured once per method (the
    # library's calls are stream-ordered and allocate nothing in a step), as a
    # solver that captures its time step would run it; --no-graph issues the
    # calls one by one.  A failed capture falls back to plain calls.
    graphs = {}
    graph_state = {"use": not a.no_graph, "error": None}

    def run_step(method):
        if graph_state["use"] and method not in graphs:
            try:
                for _ in range(2):
                    step(method)
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    step(method)
                graphs[method] = g
            except Exception as ex:  # reported in config; the plain calls below still run the step
                graph_state["use"], graph_state["error"] = False, str(ex)[:200]
                torch.cuda.synchronize()
        if graph_state["use"]:
            graphs[method].replay()
        else:
            step(method)

    def timed(method, steps, warmup, per_kernel, min_warm_s=0.0, plain=False):
        # At least `warmup` untimed steps, and at least min_warm_s of load so the
        # clock sampler sees the GPU busy around the timed region.
        t0 = time.perf_counter()
        done = 0
        direct = per_kernel or plain
        while done < warmup or time.perf_counter() - t0 < min_warm_s:
            step(method) if direct else run_step(method)
            done += 1
            if done % 16 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        if per_kernel:
            ctx.read_timing()
            ctx.timing(True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            step(method) if direct else run_step(method)
            e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        kt = ctx.read_timing() if per_kernel else {}
        ctx.timing(False)
        return ms, kt

    # headline: plain timed region (no per-kernel events), clocks sampled during it
    clk = ClockSampler(local)
    clk.start()
    ms, _ = timed(a.method, a.steps, a.warmup, False, min_warm_s=1.5)
    clocks = clk.stop()
    total_ms = max_over_ranks(sum(ms), world, dev)
    value = job_throughput(M, world, a.steps, total_ms)
    # the same step issued as plain stream-ordered calls (reported beside the headline)
    stream_calls = None
    if graph_state["use"]:
        ms_p, _ = timed(a.method, a.steps, 3, False, plain=True)
        tp = max_over_ranks(sum(ms_p), world, dev)
        stream_calls = {"value": job_throughput(M, world, a.steps, tp), "ms_per_step": tp / a.steps}

    # per-kernel pass (events around each kernel on the launching stream)
    ms_k, kt = timed(a.method, a.steps, 2, True)
    # kernels per timed phase: the exact builds also launch their double re-solve kernel
    per_phase = {"build_exact": 2, "build_exact_interp": 2, "build_exact_forcing": 2}
    launches = sum(n * per_phase.get(k, 1) for k, (n, _) in kt.items() if k != "bin_reset")
    per_launch = {k: tot / n for k, (n, tot) in kt.items() if n}
    dom = max((k for k in per_launch if k != "bin_reset"), key=lambda k: kt[k][1])
    pk, pk_src = peaks()
    vpm = len(w.vertices) / M
    byts = {k: algorithmic_bytes(k, rs, u_cells, vpm) for k in per_launch}
    ach = byts[dom] * M / (per_launch[dom] / 1e3) / 1e9 if byts.get(dom) else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": (ach / pk["hbm_gbs"]) if ach else None, "peak_source": pk_src,
            "algorithmic_bytes_per_launch": byts[dom] * M if byts.get(dom) else None,
            "traffic": traffic_for(dom, a.workload) if a.grid is None and a.bodies is None else None}
    kernels = {k: {"ms_per_launch": round(per_launch[k], 5), "launches_per_step": kt[k][0] / a.steps,
                   "gbs": (round(byts[k] * M / (per_launch[k] / 1e3) / 1e9, 1) if byts.get(k) else None)}
               for k in per_launch}

    # the other methods, same workload (reported, not the headline)
    others = {}
    for mth in methods:
        if mth == a.method:
            continue
        ms_o, _ = timed(mth, max(3, a.steps // 2), 3, False)
        _, kt_o = timed(mth, 3, 1, True)
        bname = next((b for b in ("build_" + mth + "_interp", "build_" + mth) if b in kt_o), None)
        others[mth] = {"value": M * world / (statistics.mean(ms_o) / 1e3), "ms_per_step": statistics.mean(ms_o),
                       "build_kernel": bname,
                       "build_ms": (kt_o[bname][1] / kt_o[bname][0]) if bname else None}
    # fused direct-forcing step: prep + exact build + one fused transfer pass
    ms_d, _ = timed("direct_forcing", max(3, a.steps // 2), 3, False)
    _, kt_d = timed("direct_forcing", 3, 1, True)
    kd = kt_d["direct_forcing"][1] / kt_d["direct_forcing"][0]
    bd = algorithmic_bytes("direct_forcing", rs, u_cells, vpm) * M
    others["direct_forcing"] = {
        "value": M * world / (statistics.mean(ms_d) / 1e3), "ms_per_step": statistics.mean(ms_d),
        "step": "marker_prep + build_transfer (exact) + direct_forcing (V_b = 0, dt = 1e-3)",
        "kernel_ms": kd, "algorithmic_bytes_per_launch": bd, "achieved_gbs": bd / (kd / 1e3) / 1e9,
        "frac": bd / (kd / 1e3) / 1e9 / pk["hbm_gbs"],
        "separate_interp_spread_ms": per_launch.get("interp", 0.0) + per_launch.get("spread", 0.0)}
    # the same immersed-boundary step through one call: the build kernel also interpolates and forms F
    ms_bd, _ = timed("build_direct_forcing", max(3, a.steps // 2), 3, False)
    _, kt_bd = timed("build_direct_forcing", 3, 1, True)
    others["build_direct_forcing"] = {
        "value": M * world / (statistics.mean(ms_bd) / 1e3), "ms_per_step": statistics.mean(ms_bd),
        "step": "marker_prep + build_direct_forcing (exact; U and F = (V_b - U)/dt in the build kernel, then spread)",
        "kernels_ms": {k: round(n_t[1] / n_t[0], 5) for k, n_t in kt_bd.items() if n_t[0]}}
    # the same exact step as three separate calls (build_transfer, interpolate, spread)
    if a.method == "exact":
        ms_b, _ = timed("exact_separate", max(3, a.steps // 2), 3, False)
        _, kt_b = timed("exact_separate", 3, 1, True)
        kb = {k: n_t[1] / n_t[0] for k, n_t in kt_b.items() if n_t[0]}
        others["exact_separate"] = {
            "value": M * world / (statistics.mean(ms_b) / 1e3), "ms_per_step": statistics.mean(ms_b),
            "step": "marker_prep + build_transfer (exact) + interpolate + spread",
            "build_ms": kb.get("build_exact"), "interp_ms": kb.get("interp"),
            "fused_build_interp_ms": per_launch.get("build_exact_interp")}
    # velocity gradient at the markers from the exact-MLS shape-function derivatives
    step(a.method)
    Gt = torch.empty((3, 3, M), dtype=tdt, device=dev)
    for _ in range(3):
        ctx.interpolate_gradient(T, x, u, Gt)
    torch.cuda.synchronize()
    ctx.read_timing()
    ctx.timing(True)
    for _ in range(5):
        flush.fill_(1.0)
        ctx.interpolate_gradient(T, x, u, Gt)
    torch.cuda.synchronize()
    kg = ctx.read_timing()["interp_gradient"]
    ctx.timing(False)
    kgm = kg[1] / kg[0]
    # x, home, perm, 27 gathered u cells x 3 components (touched cells), G out
    bg = (3 * rs + 8 + 3 * rs * u_cells + 9 * rs) * M
    others["interp_gradient"] = {"kernel_ms": kgm, "markers_per_s": M * world / (kgm / 1e3),
                                 "algorithmic_bytes_per_launch": bg, "achieved_gbs": bg / (kgm / 1e3) / 1e9,
                                 "step": "mls_interpolate_gradient on the exact build (9 gradient components)"}

    # coarse collision detection on the home cells of the exact build (one body index per ellipsoid)
    step(a.method)
    bf = np.asarray(w.body_faces)
    body_t = torch.as_tensor(np.repeat(np.arange(1, len(bf), dtype=np.int32), np.diff(bf)), device=dev)
    flag_t = torch.empty((M,), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(3):
        ctx.collisions(T, body_t, flag_t)
    torch.cuda.synchronize()
    ctx.read_timing()
    ctx.timing(True)
    for _ in range(5):
        flush.fill_(1.0)
        ctx.collisions(T, body_t, flag_t)
    ctx.collisions(T, body_t, flag_t, count=cnt)
    torch.cuda.synchronize()
    kc = ctx.read_timing()["collisions"]
    ctx.timing(False)
    kcm = kc[1] / kc[0]
    others["collisions"] = {"kernel_ms": kcm, "markers_per_s": M * world / (kcm / 1e3),
                            "colliding_markers": int(cnt.item()),
                            "step": "mls_collisions on the exact build's home cells, body index per ellipsoid"}
    # adaptive Lagrangian refinement of the same bodies (target element 0.8 h), then
    # the transfer step on the refined markers
    tri_t = tri
    for _ in range(2):
        xr, ar, pr, lv = ctx.refine_markers(V, tri_t, ratio=0.8)
    ctx.read_timing()
    ctx.timing(True)
    for _ in range(3):
        flush.fill_(1.0)
        xr, ar, pr, lv = ctx.refine_markers(V, tri_t, ratio=0.8)
    kr = ctx.read_timing()["refine"]
    ctx.timing(False)
    Kr = xr.shape[1]
    Tr = ctx.transfer(Kr)
    Fr = torch.randn((3, Kr), dtype=tdt, device=dev)
    Ur = torch.empty((3, Kr), dtype=tdt, device=dev)

    def refined_step():
        ctx.build_transfer(Tr, xr, ar, "exact")
        ctx.interpolate(Tr, u, Ur)
        ctx.spread(Tr, Fr, f)

    for _ in range(3):
        refined_step()
    torch.cuda.synchronize()
    evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for e0, e1 in evr:
        flush.fill_(1.0)
        e0.record(stream)
        refined_step()
        e1.record(stream)
    torch.cuda.synchronize()
    msr = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evr)
    others["refinement"] = {"base_markers": M, "refined_markers": Kr,
                            "levels": torch.bincount(lv.long(), minlength=4).tolist(),
                            "refine_ms": kr[1] / kr[0], "transfer_ms": msr,
                            "refined_markers_per_s": Kr * world / (msr / 1e3),
                            "step": "mls_refine_markers (ratio 0.8, max level 3) timed alone; build (exact) + "
                                    "interp + spread on the refined markers"}
    Tr.close()
    # exact build with the quadratic basis (m = 10) on the same markers; an
    # optional extension, so a failure here is reported and does not end the run
    try:
        cq = api.Context(w.faces, w.periodic, real=real, brick_log2=tiles, basis=10)
        Tq = cq.transfer(M)
        for _ in range(3):
            cq.build_transfer(Tq, x, area, "exact")
        torch.cuda.synchronize()
        cq.timing(True)
        for _ in range(5):
            flush.fill_(1.0)
            cq.build_transfer(Tq, x, area, "exact")
        torch.cuda.synchronize()
        kq = cq.read_timing()
        cq.timing(False)
        bq = kq["build_exact"][1] / kq["build_exact"][0]
        others["exact_quadratic"] = {
            "build_ms": bq, "markers_per_s": M * world / (bq / 1e3),
            "linear_build_ms": per_launch.get("build_exact"),
            "fp64_resolves": cq.status(Tq)["refined_fp64"],
            "step": "mls_build_transfer (exact, basis m = 10): build kernels alone, events on the stream"}
        Tq.close()
        cq.close()
    except Exception as exc:  # noqa: BLE001 - recorded in the output line
        others["exact_quadratic"] = {"error": str(exc)}
    if "surrogate" in others:
        step("surrogate")
        others["surrogate"]["fallback_rate"] = ctx.status(T)["surrogate_fallback"] / M
        others["surrogate"]["training"] = train

    # end to end through the public API with host buffers: H2D of the step's
    # vertices and forces from pinned memory, D2H of the marker velocities
    e2e = None
    if not a.no_e2e:
        U_host = torch.empty((3, M), dtype=tdt).pin_memory()
        # The library's calls are stream-ordered, so the copies overlap the
        # kernels that do not need them.  The vertices go up on a copy stream
        # in pieces of whole bodies, and each piece's markers are formed and
        # located as soon as it lands (mls_marker_prep_locate) while the next
        # piece is copied; F follows on the copy stream while the build and
        # interpolation run, and U comes down on it while the spread runs.
        cstream = torch.cuda.Stream(device=dev)
        ev_f, ev_u = torch.cuda.Event(), torch.cuda.Event()
        n_pieces = 8
        bf = np.asarray(w.body_faces)
        cut_b = sorted({int(np.searchsorted(bf, M * q // n_pieces)) for q in range(1, n_pieces)} | {len(bf) - 1})
        pieces, t0, v0 = [], 0, 0
        for b in cut_b:
            t1 = int(bf[min(b, len(bf) - 1)])
            if t1 <= t0:
                continue
            v1 = int(w.tri[:t1].max()) + 1
            pieces.append((t0, t1, v0, max(v0, v1)))
            t0, v0 = t1, max(v0, v1)
        if v0 < V.shape[0]:                                 # vertices no triangle refers to
            t_last, _, v_last, _ = pieces[-1]
            pieces[-1] = (t_last, M, v_last, V.shape[0])
        ev_v = [torch.cuda.Event() for _ in pieces]

        def e2e_step():
            stream = torch.cuda.current_stream()       # the capture stream while a graph is captured
            cstream.wait_stream(stream)
            with torch.cuda.stream(cstream):
                for (_, _, v0, v1), ev in zip(pieces, ev_v):
                    V[v0:v1].copy_(V_host[v0:v1], non_blocking=True)
                    ev.record(cstream)
                F.copy_(F_host, non_blocking=True)
                ev_f.record(cstream)
            for (t0, t1, _, _), ev in zip(pieces, ev_v):
                stream.wait_event(ev)
                ctx.marker_prep_locate(T, V, tri, x, area, begin=t0, end=t1)
            if a.method == "exact":
                ctx.build_interpolate(T, x, area, u, U, method="exact")
            else:
                ctx.build_transfer(T, x, area, a.method)
                ctx.interpolate(T, u, U)
            ev_u.record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(ev_u)
                U_host.copy_(U, non_blocking=True)
            stream.wait_event(ev_f)
            ctx.spread(T, F, f)
            stream.wait_stream(cstream)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        te = []
        for _ in range(a.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            te.append(time.perf_counter() - t0)
        # Host-timed steps: one host stall in K steps moves the mean a lot, so the
        # value is the median step (the mean and the fastest step are reported too).
        e2e = {"value": M * world / statistics.median(te), "unit": "markers/s", "statistic": "median of the K steps",
               "h2d_bytes_per_step": V_host.numel() * V_host.element_size() + F_host.numel() * F_host.element_size(),
               "d2h_bytes_per_step": U_host.numel() * U_host.element_size(),
               "ms_per_step": 1e3 * statistics.mean(te),
               "ms_per_step_median": 1e3 * statistics.median(te), "ms_per_step_min": 1e3 * min(te),
               "copies": f"pinned host buffers; vertices up on a copy stream in {len(pieces)} pieces of whole "
                         "bodies, each piece's markers formed and located as it lands; forces up after them "
                         "during build and interpolation, marker velocities down on the copy stream during "
                         "the spread"}
        # The same step (copies included) captured once into a CUDA graph and
        # replayed: what a caller that captures its time step gets.
        try:
            ge = torch.cuda.CUDAGraph()
            with torch.cuda.graph(ge):
                e2e_step()
            for _ in range(3):
                ge.replay()
            torch.cuda.synchronize()
            tg = []
            for _ in range(a.steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ge.replay()
                torch.cuda.synchronize()
                tg.append(time.perf_counter() - t0)
            e2e["graph"] = {"value": M * world / statistics.median(tg), "ms_per_step": 1e3 * statistics.mean(tg),
                            "ms_per_step_median": 1e3 * statistics.median(tg), "ms_per_step_min": 1e3 * min(tg)}
        except Exception as ex:  # reported, not fatal: the plain figure above stands
            e2e["graph"] = {"error": str(ex)[:200]}
        # Like the device-resident headline, the end-to-end value is the graph
        # replay when steps are replayed from graphs; the plain calls stay beside it.
        if graph_state["use"] and "value" in e2e["graph"]:
            g_ = e2e.pop("graph")
            keys = ("value", "ms_per_step", "ms_per_step_median", "ms_per_step_min")
            e2e["stream_calls"] = {k: e2e[k] for k in keys}
            e2e.update({k: g_[k] for k in keys})
            e2e["mode"] = "step (copies included) replayed from a CUDA graph captured once"
        else:
            e2e["mode"] = "stream-ordered calls"

    # CPU oracle on a bounded sample (rank 0, N = 1 only): its timing, and the
    # error of every method and precision mode against it on that sample.
    cpu, precision = None, None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        nb = min(a.sample_bodies, len(w.body_faces) - 1)
        ks = int(w.body_faces[nb])
        xs, as_, Fs = x[:, :ks].contiguous(), area[:ks].contiguous(), F[:, :ks].contiguous()
        with tempfile.TemporaryDirectory() as td:
            out = os.path.join(td, "s.npz")
            kw = {k: v for k, v in (("n", a.grid), ("n_bodies", a.bodies)) if v is not None}
            r = run_oracle_sample(a.workload, "exact", [0, nb], 1, out, kw, fast_too=True, dt=DT, grad=True)
            ref = dict(np.load(out))
        fk = torch.as_tensor(ref["fk"], device=dev)

        def sample_outputs(c, method, field_t):
            Ts = c.transfer(ks)
            c.build_transfer(Ts, xs, as_, method)
            uu = u.to(field_t)
            Us = c.interpolate(Ts, uu)
            fs = torch.zeros_like(uu)
            c.spread(Ts, Fs, fs)
            v = c.view(Ts)
            inv = torch.empty(ks, dtype=torch.long, device=dev)
            inv[v["perm"].long()] = torch.arange(ks, device=dev)
            phi = v["phi"][:, inv].double().cpu().numpy().T
            fv = fs.reshape(3, -1)[:, fk].double().cpu().numpy()
            nf = int(torch.count_nonzero(fs.reshape(3, -1)).item())
            out = {"phi": phi, "U": Us.double().cpu().numpy(), "f": fv, "f_nonzero_outside": nf - int(
                np.count_nonzero(fv))}
            Ts.close()
            return out

        errs = {}
        for mth in methods:
            o = sample_outputs(ctx, mth, tdt)
            errs[mth] = {"phi_vs_exact": _errs(o["phi"], ref["phi"]), "U": _errs(o["U"], ref["U"]),
                         "f": _errs(o["f"], ref["fv"])}
            if mth == "fast":
                errs[mth]["phi_vs_oracle_fast"] = _errs(o["phi"], ref["phi_fast"])
        Ts = ctx.transfer(ks)
        ctx.build_transfer(Ts, xs, as_, "exact")
        fs = torch.zeros_like(u)
        F_dfs, _ = ctx.direct_forcing(Ts, u, torch.zeros((3, ks), dtype=tdt, device=dev), DT, fs)
        errs["direct_forcing"] = {"F": _errs(F_dfs.double().cpu().numpy(), ref["F_df"]),
                                  "f": _errs(fs.reshape(3, -1)[:, fk].double().cpu().numpy(), ref["fv_df"])}
        Gs = ctx.interpolate_gradient(Ts, xs, u)
        errs["interp_gradient"] = {"G": _errs(Gs.double().cpu().numpy(), ref["G"])}
        Ts.close()
        cpu = {"value": r["markers"] / min(r["times"]), "unit": "markers/s", "cores": 1, "kind": "oracle",
               "sample": f"first {nb} bodies ({r['markers']} markers) of the same workload, prep+exact build"
                         f"+interp+spread, numpy float64, single thread",
               "err_vs_fp64_oracle": errs}
        allc = run_oracle_all_cores(a.workload, "exact", nb, kw)
        if allc:
            cpu["all_cores"] = {"value": allc[0], "unit": "markers/s", "cores": allc[1], "kind": "oracle",
                                "sample": f"{allc[1]} processes at once, each on its own {nb}-body sample; "
                                          "markers of all over the slowest process's compute time"}
        if real == "f32":
            precision = {}
            cb = api.Context(w.faces, w.periodic, real="f32", field="bf16", brick_log2=tiles)
            ub, fb = u.to(torch.bfloat16), torch.zeros(u.shape, dtype=torch.bfloat16, device=dev)
            Tb = cb.transfer(M)

            def step_b():
                cb.marker_prep(V, tri, x, area)
                cb.build_interpolate(Tb, x, area, ub, U, method="exact")
                cb.spread(Tb, F, fb)

            for _ in range(3):
                step_b()
            torch.cuda.synchronize()
            tb = []
            for _ in range(max(3, a.steps // 2)):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                step_b()
                e1.record()
                torch.cuda.synchronize()
                tb.append(e0.elapsed_time(e1))
            cb.read_timing()
            cb.timing(True)
            for _ in range(3):
                flush.fill_(1.0)
                step_b()
            kb = cb.read_timing()
            cb.timing(False)
            ob = sample_outputs(cb, "exact", torch.bfloat16)
            precision["bf16_fields"] = {"value": M / (statistics.mean(tb) / 1e3),
                                        "U": _errs(ob["U"], ref["U"]), "f": _errs(ob["f"], ref["fv"]),
                                        "bound_stated": 1e-2,
                                        "kernels_ms": {k: round(v[1] / v[0], 5) for k, v in kb.items() if v[0]}}
            c0 = api.Context(w.faces, w.periodic, real="f32", refine=0, brick_log2=tiles)
            o0 = sample_outputs(c0, "exact", torch.float32)
            precision["f32_solve_no_refinement"] = {"phi": _errs(o0["phi"], ref["phi"])}
            precision["f32_solve_one_refinement"] = {"phi": errs["exact"]["phi_vs_exact"],
                                                     "fp64_fallbacks": ctx.status(T)["refined_fp64"]}
        if "surrogate" in others:
            # The surrogate's gate (linear-reproduction residual of the raw network
            # output) at several thresholds: fallback rate and build time on the
            # whole workload, error against the double-precision oracle on the sample.
            theta = ctx.surrogate_params()
            sweep = []
            for thr in (1e-4, 1e-3, 3e-3, 1e-2, 3e-2, float("inf")):
                cs = api.Context(w.faces, w.periodic, real=real, brick_log2=tiles,
                                 residual_max=thr if thr != float("inf") else 1e30)
                cs.surrogate_params(theta)
                Tsw = cs.transfer(M)
                for _ in range(2):
                    cs.build_transfer(Tsw, x, area, "surrogate")
                torch.cuda.synchronize()
                cs.read_timing()
                cs.timing(True)
                for _ in range(3):
                    flush.fill_(1.0)
                    cs.build_transfer(Tsw, x, area, "surrogate")
                kb = cs.read_timing()["build_surrogate"]
                cs.timing(False)
                rate = cs.status(Tsw)["surrogate_fallback"] / M
                Tsw.close()
                o = sample_outputs(cs, "surrogate", tdt)
                sweep.append({"residual_max": thr if thr != float("inf") else None, "fallback_rate": rate,
                              "build_ms": kb[1] / kb[0], "phi_vs_exact": _errs(o["phi"], ref["phi"]),
                              "U": _errs(o["U"], ref["U"]), "f": _errs(o["f"], ref["fv"])})
                cs.close()
            others["surrogate"]["gate_sweep"] = sweep

    line = {
        "metric": METRIC, "value": value, "unit": "markers/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": real, "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[a.workload] if a.grid is None and a.bodies is None else
                   f"{a.workload} variant: {len(w.body_faces) - 1} bodies, {w.n[0]}x{w.n[1]}x{w.n[2]} grid",
                   "markers_per_gpu": M, "method": a.method, "grid": list(w.n),
                   "l2": "flushed by a 256 MiB write before every timed step",
                   "step": ("marker_prep + build_interpolate (build and interpolation in one call, the "
                            "interpolation inside the exact build kernel) + spread" if a.method == "exact" else
                            "marker_prep + build_interpolate (build_transfer + interpolate in turn) + spread"),
                   "graph": graph_state["use"], "graph_error": graph_state["error"], "tiles_log2": list(tiles),
                   "autotune_ms": {str(k): round(v, 4) for k, v in tune_ms.items()} if tune_ms else None,
                   "touched_cells_per_marker": round(u_cells, 4)},
        "roofline": roof, "kernels": kernels, "gpu_launches": launches, "methods": others,
        "precision": precision, "e2e": e2e, "stream_calls": stream_calls, "clocks": clocks, "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))


# ---------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    """The oracle on the host cores: each step runs it, unchanged, in one
    process per core at once, each process on its own 20-body sample of the
    workload.  The line reports what was measured: the sample's markers and the
    step's time (the slowest process's compute time), not an extrapolation to
    the whole workload."""
    if rank != 0:
        return
    w = workload(a.workload, a.grid, a.bodies)
    n_bodies = len(w.body_faces) - 1
    nb = min(20, n_bodies)
    kw = {k: v for k, v in (("n", a.grid), ("n_bodies", a.bodies)) if v is not None}
    procs, markers, times = 1, 0, []
    steps = max(1, a.steps)
    for s in range(a.warmup + steps):
        _, procs, markers, t = run_oracle_all_cores(a.workload, a.method, nb, kw, return_sample=True)
        if s >= a.warmup:
            times.append(t)
    step_s = statistics.mean(times)
    value = markers / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "markers/s", "n_gpus": world,
            "steps": steps, "warmup": a.warmup, "ms_per_step": 1e3 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[a.workload], "method": a.method,
                       "markers_per_step": markers,
                       "sample": f"each step: {procs} processes at once, each on its own {nb}-body sample of "
                                 f"the workload ({markers} markers in all); ms_per_step is the slowest "
                                 "process's compute time"},
            "cpu_baseline": {"value": value, "unit": "markers/s", "cores": procs, "kind": "oracle",
                             "sample": f"{procs} processes at once, each on its own {nb}-body sample of the "
                                       "workload, numpy float64, one thread each"},
            "e2e": {"value": value, "unit": "markers/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    a = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if a.impl == "ours" else "gloo"
        if a.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    try:
        if a.impl == "reference":
            run_reference(a, rank, world)
        else:
            run_ours(a, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
