#!/usr/bin/env python3
"""Throughput of the PL Morse-Smale segmentation on one GB300 (or N
replicas, one per GPU).

One step = one full segmentation (order keys, steepest neighbours, path
compression, MS ids) of the workload's field through the C ABI
(``ms_segment``), inputs and outputs resident in HBM.  The default workload
is a 512^3 float32 field of seeded white noise blurred by a periodic
Gaussian (sigma = 4 voxels): the shape of the paper's 512^3 strong-scaling
dataset with dense extrema.  The field (512 MiB) and the three label arrays
(1.5 GiB) are each larger than the 129 MB L2, so nothing stays cached
between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain single-threaded restatement of the paper's definitions) on a
bounded slab of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthfields as sf  # noqa: E402

METRIC = "MS-segmented vertices/s at 512³ fp32 (% HBM roofline); batched/served p99 latency"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes per vertex of the whole path: read the field once, write
# three int32 labels.
PATH_BYTES = {"f32": 16, "f16": 14}
# Algorithmic bytes per vertex of one launch of each per-vertex stage kernel:
# tile_local reads the field and writes one 16-bit pair number per vertex;
# write reads that number and writes the three int32 labels.
STAGE_BYTES = {
    "tile_local": {"f32": 4 + 2, "f16": 2 + 2},
    "write": {"f32": 2 + 12, "f16": 2 + 12},
}

WORKLOADS = {
    "noise512": dict(dims=(512, 512, 512), kind="noise", dtype="f32",
                     desc="512^3 fp32 white noise, periodic Gaussian sigma=4 (radius 16), seed 0"),
    "noise512q": dict(dims=(512, 512, 512), kind="noiseq", dtype="f32",
                      desc="512^3 fp32 sigma=4 smoothed noise quantised to 256 levels, seed 0"),
    "gauss64": dict(dims=(64, 64, 64), kind="gauss", dtype="f32",
                    desc="64^3 fp32 sum of 8 Gaussians + 1e-3 noise, seed 0"),
    "broad1024": dict(dims=(1024, 1024, 1024), kind="broad", dtype="f32",
                      desc="1024^3 fp32 two sigma=300 Gaussians + linear ramp, seed 0"),
    "broad32768": dict(dims=(32768, 32768, 1), kind="broad", dtype="f32",
                       desc="32768^2 fp32 two sigma=300 Gaussians + linear ramp, seed 0"),
    "noise256": dict(dims=(256, 256, 256), kind="noise", dtype="f32",
                     desc="256^3 fp32 sigma=4 smoothed noise, seed 0"),
    "noise384": dict(dims=(384, 384, 384), kind="noise", dtype="f32",
                     desc="384^3 fp32 sigma=4 smoothed noise, seed 0 (profiling size)"),
    "serve": dict(dims=None, kind="serve", dtype="f32",
                  desc="request loop: 64 requests (2D squares side log-uniform 512-16384, 3D cubes "
                       "side log-uniform 64-768, 50/50), fp32 sub-boxes of sigma=4 smoothed-noise "
                       "bases (16384^2 and 768^3, generated on the device), 120 GB budget; "
                       "saturation and Poisson arrivals vs the plain one-call-per-field path"),
    "index512": dict(dims=(512, 512, 512), kind="index", dtype="i32",
                     desc="marching tetrahedra index pass (codes + cell offsets) over the MS labels "
                          "of the 512^3 sigma=4 noise field (6 x 511^3 tetrahedra)"),
    "index256": dict(dims=(256, 256, 256), kind="index", dtype="i32",
                     desc="the index and geometry passes over the MS labels of the 256^3 sigma=4 noise "
                          "field (profiling size)"),
    "batch256": dict(dims=None, kind="batch", dtype="mixed",
                     desc="256 fields, dims log-uniform in [32, 256] per axis, fp32/fp16 and smoothed "
                          "noise (sigma 2-6) / 8-Gaussian sums 50/50, seed 0; one ms_segment_batch call "
                          "per step vs 256 ms_segment calls"),
}


def cache_dir():
    d = os.environ.get("MS_FIELD_CACHE") or os.path.join(tempfile.gettempdir(), "msseg_fields")
    os.makedirs(d, exist_ok=True)
    return d


def make_field(name, z0=None, z1=None):
    w = WORKLOADS[name]
    path = os.path.join(cache_dir(), f"{name}.npy")
    if os.path.exists(path):
        f = np.load(path, mmap_mode="r")
    else:
        dims = w["dims"]
        if w["kind"] == "noise":
            f = sf.smoothed_noise(dims, 0, sigma=4.0, radius=16)
        elif w["kind"] == "noiseq":
            f = sf.quantize_levels(sf.smoothed_noise(dims, 0, sigma=4.0, radius=16))
        elif w["kind"] == "gauss":
            f = sf.gaussian_sum(dims, 0)
        else:
            f = sf.broad_gaussians_ramp(dims, 0)
        if w["dtype"] == "f16":
            f = f.astype(np.float16)
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, f)
        os.replace(tmp, path)
    if z0 is not None:
        return np.ascontiguousarray(f[z0:z1])
    return np.ascontiguousarray(f)


# The sources the tiled kernels are compiled from: stored ncu traffic counts
# are used only while these are unchanged.
TILED_SOURCES = ["paper_2303_15491_gb300/csrc/ms_tiled.cu", "paper_2303_15491_gb300/csrc/ms_tiled.cuh",
                 "paper_2303_15491_gb300/csrc/ms_internal.cuh", "paper_2303_15491_gb300/csrc/fastdiv.h",
                 "include/ms.h"]


def source_hash():
    h = hashlib.sha1()
    for rel in TILED_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(rel.encode() + fh.read())
    return h.hexdigest()


def peaks():
    try:
        with open(PEAKS_PATH) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms while the
    timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x of all ranks (replicas are timed by the slowest one);
    x itself without a process group.  gloo groups reduce on the CPU."""
    if dist is None:
        return float(x)
    import torch

    if dist.get_backend() == "gloo":
        device = "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak
    scaling: every rank processes the same units)."""
    return world_size * units_per_rank / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The CPU oracle, as it stands, on bounded slabs of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    w = WORKLOADS[args.workload]
    nx, ny, nz = w["dims"]
    flat = nz == 1
    # a bounded sample per step: ref_slab planes (3D), or a block of rows of
    # as many vertices (2D)
    slab = max(1, min(ny if flat else nz, args.ref_slab * (512 * 512 // nx if flat else 1)))
    times = []
    verts = nx * slab * (1 if flat else ny)
    for step in range(args.warmup + args.steps):
        z0 = (step * slab) % max(1, (ny if flat else nz) - slab + 1)
        if flat:
            f = np.ascontiguousarray(make_field(args.workload)[0, z0:z0 + slab])
        else:
            f = make_field(args.workload, z0, z0 + slab)
        t = time.perf_counter()
        oracle.segment(f)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = verts * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "vertices/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"],
                   "sample": (f"{nx}x{slab} row block" if flat else f"z-slab {nx}x{ny}x{slab}") +
                             " per step (a different one each step)"},
        "cpu_baseline": {"value": value, "unit": "vertices/s", "cores": 1, "kind": "oracle",
                         "sample": (f"{nx}x{slab} rows" if flat else f"{nx}x{ny}x{slab} slab") +
                                   f" of {args.workload} per step"},
        "e2e": {"value": value, "unit": "vertices/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(args):
    """The oracle on a bounded sample: the first cpu_slab planes (3D), or as
    many rows as hold that many 512^2 planes' worth of vertices (2D)."""
    import oracle

    w = WORKLOADS[args.workload]
    nx, ny, nz = w["dims"]
    if nz == 1:
        rows = max(1, min(ny, args.cpu_slab * 512 * 512 // nx))
        f = np.ascontiguousarray(make_field(args.workload)[0, :rows])
        shape, n = f"{nx}x{rows} row block", nx * rows
    else:
        slab = max(1, min(nz, args.cpu_slab))
        f = make_field(args.workload, 0, slab)
        shape, n = f"{nx}x{ny}x{slab} z-slab", nx * ny * slab
    t = time.perf_counter()
    oracle.segment(f)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "vertices/s", "cores": 1, "kind": "oracle",
            "sample": f"first {shape} of {args.workload} ({n} vertices, {dt:.1f} s single-threaded)"}


def cpu_parallel_baseline(args):
    """The paper's CPU-parallel scheme (cpu_parallel: per-thread active lists,
    OpenMP) on all host cores, on the same sample as the oracle's baseline:
    one warm-up and 5 timed runs in a child process with a time limit, so
    that it can neither hang nor break this line."""
    w = WORKLOADS[args.workload]
    nx, ny, nz = w["dims"]
    if nz == 1:
        rows = max(1, min(ny, args.cpu_slab * 512 * 512 // nx))
        f = np.ascontiguousarray(make_field(args.workload)[0, :rows])
        shape = f"{nx}x{rows} row block"
    else:
        slab = max(1, min(nz, args.cpu_slab))
        f = make_field(args.workload, 0, slab)
        shape = f"{nx}x{ny}x{slab} z-slab"
    path = os.path.join(cache_dir(), f"cpu_parallel_sample_{os.getpid()}.npy")
    try:
        np.save(path, np.ascontiguousarray(f, dtype=np.float32))
        r = subprocess.run([sys.executable, "-m", "cpu_parallel", path, "5"], cwd=ROOT,
                           capture_output=True, text=True, timeout=240)
        if r.returncode != 0:
            return {"unavailable": (r.stderr.strip().splitlines() or ["failed"])[-1][:200]}
        res = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": res["vertices"] / res["median_s"], "unit": "vertices/s",
                "cores": res["threads"], "kind": "the paper's CPU-parallel scheme (OpenMP)",
                "sample": f"first {shape} of {args.workload} ({res['vertices']} vertices): median of 5 "
                          f"runs after one warm-up, {res['median_s'] * 1e3:.0f} ms"}
    except Exception as e:  # includes the time limit
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    finally:
        try:
            os.remove(path)
        except OSError:
            pass


def batch_fields():
    specs = sf.batch_specs(256, seed=0)
    out = []
    t0 = time.perf_counter()
    for i, sp in enumerate(specs):
        if i % 32 == 0:
            print(f"[bench] batch fields {i}/256 ({time.perf_counter() - t0:.0f} s)", file=sys.stderr,
                  flush=True)
        path = os.path.join(cache_dir(), f"batch256_{i:03d}.npy")
        if os.path.exists(path):
            out.append(np.load(path))
            continue
        f = sf.batch_field(sp)
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, f)
        os.replace(tmp, path)
        out.append(f)
    return out


def run_batch_bench(args):
    print(json.dumps(batch_line(args)), flush=True)
    return 0


def batch_line(args, plain_steps=None):
    """Many uneven fields per step: one ms_segment_batch call against the same
    fields through one ms_segment call each."""
    import torch

    import paper_2303_15491_gb300 as ms

    ws, rank, local = dist_env()
    torch.cuda.set_device(local if ws > 1 else 0)
    dev = torch.cuda.current_device()
    fields_np = batch_fields()
    fields = [torch.from_numpy(f).to(dev) for f in fields_np]
    outs = [[torch.empty(f.size, dtype=torch.int32, device=dev) for _ in range(3)] for f in fields_np]
    dims = [ms.dims_of(f) for f in fields_np]
    dts = [ms.dtype_code(f) for f in fields_np]
    n = int(sum(f.size for f in fields_np))
    stream = torch.cuda.Stream(device=dev)
    ctx = ms.ms_create(dev, stream)
    asc, desc, mso = [o[0] for o in outs], [o[1] for o in outs], [o[2] for o in outs]

    def batched():
        return ms.ms_segment_batch(ctx, fields, dims, dts, asc, desc, mso)

    def plain():
        for f, o in zip(fields, outs):
            ms.ms_segment(ctx, f, ms.dims_of(f), ms.dtype_code(f), o[0], o[1], o[2])

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        t = time.perf_counter()
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return max(ev0.elapsed_time(ev1), 1e3 * (time.perf_counter() - t)) / steps

    if getattr(args, "no_autotune", False):  # fixed choices (profiling runs)
        if getattr(args, "resolve_mode", None) is not None:
            ms.ms_set_tuning(ctx, resolve_mode=args.resolve_mode)
        tuning = {**ms.ms_get_tuning(ctx), "default_ms": None, "best_ms": None}
    else:
        print("[bench] fields on device; autotuning the batched call", file=sys.stderr, flush=True)
        tuning = ms.ms_batch_autotune(ctx, fields, dims, dts, asc, desc, mso)
    print(f"[bench] tuning {tuning}; timing the batched call", file=sys.stderr, flush=True)
    ms.ms_profile_enable(ctx, True)
    with ClockSampler(dev) as clk:
        t_batch = timed(batched, args.steps)
    print(f"[bench] batched {t_batch:.2f} ms/step; timing 256 single calls", file=sys.stderr,
          flush=True)
    prof = ms.ms_profile_read(ctx)
    ms.ms_profile_enable(ctx, False)
    t_plain = timed(plain, plain_steps or max(1, args.steps // 4))
    ks = batched()
    ms.ms_destroy(ctx)
    n_fields = len(fields)
    del fields, outs, asc, desc, mso
    torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": n / (t_batch / 1e3), "unit": "vertices/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batch256", "desc": WORKLOADS["batch256"]["desc"], "fields": n_fields,
                   "vertices": n, "regions_K_total": int(sum(ks)),
                   "l2": "fields 1.1 GB + labels 3.6 GB, larger than L2"},
        "plain_ms_per_step": t_plain, "speedup_vs_plain": t_plain / t_batch,
        "tuning": tuning, "tile_shape": "x".join(map(str, ms.TILE_SHAPES[tuning["shape3"]])),
        "graph_replay": prof["stages"]["graph"]["launches"] > 0,
        "gpu_launches": prof["launches"],
        "stages_ms_per_step": {k: v["ms"] / max(1, prof["calls"]) for k, v in prof["stages"].items()
                               if v["launches"] or v["ms"]},
        "clocks": clk.summary(),
    }
    return line


def device_smoothed_noise(shape, seed, dev, sigma=4.0, radius=16):
    """Seeded N(0,1) white noise on the device, filtered by a periodic
    Gaussian (sigma, truncated at radius) one axis after the other: the
    smoothed-noise recipe of the synthetic fields, generated where it is used
    so that multi-GB bases need no host round trip."""
    import torch
    import torch.nn.functional as F

    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.randn(shape, generator=g, device=dev, dtype=torch.float32)
    t = torch.arange(-radius, radius + 1, device=dev, dtype=torch.float64)
    w = torch.exp(-0.5 * (t / sigma) ** 2)
    w = (w / w.sum()).float().view(1, 1, -1)
    for ax in range(x.ndim):
        if x.shape[ax] == 1:
            continue
        y = x.movedim(ax, -1).contiguous()
        sh = y.shape
        y = y.view(-1, 1, sh[-1])
        out = torch.empty_like(y)
        rows = max(1, (1 << 27) // sh[-1])  # bound the padded temporaries
        for r0 in range(0, y.shape[0], rows):
            yy = F.pad(y[r0:r0 + rows], (radius, radius), mode="circular")
            out[r0:r0 + rows] = F.conv1d(yy, w)
        del y
        x = out.view(sh).movedim(-1, ax).contiguous()
        del out
    return x


def run_serve_bench(args):
    print(json.dumps(serve_line(args)), flush=True)
    return 0


def serve_line(args):
    """The request loop (ms_server) against the plain path on the same requests:
    (1) saturation -- all requests submitted at once -- for throughput, and
    (2) a Poisson stream at a stated rate for p50 / p99 latency, through the
    server with --slots slots and through a one-slot server (the plain path
    behind a FIFO queue)."""
    import torch

    import paper_2303_15491_gb300 as ms

    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    specs = sf.serve_specs(args.serve_requests, seed=0)
    rng = np.random.default_rng(12345)
    side2 = max(d[0] for d, _ in specs if d[2] == 1)
    side3 = max(d[0] for d, _ in specs if d[2] > 1)
    t0 = time.perf_counter()
    base2 = device_smoothed_noise((side2, side2), 1, dev)
    base3 = device_smoothed_noise((side3, side3, side3), 2, dev)
    reqs = []
    for dims, _ in specs:
        s_ = dims[0]
        if dims[2] == 1:
            y0, x0 = (int(v) for v in rng.integers(0, side2 - s_ + 1, size=2))
            f = base2[y0:y0 + s_, x0:x0 + s_].contiguous()
        else:
            z0, y0, x0 = (int(v) for v in rng.integers(0, side3 - s_ + 1, size=3))
            f = base3[z0:z0 + s_, y0:y0 + s_, x0:x0 + s_].contiguous()
        outs = [torch.empty(f.numel(), dtype=torch.int32, device=dev) for _ in range(3)]
        reqs.append((f, tuple(dims), outs))
    del base2, base3
    torch.cuda.synchronize()
    nvert = [int(f.numel()) for f, _, _ in reqs]
    total = int(sum(nvert))
    print(f"[bench] {len(reqs)} requests, {total / 1e9:.2f} G vertices on device "
          f"({time.perf_counter() - t0:.0f} s)", file=sys.stderr, flush=True)

    # ---- plain path: one ms_segment call after the other on one context
    stream = torch.cuda.Stream(device=dev)
    ctx = ms.ms_create(dev, stream)
    for f, dims, o in reqs:  # warm: scratch grows to the largest request
        ms.ms_segment(ctx, f, dims, ms.MS_F32, *o)
    plain_k = []
    service = []
    ms.ms_profile_enable(ctx, True)
    t = time.perf_counter()
    for f, dims, o in reqs:
        ti = time.perf_counter()
        ms.ms_segment(ctx, f, dims, ms.MS_F32, *o)  # returns after completion
        service.append(time.perf_counter() - ti)
        plain_k.append(ms.ms_last_region_count(ctx))
    t_plain = time.perf_counter() - t
    plain_launches = ms.ms_profile_read(ctx)["launches"]
    ms.ms_destroy(ctx)

    budget = int(args.serve_budget_gb * (1 << 30))

    def run_stream(slots, arrivals):
        """Submit request j at arrivals[j] (seconds from the start; None = all at
        once); returns (makespan s, latencies ms, stats, region counts)."""
        srv = ms.ms_server_create(dev, budget, slots)
        try:
            # warm every slot's scratch: `slots` copies of the largest 2D and of
            # the largest 3D request at once (an idle slot takes one each)
            for big in (max((r for r in reqs if r[1][2] == 1), key=lambda r: r[0].numel()),
                        max((r for r in reqs if r[1][2] > 1), key=lambda r: r[0].numel())):
                f, dims, _ = big
                tmp = [[torch.empty(f.numel(), dtype=torch.int32, device=dev) for _ in range(3)]
                       for _ in range(slots)]
                torch.cuda.synchronize()
                ts = [ms.ms_server_submit(srv, f, dims, ms.MS_F32, *o) for o in tmp]
                for tk in ts:
                    ms.ms_server_wait(srv, tk, -1)
                del tmp
            base = ms.ms_server_stats(srv)
            order = list(range(len(arrivals)))
            tickets, sub_t = [None] * len(order), [0.0] * len(order)
            lat, ks, pending = [0.0] * len(order), [0] * len(order), {}
            start = time.perf_counter()
            for j in order:
                i = j % len(reqs)
                if i in pending:  # the previous use of request i's buffers must be done
                    jp = pending.pop(i)
                    st, ks[jp], lat[jp] = ms.ms_server_wait(srv, tickets[jp], -1)
                    assert st == 0, ms.STATUS[st]
                if arrivals[j] is not None:
                    delay = start + arrivals[j] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                f, dims, o = reqs[i]
                sub_t[j] = time.perf_counter() - start
                tickets[j] = ms.ms_server_submit(srv, f, dims, ms.MS_F32, *o)
                pending[i] = j
            for i, jp in pending.items():
                st, ks[jp], lat[jp] = ms.ms_server_wait(srv, tickets[jp], -1)
                assert st == 0, ms.STATUS[st]
            makespan = max(sub_t[j] + lat[j] / 1e3 for j in order)
            stats = ms.ms_server_stats(srv)
            stats["launches"] -= base["launches"]
        finally:
            ms.ms_server_destroy(srv)
        return makespan, lat, stats, ks

    def pct(xs, q):
        return float(np.percentile(np.asarray(xs), q))

    # ---- saturation: every request submitted at once, passes times over
    n_sat = len(reqs) * args.serve_passes
    with ClockSampler(dev) as clk:
        sat_t, sat_lat, sat_stats, sat_k = run_stream(args.slots, [None] * n_sat)
    sat_vps = total * args.serve_passes / sat_t
    plain_vps = total / t_plain
    print(f"[bench] plain {t_plain * 1e3:.1f} ms/pass, saturated server "
          f"{sat_t * 1e3 / args.serve_passes:.1f} ms/pass", file=sys.stderr, flush=True)
    assert sat_k[:len(reqs)] == plain_k, "served region counts differ from the plain path"

    # ---- Poisson arrivals at rho x the plain path's request capacity
    rate = args.serve_load * len(reqs) / t_plain  # requests per second
    gaps = np.random.default_rng(777).exponential(1.0 / rate, size=n_sat)
    arrivals = list(np.cumsum(gaps) - gaps[0])
    p_t, p_lat, p_stats, _ = run_stream(args.slots, arrivals)
    q_t, q_lat, _, _ = run_stream(1, arrivals)
    line = {
        "metric": METRIC, "value": sat_vps, "unit": "vertices/s", "n_gpus": 1,
        "steps": args.serve_passes, "warmup": 1, "ms_per_step": sat_t * 1e3 / args.serve_passes,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "serve", "desc": WORKLOADS["serve"]["desc"], "requests": len(reqs),
                   "vertices_per_pass": total, "slots": args.slots,
                   "budget_bytes": budget, "l2": "inputs and labels larger than L2"},
        "plain": {"ms_per_pass": t_plain * 1e3, "vertices_per_s": plain_vps,
                  "service_ms_p50": 1e3 * pct(service, 50), "service_ms_p99": 1e3 * pct(service, 99)},
        "speedup_vs_plain": sat_vps / plain_vps,
        "saturated": {"latency_ms_p50": pct(sat_lat, 50), "latency_ms_p99": pct(sat_lat, 99),
                      "peak_bytes": sat_stats["peak_bytes"]},
        "poisson": {"rate_req_per_s": rate, "load_vs_plain_capacity": args.serve_load,
                    "requests": n_sat,
                    "served": {"latency_ms_p50": pct(p_lat, 50), "latency_ms_p99": pct(p_lat, 99),
                               "vertices_per_s": total * args.serve_passes / p_t,
                               "peak_bytes": p_stats["peak_bytes"]},
                    "plain_fifo": {"latency_ms_p50": pct(q_lat, 50), "latency_ms_p99": pct(q_lat, 99),
                                   "vertices_per_s": total * args.serve_passes / q_t}},
        "gpu_launches": sat_stats["launches"],
        "plain_gpu_launches": plain_launches,
        "clocks": clk.summary(),
    }
    del reqs
    torch.cuda.empty_cache()
    return line


def run_index_bench(args):
    """The index pass after the segmentation (ms_simplex_index) on the MS labels
    of the 512^3 (index256: 256^3) noise field: per cell, labels in (4 B, each
    vertex once), 6 tetrahedron codes (6 B) and one offset (8 B) out; then the
    geometry pass (region separators) into the slots it made."""
    import torch

    import paper_2303_15491_gb300 as ms

    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    dims = WORKLOADS[args.workload]["dims"]
    field = torch.from_numpy(make_field("noise512" if dims[0] == 512 else "noise256")).to(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = ms.ms_create(dev, stream)
    asc, desc, labels, _ = ms.segment(ctx, field)
    del asc, desc, field
    cells, per = ms.simplex_cells(dims)
    codes = torch.empty(cells * per, dtype=torch.uint8, device=dev)
    offs = torch.empty(cells, dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        total = ms.ms_simplex_index(ctx, labels, dims, codes, offs)
    torch.cuda.synchronize()
    ms.ms_profile_enable(ctx, True)
    with ClockSampler(dev) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        t = time.perf_counter()
        for _ in range(args.steps):
            total = ms.ms_simplex_index(ctx, labels, dims, codes, offs)
        ev1.record(stream)
        torch.cuda.synchronize()
        host_ms = 1e3 * (time.perf_counter() - t)
    prof = ms.ms_profile_read(ctx)
    ms.ms_profile_enable(ctx, False)
    ms_per = max(ev0.elapsed_time(ev1), host_ms) / args.steps
    kern_ms = prof["stages"]["tile_local"]["ms"] / max(1, prof["calls"])
    hbm, peak_kind = peaks()
    alg = 18 * cells
    # the geometry pass (region separators) into the slots the index pass made:
    # labels and offsets in, 9 floats + 2 labels out per triangle
    pts = torch.empty((total, 3, 3), dtype=torch.float32, device=dev)
    prs = torch.empty((total, 2), dtype=torch.int32, device=dev)
    for _ in range(2):
        ms.ms_simplex_geometry(ctx, labels, dims, offs, total, pts, prs)
    ms.ms_profile_enable(ctx, True)
    geo_steps = max(1, args.steps // 4)
    for _ in range(geo_steps):
        ms.ms_simplex_geometry(ctx, labels, dims, offs, total, pts, prs)
    gprof = ms.ms_profile_read(ctx)
    ms.ms_profile_enable(ctx, False)
    geo_ms = gprof["stages"]["write"]["ms"] / max(1, gprof["calls"])
    geo_bytes = 12 * cells + 44 * total
    del pts, prs
    # CPU baseline: the oracle on a z-slab of the labels
    import oracle

    slab = 17
    lab_np = labels.view(dims[2], dims[1], dims[0])[:slab].cpu().numpy()
    t = time.perf_counter()
    oracle.simplex_index(lab_np, (dims[0], dims[1], slab))
    cpu_s = time.perf_counter() - t
    ms.ms_destroy(ctx)
    line = {
        "metric": "tetrahedra indexed/s (marching tetrahedra index pass)", "value": cells * per / (ms_per / 1e3),
        "unit": "tetrahedra/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "i32", "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "cells": cells,
                   "tetrahedra": cells * per, "elements_total": total,
                   "l2": ("labels 512 MiB, codes 800 MB, offsets 1.07 GB: larger than L2" if dims[0] == 512
                          else "labels 64 MiB (L2-resident), codes 100 MB, offsets 134 MB")},
        "roofline": {"bound": "hbm", "kernel": "index pass (k_simplex_index, one launch)", "achieved": alg / (kern_ms / 1e3) / 1e9,
                     "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": alg / (kern_ms / 1e3) / 1e9 / hbm, "traffic": None,
                     "alg_bytes_per_cell": 18, "avg_launch_ms": kern_ms},
        "gpu_launches": prof["launches"],
        "geometry": {"kernel": "region separators", "ms": geo_ms, "triangles": total,
                     "alg_bytes": geo_bytes, "achieved_gbs": geo_bytes / (geo_ms / 1e3) / 1e9,
                     "frac": geo_bytes / (geo_ms / 1e3) / 1e9 / hbm,
                     "note": "labels 4 B + offset 8 B per cell in, 36 B of points + 8 B of labels "
                             "per triangle out"},
        "cpu_baseline": {"value": (dims[0] - 1) * (dims[1] - 1) * (slab - 1) * per / cpu_s,
                         "unit": "tetrahedra/s", "cores": 1, "kind": "oracle",
                         "sample": f"{dims[0]}x{dims[1]}x{slab} slab ({cpu_s:.1f} s single-threaded)"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def extra(name, fn):
    """One sub-measurement of the default run; a failure is reported in the
    line instead of ending the run."""
    t = time.perf_counter()
    print(f"[bench] {name} ...", file=sys.stderr, flush=True)
    try:
        out = fn()
    except Exception as e:  # reported, not hidden: the key says what failed
        out = {"unavailable": f"{type(e).__name__}: {e}"[:300]}
    out["wall_s"] = round(time.perf_counter() - t, 1)
    return out


def quantised_summary(args, f_np):
    """The 512^3 field quantised to 256 levels (exact ties), one field per
    call, timed like the main workload over fewer steps."""
    import torch

    import paper_2303_15491_gb300 as ms

    fq = sf.quantize_levels(np.asarray(f_np))
    dev = torch.cuda.current_device()
    n = fq.size
    field = torch.from_numpy(fq).to(dev)
    outs = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(3)]
    stream = torch.cuda.Stream(device=dev)
    ctx = ms.ms_create(dev, stream)
    dims = ms.dims_of(fq)
    try:
        for _ in range(args.warmup):
            ms.ms_segment(ctx, field, dims, ms.MS_F32, *outs)
        steps = 20
        torch.cuda.synchronize()
        ms.ms_profile_enable(ctx, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            ms.ms_segment(ctx, field, dims, ms.MS_F32, *outs)
        ev1.record(stream)
        torch.cuda.synchronize()
        prof = ms.ms_profile_read(ctx)
        t = ev0.elapsed_time(ev1) / steps
        k = ms.ms_last_region_count(ctx)
    finally:
        ms.ms_destroy(ctx)
        del field, outs
        torch.cuda.empty_cache()
    hbm, _ = peaks()
    return {"workload": "noise512q", "desc": WORKLOADS["noise512q"]["desc"], "steps": steps,
            "ms_per_step": t, "vertices_per_s": n / (t / 1e3), "regions_K": k,
            "path_frac": PATH_BYTES["f32"] * n / (t / 1e3) / 1e9 / hbm,
            "stages_ms_per_step": {kk: v["ms"] / max(1, prof["calls"])
                                   for kk, v in prof["stages"].items() if v["launches"] or v["ms"]}}


def persistence_summary(args, f_np):
    """Persistence pairs of the workload field's minima and maxima from its
    segmentation (ms_persistence, Sec. 4.1), wall time per call (the call
    reads counts back between its steps), median of 5 after one untimed."""
    import torch

    import paper_2303_15491_gb300 as ms

    dev = torch.cuda.current_device()
    field = torch.from_numpy(np.asarray(f_np)).to(dev)
    ctx = ms.ms_create(dev, torch.cuda.Stream(device=dev))
    out = {"workload": args.workload, "reps": 5}
    try:
        asc, desc, _, _ = ms.segment(ctx, field)
        dims, dt = ms.dims_of(field), ms.dtype_code(field)
        for name, direction, lab in (("minima", -1, asc), ("maxima", 1, desc)):
            ext, death, info = ms.persistence(ctx, field, lab, direction)
            cap = info["n_extrema"]
            times = []
            for _ in range(5):
                torch.cuda.synchronize()
                t = time.perf_counter()
                info = ms.ms_persistence(ctx, field, dims, dt, lab, direction, ext, death, cap)
                times.append(1e3 * (time.perf_counter() - t))
            out[name] = {"ms": float(np.median(times)), "extrema": info["n_extrema"],
                         "basin_edges": info["basin_edges"], "rounds": info["rounds"],
                         "finish_edges": info["finish_edges"]}
    finally:
        ms.ms_destroy(ctx)
        del field
        torch.cuda.empty_cache()
    return out


def batched_summary(args):
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = 10, 3
    ln = batch_line(sub, plain_steps=2)
    return {"workload": "batch256", "desc": WORKLOADS["batch256"]["desc"], "steps": sub.steps,
            "ms_per_step": ln["ms_per_step"], "vertices_per_s": ln["value"],
            "plain_ms_per_step": ln["plain_ms_per_step"], "speedup_vs_plain": ln["speedup_vs_plain"],
            "fields": ln["config"]["fields"], "vertices": ln["config"]["vertices"],
            "regions_K_total": ln["config"]["regions_K_total"], "tuning": ln["tuning"],
            "tile_shape": ln["tile_shape"],
            "graph_replay": ln["graph_replay"], "stages_ms_per_step": ln["stages_ms_per_step"],
            "note": "10 timed batched steps, 2 timed rounds of 256 single calls (reduced counts)"}


def served_summary(args):
    sub = argparse.Namespace(**vars(args))
    sub.serve_passes = 4
    ln = serve_line(sub)
    return {"workload": "serve", "desc": WORKLOADS["serve"]["desc"], "passes": sub.serve_passes,
            "slots": ln["config"]["slots"], "budget_bytes": ln["config"]["budget_bytes"],
            "saturated_vertices_per_s": ln["value"], "speedup_vs_plain": ln["speedup_vs_plain"],
            "plain": ln["plain"], "saturated": ln["saturated"], "poisson": ln["poisson"],
            "note": "4 passes of 64 requests (256 requests) per stream instead of 16 (reduced count)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="noise512", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--cpu-slab", type=int, default=48)
    ap.add_argument("--ref-slab", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the quantised, batched, served and persistence sub-measurements of "
                         "the default run")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch256: time the default launch choices (no autotuning run first)")
    ap.add_argument("--resolve-mode", type=int, choices=[-1, 0, 1], default=None,
                    help="batch256 with --no-autotune: resolve by tile (0), flat (1) or by tile count (-1)")
    ap.add_argument("--persistence-only", action="store_true",
                    help="time only the persistence pairing of the workload's field (a profiling aid)")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-passes", type=int, default=16)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.persistence_only:
        if args.impl == "reference" or WORKLOADS[args.workload]["kind"] not in ("noise", "noiseq", "gauss", "broad"):
            print(json.dumps({"impl": args.impl, "unavailable": "--persistence-only times the GPU pairing of "
                              "one field workload"}))
            return 0
        import torch

        torch.cuda.set_device(0)
        print(json.dumps({"persistence": persistence_summary(args, make_field(args.workload))}))
        return 0
    if args.workload in ("index512", "index256"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the index pass has no separate "
                              "reference arm; its CPU baseline is in the line's cpu_baseline"}))
            return 0
        return run_index_bench(args)
    if args.workload == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no CPU "
                              "reference arm; the oracle arm runs on the 512^3 workload"}))
            return 0
        return run_serve_bench(args)
    if args.impl == "reference" and args.workload != "batch256":
        return run_reference(args)
    if args.workload == "batch256":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU "
                              "reference arm; the oracle arm runs on the 512^3 workload"}))
            return 0
        return run_batch_bench(args)

    import torch

    import paper_2303_15491_gb300 as ms

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    w = WORKLOADS[args.workload]
    f_np = make_field(args.workload)
    dims = w["dims"]
    n = int(np.prod(dims))
    dtype = ms.MS_F16 if w["dtype"] == "f16" else ms.MS_F32
    field = torch.from_numpy(f_np).to(dev)
    asc = torch.empty(n, dtype=torch.int32, device=dev)
    desc = torch.empty_like(asc)
    msid = torch.empty_like(asc)
    stream = torch.cuda.Stream(device=dev)
    ctx = ms.ms_create(dev, stream)  # the library launches on this stream

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        ms.ms_segment(ctx, field, dims, dtype, asc, desc, msid)
    k_regions = ms.ms_last_region_count(ctx)

    # ---- device-resident timed region.  A field whose input and labels are
    # not well above L2 gets L2 flushed before every step (a write of twice
    # L2, outside the per-step events), and the time is the sum of the steps.
    esz = 2 if w["dtype"] == "f16" else 4
    io_bytes = n * esz + 3 * n * 4
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0) or (129 << 20))
    flush_buf = (torch.empty(2 * l2_bytes, dtype=torch.uint8, device=dev) if io_bytes < 4 * l2_bytes
                 else None)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms.ms_profile_enable(ctx, True)
    with ClockSampler(dev) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        # events on the stream the library's kernels are launched on, around
        # every step for the per-step statistics
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
        ev0.record(stream)
        t_host = time.perf_counter()
        for i in range(args.steps):
            if flush_buf is not None:
                with torch.cuda.stream(stream):
                    flush_buf.fill_(i & 255)
            step_ev[i][0].record(stream)
            ms.ms_segment(ctx, field, dims, dtype, asc, desc, msid)
            step_ev[i][1].record(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_host = time.perf_counter() - t_host
    prof = ms.ms_profile_read(ctx)
    ms.ms_profile_enable(ctx, False)
    barrier()
    torch.cuda.synchronize()
    # per-step times: median, and the paper's protocol (10 runs, the best and
    # the worst dropped, the mean of the other 8) over the last 10 steps
    per_step = [a.elapsed_time(b) for a, b in step_ev]
    if flush_buf is None:
        local_ms = max(ev0.elapsed_time(ev1), 1e3 * t_host)
        l2_note = (f"inputs larger than L2 (field {n * esz / 2**20:.0f} MiB, labels 3 x {n * 4 / 2**20:.0f} MiB "
                   f"> {l2_bytes / 2**20:.0f} MiB L2)")
    else:
        local_ms = sum(per_step)
        l2_note = (f"L2 flushed before every step (a {2 * l2_bytes / 2**20:.0f} MiB write outside the step's "
                   f"events; field and labels {io_bytes / 2**20:.1f} MiB); time = sum of the per-step events")
        del flush_buf
    elapsed_ms = max_over_ranks(local_ms, dist, dev)
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(n * args.steps, ws, elapsed_ms / 1e3)
    step_stats = {"median_ms": statistics.median(per_step), "min_ms": min(per_step),
                  "max_ms": max(per_step)}
    if len(per_step) >= 10:
        last = sorted(per_step[-10:])
        step_stats["paper_protocol_ms"] = sum(last[1:-1]) / 8

    # ---- end to end through ms_segment_host (pinned host memory)
    e2e_value = e2e_single = None
    if args.e2e_steps > 0:
        h_field = torch.from_numpy(f_np).pin_memory()
        h_asc = torch.empty(n, dtype=torch.int32).pin_memory()
        h_desc = torch.empty_like(h_asc).pin_memory()
        h_ms = torch.empty_like(h_asc).pin_memory()
        ms.ms_segment_host(ctx, h_field, dims, dtype, h_asc, h_desc, h_ms)  # warm the io buffers
        barrier()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            ms.ms_segment_host(ctx, h_field, dims, dtype, h_asc, h_desc, h_ms)
        single_s = max_over_ranks(time.perf_counter() - t, dist, dev)
        e2e_single = whole_job_rate(n * args.e2e_steps, ws, single_s)
        # the pipelined host path: step s+1's upload and step s-1's download
        # overlap step s's segmentation (every step's copies are in the region)
        k_steps = args.e2e_steps
        many = lambda: ms.ms_segment_host_many(ctx, [h_field] * k_steps, [dims] * k_steps,
                                               [dtype] * k_steps, [h_asc] * k_steps,
                                               [h_desc] * k_steps, [h_ms] * k_steps)
        many()  # warm the second buffer set and its captured plan
        barrier()
        t = time.perf_counter()
        many()
        e2e_s = max_over_ranks(time.perf_counter() - t, dist, dev)
        e2e_value = whole_job_rate(n * k_steps, ws, e2e_s)

    # ---- roofline of the dominant kernel and of the whole path.  The
    # headline figure is the path's algorithmic bytes (field in, three labels
    # out: 16 B a vertex) over one launch of the dominant kernel; the bytes the
    # kernel itself must move (its stage figure) are reported beside it.
    hbm, peak_kind = peaks()
    stages = prof["stages"]
    dom = max(("tile_local", "write"), key=lambda s: stages[s]["ms"])
    launches = max(1, stages[dom]["launches"])
    per_launch_s = stages[dom]["ms"] / 1e3 / launches
    alg_bytes = PATH_BYTES[w["dtype"]] * n
    achieved = alg_bytes / per_launch_s / 1e9 if per_launch_s > 0 else None
    stage_bytes = STAGE_BYTES[dom][w["dtype"]] * n
    stage_gbs = stage_bytes / per_launch_s / 1e9 if per_launch_s > 0 else None
    traffic = None
    warp_inst = None  # ncu's executed warp instructions per launch, for the issue roofline
    tpath = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if os.path.exists(tpath):
        try:
            tj = json.load(open(tpath))
            ent = tj.get(dom)
            if ent and ent.get("csrc_sha1") == source_hash() and ent.get("workload") == args.workload:
                traffic = ent["dram_bytes_per_launch"]
                warp_inst = ent.get("warp_inst_per_launch")
        except Exception:
            traffic = None
    path_gbs = PATH_BYTES[w["dtype"]] * n / (ms_per_step / 1e3) / 1e9
    clocks = clk.summary()
    # The tiled kernels are bound by instruction issue, not DRAM: beside the
    # HBM roofline, the executed warp instructions (ncu) per launch time
    # against the issue peak -- four schedulers an SM, one warp instruction a
    # cycle each, at the SM clock sampled during the timed region.
    issue = None
    if warp_inst and per_launch_s > 0:
        sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_wi = sms * 4 * sm_mhz * 1e6
        issue = {"kernel": dom, "warp_inst_per_launch": warp_inst,
                 "achieved_warp_inst_per_s": warp_inst / per_launch_s, "peak_warp_inst_per_s": peak_wi,
                 "frac": warp_inst / per_launch_s / peak_wi,
                 "peak_from": f"{sms} SMs x 4 schedulers x 1 warp instruction a cycle x {sm_mhz:.0f} MHz"}

    # what limits the dominant kernel: the larger of its DRAM fraction (the
    # bytes it moves itself) and its instruction-issue fraction
    hbm_frac = (traffic / per_launch_s / 1e9 / hbm) if (traffic and per_launch_s > 0) else (
        stage_gbs / hbm if stage_gbs else 0.0)
    if issue and issue["frac"] > hbm_frac:
        limiter = (f"instruction issue: {issue['frac']:.0%} of the issue peak against "
                   f"{hbm_frac:.0%} of HBM for the bytes the kernel moves")
    else:
        limiter = f"HBM: {hbm_frac:.0%} of the copy peak for the bytes the kernel moves"
    line = {
        "metric": METRIC, "value": value, "unit": "vertices/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "dims": list(dims),
                   "input_dtype": w["dtype"], "regions_K": k_regions,
                   "l2": l2_note,
                   "parallelism": f"replicas x{ws} (no data-path collective)"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": None if achieved is None else achieved / hbm,
                     "traffic": traffic,
                     "alg_bytes_per_vertex": PATH_BYTES[w["dtype"]],
                     "avg_launch_ms": per_launch_s * 1e3,
                     "limiter": limiter},
        "stage_roofline": {"kernel": dom, "alg_bytes_per_vertex": STAGE_BYTES[dom][w["dtype"]],
                           "achieved": stage_gbs, "peak": hbm, "unit": "GB/s",
                           "frac": None if stage_gbs is None else stage_gbs / hbm},
        "path_roofline": {"alg_bytes_per_vertex": PATH_BYTES[w["dtype"]], "achieved": path_gbs,
                          "peak": hbm, "unit": "GB/s", "frac": path_gbs / hbm},
        "issue_roofline": issue,
        "step_ms": step_stats,
        "stages_ms_per_step": {k: v["ms"] / max(1, prof["calls"]) for k, v in stages.items()
                               if v["launches"] or v["ms"]},
        "gpu_launches": prof["launches"],
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": "vertices/s", "h2d_bytes_per_step": n * esz,
            "d2h_bytes_per_step": 3 * n * 4,
            "api": f"ms_segment_host_many over {args.e2e_steps} steps, pinned host buffers (each step's "
                   "upload and label download overlap the neighbouring steps' work)",
            "single_call": {"value": e2e_single, "unit": "vertices/s",
                            "api": "ms_segment_host, one synchronous call a step"}},
        "clocks": clocks,
    }
    ms.ms_destroy(ctx)
    del field, asc, desc, msid
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
        line["cpu_parallel_baseline"] = cpu_parallel_baseline(args)
    if rank == 0 and ws == 1 and args.workload == "noise512" and not args.no_extras:
        # the metric's other halves, measured in the same run: the quantised
        # 512^3 variant, the 256-field batch and the request loop
        line["quantised"] = extra("quantised", lambda: quantised_summary(args, f_np))
        line["batched"] = extra("batched", lambda: batched_summary(args))
        line["served"] = extra("served", lambda: served_summary(args))
        line["persistence"] = extra("persistence", lambda: persistence_summary(args, f_np))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
