"""Benchmark of the octree-construction hot path (one step = every stage of one
plain build: bounds + preview, count grid, chunk merge, stable distribution,
chunk octrees + LOD selection, final LOD layout) on synthetic clouds.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is whole-job throughput in Gpts/s with
the cloud resident in HBM (N GPUs build N replicas: weak scaling, no data-path
collective); `e2e` is the same metric through the C-ABI calls with the input in
pinned host memory copied in and the node table read back every step.  The
workload defaults to the 1B-point uniform cloud (10^9 points, g = 7, s = 7,
L_max = 8, T = 5e6, C = 5e4), the largest single-GPU configuration; the
roofline names the kernel with the largest device time in the step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator, n, seed, grid_log2, sub_log2, max_level, chunk_threshold, node_capacity)
    "lidar-100M": ("lidar", 100_000_000, 2, 7, 7, 15, 100_000, 20_000),
    "uniform-1M": ("uniform", 1_000_000, 1, 7, 7, 15, 100_000, 20_000),
    "uniform-1B": ("uniform", 1_000_000_000, 3, 7, 7, 8, 5_000_000, 50_000),
    "lidar-10M": ("lidar", 10_000_000, 2, 7, 7, 15, 100_000, 20_000),
    # the 1B parameters at 100M points: 512 chunks (the one-sweep distribution), 1.6 GB resident
    "uniform-100M": ("uniform", 100_000_000, 3, 7, 7, 8, 500_000, 50_000),
    # 256 clouds, sizes log-uniform in [1e4, 2e7], uniform or LiDAR generator per cloud (seed 1000 + i)
    "batched-256": ("batch", 256, 1000, 7, 7, 15, 100_000, 20_000),
    # 32 LiDAR requests, sizes log-uniform in [1e6, 5e8], Poisson arrivals 4/s, 24 GB device budget (seed 5000 + i)
    "served-32": ("served", 32, 5000, 7, 7, 15, 100_000, 20_000),
    # spatially constrained random preview of the 100M LiDAR cloud: one point per occupied level-7 cell
    "spatial-preview-100M": ("spatial", 100_000_000, 2, 7, 7, 15, 100_000, 20_000),
    # headless frame of the 100M LiDAR octree: node selection + rasterisation at 1920x1080
    "render-100M": ("render", 100_000_000, 2, 7, 7, 15, 100_000, 20_000),
}
DEFAULT_WORKLOAD = "uniform-1B"
RENDER_W, RENDER_H, RENDER_MIN_PX = 1920, 1080, 30.0
STAGES = ["bounds_decimate", "count", "merge", "distribute", "octree", "subsample"]
# the method's mandatory HBM bytes per point (read and write passes of its
# definition): bounds + preview 17 (read 16; a 16-byte record for 1 point in
# 16), count 16, distribute 32 (read 16, write 16), chunk octrees + LOD 32 (one
# read and one final write of each point) -- 97 in all -- plus the count grid's
# fixed 3 * 4 * 8^g bytes (written, read by the merge, LUT written)
ALG_PER_POINT = 97
FIXED_BYTES = {"merge": 3 * 4 * (1 << 21)}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one call's
# launches of a kernel, from one ncu capture of the workload, valid while the
# sources that kernel is built from hash to the recorded value (a changed
# kernel reports null)
_COMMON = ["fp_common.cuh", "fp_internal.cuh", "fp_scan.cuh"]   # (fp_api.cu: argument checks, no kernel)
_OCT = _COMMON + ["fp_sort.cuh", "fp_seg.cuh", "fp_octree.cu"]
KERNEL_FILES = {
    "bounds_decimate": _COMMON + ["fp_core.cu"],
    "count": _COMMON + ["fp_core.cu"],
    "distribute": _COMMON + ["fp_sort.cuh", "fp_seg.cuh", "fp_sort.cu", "fp_seg.cu"],
    "cell_group": _OCT, "units": _OCT, "resolve": _OCT,
    "owner_scatter": _OCT + ["fp_seg.cu"],
}
# uniform-100M: one-kernel captures of the first launch (the distribution: its counting
# pass and sweep; the table and scan launches move under 20 MB), with the hash of the
# kernel's sources at the capture (profiles/kernels_uniform100M.md); uniform-1B has the
# same per-point structure (512 chunks, the same node levels) and ten times the points
_T100 = {"bounds_decimate": (1.698e9, "745ecb4644c62907"), "count": (1.977e9, "745ecb4644c62907"),
         "distribute": (0.617e9 + 3.803e9, "6f0641cb0d48e153"),
         "cell_group": (4.424e9, "f33f4efb97ca77c1"), "units": (2.467e9, "f33f4efb97ca77c1"),
         "resolve": (0.844e9, "f33f4efb97ca77c1"), "owner_scatter": (3.806e9, "78b841f4a17e80b4")}
NCU_TRAFFIC = {}
for _k, (_b, _h) in _T100.items():
    NCU_TRAFFIC[("uniform-100M", _k)] = (_b, _h)
    NCU_TRAFFIC[("uniform-1B", _k)] = (10 * _b, _h)


def sources_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_FILES[kernel]:
        with open(os.path.join(ROOT, "paper_2302_05002_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel):
    rec = NCU_TRAFFIC.get((workload, kernel))
    if rec is None:
        return None
    try:
        return rec[0] if sources_hash(kernel) == rec[1] else None
    except OSError:
        return None


def replica_rate(ms, n, world, device):
    """Replicas only (every rank builds its own cloud of n points, nothing is
    exchanged): the step time of the job is the slowest rank's, and the job
    processed n * world points in it.  Returns (max ms over ranks, Gpts/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, n * world / (ms * 1e-3) / 1e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def count_kernels_captured(run, stream):
    """Kernels one call of run() enqueues: the call is captured into a CUDA graph
    (relaxed mode; nothing executes) and the graph's kernel nodes are counted."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so.13")
    h = ctypes.c_void_p(stream.cuda_stream)
    if rt.cudaStreamBeginCapture(h, ctypes.c_int(2)) != 0:   # cudaStreamCaptureModeRelaxed
        raise RuntimeError("begin capture failed")
    graph = ctypes.c_void_p()
    try:
        run()
    finally:
        rc = rt.cudaStreamEndCapture(h, ctypes.byref(graph))
    if rc != 0 or not graph.value:
        rt.cudaGetLastError()
        raise RuntimeError("capture failed (%d)" % rc)
    try:
        num = ctypes.c_size_t(0)
        if rt.cudaGraphGetNodes(graph, None, ctypes.byref(num)) != 0:
            raise RuntimeError("graph nodes query failed")
        nodes = (ctypes.c_void_p * max(1, num.value))()
        if rt.cudaGraphGetNodes(graph, nodes, ctypes.byref(num)) != 0:
            raise RuntimeError("graph nodes query failed")
        kernels = 0
        for i in range(num.value):
            t = ctypes.c_int(-1)
            if rt.cudaGraphNodeGetType(ctypes.c_void_p(nodes[i]), ctypes.byref(t)) == 0 and t.value == 0:
                kernels += 1   # cudaGraphNodeTypeKernel
        return kernels
    finally:
        rt.cudaGraphDestroy(graph)


def count_kernels(run, torch, stream=None):
    """Kernels one call of run() launches: counted from a captured graph when
    possible, else from the profiler's device activity."""
    if stream is not None:
        try:
            k = count_kernels_captured(run, stream)
            torch.cuda.synchronize()
            if k:
                return k
        except Exception as ex:
            print("gpu_launches: capture count failed: %r" % (ex,), file=sys.stderr)
            torch.cuda.synchronize()
    try:
        from torch.profiler import ProfilerActivity, profile
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]) as pr:
            run()
            torch.cuda.synchronize()
        names = []
        for e in pr.events():
            dt = getattr(e, "device_type", None)
            if dt is None or "CUDA" not in str(dt):
                continue
            if e.name.startswith(("Memset", "Memcpy", "cuda", "Activity")):
                continue
            names.append(e.name)
        if not names:
            print("gpu_launches: profiler saw no kernels", file=sys.stderr)
            return None
        return len(names)
    except Exception as ex:  # reported, not fatal: the count is informational
        print("gpu_launches: profiler failed: %r" % (ex,), file=sys.stderr)
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_cloud(kind, n, seed, out_tensor):
    import synth
    if kind == "lidar":
        synth.lidar_into(out_tensor.data_ptr(), n, seed)
    else:
        synth.uniform_into(out_tensor.data_ptr(), n, seed)


def oracle_rate(kind, seed, wl, budget_s):
    """Oracle (single thread, plain C) on the first points of the same workload:
    returns (points/s, sample size, seconds, cores)."""
    import numpy as np

    import oracle
    import synth
    _, _, _, g, s, lmax, T, C = wl
    prm = oracle.params(g, s, lmax, 16, T, C)
    gen = synth.lidar if kind == "lidar" else synth.uniform
    n = 20_000
    while True:
        pts = gen(n, seed)
        t0 = time.perf_counter()
        oracle.build_all(pts, prm)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 8 or n >= min(4_000_000, wl[1]):
            break
        n = int(min(4_000_000, wl[1], n * max(2.0, budget_s / 4 / max(dt, 1e-3))))
    return n / dt, n, dt, 1


def run_reference(args, wl, rank):
    if rank != 0:
        return
    kind, n, seed = wl[0], wl[1], wl[2]
    budget = float(os.environ.get("FP_ORACLE_BUDGET_S", "12"))
    rates, samples = [], []
    for _ in range(args.warmup):
        oracle_rate(kind, seed, wl, budget / 4)
    for _ in range(args.steps):
        r, ns, dt, cores = oracle_rate(kind, seed, wl, budget)
        rates.append(r)
        samples.append(ns)
    v = statistics.median(rates) / 1e9
    line = {"impl": "reference", "metric": "octree build throughput (Gpts/s)", "value": v, "unit": "Gpts/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "points": n},
            "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
                             "sample": "first %d points of the %s workload, same parameters" % (samples[-1], args.workload)},
            "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched workload
def batch_sizes(count, seed):
    """Cloud sizes log-uniform in [1e4, 2e7] and generator per cloud, from a seeded generator."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(1e4), np.log(2e7), count))).astype(np.int64)
    kinds = np.where(rng.random(count) < 0.5, "uniform", "lidar")
    return [int(x) for x in sizes], [str(k) for k in kinds]


def run_batched(args, wl, rank, world, local):   # returns the JSON line (rank 0)
    """256 clouds built three ways on the same GPU: the plain calls cloud after
    cloud on one stream; fp_build_batched on lanes (every pass per cloud); and
    fp_build_batched_ex with the tuner's options (grid per cloud, lanes, fused
    first passes, their block and table sizes), each batch captured into one
    CUDA graph.  value = all points / tuned batched time."""
    import torch

    from paper_2302_05002_gb300 import fastpoints as fp
    from paper_2302_05002_gb300 import tune

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _, count, seed0, g, s, lmax, T, C = wl
    sizes, kinds = batch_sizes(count, seed0)
    total = sum(sizes)
    base = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T, node_capacity=C)
    host = []
    for i, (n, kind) in enumerate(zip(sizes, kinds)):
        h = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
        make_cloud(kind, n, seed0 + i, h)
        host.append(h)
    pts = [h.to(dev) for h in host]
    st = torch.cuda.Stream(dev)

    # plain: the seven calls per cloud, one cloud after another, one stream, configured grid
    plain_clouds = [(p, base) for p in pts]
    plain_outs = [fp.cloud_outputs(p, base) for p in pts]
    plain_descs = fp.batch_descs(plain_clouds, plain_outs)
    ws_plain = torch.empty(max(fp.batch_workspace_size(plain_descs, count, 1), 1), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def run_plain():
        for i in range(count):
            fp.plain_calls(plain_descs[i], ws_plain, stream=st)

    # batched: grid per cloud by the tuner, lanes by the tuner, one graph
    def sample(n):
        h = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
        make_cloud("lidar", n, 999, h)
        return h.to(dev)

    tuner = tune.BatchTuner(sample, stream=st)
    clouds = tuner.tune_params(plain_clouds)
    outs = [fp.cloud_outputs(p, prm) for p, prm in clouds]
    descs = fp.batch_descs(clouds, outs)
    ws_need = max(max(fp.batch_workspace_size(descs, count, L) for L in (4, 8, 16, 32)),
                  max(fp.batch_workspace_size_ex(descs, count, fp.batch_opts(L, 1)) for L in (4, 8, 16, 32)))
    ws = torch.empty(max(ws_need, 1), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()   # the outputs' zero fills (default stream) land before the lanes write them
    lanes = tuner.tune_lanes(lambda L: fp.fp_build_batched(descs, count, L, ws, stream=st))
    opts = tuner.tune_opts(lambda o: fp.fp_build_batched_ex(descs, count, o, ws, stream=st), lanes)

    def capture(o):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=st, capture_error_mode="relaxed"):
            fp.fp_build_batched_ex(descs, count, o, ws, stream=st)
        return gr

    graph = capture(opts)
    lanes_opts = fp.batch_opts(lanes, 0)   # the lanes alone (every pass per cloud), for comparison
    graph_lanes = capture(lanes_opts)

    for _ in range(max(3, args.warmup)):
        run_plain()
        graph_lanes.replay()
        graph.replay()
    torch.cuda.synchronize()
    assert fp.get_device_error(stream=st) == 0, "device error word set"
    # every cloud's octree equals the plain build's (the grid changes only the chunking)
    same = True
    for o, r in zip(outs, plain_outs):
        M = int(r["num_nodes"].item())
        same &= M == int(o["num_nodes"].item()) and torch.equal(o["nodes"][:M], r["nodes"][:M]) and \
            torch.equal(o["final_perm"], r["final_perm"])
    assert same, "batched octrees differ from the plain builds"

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        e0.record(st)
        for _ in range(args.steps):
            run_plain()
        e1.record(st)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / args.steps

    with torch.cuda.stream(st):
        e0.record(st)
        for _ in range(args.steps):
            graph_lanes.replay()
        e1.record(st)
    torch.cuda.synchronize()
    lanes_ms = e0.elapsed_time(e1) / args.steps

    launches = count_kernels(lambda: fp.fp_build_batched_ex(descs, count, opts, ws, stream=st), torch, st)
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    with torch.cuda.stream(st):
        e0.record(st)
        for _ in range(args.steps):
            graph.replay()
        e1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    value = total / (ms * 1e-3) / 1e9
    plain_value = total / (plain_ms * 1e-3) / 1e9

    # end to end: every cloud copied in from pinned host memory, batch, node tables read back
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        with torch.cuda.stream(st):
            for p, h in zip(pts, host):
                p.copy_(h, non_blocking=True)
            fp.fp_build_batched_ex(descs, count, opts, ws, stream=st)
            nums = torch.stack([o["num_nodes"][0] for o in outs]).cpu()
            d2h = 0
            for o, M in zip(outs, nums.tolist()):
                o["nodes"][:M].cpu()
                d2h += M * 40 + 4
            st.synchronize()
    e2e_ms = (time.perf_counter() - te0) * 1e3 / e2e_steps
    peak, peak_kind = measured_peaks()
    alg = ALG_PER_POINT * total + FIXED_BYTES["merge"] * count
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = batch_oracle_rate(sizes, kinds, seed0, wl, float(os.environ.get("FP_ORACLE_BUDGET_S", "12")))
        gs = {}
        for _, prm in clouds:
            gs[prm.grid_log2] = gs.get(prm.grid_log2, 0) + 1
        line = {
            "metric": "batched octree build throughput (Gpts/s)", "value": value, "unit": "Gpts/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "clouds": count, "points": total, "min_points": min(sizes),
                       "max_points": max(sizes), "lanes": lanes, "grid_log2_per_cloud": gs,
                       "fused_first_passes": bool(opts.fused_first), "count_threads": opts.count_threads,
                       "count_slots": opts.count_slots,
                       "lanes_only_ms_per_step": lanes_ms, "lanes_only_gpts": total / (lanes_ms * 1e-3) / 1e9,
                       "chunk_threshold": T, "node_capacity": C, "max_level": lmax, "sub_log2": s,
                       "plain_ms_per_step": plain_ms, "plain_gpts": plain_value,
                       "batched_over_plain": value / plain_value, "graph": "one CUDA graph per batch",
                       "l2": "inputs (%.1f GB) larger than L2" % (16 * total / 1e9)},
            "e2e": {"value": total / (e2e_ms * 1e-3) / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": 16 * total,
                    "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "hbm", "kernel": "whole batch", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": alg / (ms * 1e-3) / 1e9 / peak,
                         "traffic": None, "alg_bytes_per_launch": alg},
            "clocks": clocks,
            "gpu_launches": launches * args.steps if launches else None,
            "cpu_baseline": cpu,
            "tuner": tuner.log[-12:],
        }
        return line


def batch_oracle_rate(sizes, kinds, seed0, wl, budget_s):
    """Oracle (single thread) over the batch's clouds, smallest first, within the budget."""
    import oracle
    import synth
    _, _, _, g, s, lmax, T, C = wl
    prm = oracle.params(g, s, lmax, 16, T, C)
    done, t_all, used = 0, 0.0, 0
    for i in sorted(range(len(sizes)), key=lambda k: sizes[k]):
        gen = synth.lidar if kinds[i] == "lidar" else synth.uniform
        pts = gen(sizes[i], seed0 + i)
        t0 = time.perf_counter()
        oracle.build_all(pts, prm)
        t_all += time.perf_counter() - t0
        done += sizes[i]
        used += 1
        if t_all >= budget_s:
            break
    return {"value": done / t_all / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
            "sample": "the %d smallest clouds of the batch (%d points), %.1f s" % (used, done, t_all)}


def run_batched_reference(args, wl, rank):
    if rank != 0:
        return
    sizes, kinds = batch_sizes(wl[1], wl[2])
    budget = float(os.environ.get("FP_ORACLE_BUDGET_S", "12"))
    rates = []
    for _ in range(args.warmup):
        batch_oracle_rate(sizes, kinds, wl[2], wl, budget / 4)
    for _ in range(args.steps):
        cpu = batch_oracle_rate(sizes, kinds, wl[2], wl, budget)
        rates.append(cpu["value"])
    v = statistics.median(rates)
    cpu["value"] = v
    line = {"impl": "reference", "metric": "batched octree build throughput (Gpts/s)", "value": v,
            "unit": "Gpts/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "clouds": wl[1], "points": sum(sizes)}, "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ served workload
def run_spatial(args, wl, rank, world, local):
    """Bounds + spatially constrained preview (fp_bounds, fp_preview_spatial) of
    a resident cloud per step; e2e adds the cloud's copy in and the preview's
    copy out."""
    import torch

    from paper_2302_05002_gb300 import fastpoints as fp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _, n, seed, level = wl[0], wl[1], wl[2], wl[3]
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    make_cloud("lidar", n, seed, host)
    pts = host.to(dev)
    st = torch.cuda.Stream(dev)
    cap = min(n, 1 << (3 * level))
    out = torch.empty((cap, 4), dtype=torch.int32, device=dev)
    cube = torch.empty(8, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    prm = fp.params(grid_log2=level, sub_log2=level, max_level=level)
    ws = torch.empty(max(fp.workspace_size("preview_spatial", n, prm), fp.workspace_size("bounds", n)),
                     dtype=torch.uint8, device=dev)
    L, P, S = fp.load(), fp._ptr, fp._stream(st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(src, record=False):
        if record:
            ev[0].record(st)
        fp._check(L.fp_bounds(P(src), n, P(cube), P(ws), ws.numel(), S), "fp_bounds")
        if record:
            ev[1].record(st)
        fp._check(L.fp_preview_spatial(P(src), n, P(cube), level, 0, P(out), cap, P(cnt), P(ws), ws.numel(), S),
                  "fp_preview_spatial")
        if record:
            ev[2].record(st)

    for _ in range(max(3, args.warmup)):
        step(pts)
    torch.cuda.synchronize()
    assert fp.get_device_error(stream=st) == 0
    launches = count_kernels(lambda: step(pts), torch, st)
    clk = ClockSampler(local)
    clk.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sp_ms = []
    t0.record(st)
    for _ in range(args.steps):
        step(pts, True)
        st.synchronize()
        sp_ms.append(ev[1].elapsed_time(ev[2]))
    t1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1) / args.steps
    k = int(cnt.item())
    # e2e: pinned cloud in, preview out
    e2e_pts = torch.empty_like(pts)
    out_host = torch.empty((cap, 4), dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    te = time.perf_counter()
    reps = max(1, min(args.steps, 3))
    for _ in range(reps):
        with torch.cuda.stream(st):
            e2e_pts.copy_(host, non_blocking=True)
            step(e2e_pts)
            kk = int(cnt.item())
            out_host[:kk].copy_(out[:kk], non_blocking=True)
            st.synchronize()
    e2e_ms = (time.perf_counter() - te) * 1e3 / reps
    peak, peak_kind = measured_peaks()
    sp = statistics.median(sp_ms)
    alg = 32 * n + 16 * k + 2 * 8 * (1 << (3 * level))   # two reads of the cloud, the kept points, the table
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = spatial_oracle_rate(n, seed, level, float(os.environ.get("FP_ORACLE_BUDGET_S", "12")))
        line = {
            "metric": "spatial preview throughput (Gpts/s)", "value": n / (ms * 1e-3) / 1e9, "unit": "Gpts/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "points": n, "level": level, "kept": k,
                       "parallelism": "single", "l2": "inputs (%.1f GB) larger than L2" % (16 * n / 1e9)},
            "e2e": {"value": n / (e2e_ms * 1e-3) / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 16 * k + 8},
            "roofline": {"bound": "hbm", "kernel": "fp_preview_spatial (cell minima + compaction)",
                         "achieved": alg / (sp * 1e-3) / 1e9, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": alg / (sp * 1e-3) / 1e9 / peak, "traffic": None, "alg_bytes_per_launch": alg},
            "stage_ms": {"bounds": ms - sp, "preview_spatial": sp},
            "clocks": clocks, "gpu_launches": launches * args.steps if launches else None, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def render_camera(fp, host_np):
    import numpy as np
    lo = np.array([host_np[:, a].min() for a in range(3)], np.float64)
    hi = np.array([host_np[:, a].max() for a in range(3)], np.float64)
    c, size = (lo + hi) / 2, float((hi - lo).max())
    m = fp.view_projection(c + np.array([0.45, -0.6, 0.25]) * size, c, fovy_deg=60, aspect=RENDER_W / RENDER_H,
                           near=size * 1e-3, far=size * 10)
    return fp.camera(m, RENDER_W, RENDER_H, RENDER_MIN_PX), m


def run_render(args, wl, rank, world, local):
    """One headless frame per step of the resident octree of the 100M LiDAR
    cloud: fp_select_nodes + fp_rasterize at 1920x1080.  value = drawn points
    per second; e2e adds reading the framebuffer back to the host."""
    import torch

    from paper_2302_05002_gb300 import fastpoints as fp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _, n, seed, g, s, lmax, T, C = wl
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    make_cloud("lidar", n, seed, host)
    pts = host.to(dev)
    prm = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T, node_capacity=C)
    r = fp.build_octree(pts, prm)
    torch.cuda.synchronize()
    M = int(r["num_nodes"].item())
    nodes = r["nodes"][:M].contiguous()
    cam, m = render_camera(fp, host.numpy())
    st = torch.cuda.Stream(dev)
    ws = torch.empty(fp.render_workspace_size(M), dtype=torch.uint8, device=dev)
    fb = torch.empty((RENDER_H, RENDER_W), dtype=torch.int64, device=dev)
    ids = torch.empty(M, dtype=torch.int32, device=dev)
    nsel = torch.zeros(1, dtype=torch.int32, device=dev)
    npts = torch.zeros(1, dtype=torch.int64, device=dev)
    L, P, S = fp.load(), fp._ptr, fp._stream(st)
    import ctypes
    cref = ctypes.byref(cam)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(record=False):
        if record:
            ev[0].record(st)
        fp._check(L.fp_select_nodes(P(nodes), P(r["num_nodes"]), M, P(r["cube"]), cref, P(ids), P(nsel), P(npts),
                                    P(ws), ws.numel(), S), "fp_select_nodes")
        if record:
            ev[1].record(st)
        fp._check(L.fp_rasterize(P(nodes), P(ids), P(nsel), M, P(r["final"]), n, cref, P(fb), P(ws), ws.numel(), S),
                  "fp_rasterize")
        if record:
            ev[2].record(st)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    assert fp.get_device_error(stream=st) == 0
    launches = count_kernels(lambda: step(), torch, st)
    drawn = int(npts.item())
    clk = ClockSampler(local)
    clk.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sel_ms, ras_ms = [], []
    t0.record(st)
    for _ in range(args.steps):
        step(True)
        st.synchronize()
        sel_ms.append(ev[0].elapsed_time(ev[1]))
        ras_ms.append(ev[1].elapsed_time(ev[2]))
    t1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = t0.elapsed_time(t1) / args.steps
    fb_host = torch.empty((RENDER_H, RENDER_W), dtype=torch.int64, pin_memory=True)
    te = time.perf_counter()
    reps = max(1, min(args.steps, 5))
    for _ in range(reps):
        with torch.cuda.stream(st):
            step()
            fb_host.copy_(fb, non_blocking=True)
            st.synchronize()
    e2e_ms = (time.perf_counter() - te) * 1e3 / reps
    peak, peak_kind = measured_peaks()
    ras = statistics.median(ras_ms)
    alg = 16 * drawn + 2 * 8 * RENDER_W * RENDER_H + 40 * M   # drawn points, framebuffer set + read-modify, nodes
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = render_oracle_rate(fp, r, M, m)
        line = {
            "metric": "rendered points per second (Gpts/s)", "value": drawn / (ms * 1e-3) / 1e9, "unit": "Gpts/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {"workload": args.workload, "points": n, "nodes": M, "drawn_nodes": int(nsel.item()),
                       "drawn_points": drawn, "width": RENDER_W, "height": RENDER_H, "min_node_px": RENDER_MIN_PX,
                       "fps": 1e3 / ms, "parallelism": "single",
                       "l2": "drawn points (%.2f GB) larger than L2" % (16 * drawn / 1e9)},
            "e2e": {"value": drawn / (e2e_ms * 1e-3) / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 8 * RENDER_W * RENDER_H},
            "roofline": {"bound": "hbm", "kernel": "fp_rasterize", "achieved": alg / (ras * 1e-3) / 1e9, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": alg / (ras * 1e-3) / 1e9 / peak,
                         "traffic": None, "alg_bytes_per_launch": alg},
            "stage_ms": {"select": statistics.median(sel_ms), "rasterize": ras},
            "clocks": clocks, "gpu_launches": launches * args.steps if launches else None, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def render_oracle_rate(fp, r, M, m):
    """The oracle's selection and rasterisation of the same frame (node table
    and final points copied to the host)."""
    import numpy as np

    import oracle
    nodes = fp.nodes_to_host(r["nodes"], r["num_nodes"])
    fin = r["final"].cpu().numpy().view(np.uint8).reshape(-1, 16).copy().view(oracle.POINT).reshape(-1)
    cube = r["cube"].cpu().numpy().view(np.uint8).copy().view(oracle.CUBE)
    cam = oracle.camera(m, RENDER_W, RENDER_H, RENDER_MIN_PX)
    t0 = time.perf_counter()
    sel = oracle.render_select(nodes, cube, cam)
    oracle.rasterize(nodes, sel, fin, cam)
    dt = time.perf_counter() - t0
    drawn = int(nodes["n_own"][sel].astype(np.int64).sum())
    return {"value": drawn / dt / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
            "sample": "the whole frame (%d drawn points), %.1f s" % (drawn, dt)}


def run_render_reference(args, wl, rank):
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth
    from paper_2302_05002_gb300 import fastpoints as fp
    # the oracle builds a bounded prefix of the cloud and renders one frame of it
    n = 2_000_000
    pts = synth.lidar(n, wl[2])
    _, _, _, g, s, lmax, T, C = wl
    cube = oracle.bounds(pts)
    t = oracle.octree_lod(pts, cube, oracle.params(g, s, lmax, 16, T, C))
    _, m = render_camera(fp, pts.view(np.int32).reshape(-1, 4))
    cam = oracle.camera(m, RENDER_W, RENDER_H, RENDER_MIN_PX)
    rates = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        sel = oracle.render_select(t["nodes"], cube, cam)
        oracle.rasterize(t["nodes"], sel, t["final_pts"], cam)
        dt = time.perf_counter() - t0
        rates.append(int(t["nodes"]["n_own"][sel].astype(np.int64).sum()) / dt / 1e9)
    v = statistics.median(rates)
    print(json.dumps({"impl": "reference", "metric": "rendered points per second (Gpts/s)", "value": v,
                      "unit": "Gpts/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "fp32", "data": "synthetic",
                      "config": {"workload": args.workload, "points": wl[1], "width": RENDER_W, "height": RENDER_H},
                      "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
                                       "sample": "one frame of the octree of the first %d points" % n},
                      "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def spatial_oracle_rate(n, seed, level, budget_s):
    import oracle
    import synth
    m = 1_000_000
    while True:
        pts = synth.lidar(m, seed)
        t0 = time.perf_counter()
        oracle.preview_spatial(pts, oracle.bounds(pts), level)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 4 or m >= min(n, 64_000_000):
            break
        m *= 2
    return {"value": m / dt / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
            "sample": "first %d points of the LiDAR cloud, bounds + spatial preview, %.1f s" % (m, dt)}


def run_spatial_reference(args, wl, rank):
    if rank != 0:
        return
    budget = float(os.environ.get("FP_ORACLE_BUDGET_S", "12"))
    rates = [spatial_oracle_rate(wl[1], wl[2], wl[3], budget / 2)["value"] for _ in range(max(1, args.steps))]
    v = statistics.median(rates)
    cpu = spatial_oracle_rate(wl[1], wl[2], wl[3], budget / 2)
    print(json.dumps({"impl": "reference", "metric": "spatial preview throughput (Gpts/s)", "value": v,
                      "unit": "Gpts/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "int32", "data": "synthetic",
                      "config": {"workload": args.workload, "points": wl[1], "level": wl[3]},
                      "cpu_baseline": dict(cpu, value=v),
                      "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def served_plan(count, seed):
    """Request sizes (log-uniform in [1e6, 5e8]) and arrival offsets (Poisson, 4/s)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(1e6), np.log(5e8), count))).astype(np.int64)
    arrivals = np.cumsum(rng.exponential(0.25, count)) - 0.25
    return [int(x) for x in sizes], [max(0.0, float(t)) for t in arrivals]


def host_mem_available():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return None


def run_served(args, wl, rank, world, local):   # returns the JSON line (rank 0)
    """Poisson-arriving LiDAR clouds served under a 24 GB device budget
    (serve.Server): p50/p99 time to preview and to the full octree, aggregate
    points/s; the same clouds submitted at once (saturated); and the plain
    per-cloud builds back to back (copy in, seven calls) on the same GPU."""
    import torch

    from paper_2302_05002_gb300 import fastpoints as fp
    from paper_2302_05002_gb300 import serve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _, count, seed0, g, s, lmax, T, C = wl
    sizes, arrivals = served_plan(count, seed0)
    note = None
    avail = host_mem_available()
    need = sum(sizes) * 18 + 40 * max(sizes)
    if avail is not None and need > 0.7 * avail:   # shrink every cloud alike to fit the host
        f = 0.7 * avail / need
        sizes = [max(1_000_000, int(x * f)) for x in sizes]
        note = "sizes scaled by %.3f to fit %.0f GB of host memory" % (f, avail / 1e9)
    budget, piece = 24 << 30, 1 << 23

    def prm_for(n):
        return fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16,
                         chunk_threshold=5_000_000 if n >= 200_000_000 else T, node_capacity=C)

    hosts, prev_bufs, prms = [], [], []
    for i, n in enumerate(sizes):
        h = torch.empty((n, 4), dtype=torch.int32).pin_memory()
        make_cloud("lidar", n, seed0 + i, h)
        hosts.append(h)
        prms.append(prm_for(n))
        prev_bufs.append(torch.empty(serve.preview_slots_shape(n, piece, 16), dtype=torch.int32).pin_memory())
    ooc = [n for n, p in zip(sizes, prms) if serve.incore_need(n, p) > budget * 3 // 4]
    ooc_max = max(ooc) if ooc else 0
    ooc_prm = prm_for(ooc_max) if ooc_max else None

    srv_pools = serve.Server(budget_bytes=budget, piece_points=piece, device=local, ooc_max_points=ooc_max,
                             ooc_prm=ooc_prm)   # pinned host pools, made once before the clock
    srv_pools.close()
    pools = srv_pools.ooc_free

    def serve_run(offsets, one_at_a_time=False):
        srv = serve.Server(budget_bytes=budget, piece_points=piece, device=local, ooc_slots=0)
        srv.ooc_free, srv.ooc_slots = list(pools), len(pools)
        reqs = [serve.Request(i, hosts[i], prms[i], preview_host=prev_bufs[i]) for i in range(count)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, (r, off) in enumerate(zip(reqs, offsets)):
            wait = t0 + off - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            srv.submit(r)
            if one_at_a_time:
                srv.drain(i + 1)
        srv.drain(count)
        srv.close()
        errs = [r.error for r in reqs if r.error]
        assert not errs, errs[0]
        t_end = max(r.t_done for r in reqs)
        for r in reqs:
            r.result = None
        torch.cuda.empty_cache()
        return reqs, t0, t_end, srv.peak_active

    # warm: the smallest request alone
    k = min(range(count), key=lambda i: sizes[i])
    srv = serve.Server(budget_bytes=budget, piece_points=piece, device=local)
    r = serve.Request(k, hosts[k], prms[k], preview_host=prev_bufs[k])
    srv.submit(r)
    srv.drain(1)
    srv.close()
    assert r.error is None, r.error

    clk = ClockSampler(local)
    clk.start()
    reqs, t0, t_end, peak = serve_run(arrivals)
    clocks = clk.stop()
    ttp = [(r.t_preview - r.arrival) * 1e3 for r in reqs]
    ttf = [(r.t_done - r.arrival) * 1e3 for r in reqs]
    total = sum(sizes)
    served_rate = total / (t_end - t0)
    sreqs, s0, s_end, speak = serve_run([0.0] * count)
    saturated_rate = total / (s_end - s0)
    # the same requests through the same budgeted path, one after another
    breqs, b0, b_end, _ = serve_run([0.0] * count, one_at_a_time=True)
    budget_plain_rate = total / (b_end - b0)

    # plain: each cloud in turn, copied in, the seven calls, resident result
    torch.cuda.synchronize()
    tp0 = time.perf_counter()
    for h, p in zip(hosts, prms):
        pts = h.to(dev, non_blocking=True)
        r = fp.build_octree(pts, p)
        del r, pts
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - tp0
    torch.cuda.empty_cache()
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = served_oracle_rate(sizes, seed0, wl, float(os.environ.get("FP_ORACLE_BUDGET_S", "12")))
        p50 = serve.percentile(ttp, 0.5)
        line = {
            "metric": "served time to preview p50 (ms)", "value": p50, "unit": "ms", "n_gpus": world,
            "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "requests": count, "points": total, "min_points": min(sizes),
                       "max_points": max(sizes), "arrival_rate_per_s": 4, "budget_gb": budget / 2 ** 30,
                       "piece_points": piece, "out_of_core_requests": len(ooc), "peak_in_flight": peak,
                       "size_note": note,
                       "l2": "inputs (%.1f GB) larger than L2" % (16 * total / 1e9)},
            "served": {"time_to_preview_ms": {"p50": p50, "p99": serve.percentile(ttp, 0.99)},
                       "time_to_full_octree_ms": {"p50": serve.percentile(ttf, 0.5),
                                                  "p99": serve.percentile(ttf, 0.99)},
                       "aggregate_gpts": served_rate / 1e9, "span_s": t_end - t0},
            "saturated": {"aggregate_gpts": saturated_rate / 1e9, "peak_in_flight": speak,
                          "span_s": s_end - s0},
            "plain_budgeted": {"aggregate_gpts": budget_plain_rate / 1e9, "span_s": b_end - b0,
                               "note": "the same requests and path under the same budget, one at a time"},
            "served_over_plain_budgeted": saturated_rate / budget_plain_rate,
            "plain": {"aggregate_gpts": total / plain_s / 1e9, "span_s": plain_s,
                      "note": "per cloud: copy in, the seven calls in core without the budget, one after another"},
            "e2e": {"value": saturated_rate / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": 16 * total,
                    "d2h_bytes_per_step": None},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        return line


def served_oracle_rate(sizes, seed0, wl, budget_s):
    import oracle
    import synth
    _, _, _, g, s, lmax, T, C = wl
    prm = oracle.params(g, s, lmax, 16, T, C)
    i = min(range(len(sizes)), key=lambda k: sizes[k])
    n = min(sizes[i], 2_000_000)
    pts = synth.lidar(n, seed0 + i)
    t0 = time.perf_counter()
    oracle.build_all(pts, prm)
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e9, "unit": "Gpts/s", "cores": 1, "kind": "oracle",
            "sample": "first %d points of the smallest request, %.1f s" % (n, dt)}


def run_served_reference(args, wl, rank):
    if rank != 0:
        return
    sizes, _ = served_plan(wl[1], wl[2])
    cpu = served_oracle_rate(sizes, wl[2], wl, float(os.environ.get("FP_ORACLE_BUDGET_S", "12")))
    line = {"impl": "reference", "metric": "served octree build throughput (Gpts/s)", "value": cpu["value"],
            "unit": "Gpts/s", "n_gpus": args.gpus, "steps": 1, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "requests": wl[1]}, "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true",
                    help="the default run without the batched and served summaries")
    ap.add_argument("--quick", action="store_true",
                    help="warm-up and timed steps only (no per-kernel times, leaf-grouped or e2e runs): "
                         "the form the ncu captures use")
    ap.add_argument("--leaf-grouped", action="store_true",
                    help="the timed step also writes the optional leaf-grouped layout")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if wl[0] == "served":
        if args.impl == "reference":
            run_served_reference(args, wl, rank)
        else:
            emit(run_served(args, wl, rank, world, local))
        return
    if wl[0] == "render":
        if args.impl == "reference":
            run_render_reference(args, wl, rank)
        else:
            run_render(args, wl, rank, world, local)
        return
    if wl[0] == "spatial":
        if args.impl == "reference":
            run_spatial_reference(args, wl, rank)
        else:
            run_spatial(args, wl, rank, world, local)
        return
    if wl[0] == "batch":
        if args.impl == "reference":
            run_batched_reference(args, wl, rank)
        else:
            emit(run_batched(args, wl, rank, world, local))
        return
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    line = run_plain(args, wl, rank, world, local)
    if line is not None and world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_extras:
        line["configs"] = extra_configs(args, local)
    emit(line)


def emit(line):
    if line is not None:
        print(json.dumps(line), flush=True)


def extra_configs(args, local):
    """The batched and served workloads, measured in the same run as the
    headline (one GPU): a summary of each one's own line."""
    import copy

    import torch
    out = {}
    for name, fn, keys in (("batched-256", run_batched,
                            ("value", "unit", "ms_per_step", "e2e", "clocks", "gpu_launches", "tuner")),
                           ("served-32", run_served,
                            ("value", "unit", "metric", "served", "saturated", "plain", "plain_budgeted",
                             "served_over_plain_budgeted", "clocks"))):
        torch.cuda.empty_cache()
        sub = copy.copy(args)
        sub.workload, sub.warmup, sub.no_cpu_baseline = name, 3, True
        sub.steps = 3 if name.startswith("batched") else 1
        t0 = time.perf_counter()
        try:
            r = fn(sub, WORKLOADS[name], 0, 1, local)
        except Exception as ex:   # reported in the line; the headline stands
            out[name] = {"error": repr(ex)[:300]}
            continue
        d = {k: r.get(k) for k in keys}
        c = r["config"]
        if name.startswith("batched"):
            d.update({k: c.get(k) for k in ("clouds", "points", "lanes", "fused_first_passes", "count_threads",
                                            "count_slots", "plain_gpts", "lanes_only_gpts", "batched_over_plain")})
        else:
            d.update({k: c.get(k) for k in ("requests", "points", "out_of_core_requests", "peak_in_flight")})
        d["wall_s"] = time.perf_counter() - t0
        out[name] = d
    return out


def kernel_alg_bytes(kernel, n):
    """Algorithmic bytes of one call's launches of a kernel: its share of the
    method's mandatory per-point traffic (97 B/pt in all, plus the 25.2 MB of
    the count grid): bounds + preview 17 (read 16, preview write 1), count 16,
    distribute 32 (read 16, write 16), chunk octrees + LOD 32 (one read and one
    final write of each point) charged to the final-layout scatter, which does
    both.  The other kernels of the octree stage move intermediates only."""
    return {"bounds_decimate": 17, "count": 16, "distribute": 32, "owner_scatter": 32}.get(kernel, 0) * n


def run_plain(args, wl, rank, world, local):
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2302_05002_gb300 import fastpoints as fp

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    kind, n, seed, g, s, lmax, T, C = wl
    prm = fp.params(grid_log2=g, sub_log2=s, max_level=lmax, decim_modulus=16, chunk_threshold=T, node_capacity=C)
    dev = torch.device("cuda", local)

    # input: generated on the host (pinned), copied in once; a replica per rank
    host = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    make_cloud(kind, n, seed, host)
    pts = host.to(dev, non_blocking=False)
    st = torch.cuda.Stream(dev)

    # every output and workspace allocated once
    cells = 1 << (3 * g)
    ncap = fp.node_capacity_bound(n, prm)
    O = dict(
        cube=torch.empty(8, dtype=torch.int32, device=dev),
        prev=torch.empty((fp._preview_cap(n, 16), 4), dtype=torch.int32, device=dev),
        prev_n=torch.zeros(1, dtype=torch.int64, device=dev),
        counts=torch.empty(cells, dtype=torch.int32, device=dev),
        chunks=torch.empty((cells, 2), dtype=torch.int64, device=dev),
        num_chunks=torch.zeros(1, dtype=torch.int32, device=dev),
        lut=torch.empty(cells, dtype=torch.int32, device=dev),
        offsets=torch.empty(cells + 1, dtype=torch.int64, device=dev),
        dist=torch.empty_like(pts), perm=torch.empty(n, dtype=torch.int32, device=dev),
        cells=torch.empty(n, dtype=torch.int32, device=dev),
        nodes=torch.zeros((ncap, 5), dtype=torch.int64, device=dev),
        num_nodes=torch.zeros(1, dtype=torch.int32, device=dev),
        owner=torch.empty(n, dtype=torch.int32, device=dev),
        final=torch.empty_like(pts), final_perm=torch.empty(n, dtype=torch.int32, device=dev),
    )
    leaf = dict(leaf=torch.empty_like(pts), leaf_perm=torch.empty(n, dtype=torch.int32, device=dev)) \
        if args.leaf_grouped else None
    ws_need = max(fp.workspace_size(k, n, prm) for k in ("bounds_decimate", "merge", "distribute", "octree",
                                                         "subsample"))
    ws = torch.empty(ws_need, dtype=torch.uint8, device=dev)
    L = fp.load()
    P = lambda t: fp._ptr(t)
    S = fp._stream(st)
    prm_ref = ctypes.byref(prm)

    def stage_calls(src, with_leaf):
        lp = P(leaf["leaf"]) if with_leaf else None
        lpp = P(leaf["leaf_perm"]) if with_leaf else None
        return [
            ("bounds_decimate", lambda: L.fp_bounds_decimate(P(src), n, P(O["cube"]), 0, 16, P(O["prev"]),
                                                             O["prev"].shape[0], P(O["prev_n"]), P(ws), ws.numel(), S)),
            ("count", lambda: L.fp_count_cells(P(src), n, P(O["cube"]), g, P(O["counts"]), 0, P(O["cells"]), None,
                                               0, S)),
            ("merge", lambda: L.fp_merge_chunks(P(O["counts"]), g, T, P(O["chunks"]), P(O["num_chunks"]),
                                                P(O["lut"]), P(O["offsets"]), P(ws), ws.numel(), S)),
            ("distribute", lambda: L.fp_distribute_cells(P(src), P(O["cells"]), n, P(O["cube"]), g, P(O["lut"]),
                                                         P(O["offsets"]), P(O["num_chunks"]), P(O["dist"]),
                                                         P(O["perm"]), P(ws), ws.numel(), S)),
            ("octree", lambda: L.fp_build_chunk_octree(P(O["dist"]), P(O["perm"]), n, P(O["cube"]), P(O["chunks"]),
                                                       P(O["num_chunks"]), P(O["offsets"]), P(O["counts"]), prm_ref,
                                                       P(O["nodes"]), ncap, P(O["num_nodes"]), lp, lpp,
                                                       P(O["owner"]), P(ws), ws.numel(), S)),
            ("subsample", lambda: L.fp_subsample(P(O["nodes"]), P(O["num_nodes"]), ncap, P(O["dist"]), P(O["perm"]),
                                                 P(O["owner"]), n, P(O["chunks"]), P(O["num_chunks"]),
                                                 P(O["offsets"]), P(O["final"]), P(O["final_perm"]), P(ws),
                                                 ws.numel(), S)),
        ]

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(STAGES) + 1)]

    def step(calls, record=False):
        with torch.cuda.stream(st):
            if record:
                ev[0].record(st)
            for k, (name, f) in enumerate(calls):
                rc = f()
                if rc != 0:
                    raise RuntimeError("%s failed with status %d" % (name, rc))
                if record:
                    ev[k + 1].record(st)

    def capture(calls):
        g_ = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_, stream=st, capture_error_mode="relaxed"):
            step(calls)
        return g_

    calls = stage_calls(pts, False)
    for _ in range(max(3, args.warmup)):
        step(calls)
    torch.cuda.synchronize()
    err = fp.get_device_error(stream=st)
    assert err == 0, "device error word set: %#x (sites %#x)" % (err, fp.get_device_error_sites(stream=st))

    # kernels per step (counted from a captured graph, one step outside the timed region)
    launches_per_step = count_kernels(lambda: step(calls), torch, st)

    # the step captured once into a CUDA graph and replayed: its few hundred
    # launches cost one graph launch (the calls enqueue no host synchronisation)
    graph = capture(calls)
    with torch.cuda.stream(st):
        graph.replay()
    torch.cuda.synchronize()
    assert fp.get_device_error(stream=st) == 0, "device error word set after graph replay"
    # inputs smaller than L2 (129 MB): L2 flushed between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if 16 * n < (256 << 20) else None

    def timed_graph(gr, steps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(steps):
            if flush is not None:
                flush.fill_(1)
            with torch.cuda.stream(st):
                t0.record(st)
                gr.replay()
                t1.record(st)
            t1.synchronize()
            tot += t0.elapsed_time(t1)
        return tot / steps

    clk = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    ms = timed_graph(graph, args.steps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    # per-stage times: the same steps with plain launches and events between the calls
    stage_ms = {k: [] for k in STAGES}
    for _ in range(args.steps):
        if flush is not None:
            flush.fill_(1)
        step(calls, True)
        st.synchronize()
        for k, name in enumerate(STAGES):
            stage_ms[name].append(ev[k].elapsed_time(ev[k + 1]))
    # per-kernel times: events the library records around the kernel's launches
    # (fp_time_kernel), on the launching stream, plain launches
    kev = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
    with torch.cuda.stream(st):
        kev[0].record(st)
        kev[1].record(st)
    kernel_ms = {}
    for kname in ([] if args.quick else [k for k in fp.KERNEL if k != "none"]):
        vals = []
        for _ in range(args.steps):
            if flush is not None:
                flush.fill_(1)
            fp.time_kernel(kname, kev[0], kev[1])
            with torch.cuda.stream(st):
                kev[0].record(st)   # a kernel the step does not launch reads 0
                kev[1].record(st)
            step(calls)
            fp.time_kernel("none")
            st.synchronize()
            vals.append(kev[0].elapsed_time(kev[1]))
        kernel_ms[kname] = statistics.median(vals)
    ms, value = replica_rate(ms, n, world, dev)

    # the same step with the optional leaf-grouped layout (fp_build_chunk_octree's d_leaf_pts)
    leaf_ms = None
    if leaf is None and not args.quick:
        leaf = dict(leaf=torch.empty_like(pts), leaf_perm=torch.empty(n, dtype=torch.int32, device=dev))
        g_leaf = capture(stage_calls(pts, True))
        with torch.cuda.stream(st):
            g_leaf.replay()
        torch.cuda.synchronize()
        leaf_ms = timed_graph(g_leaf, args.steps)
        del g_leaf, leaf
        leaf = None
        torch.cuda.synchronize()
        assert fp.get_device_error(stream=st) == 0

    # end to end through the C ABI: every step copies its cloud in from pinned
    # host memory and reads its node table (and node count) back into pinned
    # memory.  The copy of cloud i + 1 runs on a side stream under the build of
    # cloud i (two device input buffers, each with its captured step); nothing
    # waits on the host until the last step.  Two untimed steps of the same
    # loop warm the host link first (the first copies out of a freshly pinned
    # buffer run several times slower than the later ones).
    e2e_bufs = [pts, torch.empty_like(pts)]
    e2e_graphs = [graph, capture(stage_calls(e2e_bufs[1], False))]
    nodes_host = [torch.empty_like(O["nodes"], device="cpu").pin_memory() for _ in range(2)]
    nn_host = [torch.empty(1, dtype=torch.int32).pin_memory() for _ in range(2)]
    cs = torch.cuda.Stream(dev)
    e2e_steps = 1 if args.quick else min(max(4, args.steps), 10)
    copied = [torch.cuda.Event() for _ in range(2)]
    built = [torch.cuda.Event() for _ in range(2)]
    h2d_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    b_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    t_origin = torch.cuda.Event(enable_timing=True)

    def copy_in(k):
        c0, c1 = h2d_ev[k]
        with torch.cuda.stream(cs):
            if k >= 2:
                cs.wait_event(built[k % 2])   # the buffer's previous cloud is built
            c0.record(cs)
            e2e_bufs[k % 2].copy_(host, non_blocking=True)
            c1.record(cs)
            copied[k % 2].record(cs)

    def e2e_loop(steps):
        copy_in(0)
        for k in range(steps):
            if k + 1 < steps:
                copy_in(k + 1)
            with torch.cuda.stream(st):
                st.wait_event(copied[k % 2])
                b_ev[k][0].record(st)
                e2e_graphs[k % 2].replay()
                b_ev[k][1].record(st)
                built[k % 2].record(st)
                nn_host[k % 2].copy_(O["num_nodes"], non_blocking=True)
                nodes_host[k % 2].copy_(O["nodes"], non_blocking=True)

    torch.cuda.synchronize()
    if not args.quick:
        e2e_loop(min(2, e2e_steps))
        torch.cuda.synchronize()
    te0 = time.perf_counter()
    t_origin.record(st)
    e2e_loop(e2e_steps)
    st.synchronize()
    e2e_ms = (time.perf_counter() - te0) * 1e3 / e2e_steps
    d2h = O["nodes"].numel() * 8 + 4
    M = int(nn_host[(e2e_steps - 1) % 2].item())
    assert M == int(O["num_nodes"].item()) and fp.get_device_error(stream=st) == 0
    e2e_value = n * world / (e2e_ms * 1e-3) / 1e9
    # the host link's rate for these copies: it varies from host to host
    h2d_gbs = 16 * n / (statistics.median(c0.elapsed_time(c1) for c0, c1 in h2d_ev) * 1e-3) / 1e9
    # device timeline of the loop (ms from its start): copy k and build k, start and end
    timeline = [[round(t_origin.elapsed_time(e), 2) for e in (h2d_ev[k][0], h2d_ev[k][1], b_ev[k][0], b_ev[k][1])]
                for k in range(e2e_steps)]
    del e2e_bufs, e2e_graphs

    peak, peak_kind = measured_peaks()
    med = {k: statistics.median(v) for k, v in stage_ms.items()}
    if not kernel_ms:   # --quick: no per-kernel times, the distribution stands in
        kernel_ms = {"distribute": statistics.median(stage_ms["distribute"])}
    dom = max(kernel_ms, key=lambda k: kernel_ms[k])
    alg = kernel_alg_bytes(dom, n)
    achieved = alg / (kernel_ms[dom] * 1e-3) / 1e9
    kernels = {}
    for k, v in sorted(kernel_ms.items(), key=lambda kv: -kv[1]):
        if v <= 0:
            continue
        b = kernel_alg_bytes(k, n)
        kernels[k] = {"ms": v, "share_of_step": v / ms, "alg_bytes": b,
                      "frac": (b / (v * 1e-3) / 1e9 / peak) if b else 0.0,
                      "traffic": ncu_traffic(args.workload, k)}
    # the method's mandatory bytes: 97 per point plus the count grid's 25.2 MB
    step_alg = ALG_PER_POINT * n + FIXED_BYTES["merge"]
    # a dominant kernel that moves none of those bytes (it groups or orders
    # intermediates) has frac 0: its measured DRAM rate and the kernel with the
    # largest fraction are named beside it
    dom_traffic = ncu_traffic(args.workload, dom)
    dom_note = {}
    if not alg:
        best = max(kernels, key=lambda k: kernels[k]["frac"]) if kernels else None
        dom_note = {"note": "moves intermediates only (none of the 97 B/pt)",
                    "traffic_frac": (dom_traffic / (kernel_ms[dom] * 1e-3) / 1e9 / peak) if dom_traffic else None,
                    "largest_frac_kernel": best, "largest_frac": kernels[best]["frac"] if best else None}
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            r, ns, dt, cores = oracle_rate(kind, seed, wl, float(os.environ.get("FP_ORACLE_BUDGET_S", "12")))
            cpu = {"value": r / 1e9, "unit": "Gpts/s", "cores": cores, "nproc": os.cpu_count(), "kind": "oracle",
                   "sample": "first %d points of the %s workload, same parameters, %.1f s, one thread" %
                             (ns, args.workload, dt)}
        line = {
            "metric": "octree build throughput (Gpts/s)", "value": value, "unit": "Gpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "points": n, "grid_log2": g, "sub_log2": s, "max_level": lmax,
                       "chunk_threshold": T, "node_capacity": C, "nodes": M,
                       "chunks": int(O["num_chunks"].item()), "parallelism": "replicas" if world > 1 else "single",
                       "launch": "one CUDA graph per step",
                       "outputs": "cube, preview, count grid (+ each point's cell, handed to the distribution), "
                                  "chunks, LUT, offsets, distributed points + perm, "
                                  "node table, owner per point, final LOD layout + perm" +
                                  (", leaf-grouped points + perm" if args.leaf_grouped else ""),
                       "l2": ("inputs (%.1f GB) larger than L2" % (16 * n / 1e9)) if flush is None else
                             "L2 flushed between steps (256 MB written)"},
            "e2e": {"value": e2e_value, "unit": "Gpts/s", "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": d2h,
                    "h2d_gbs": h2d_gbs, "steps": e2e_steps, "timeline_ms": timeline,
                    "overlap": "copy of cloud i+1 on a side stream under the build of cloud i; node table and "
                               "count read back asynchronously"},
            "roofline": dict({"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                              "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                              "frac_of_8tbs": achieved / 8000.0, "traffic": dom_traffic,
                              "alg_bytes_per_launch": alg, "ms": kernel_ms[dom]}, **dom_note),
            "step_roofline": {"alg_bytes": step_alg, "alg_bytes_per_point": ALG_PER_POINT,
                              "achieved_gbs": step_alg / (ms * 1e-3) / 1e9,
                              "frac": step_alg / (ms * 1e-3) / 1e9 / peak,
                              "frac_of_8tbs": step_alg / (ms * 1e-3) / 1e9 / 8000.0},
            "stage_ms": med,
            "kernels": kernels,
            "with_leaf_grouped": None if leaf_ms is None else
            {"ms_per_step": leaf_ms, "value": n * world / (leaf_ms * 1e-3) / 1e9,
             "note": "the same step also writing the optional leaf-grouped layout"},
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps if launches_per_step else None,
            "cpu_baseline": cpu,
        }
    else:
        line = None
    if world > 1:
        dist.destroy_process_group()
    return line


if __name__ == "__main__":
    main()
