"""End-to-end Morse-Smale complex 1-skeleton throughput on GB300 (Mvoxel/s).

One step = the whole hot path (lower-star gradient, critical cells, saddle-extremum arcs,
saddle-saddle reachability, DAG minor, D* path counts) over one synthetic volume, through
the library's C ABI.  The default workload is the 256^3 float32 Gaussian random field with
P(k) ~ k^-3 (seed 1).  The timed region starts with the field resident in HBM; the L2 is
flushed (a 256 MB write) before every timed step.  A second pass times the same steps
end to end from pinned host memory (H2D of the field, D2H of the whole 1-skeleton every step),
with two plans on two streams taking the steps in turn so that copies overlap compute.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the plain CPU oracle (the only other implementation of this path)
on bounded crops of the same workload on the host cores.  With N > 1 (torchrun) every rank
runs an independent replica on its own GPU (the path does not shard; no collective is on
the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "grf256": "256^3 float32 Gaussian random field, P(k) ~ k^-3, zero mean, unit variance, seed 1",
    "blobs512": "512^3 float32 sum of 2000 Gaussian blobs (sigma 2-20, amplitude U[-1,1]) + N(0,1e-3), seed 2",
    "cos32": "32^3 float32 cos(2 pi x/16)+cos(2 pi y/16)+cos(2 pi z/16) + U[0,1e-3], seed 0",
    "batch64": "64 float32 GRFs, P(k) ~ k^-2.5, seeds 100-163, each axis uniform in 48-192",
    "serve500": "500 requests over 8 advected k^-3 GRF streams sized 64^3-384^3, Poisson 200 req/s, 8 GiB admission",
}
METRIC = "end-to-end MS-complex Mvoxel/s on 1 GB300 (batched vs plain) + per-stage HBM GB/s"
L2_FLUSH_BYTES = 256 << 20
REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
           0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
           0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


E2E_LANES = 3  # plans in flight in the end-to-end leg


def _rounded(d):
    """Floats in a (nested) dict to 6 significant digits, for the JSON line."""
    if isinstance(d, dict):
        return {k: _rounded(v) for k, v in d.items()}
    return float(f"{d:.6g}") if isinstance(d, float) else d


def _num_sms():
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _field(name):
    from synth import fields

    return fields.config_field(name)


# ---------------------------------------------------------------------------------------
# clocks during the timed region
class ClockSampler:
    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        time.sleep(0.15)
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                active = int(parts[3], 16)
            except Exception:
                continue
            for bit, name in REASONS.items():
                if active & bit and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
def _traffic_record(kernel):
    """DRAM bytes per unit of one ncu capture, if the kernel's sources are unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
    except Exception:
        return None
    h = hashlib.sha256()
    for rel in rec["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return rec


def aggregate_replicas(ms_local, e2e_local, voxels_per_rank, dist=None, device="cpu"):
    """Replicas only: every rank times the same per-GPU work; the job's step time is the
    slowest rank's, and throughput counts the voxels of all ranks (weak scaling)."""
    import torch

    world = 1
    ms, e2e = float(ms_local), float(e2e_local)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms, e2e], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e = float(t[0]), float(t[1])
    return {"world": world, "ms": ms, "e2e_ms": e2e, "value": world * voxels_per_rank / (ms / 1e3) / 1e6,
            "e2e_value": world * voxels_per_rank / (e2e / 1e3) / 1e6}


def cpu_baseline(field, min_seconds=10.0, max_runs=64):
    """The oracle as it stands, single-threaded, on bounded crops of the workload: successive
    64 x 96 x 96 blocks of the field (cycling when there are fewer), until about min_seconds of
    oracle time have passed."""
    import numpy as np

    import oracle

    nz, ny, nx = field.shape
    origins = [(z, y, x) for z in range(0, nz, 64) for y in range(0, ny, 96) for x in range(0, nx, 96)]
    nvox = 0
    runs = 0
    dt = 0.0
    while runs < max_runs and (runs == 0 or dt < min_seconds):
        z, y, x = origins[runs % len(origins)]
        crop = np.ascontiguousarray(field[z:z + 64, y:y + 96, x:x + 96])
        t = time.perf_counter()
        oracle.compute_all(crop)
        dt += time.perf_counter() - t
        nvox += crop.size
        runs += 1
    what = "the whole field" if len(origins) == 1 and field.shape[0] <= 64 and ny <= 96 and nx <= 96 \
        else "blocks of at most 64x96x96"
    return {"value": nvox / dt / 1e6, "unit": "Mvoxel/s", "cores": 1, "kind": "oracle",
            "sample": f"full pipeline on {what}, {runs} oracle run(s) over {nvox} voxels in {dt:.1f} s "
                      f"on {os.cpu_count()} host cores (oracle uses 1)"}


def _oracle_crop(v):
    import oracle
    oracle.compute_all(v)
    return v.size


def cpu_baseline_batch(vols, edge=40):
    """The oracle as it stands over the batch workload's 64 volumes, one process per host core
    (spawned, so no process inherits a CUDA context), each volume cropped to its first edge^3 corner
    so that the leg stays bounded."""
    import multiprocessing as mp

    import numpy as np

    crops = [np.ascontiguousarray(v[:edge, :edge, :edge]) for v in vols]
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_crop, crops[:cores])  # workers started and the oracle loaded
        t = time.perf_counter()
        nvox = sum(pool.map(_oracle_crop, crops, chunksize=1))
        dt = time.perf_counter() - t
    return {"value": nvox / dt / 1e6, "unit": "Mvoxel/s", "cores": cores, "kind": "oracle",
            "sample": f"the {len(crops)} volumes cropped to their first {edge}^3 corner ({nvox} voxels), one "
                      f"process per host core, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle

    f = _field(args.workload)
    crop = np.ascontiguousarray(f[:48, :48, :48])
    for _ in range(args.warmup):
        oracle.compute_all(crop)
    times = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.compute_all(crop)
        times.append(time.perf_counter() - t)
    total = time.perf_counter() - t0
    ms = 1e3 * total / args.steps
    value = crop.size / (total / args.steps) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32-compare/u64-count", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "sample": "48^3 corner crop per step (the oracle cannot run the full volume in a bench step)"},
            "cpu_baseline": {"value": value, "unit": "Mvoxel/s", "cores": 1, "kind": "oracle",
                             "sample": f"48^3 corner crop ({crop.size} voxels) per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": "Mvoxel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2009_03707_gb300 import msc

    f = _field(args.workload)
    nz, ny, nx = f.shape
    nvox = f.size
    plan = msc.Plan((nx, ny, nz), no_graph=args.no_graph, gradient_tile=args.gradient_tile)
    d_field = torch.from_numpy(f).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.fill_(1.0)
        msc.msc_compute(plan, d_field)
    torch.cuda.synchronize()
    stats = msc.msc_get_stats(plan)

    # ---- device-resident timing -------------------------------------------------------
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    step_ms, stage_ms, kernel_ms = [], [], {"gradient_kernel": [], "rows_thread": []}
    launches = 0
    barrier()
    with ClockSampler(uuid) as clk:
        t_region = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(2.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            msc.msc_compute(plan, d_field)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            st = msc.msc_get_stats(plan)
            launches += int(st["n_launches"])
            stage_ms.append(st)
            kernel_ms["gradient_kernel"].append(st["ms_gradient_kernel"])
            kernel_ms["rows_thread"].append(st["ms_rows_kernel"])
        barrier()
        wall = time.perf_counter() - t_region
    ms_local = sum(step_ms) / len(step_ms)

    # ---- end to end from pinned host memory -------------------------------------------
    # Every step copies its field in from pinned host memory, runs the pass and reads the whole
    # 1-skeleton back into pinned host memory.  E2E_LANES plans on as many streams take the steps in
    # turn through the public asynchronous entry points: step i's pass is enqueued
    # (msc_compute_async), then the oldest pass still out, step i - E2E_LANES + 1, is waited for
    # (msc_compute_wait) and its results are copied out on its stream, and the field of step i+1
    # goes up into that plan's buffer behind them.  So the device always has the next passes queued
    # while the host collects an earlier one; a plan's result buffers are reused E2E_LANES steps
    # later, on the same stream, after their copies.
    h_field = torch.from_numpy(f).pin_memory()
    counts = stats["counts"]
    lanes = []
    for x in range(E2E_LANES):
        # several passes in flight fill the device: each plan replays its pass as one chain
        pl = msc.Plan((nx, ny, nz), no_graph=args.no_graph, gradient_tile=args.gradient_tile, serial_pass=True)
        lanes.append({"plan": pl, "field": d_field if x == 0 else torch.empty_like(d_field),
                      "stream": stream if x == 0 else torch.cuda.Stream(), "out": {}})

    def d2h(lane, name, t):
        n = t.numel() * t.element_size()
        buf = lane["out"].get(name)
        if buf is None or buf.numel() < n:
            buf = lane["out"][name] = torch.empty(max(n, 1), dtype=torch.uint8, pin_memory=True)
        if n:
            buf[:n].copy_(t.view(torch.uint8).reshape(-1), non_blocking=True)
        return n

    def upload(lane):
        with torch.cuda.stream(lane["stream"]):
            lane["field"].copy_(h_field, non_blocking=True)

    def issue(lane):
        with torch.cuda.stream(lane["stream"]):
            msc.msc_compute_async(lane["plan"], lane["field"])

    def collect(lane):
        with torch.cuda.stream(lane["stream"]):
            msc.msc_compute_wait(lane["plan"])
            _, cells = msc.msc_critical(lane["plan"])
            amin, amax, _, _ = msc.msc_extremum_arcs(lane["plan"])
            rowptr, col, cnt = msc.msc_saddle_arcs(lane["plan"])
            n = sum(d2h(lane, f"cells{k}", cells[k]) for k in range(4))
            n += d2h(lane, "amin", amin) + d2h(lane, "amax", amax)
            n += d2h(lane, "rowptr", rowptr) + d2h(lane, "col", col) + d2h(lane, "cnt", cnt)
        return n

    def run_e2e(k):
        L = len(lanes)
        upload(lanes[0])
        n = 0
        for i in range(k):
            issue(lanes[i % L])
            nxt = lanes[(i + 1) % L]
            if i - L + 1 >= 0:
                n = collect(nxt)  # pass i - L + 1 ran on the lane that takes step i + 1
            if i + 1 < k:
                upload(nxt)
        for i in range(max(k - L + 1, 0), k):  # the passes still out
            n = collect(lanes[i % L])
        return n

    warm = max(args.warmup, E2E_LANES)  # every plan warm (its graph captured)
    for _ in range(2):
        run_e2e(warm)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lanes[0]["stream"])
    for lane in lanes[1:]:
        lane["stream"].wait_event(e0)
    bo = run_e2e(args.steps)  # the first field's upload is inside the timed region
    for lane in lanes[1:]:
        done = torch.cuda.Event()
        done.record(lane["stream"])
        lanes[0]["stream"].wait_event(done)
    e1.record(lanes[0]["stream"])
    e1.synchronize()
    e2e_ms = [e0.elapsed_time(e1) / args.steps]
    agg = aggregate_replicas(ms_local, sum(e2e_ms) / len(e2e_ms), nvox, dist, device="cuda")
    ms, value = agg["ms"], agg["value"]

    if rank != 0:
        dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ----------------------------------------------
    peak, peak_kind = _peaks()
    last = stage_ms[-1]
    km = {k: statistics.median(v) for k, v in kernel_ms.items()}
    algo = {"gradient_kernel": 8.0 * nvox,
            "rows_thread": 17.0 * (counts[1] + last["n_frontier_entries"]) + 12.0 * last["nnz_Dstar"]}
    units = {"gradient_kernel": nvox, "rows_thread": counts[1] + last["n_frontier_entries"]}
    dom = max(km, key=km.get)
    achieved = algo[dom] / (km[dom] / 1e3) / 1e9 if km[dom] > 0 else None
    rec = _traffic_record(dom)
    traffic = None
    if rec and rec.get("workload") == args.workload:
        traffic = rec["bytes_per_unit"] * units[dom]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic, "peak_kind": peak_kind,
                "kernel_ms": km[dom], "algorithmic_bytes": algo[dom]}
    # the lower-star pairing is a sequential loop per vertex: beside the HBM figure, the warp
    # instructions it issues (counted once by ncu, profiles/traffic.json) per second of the live
    # kernel time, against the SMs' issue rate at the clock sampled during the run
    grec = _traffic_record("gradient_kernel")
    sm_mhz = (clk.summary() or {}).get("sm_mhz")
    if grec and grec.get("workload") == args.workload and grec.get("warp_inst_per_unit") and sm_mhz and km["gradient_kernel"] > 0:
        inst = grec["warp_inst_per_unit"] * nvox
        got = inst / (km["gradient_kernel"] / 1e3) / 1e9
        top = _num_sms() * 4 * float(sm_mhz) / 1e3
        roofline["issue"] = {"kernel": "gradient_kernel", "warp_inst": inst, "achieved": got, "peak": top,
                             "unit": "G warp-instructions/s", "frac": got / top,
                             "peak_basis": "4 schedulers x 1 instruction/clock per SM at the sampled SM clock"}

    def med(key):
        return statistics.median(s[key] for s in stage_ms)

    stage_bytes = {"gradient": 8.0 * nvox, "critical": 1.0 * nvox + 4.0 * sum(counts),
                   "extremum": 4.0 * nvox + 8.0 * nvox, "reachability": 4.0 * last["n_reachable"],
                   "minor": 17.0 * (counts[1] + last["n_junctions"]),
                   "path_count": algo["rows_thread"]}
    stages = {}
    for name in stage_bytes:
        t = med("ms_" + name)
        stages[name] = {"ms": t, "GB/s": stage_bytes[name] / (t / 1e3) / 1e9 if t > 0 else None}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-compare/u64-count", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "dims": [nx, ny, nz],
                   "voxels_per_step": nvox, "parallelism": f"replicas x{world}",
                   "l2": "flushed before every timed step (256 MB write)",
                   "critical_counts": counts, "nnz_Dstar": last["nnz_Dstar"], "n_iter": last["n_iter"],
                   "graph": {k: last[k] for k in ("n_reachable", "n_bfs_levels", "n_junctions", "nnz_A", "nnz_B",
                                                  "nnz_Bstar", "nnz_D", "n_pointer_jumps", "n_frontier_entries")},
                   "max_path_count": str(last["max_path_count"]),
                   "gradient_tile": "x".join(str(v) for v in (32, last["gradient_tile"] & 0xFF,
                                                             (last["gradient_tile"] >> 8) & 0xFF))
                   + f" vertices, {last['gradient_tile'] >> 16} threads (autotuned)",
                   "path_count_method": {1: "row-wise products", 2: "junction waves"}.get(
                       last["path_count_method"], "?") + " (chosen automatically)",
                   "diagnostics": _rounded(msc.diagnostics(last))},
        "e2e": {"value": agg["e2e_value"], "unit": "Mvoxel/s",
                "h2d_bytes_per_step": int(f.nbytes), "d2h_bytes_per_step": int(bo)},
        "gpu_launches": launches,
        "roofline": roofline,
        "stages": stages,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(f)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batch(args):
    """Batching workload: 64 uneven volumes, one batched submission vs 64 sequential runs."""
    import torch

    from paper_2009_03707_gb300 import msc
    from synth import fields

    vols = fields.batch_volumes(64)
    dev = [torch.from_numpy(v).cuda() for v in vols]
    nvox = sum(v.size for v in vols)
    plans = [msc.Plan((v.shape[2], v.shape[1], v.shape[0])) for v in vols]
    for _ in range(args.warmup):  # allocates every plan's buffers
        for p, d in zip(plans, dev):
            msc.msc_compute(p, d)
    torch.cuda.synchronize()
    plain, batched = [], []
    batch = msc.Batch(n_workers=args.workers)
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for p, d in zip(plans, dev):
            msc.msc_compute(p, d)
        torch.cuda.synchronize()
        plain.append(time.perf_counter() - t)
        t = time.perf_counter()
        ticket, _ = batch.msc_batch_submit(dev, plans)
        st = batch.msc_batch_wait(ticket)
        torch.cuda.synchronize()
        batched.append(time.perf_counter() - t)
        assert st == 0, st
    batch.close()
    tp, tb = statistics.median(plain), statistics.median(batched)
    line = {"metric": METRIC, "value": nvox / tb / 1e6, "unit": "Mvoxel/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tb, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-compare/u64-count", "data": "synthetic",
            "config": {"workload": f"batch64: {WORKLOADS['batch64']}", "voxels_per_step": nvox,
                       "workers": args.workers, "timing": "host wall clock around each pass, device synced"},
            "plain": {"value": nvox / tp / 1e6, "unit": "Mvoxel/s", "ms_per_step": 1e3 * tp,
                      "how": "64 msc_compute calls one after another on one stream"},
            "batched_over_plain": tp / tb}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batch(vols)
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload: Poisson arrivals over 8 advected streams, HBM-budget admission."""
    import threading

    import torch

    from paper_2009_03707_gb300 import msc
    from synth import fields

    streams = fields.serving_streams()
    trace = fields.request_trace()
    if args.requests:
        trace = trace[:args.requests]
    budget = 8 << 30
    batch = msc.Batch(n_workers=args.workers, hbm_budget_bytes=budget)
    plans = [None] * len(streams)
    for s in range(len(streams)):  # warm-up: one step per stream creates and sizes its plan
        ticket, out = batch.msc_batch_submit([streams[s].step_device(0)], [plans[s]])
        plans[s] = out[0]
        assert batch.msc_batch_wait(ticket) == 0
    torch.cuda.synchronize()
    done_at, lock = {}, threading.Lock()
    pending = []
    stop = threading.Event()

    def poller():
        while not stop.is_set() or pending:
            with lock:
                items = list(pending)
            for i, ticket in items:
                ok, status = batch.msc_poll(ticket)
                if ok:
                    assert status == 0, status
                    with lock:
                        done_at[i] = time.perf_counter()
                        pending.remove((i, ticket))
            time.sleep(0.0002)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    arrive = {}
    for i, (at, s, step) in enumerate(trace):
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        arrive[i] = t0 + at
        field = streams[s].step_device(step + 1)
        ticket, _ = batch.msc_batch_submit([field], [plans[s]])
        with lock:
            pending.append((i, ticket))
    while True:
        with lock:
            if not pending:
                break
        time.sleep(0.001)
    stop.set()
    th.join()
    t_end = max(done_at.values())
    batch.close()
    lat = sorted(1e3 * (done_at[i] - arrive[i]) for i in done_at)
    nvox = sum(streams[s].size ** 3 for _, s, _ in trace)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]
    line = {"metric": METRIC, "value": nvox / (t_end - t0) / 1e6, "unit": "Mvoxel/s", "n_gpus": 1,
            "steps": len(trace), "warmup": len(streams), "ms_per_step": 1e3 * (t_end - t0) / len(trace),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32-compare/u64-count",
            "data": "synthetic",
            "config": {"workload": f"serve500: {WORKLOADS['serve500']}", "requests": len(trace),
                       "voxels": nvox, "workers": args.workers, "hbm_budget_bytes": budget,
                       "offered_mvoxel_s": nvox / trace[-1][0] / 1e6,
                       "inputs": "synthesised on the GPU at arrival (Fourier shift of each stream's base field)"},
            "latency_ms": {"p50": p50, "p99": p99, "max": lat[-1], "mean": sum(lat) / len(lat)}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["msc", "reference"], default="msc")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="grf256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workers", type=int, default=8, help="batch/serve worker streams")
    ap.add_argument("--requests", type=int, default=0, help="serve500: truncate the request trace")
    ap.add_argument("--no-graph", action="store_true",
                    help="run every pass synchronised between stages instead of replaying its CUDA graph "
                         "(same kernels; profilers list each launch)")
    ap.add_argument("--gradient-tile", type=int, default=0, help="force a lower-star tile variant (1..9)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps are required")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "serve500":
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
