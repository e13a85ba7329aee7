"""End-to-end Morse-Smale complex 1-skeleton throughput on GB300 (Mvoxel/s).

One step = the whole hot path (lower-star gradient, critical cells, saddle-extremum arcs,
saddle-saddle reachability, DAG minor, D* path counts) over one synthetic volume, through
the library's C ABI.  The default workload is the 256^3 float32 Gaussian random field with
P(k) ~ k^-3 (seed 1).  The timed region starts with the field resident in HBM; the L2 is
flushed (a 256 MB write) before every timed step.  A second pass times the same steps
end to end from pinned host memory: the field goes up every step, and every output of the
pass (critical lists, both arc arrays, both label arrays, D* CSR) comes back through
msc_copy_to_host into caller-owned pinned buffers, with three plans on three streams taking
the steps in turn so that copies overlap compute.  That pass is timed five times and the median
is reported (the host copies share the machine's host memory with other jobs).

The default run adds the metric's other workloads to the same JSON line ("legs"), each with
the clocks sampled while it ran: the 256^3 pass's on-request outputs (D* by 2-saddle, the host
1-skeleton, the cells along both kinds of arcs) and its simplification at 5 % of the field's
range; the 512^3 blob field (the largest single volume); the
64-volume uneven batch as one submission against the same volumes one msc_compute at a time;
and the serving trace (the first 200 requests of the Poisson stream) through the
continuous-batching runtime against the same trace served one request at a time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--no-legs]
  python bench.py --workload blobs512 | batch64 | serve500 | cos32

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
    "serve500": "500 requests over 8 advected k^-3 GRF streams sized 64^3-384^3, Poisson 200 req/s, HBM-budget admission",
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
E2E_REPEATS = 5  # timed runs of the end-to-end leg (the median is reported)
# every output of a pass, copied to the host by the end-to-end leg (msc_copy_to_host selectors)
E2E_OUTPUTS = ("cells0", "cells1", "cells2", "cells3", "min_arcs", "max_arcs", "vertex_min", "cube_max",
               "dstar_rowptr", "dstar_col", "dstar_count")


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

    def d2h(lane, what):
        """One output into the lane's caller-owned pinned buffer through msc_copy_to_host."""
        n = msc.msc_copy_to_host_size(lane["plan"], what)
        buf = lane["out"].get(what)
        if buf is None or buf.numel() < n:
            buf = lane["out"][what] = torch.empty(max(n, 1), dtype=torch.uint8, pin_memory=True)
        return msc.msc_copy_to_host_into(lane["plan"], what, buf) if n else 0

    def upload(lane):
        with torch.cuda.stream(lane["stream"]):
            lane["field"].copy_(h_field, non_blocking=True)

    def issue(lane):
        with torch.cuda.stream(lane["stream"]):
            msc.msc_compute_async(lane["plan"], lane["field"])

    def collect(lane):
        with torch.cuda.stream(lane["stream"]):
            msc.msc_compute_wait(lane["plan"])
            return sum(d2h(lane, what) for what in E2E_OUTPUTS)

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
    # three timed runs of K steps each; the median counts (the host copies share the machine's
    # host memory and its link to the GPU with other jobs, so one run can be disturbed)
    e2e_ms = []
    for _ in range(E2E_REPEATS):
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
        e2e_ms.append(e0.elapsed_time(e1) / args.steps)
    agg = aggregate_replicas(ms_local, statistics.median(e2e_ms), nvox, dist, device="cuda")
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
        gbs = stage_bytes[name] / (t / 1e3) / 1e9 if t > 0 else None
        stages[name] = {"ms": t, "GB/s": gbs, "frac": gbs / peak if gbs else None}
    # the whole pass: every stage's algorithmic bytes over the step time
    total_bytes = sum(stage_bytes.values())
    stages["end_to_end"] = {"ms": ms, "GB/s": total_bytes / (ms / 1e3) / 1e9,
                            "frac": total_bytes / (ms / 1e3) / 1e9 / peak,
                            "note": "sum of the stages' algorithmic bytes over the device-resident step time"}
    # both candidates for the dominant kernel, each against its own algorithmic bytes
    kernels = {}
    for k in km:
        a = algo[k] / (km[k] / 1e3) / 1e9 if km[k] > 0 else None
        kernels[k] = {"ms": km[k], "algorithmic_bytes": algo[k], "achieved": a, "frac": a / peak if a else None}
    roofline["kernels"] = kernels

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
                "h2d_bytes_per_step": int(f.nbytes), "d2h_bytes_per_step": int(bo),
                "runs_mvoxel_s": [nvox / (t / 1e3) / 1e6 for t in e2e_ms],
                "copies_declared": True, "outputs": list(E2E_OUTPUTS), "passes_in_flight": E2E_LANES,
                "how": (f"msc_compute_async / msc_compute_wait on {E2E_LANES} plans ({E2E_LANES} passes in "
                        "flight); each step's field uploaded from pinned host memory inside the timed "
                        "region; every output read back with msc_copy_to_host into caller-owned pinned "
                        f"buffers; median of {E2E_REPEATS} runs of {args.steps} steps")},
        "gpu_launches": launches,
        "roofline": roofline,
        "stages": stages,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(f)
    if world == 1 and args.workload == "grf256" and not args.no_legs:
        # the other workloads of the metric, in the same run: simplification of this pass's complex,
        # the largest single volume, batched against one volume at a time, served against one
        # request at a time
        legs = {}
        want = set(args.legs.split(","))
        if "outputs" in want:
            legs["outputs"] = leg_outputs(msc, torch, plan, d_field, uuid)
        if "simplify" in want:
            legs["simplify"] = leg_simplify(msc, torch, plan, d_field, f, uuid)
        del lanes, plan, d_field
        torch.cuda.empty_cache()
        if "blobs512" in want:
            legs["blobs512"] = leg_single(msc, torch, "blobs512", steps=5, warmup=3, uuid=uuid)
        if "batch64" in want:
            legs["batch64"] = leg_batch(msc, torch, steps=3, workers=args.workers, uuid=uuid,
                                        with_cpu=not args.no_cpu_baseline)
        if "serve" in want:
            legs["serve"] = leg_serve(msc, torch, args.requests, args.workers, args.serve_budget, uuid)
        line["legs"] = legs
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _events_ms(torch, fn, reps):
    """Median over reps of fn() bracketed by CUDA events on the current stream, device synced on
    both sides (fn may leave the stream and wait on the host: the events then see the wall time
    the stream spent, idle gaps included)."""
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def leg_simplify(msc, torch, plan, d_field, f, uuid, frac=0.05, reps=3):
    """Simplification of the pass's 1-skeleton at a persistence threshold of `frac` of the field's
    range (the paper's 5 %), on the GPU in rounds of independent cancellations; timed by CUDA events
    around msc_simplify (which synchronises once per round), median of reps."""
    counts, _ = msc.msc_critical(plan)
    threshold = frac * float(f.max() - f.min())
    msc.msc_simplify(plan, d_field, threshold)  # builds the host-side graph once; warm
    res = {}

    def run():
        res.update(msc.msc_simplify(plan, d_field, threshold))

    with ClockSampler(uuid) as clk:
        ms = _events_ms(torch, run, reps)
    return {"threshold": threshold, "threshold_fraction_of_range": frac, "ms": ms, "rounds": res["n_rounds"],
            "cancelled_pairs": res["n_cancelled"], "critical_before": counts, "critical_after": res["counts"],
            "arcs_after": int(res["adj"].numel() // 2),
            "how": "msc_simplify on the 256^3 pass's complex (rounds of independent least-key cancellations)",
            "clocks": clk.summary()}


def leg_outputs(msc, torch, plan, d_field, uuid, reps=3):
    """The on-request outputs of the 256^3 pass, each built on its first call after a pass and timed by
    CUDA events around that call (every call synchronises): D* by 2-saddle (CSC), the 1-skeleton's
    adjacency (built on the device; the size query, so no host copy), the cells along the
    saddle-extremum arcs, and the cells along the
    saddle-saddle arcs of count 1 (after a row-wise pass this runs the junction waves once more for
    the rows of J).  A fresh pass (untimed) before each rep; median of reps."""
    calls = {"dstar_csc": lambda: msc.msc_saddle_arcs_csc(plan),
             "complex_graph": lambda: msc.msc_complex_graph_size(plan),
             "arc_geometry": lambda: msc.msc_arc_geometry(plan),
             "saddle_arc_geometry": lambda: msc.msc_saddle_arc_geometry(plan)}
    times = {k: [] for k in calls}
    got = {}
    with ClockSampler(uuid) as clk:
        for _ in range(reps):
            msc.msc_compute(plan, d_field)
            torch.cuda.synchronize()
            stream = torch.cuda.current_stream()
            for k, fn in calls.items():
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                got[k] = fn()
                e1.record(stream)
                e1.synchronize()
                times[k].append(e0.elapsed_time(e1))
    cnt = got["saddle_arc_geometry"]
    _, dstar_col, dstar_cnt = msc.msc_saddle_arcs(plan)
    sizes = {"dstar_csc": {"nnz": int(got["dstar_csc"][1].numel())},
             "complex_graph": {"nodes": got["complex_graph"][0], "adjacency": got["complex_graph"][1]},
             "arc_geometry": {"arcs": int(got["arc_geometry"][0].numel() - 1), "cells": int(got["arc_geometry"][1].numel())},
             "saddle_arc_geometry": {"entries": int(cnt[0].numel() - 1), "count_one": int((dstar_cnt == 1).sum()),
                                     "cells": int(cnt[1].numel())}}
    out = {k: dict(ms=statistics.median(v), **sizes[k]) for k, v in times.items()}
    out["how"] = ("each call's first build after a fresh 256^3 pass, CUDA events around the call, median of "
                  f"{reps}; the 1-skeleton as msc_complex_graph's size query (built on the device, not copied)")
    out["clocks"] = clk.summary()
    return out


def leg_single(msc, torch, name, steps, warmup, uuid):
    """A single-volume workload timed like the main leg (device-resident, L2 flushed per step)."""
    f = _field(name)
    nz, ny, nx = f.shape
    plan = msc.Plan((nx, ny, nz))
    d = torch.from_numpy(f).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        msc.msc_compute(plan, d)

    def step():
        flush.fill_(3.0)
        msc.msc_compute(plan, d)

    with ClockSampler(uuid) as clk:
        ms = _events_ms(torch, step, steps)  # the flush write is inside; it takes ~0.05 ms
    st = msc.msc_get_stats(plan)
    return {"workload": f"{name}: {WORKLOADS[name]}", "value": f.size / (ms / 1e3) / 1e6, "unit": "Mvoxel/s",
            "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "stages_ms": {k: st["ms_" + k] for k in ("gradient", "critical", "extremum", "reachability", "minor",
                                                    "path_count")},
            "gradient_kernel_ms": st["ms_gradient_kernel"],
            "path_count_method": {1: "row-wise products", 2: "junction waves"}.get(st["path_count_method"], "?"),
            "n_iter": st["n_iter"], "n_bfs_levels": st["n_bfs_levels"], "max_path_count": str(st["max_path_count"]),
            "clocks": clk.summary()}


def leg_batch(msc, torch, steps, workers, uuid, with_cpu=False):
    """Batching: 64 uneven volumes as one submission (one group graph, one launch) against the same
    64 volumes one msc_compute at a time on one stream, each on its own default plan.  Both arms
    are timed by CUDA events on the launching stream around the whole 64-volume job."""
    from synth import fields

    vols = fields.batch_volumes(64)
    dev = [torch.from_numpy(v).cuda() for v in vols]
    nvox = sum(v.size for v in vols)
    single = [msc.Plan((v.shape[2], v.shape[1], v.shape[0])) for v in vols]
    batch = msc.Batch(n_workers=workers)
    ticket, grouped = batch.msc_batch_submit(dev)  # the runtime's own plans: one job per volume
    assert batch.msc_batch_wait(ticket) == 0
    for _ in range(2):  # group capture, then a replay; the single plans capture their graphs
        ticket, _ = batch.msc_batch_submit(dev, grouped)
        assert batch.msc_batch_wait(ticket) == 0
        for p, d in zip(single, dev):
            msc.msc_compute(p, d)

    def one_at_a_time():
        for p, d in zip(single, dev):
            msc.msc_compute(p, d)

    def batched():
        t, _ = batch.msc_batch_submit(dev, grouped)
        assert batch.msc_batch_wait(t) == 0

    with ClockSampler(uuid) as clk:
        t_one = _events_ms(torch, one_at_a_time, steps)
        t_bat = _events_ms(torch, batched, steps)
    batch.close()
    out = {"workload": f"batch64: {WORKLOADS['batch64']}", "voxels": nvox,
           "batched": {"value": nvox / t_bat * 1e-3, "unit": "Mvoxel/s", "ms": t_bat,
                       "how": "one msc_batch_submit of the 64 volumes (a CUDA graph with a branch per volume, "
                              "one launch) and msc_batch_wait"},
           "one_at_a_time": {"value": nvox / t_one * 1e-3, "unit": "Mvoxel/s", "ms": t_one,
                             "how": "64 msc_compute calls one after another on one stream (each a replayed "
                                    "graph and a host wait)"},
           "batched_over_one_at_a_time": t_one / t_bat, "repetitions": steps,
           "timing": "CUDA events on the launching stream around each 64-volume job, median",
           "clocks": clk.summary()}
    if with_cpu:
        out["cpu_baseline"] = cpu_baseline_batch(vols)
    return out


def _serve_arm(msc, torch, trace, inputs, plans, batch, saturated):
    """Runs the request trace; batch None = one request at a time (msc_compute in arrival order).
    Returns per-request (arrival, completion) host times relative to the start."""
    import threading

    n = len(trace)
    arrive = [0.0 if saturated else at for at, _, _ in trace]
    done = [None] * n
    torch.cuda.synchronize()
    if batch is None:
        t0 = time.perf_counter()
        for i, (_, s, _) in enumerate(trace):
            wait = arrive[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            msc.msc_compute(plans[s], inputs[i])
            done[i] = time.perf_counter() - t0
        return arrive, done
    pending, lock, stop = [], threading.Lock(), threading.Event()

    def poller():
        while not stop.is_set() or pending:
            with lock:
                items = list(pending)
            for i, ticket in items:
                ok, status = batch.msc_poll(ticket)
                if ok:
                    assert status == 0, status
                    with lock:
                        done[i] = time.perf_counter() - t0
                        pending.remove((i, ticket))
            time.sleep(0.0001)

    th = threading.Thread(target=poller)
    t0 = time.perf_counter()
    th.start()
    for i, (_, s, _) in enumerate(trace):
        wait = arrive[i] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ticket, _ = batch.msc_batch_submit([inputs[i]], [plans[s]])
        with lock:
            pending.append((i, ticket))
    while True:
        with lock:
            if not pending:
                break
        time.sleep(0.0005)
    stop.set()
    th.join()
    return arrive, done


def _serve_summary(trace, sizes, arrive, done):
    nvox = sum(sizes[s] ** 3 for _, s, _ in trace)
    lat = sorted(1e3 * (d - a) for a, d in zip(arrive, done))
    span = max(done) - min(arrive)
    return {"value": nvox / span / 1e6, "unit": "Mvoxel/s", "span_s": span,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1], "mean": sum(lat) / len(lat)}}


def leg_serve(msc, torch, n_requests, workers, budget, uuid):
    """Serving: the first n_requests of the Poisson trace (200 req/s over the 8 advected streams),
    each request's field synthesised on the device before the timed region, served by the
    continuous-batching runtime (HBM-budget admission, each stream keeping its plan on the device)
    and, on the same trace, one request at a time in arrival order on default plans; both arms also
    with every request available at once (saturated)."""
    from synth import fields

    streams = fields.serving_streams()
    sizes = [st.size for st in streams]
    trace = fields.request_trace()[:n_requests]
    inputs = [streams[s].step_device(step + 1) for _, s, step in trace]
    single = [msc.Plan((n, n, n)) for n in sizes]
    batch = msc.Batch(n_workers=workers, hbm_budget_bytes=budget)
    served = [None] * len(streams)
    for s in range(len(streams)):  # each stream's plans: first pass, graph capture
        for _ in range(2):
            ticket, out = batch.msc_batch_submit([inputs[s]], [served[s]])
            served[s] = out[0]
            assert batch.msc_batch_wait(ticket) == 0
            msc.msc_compute(single[s], inputs[s])
    torch.cuda.synchronize()
    res = {}
    with ClockSampler(uuid) as clk:
        for mode, sat in (("poisson", False), ("saturated", True)):
            a, d = _serve_arm(msc, torch, trace, inputs, served, batch, sat)
            res[f"served_{mode}"] = _serve_summary(trace, sizes, a, d)
            a, d = _serve_arm(msc, torch, trace, inputs, single, None, sat)
            res[f"one_at_a_time_{mode}"] = _serve_summary(trace, sizes, a, d)
    batch.close()
    nvox = sum(sizes[s] ** 3 for _, s, _ in trace)
    res.update({"workload": f"serve: {WORKLOADS['serve500']} (first {len(trace)} requests)",
                "requests": len(trace), "voxels": nvox, "workers": workers, "hbm_budget_bytes": budget,
                "offered_mvoxel_s": nvox / trace[-1][0] / 1e6,
                "inputs": "every request's field synthesised on the GPU before the timed region",
                "timing": "host clock from the first arrival to the last completion; latency = completion - "
                          "arrival; saturated = every request available at t = 0",
                "served_over_one_at_a_time": {m: res[f"one_at_a_time_{m}"]["span_s"] / res[f"served_{m}"]["span_s"]
                                              for m in ("poisson", "saturated")},
                "clocks": clk.summary()})
    return res


def _standalone_line(args, leg, value, ms, steps):
    return {"metric": METRIC, "value": value, "unit": "Mvoxel/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-compare/u64-count", "data": "synthetic",
            "config": {"workload": leg["workload"]}, "leg": leg, "clocks": leg.get("clocks")}


def run_multi(args):
    """--workload batch64 | serve500 alone: the leg's JSON line."""
    import torch

    from paper_2009_03707_gb300 import msc

    torch.cuda.set_device(0)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        pass
    if args.workload == "batch64":
        leg = leg_batch(msc, torch, args.steps, args.workers, uuid, with_cpu=not args.no_cpu_baseline)
        line = _standalone_line(args, leg, leg["batched"]["value"], leg["batched"]["ms"], args.steps)
    else:
        leg = leg_serve(msc, torch, args.requests, args.workers, args.serve_budget, uuid)
        line = _standalone_line(args, leg, leg["served_poisson"]["value"],
                                1e3 * leg["served_poisson"]["span_s"] / leg["requests"], leg["requests"])
    if "cpu_baseline" in leg:
        line["cpu_baseline"] = leg.pop("cpu_baseline")
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
    ap.add_argument("--requests", type=int, default=200, help="serving: the first R requests of the 500-request trace")
    ap.add_argument("--serve-budget", type=int, default=24 << 30, help="serving: HBM admission budget in bytes")
    ap.add_argument("--no-legs", action="store_true",
                    help="grf256: skip the legs that the default run adds")
    ap.add_argument("--legs", default="outputs,simplify,blobs512,batch64,serve",
                    help="grf256: the legs to add (comma-separated subset of the default)")
    ap.add_argument("--no-graph", action="store_true",
                    help="run every pass synchronised between stages instead of replaying its CUDA graph "
                         "(same kernels; profilers list each launch)")
    ap.add_argument("--gradient-tile", type=int, default=0, help="force a lower-star tile variant (1..9)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps are required")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("batch64", "serve500"):
        run_multi(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
