#!/usr/bin/env python
"""Throughput benchmark of the GB300 stereo path.  Prints ONE JSON line (rank 0).

Workload: 1242x375 driving-shaped synthetic pairs (ground plane + 40 boxes,
noise sigma 3, 5% unmatched pixels), N_D = 128, 3 refine+resample iterations,
8x8 initial cells.  One step = one batch of distinct pairs through the whole
method (census, FAST bins, epipolar match, host Delaunay, raster, fused
validate, resample + match) via the request API with continuous batching.
Inputs are resident in HBM when a step starts; L2 is flushed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]

--impl reference times the CPU oracle (the plain restatement of the method)
on the same workload, one pair per step, on the host cores.  With N > 1 the
pairs shard across ranks (independent replicas, no collective on the data
path); the timed region is bracketed by barriers and the max over ranks.
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
os.environ.setdefault("STEREO_SCENE_CACHE", os.path.join(tempfile.gettempdir(), "stereo_scenes"))

WORKLOAD = "driving_1242x375"
PRM = dict(t_lo=4, t_hi=8, t_grad=8, t_fast=20, kp_per_bin=4, uniq_margin=2)
METRIC = "Mpix/s"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def _workload_config(batch, W, H, p, window=0):
    kind = "driving-shaped" if WORKLOAD.startswith("driving") else "polygon-scene"
    return {"workload": f"{W}x{H} {kind} synthetic pairs, dmax {p.dmax}, {p.iters} iterations, "
                        f"{p.cell}x{p.cell} initial cells, " + (f"{batch} distinct pairs per step" if batch > 1 else "1 pair per step"),
            "pairs_per_step": batch, "batch_window_us": window, "W": W, "H": H, "dmax": p.dmax, "iters": p.iters, "cell": p.cell,
            "l2": "flushed between steps (256 MiB write), flush outside the timed spans",
            "omega": "dense (t_grad 0)" if PRM["t_grad"] == 0 else f"semi-dense (t_grad {PRM['t_grad']})",
            "parallelism": "replicas: pairs sharded across ranks, no data-path collective"}


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is running (its first line is out)
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import oracle
    import scenes
    oracle.build()
    pairs = scenes.config_pairs(WORKLOAD, n=1)
    p = pairs[0]
    H, W = p.left.shape
    # one pair per step takes the oracle about 2.3 s: the run is bounded to 20 steps and one
    # warm-up (under a minute) whatever --steps asks for; the line reports what ran
    steps, warm = max(1, min(args.steps, 20)), min(args.warmup, 1)
    for _ in range(warm):
        oracle.run(p.left, p.right, p.dmax, p.iters, p.cell, **PRM)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.run(p.left, p.right, p.dmax, p.iters, p.cell, **PRM)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = W * H * steps / tot / 1e6
    cfg = _workload_config(1, W, H, p)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": args.gpus,
           "steps": steps, "warmup": warm, "steps_requested": args.steps, "ms_per_step": 1e3 * tot / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/f32",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                            "sample": f"one {W}x{H} pair per step, whole method, single thread"},
           "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ replicas across ranks
def rank_shard(rank, batch):
    """First pair index and count of a rank: every rank runs its own distinct pairs (no shared data)."""
    return rank * batch, batch


def max_over_ranks(value, world, dist=None, device="cpu"):
    """The step time that counts is the slowest rank's (all ranks start after a barrier)."""
    if world <= 1 or dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(px_per_rank_step, steps, world, max_ms):
    """Pixels all ranks processed divided by the slowest rank's time."""
    return world * px_per_rank_step * steps / (max_ms / 1e3) / 1e6


# Kernel timing: CUDA events around the launches of every PROFILE_EVERY-th GPU round.  The event
# nodes lengthen a round by tens of microseconds, so timing every round slows the workload it
# measures; the mean launch time comes from the timed rounds and totals scale to all launches.
PROFILE_EVERY = 4

# ------------------------------------------------------------------ our arm
def _source_hash(kind=None):
    """Hash of the sources a kernel kind is built from (the mesh pass lives in retess.cu)."""
    h = hashlib.sha256()
    main = "retess.cu" if kind == "mesh" else "kernels.cu"
    for f in (f"paper_1511_00758_gb300/csrc/{main}", "paper_1511_00758_gb300/csrc/internal.h"):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kind, algo_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu capture of this kernel kind, scaled from the
    captured launch to this run's average launch by algorithmic bytes (traffic grows in proportion);
    None when there is no capture or the kernel source changed since it was taken."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        e = d[kind]
        if e.get("source_hash") != _source_hash(kind) or not algo_bytes_per_launch:
            return None
        return e["dram_bytes"] * algo_bytes_per_launch / e["algorithmic_bytes"]
    except Exception:
        return None


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1511_00758_gb300 as S
    import scenes

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    S.load()
    B = args.batch
    first, count = rank_shard(rank, B)
    pairs = scenes.config_pairs(WORKLOAD, n=count, first=first)
    H, W = pairs[0].left.shape
    p0 = pairs[0]
    px_step = W * H * B
    dev_in = [(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda()) for p in pairs]
    host_in = []
    for p in pairs:
        l = torch.from_numpy(p.left).pin_memory()
        r = torch.from_numpy(p.right).pin_memory()
        host_in.append((l, r))
    host_out = [(torch.empty((H, W), dtype=torch.float32).pin_memory(),
                 torch.empty((H, W), dtype=torch.uint8).pin_memory()) for _ in pairs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ncpu = os.cpu_count() or 1
    # one core stays free for the scheduler thread and this client thread (measured faster)
    threads = args.host_threads or max(1, min(B, ncpu // max(1, world) - 1))
    budget = int(0.5 * 2**30) + B * S.request_bytes(W, H, p0.dmax, p0.iters, p0.cell)
    ctx = S.Context(device=local, mem_budget_bytes=budget, max_slots=B, max_queue=4 * B, host_threads=threads,
                    profile=PROFILE_EVERY, batch_window_us=args.window_us, autotune=0 if args.no_autotune else 1,
                    tune_w=W, tune_h=H, host_mesh=1 if args.host_mesh else 0, **PRM)
    stream = ctx.stream

    host_ms = {"submit": 0.0, "poll": 0.0, "steps": 0}

    def one_step(host=False):
        lat = []
        ins = host_in if host else dev_in
        t0 = time.perf_counter()
        # host leg: the library writes D_f and C_f into page-locked host buffers named at
        # submit, in the GPU round that finishes each request
        tickets = ctx.submit_batch([(l, r, W, H, p.dmax, p.iters, p.cell, 0, (o[0], o[1], None) if host else None)
                                    for (l, r), p, o in zip(ins, pairs, host_out)])
        t1 = time.perf_counter()
        if len(tickets) != len(pairs):
            raise RuntimeError(f"only {len(tickets)} of {len(pairs)} pairs taken")
        for r in ctx.poll_batch(tickets):
            if r.status != 0:
                raise RuntimeError(f"request failed: {r.status}")
            lat.append(r.latency_ms)
        ctx.release_batch(tickets)
        if not host:
            host_ms["submit"] += 1e3 * (t1 - t0)
            host_ms["poll"] += 1e3 * (time.perf_counter() - t1)
            host_ms["steps"] += 1
        return lat

    def timed(nsteps, host=False):
        spans, lats = [], []
        for _ in range(nsteps):
            flush.fill_(1)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lats += one_step(host)
            e1.record(stream)
            e1.synchronize()
            spans.append(e0.elapsed_time(e1))
        return spans, lats

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    host_ms.update(submit=0.0, poll=0.0, steps=0)
    s0 = ctx.stats()
    clocks = Clocks(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]
                    if os.environ.get("CUDA_VISIBLE_DEVICES") else local)
    clocks.start()
    spans, lats = timed(args.steps)
    clk = clocks.stop()
    s1 = ctx.stats()
    max_ms = max_over_ranks(sum(spans), world, dist if world > 1 else None, device="cuda")
    value = whole_job_mpix_s(px_step, args.steps, world, max_ms)

    # roofline of the dominant kernel kind, from the CUDA events recorded inside the timed region
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    per = {}
    timed_launches = {}
    for i, name in enumerate(S.KINDS):
        nl = s1.kind_launches[i] - s0.kind_launches[i]
        nt = s1.kind_timed[i] - s0.kind_timed[i]
        mt = s1.kind_ms[i] - s0.kind_ms[i]
        # the timed launches (every PROFILE_EVERY-th round) give the mean; all launches the total
        per[name] = (nl, mt / nt * nl if nt else 0.0, s1.kind_bytes[i] - s0.kind_bytes[i])
        timed_launches[name] = nt
    # a separate clear launch (if any) belongs to the raster pass over the same map
    rc, rr = per.pop("raster_clear"), per.pop("raster")
    per["raster"] = (rr[0], rc[1] + rr[1], rc[2] + rr[2])
    dominant = max(per, key=lambda n: per[n][1])
    with_bytes = [n for n in sorted(per, key=lambda n: -per[n][1]) if per[n][2] > 0]
    rk = dominant if per[dominant][2] > 0 else with_bytes[0]
    nl, kms, kbytes = per[rk]
    achieved = (kbytes / nl) / (kms / nl * 1e-3) / 1e9 if nl and kms > 0 else None
    names = {"validate": "k_validate (cost evaluation + refinement, fused)",
             "raster": "k_raster (lookup table + interpolation, hull-interval clear fused)",
             "census": "k_census", "fast_score": "k_fast_score", "fill": "k_fill_cells",
             "mesh": "k_mesh_pass (re-tessellation: insertion + flips, planes, raster lists; a cluster per pair)"}
    roofline = {"kernel": names.get(rk, rk), "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "peak_source": "measured" if peaks else "fallback",
                "traffic": _traffic(rk, kbytes / nl if nl else None), "launches": nl, "avg_launch_us": 1e3 * kms / nl if nl else None,
                "algorithmic_bytes_per_launch": kbytes / nl if nl else None,
                "share_of_kernel_time": kms / max(1e-9, sum(v[1] for v in per.values())),
                "dominant_kernel": dominant, "pairs_per_launch_mean": None}
    other = {}
    for n in with_bytes:
        if n == rk:
            continue
        l_, m_, b_ = per[n]
        if l_ and m_ > 0:
            other[n] = {"gbs": (b_ / l_) / (m_ / l_ * 1e-3) / 1e9, "frac": (b_ / l_) / (m_ / l_ * 1e-3) / 1e9 / peak,
                        "avg_launch_us": 1e3 * m_ / l_, "traffic": _traffic(n, b_ / l_)}
    roofline["other_kernels"] = other
    roofline["timed_launches"] = timed_launches.get(rk, 0) + (timed_launches.get("raster_clear", 0) if rk == "raster" else 0)
    roofline["timing"] = (f"CUDA events around the launches of every {PROFILE_EVERY}th round (event nodes lengthen "
                          "a round); mean launch time from those, totals scaled to all launches")
    kinds = {}
    for i, name in enumerate(S.KINDS):
        nl = s1.kind_launches[i] - s0.kind_launches[i]
        nt = s1.kind_timed[i] - s0.kind_timed[i]
        mt = s1.kind_ms[i] - s0.kind_ms[i]
        kb = s1.kind_bytes[i] - s0.kind_bytes[i]
        kinds[name] = {"launches": nl, "timed": nt, "ms": round(mt / nt * nl, 4) if nt else 0.0,
                       "algorithmic_bytes_per_launch": kb / nl if nl else None}
    tuning = ctx.tuning()
    rounds = s1.gpu_rounds - s0.gpu_rounds
    round_stats = {"rounds_per_step": rounds / args.steps,
                   "submit_ms_per_step": host_ms["submit"] / max(1, host_ms["steps"]),
                   "poll_wait_ms_per_step": host_ms["poll"] / max(1, host_ms["steps"]),
                   "round_wall_ms": (s1.round_ms - s0.round_ms) / max(1, rounds),
                   "graph_ms": (s1.graph_ms - s0.graph_ms) / max(1, rounds),
                   "exec_ms": (s1.exec_ms - s0.exec_ms) / max(1, rounds),
                   "instantiations_per_step": (s1.graph_instantiations - s0.graph_instantiations) / args.steps,
                   "scheduler_busy": (s1.round_ms - s0.round_ms) / max(1e-9, sum(spans))}
    launches = s1.kernel_launches - s0.kernel_launches
    if launches:
        roofline["pairs_per_launch_mean"] = (s1.batched_pairs - s0.batched_pairs) / launches
    mp = s1.mesh_passes - s0.mesh_passes
    mesh_stats = {"path": "host" if args.host_mesh else "device",
                  "device_passes_per_step": mp / args.steps,
                  "insert_rounds_per_pass": (s1.mesh_insert_rounds - s0.mesh_insert_rounds) / max(1, mp),
                  "flip_rounds_per_pass": (s1.mesh_flip_rounds - s0.mesh_flip_rounds) / max(1, mp),
                  "flips_per_pass": (s1.mesh_flips - s0.mesh_flips) / max(1, mp),
                  "points_per_pass": (s1.mesh_points - s0.mesh_points) / max(1, mp),
                  "edge_points_per_pass": (s1.mesh_edge_points - s0.mesh_edge_points) / max(1, mp)}

    # end to end through the public API with host buffers, copies inside the span
    one_step(host=True)  # untimed: the host leg's first round
    e2e_spans, _ = timed(max(1, min(args.steps, 20)), host=True)
    e2e = {"value": px_step * len(e2e_spans) / (sum(e2e_spans) / 1e3) / 1e6, "unit": "Mpix/s",
           "h2d_bytes_per_step": 2 * px_step, "d2h_bytes_per_step": 5 * px_step}
    mesh_ms = (s1.host_mesh_ms - s0.host_mesh_ms) / max(1, (s1.requests_done - s0.requests_done))
    ctx.close()

    # plain per-pair path: one request in flight, one host thread
    plain = None
    if not args.no_plain:
        pctx = S.Context(device=local, mem_budget_bytes=budget, max_slots=1, max_queue=4 * B, host_threads=1,
                         autotune=0 if args.no_autotune else 1, tune_w=W, tune_h=H,
                         host_mesh=1 if args.host_mesh else 0, **PRM)
        ctx_plain = pctx
        nplain = min(B, 4)

        def plain_step():
            for (l, r), p in list(zip(dev_in, pairs))[:nplain]:
                tk = ctx_plain.submit(l, r, W, H, p.dmax, p.iters, p.cell)
                ctx_plain.poll(tk)
                ctx_plain.release(tk)
        plain_step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(pctx.stream)
        plain_step()
        e1.record(pctx.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        plain = {"value": W * H * nplain / (ms / 1e3) / 1e6, "unit": "Mpix/s",
                 "pairs_per_s": nplain / (ms / 1e3), "pairs_timed": nplain}
        pctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        n = 0
        while True:
            oracle.run(p0.left, p0.right, p0.dmax, p0.iters, p0.cell, **PRM)
            n += 1
            if time.perf_counter() - t0 > 8.0 or n >= 3:
                break
        dt = time.perf_counter() - t0
        cpu = {"value": W * H * n / dt / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} x the first {W}x{H} pair of the workload, whole method, single thread"}

    if rank == 0:
        lats.sort()
        out = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "u8/f32", "data": "synthetic",
               "config": _workload_config(B, W, H, p0, args.window_us),
               "pairs_per_s": world * B * args.steps / (max_ms / 1e3),
               "latency_ms": {"p50": lats[len(lats) // 2], "p99": lats[min(len(lats) - 1, int(0.99 * len(lats)))]},
               "host_mesh_ms_per_pair": mesh_ms, "host_threads": threads,
               "plain": plain, "roofline": roofline, "kernels": kinds, "rounds": round_stats, "mesh": mesh_stats, "tuning": tuning,
               "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": clk}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ other workloads
def _make_ctx(S, local, pairs, slots, threads, window_us=0, profile=PROFILE_EVERY):
    need = sum(S.request_bytes(p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell) for p in pairs[:slots])
    big = max(pairs, key=lambda p: p.left.size)  # the tuning round uses the largest frame
    return S.Context(device=local, mem_budget_bytes=int(0.5 * 2**30) + need, max_slots=slots, max_queue=4096,
                     host_threads=threads, profile=profile, batch_window_us=window_us, autotune=1,
                     tune_w=big.left.shape[1], tune_h=big.left.shape[0], **PRM)


def run_batch_workload(args, name):
    """One step = every pair of the workload through the batched engine."""
    import torch

    import paper_1511_00758_gb300 as S
    import scenes
    S.load()
    torch.cuda.set_device(0)
    pairs = scenes.mixed_pairs(64) if name == "mixed" else (scenes.large_pairs(16) if name == "large"
                                                            else scenes.burst_pairs(32))
    dev = [(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda()) for p in pairs]
    threads = max(1, (os.cpu_count() or 1) - 1)  # one core for the scheduler and this thread
    ctx = _make_ctx(S, 0, pairs, len(pairs), threads, args.window_us)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        lat = []
        ts = [ctx.submit(l, r, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell) for (l, r), p in zip(dev, pairs)]
        for t in ts:
            res = ctx.poll(t)
            if res.status != 0:
                raise RuntimeError(f"request failed: {res.status}")
            lat.append(res.latency_ms)
            ctx.release(t)
        return lat
    for _ in range(args.warmup):
        step()
    s0 = ctx.stats()
    spans, lats = [], []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        lats += step()
        e1.record(ctx.stream)
        e1.synchronize()
        spans.append(e0.elapsed_time(e1))
    s1 = ctx.stats()
    ctx.close()
    px = sum(p.left.size for p in pairs)
    tot = sum(spans) / 1e3
    lats.sort()
    k = 6  # validate
    nl = s1.kind_launches[k] - s0.kind_launches[k]
    nt = s1.kind_timed[k] - s0.kind_timed[k]
    kms = (s1.kind_ms[k] - s0.kind_ms[k]) / nt * nl if nt else 0.0  # all launches, from the timed ones
    kb = s1.kind_bytes[k] - s0.kind_bytes[k]
    desc = {"mixed": "64 uneven pairs (16 each of 320x240, 640x480, 1242x375 driving, 1280x720), dmax 64-128, "
                     "3 iterations, 16x16 cells, one batch per step",
            "large": "16 pairs of 2048x1536, 30-plane scenes, dmax 256, 5 iterations, 4x4 initial cells",
            "burst": "32 concurrent 1920x1080 streams arriving together, dmax 128, 2 iterations, 16x16 cells"}[name]
    out = {"metric": METRIC, "value": px * args.steps / tot / 1e6, "unit": "Mpix/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
           "higher_is_better": True, "data": "synthetic", "config": {"workload": desc, "pairs_per_step": len(pairs)},
           "pairs_per_s": len(pairs) * args.steps / tot,
           "latency_ms": {"p50": lats[len(lats) // 2], "p99": lats[min(len(lats) - 1, int(0.99 * len(lats)))]},
           "host_mesh_ms_per_pair": (s1.host_mesh_ms - s0.host_mesh_ms) / max(1, s1.requests_done - s0.requests_done),
           "validate_gbs": (kb / (kms * 1e-3) / 1e9) if kms > 0 else None,
           "validate_pairs_per_launch": (s1.batched_pairs - s0.batched_pairs) / max(1, s1.kernel_launches - s0.kernel_launches),
           "gpu_launches": s1.kernel_launches - s0.kernel_launches}
    out["cpu_baseline"] = None if args.no_cpu else _oracle_all_cores(name, pairs)
    print(json.dumps(out))
    return 0


def _oracle_all_cores(name, pairs):
    """The oracle, one pair per thread on min(pairs, cores) host cores (the C oracle releases the
    interpreter lock), over pairs spread evenly through the workload: a bounded sample of it."""
    if name == "large":
        return {"value": None, "unit": "Mpix/s", "cores": 0, "kind": "oracle",
                "sample": "not run: the oracle's gift-wrapping triangulation is O(n^2) in the support points, "
                          "and cells down to 1x1 make millions of them per pair (hours per pair)"}
    import threading

    import oracle
    oracle.build()
    ncore = max(1, min(len(pairs), os.cpu_count() or 1))
    step = max(1, len(pairs) // ncore)
    sample = pairs[::step][:ncore]
    th = [threading.Thread(target=oracle.run, args=(p.left, p.right, p.dmax, p.iters, p.cell), kwargs=PRM)
          for p in sample]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    dt = time.perf_counter() - t0
    return {"value": sum(p.left.size for p in sample) / dt / 1e6, "unit": "Mpix/s", "cores": ncore,
            "kind": "oracle", "sample": f"{len(sample)} pairs spread through the workload, one per thread on "
                                        f"{ncore} host cores, whole method"}


def run_kernel(args, which):
    """One kernel alone on a 4096x4096 frame (inputs larger than L2) through the stage entry points:
    random images, their census, and a smooth slanted D_it field; CUDA events on the launching stream."""
    import torch

    import paper_1511_00758_gb300 as S
    S.load()
    torch.cuda.set_device(0)
    W = H = args.kernel_size
    g = torch.Generator(device="cuda").manual_seed(0x5EED0006)
    L = torch.randint(0, 256, (H, W), dtype=torch.uint8, device="cuda", generator=g)
    R = torch.roll(L, shifts=-5, dims=1).contiguous()
    cL = torch.empty((H, W), dtype=torch.int32, device="cuda")
    cR = torch.empty_like(cL)
    om = torch.empty((H, (W + 31) // 32), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    S.census(L, R, W, H, PRM["t_grad"], cL, cR, om, stream)
    vv, uu = torch.meshgrid(torch.arange(H, device="cuda", dtype=torch.float32),
                            torch.arange(W, device="cuda", dtype=torch.float32), indexing="ij")
    Dit = (5.0 + 0.001 * uu + 0.002 * vv).contiguous()
    Df = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    Cf = torch.full((H, W), PRM["t_hi"], dtype=torch.uint8, device="cuda")
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    sz = max(1, args.cell)  # cell side of the resample records (--cell 0: the last pass, no records)
    nc = -(-W // sz) * -(-H // sz)
    cg = torch.empty(nc, dtype=torch.int32, device="cuda") if args.cell > 0 else None
    cb = torch.empty(nc, dtype=torch.int32, device="cuda") if args.cell > 0 else None
    # a mesh for the raster: a jittered lattice of support points, triangulated on the host
    import numpy as np
    rng = np.random.default_rng(6)
    step = args.mesh_step
    P = np.array([(min(W - 1, u + int(rng.integers(0, step))), min(H - 1, v + int(rng.integers(0, step))))
                  for v in range(0, H, step) for u in range(0, W, step)], np.int32)
    P = np.unique(P, axis=0)
    P = np.ascontiguousarray(P[np.lexsort((P[:, 0], P[:, 1]))])
    tri = np.zeros((2 * len(P) + 8, 3), np.int32)
    T = S.delaunay(P, len(P), tri, len(tri))
    D = (5.0 + 0.001 * P[:, 0] + 0.002 * P[:, 1]).astype(np.float32)
    abc = np.zeros((T, 3), np.float32)
    S.planes(P, D, tri[:T], T, abc)
    tuv = torch.from_numpy(np.ascontiguousarray(P[tri[:T]].reshape(-1, 6))).cuda()
    tabc = torch.from_numpy(abc).cuda()
    nbytes = S.raster_scratch_bytes(T)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    Dit2 = torch.empty_like(Dit)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")

    def once():
        if which == "validate":
            if cg is not None:
                cg.fill_(-1)
                cb.fill_(-1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if args.plain_kernel:
                S.validate(cL, cR, om, Dit, W, H, sz, PRM["t_lo"], PRM["t_hi"], 0, Df, Cf, mask, cg, cb, stream)
            else:
                S.validate_bulk(cL, cR, om, Dit, W, H, sz, PRM["t_lo"], PRM["t_hi"], 0, Df, Cf, mask, cg, cb, err,
                                stream)
            e1.record(stream)
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.raster(tuv, tabc, T, W, H, None, Dit2, scratch, nbytes, stream)
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)
    for _ in range(args.warmup):
        once()
    ms = [once() for _ in range(args.steps)]
    avg = sum(ms) / len(ms)
    px = W * H
    algo = px * (19.125 if which == "validate" else 8.0)  # raster: clear + write of D_it
    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    if which == "validate" and not args.plain_kernel and int(err.item()) != 0:
        raise RuntimeError("a bounded wait of the bulk validate kernel gave up")
    out = {"kernel": ("k_validate" if args.plain_kernel else "k_validate_bulk") if which == "validate"
           else "k_raster_clear + k_raster (D_it only)",
           "frame": f"{W}x{H}", "pixels": px, "triangles": T if which == "raster" else None,
           "cell": args.cell if which == "validate" else None,
           "algorithmic_bytes": algo, "avg_us": 1e3 * avg, "gbs": algo / (avg * 1e-3) / 1e9,
           "frac": algo / (avg * 1e-3) / 1e9 / peak, "peak": peak, "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(out))
    return 0


def run_serving(args):
    """Eight camera streams with Poisson arrivals at 120 Hz each; requests are admitted as slots and
    memory free up; latency is submit -> result ready."""
    import queue
    import threading

    import numpy as np
    import torch

    import paper_1511_00758_gb300 as S
    import scenes
    S.load()
    torch.cuda.set_device(0)
    streams = scenes.serving_streams()
    host = [(torch.from_numpy(p.left).pin_memory(), torch.from_numpy(p.right).pin_memory()) for p in streams]
    threads = max(1, (os.cpu_count() or 1) - 1)  # one core for the scheduler and this thread
    ctx = _make_ctx(S, 0, streams * 2, 16, threads, window_us=0, profile=0)
    rng = np.random.default_rng(0x5EED0004)
    arrivals = []
    for sid in range(len(streams)):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / args.rate_hz)
            if t >= args.duration_s:
                break
            arrivals.append((t, sid))
    arrivals.sort()
    done_q = queue.Queue()
    lat, errors = [], []

    def poller():
        while True:
            item = done_q.get()
            if item is None:
                return
            ticket = item
            res = ctx.poll(ticket)
            if res.status != 0:
                errors.append(res.status)
            lat.append(res.latency_ms)
            ctx.release(ticket)
    th = threading.Thread(target=poller)
    th.start()
    busy = 0
    t0 = time.perf_counter()
    for at, sid in arrivals:
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        p = streams[sid]
        l, r = host[sid]
        while True:
            try:
                tk = ctx.submit(l, r, p.left.shape[1], p.left.shape[0], p.dmax, p.iters, p.cell, stream_id=sid)
                break
            except S.StereoError as e:
                if e.code != -3:
                    raise
                busy += 1
                time.sleep(0.0005)
        done_q.put(tk)
    done_q.put(None)
    th.join()
    wall = time.perf_counter() - t0
    st = ctx.stats()
    ctx.close()
    lat.sort()
    px = sum(streams[sid].left.size for _, sid in arrivals)
    out = {"metric": "p50/p99 latency and throughput under Poisson arrivals", "unit": "ms",
           "config": {"workload": f"8 streams (4 x 640x480 dmax 64, 4 x 1280x720 dmax 128), Poisson "
                                  f"{args.rate_hz} Hz per stream for {args.duration_s} s, 2 iterations, 16x16 cells, "
                                  "host input buffers, 16 slots"},
           "requests": len(arrivals), "failed": len(errors), "busy_retries": busy,
           "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                          "max": lat[-1]},
           "throughput_pairs_per_s": len(arrivals) / wall, "throughput_mpix_s": px / wall / 1e6,
           "offered_pairs_per_s": len(arrivals) / args.duration_s,
           "mean_pairs_per_launch": st.batched_pairs / max(1, st.kernel_launches), "gpu_rounds": st.gpu_rounds}
    print(json.dumps(out))
    return 0


def accuracy(D_f, C_f, mask, gt, occ, t_hi):
    """Error-rate protocol of the paper's accuracy table, on synthetic ground
    truth: over the valid (C_f < t_hi), non-occluded pixels of Omega_I (mask
    bit 0), the share within tau px of the truth, tau = 2..5; and the density,
    the share of non-occluded Omega_I pixels that are valid."""
    import numpy as np
    sel = ((mask & 1) != 0) & ~occ
    ok = (C_f < t_hi) & sel
    nv = max(1, int(ok.sum()))
    err = np.abs(D_f - gt)
    out = {f"lt{t}px": float(((err < t) & ok).sum() / nv) for t in (2, 3, 4, 5)}
    out["density"] = float(ok.sum() / max(1, int(sel.sum())))
    return out


def run_sweep(args):
    """The paper's runtime table as a workload: 320x240 .. 1920x1080, 1 / 2 / 4
    iterations, 4 pairs per point through the batched engine; per point the time
    per pair and the error rates of the accuracy protocol on synthetic truth."""
    import numpy as np
    import torch

    import paper_1511_00758_gb300 as S
    import scenes
    S.load()
    torch.cuda.set_device(0)
    threads = max(1, (os.cpu_count() or 1) - 1)  # one core for the scheduler and this thread
    rows = []
    for W, H, dmax in scenes.SWEEP_SIZES:
        pairs = scenes.sweep_pairs(W, H, dmax, 4)
        dev = [(torch.from_numpy(p.left).cuda(), torch.from_numpy(p.right).cuda()) for p in pairs]
        ctx = _make_ctx(S, 0, pairs, len(pairs), threads, args.window_us)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        for iters in (1, 2, 4):
            def step(keep=False):
                ts = ctx.submit_batch([(l, r, W, H, dmax, iters, p.cell) for (l, r), p in zip(dev, pairs)])
                if len(ts) != len(pairs):
                    raise RuntimeError("the batch was not taken whole")
                res = []
                for r in ctx.poll_batch(ts):
                    if r.status != 0:
                        raise RuntimeError(f"request failed: {r.status}")
                    if keep:
                        o = ctx.result_tensors(r)
                        res.append({k: o[k].cpu().numpy() for k in ("D_f", "C_f", "mask")})
                ctx.release_batch(ts)
                return res
            step()
            spans = []
            s0 = ctx.stats()
            for _ in range(max(1, args.steps)):
                flush.fill_(1)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                step()
                e1.record(ctx.stream)
                e1.synchronize()
                spans.append(e0.elapsed_time(e1))
            s1 = ctx.stats()
            nsteps = max(1, args.steps)
            kern = {}
            for i, name in enumerate(S.KINDS):
                nl, nt = s1.kind_launches[i] - s0.kind_launches[i], s1.kind_timed[i] - s0.kind_timed[i]
                if nl and nt:
                    kern[name] = round((s1.kind_ms[i] - s0.kind_ms[i]) / nt * nl / nsteps, 4)
            res = step(keep=True)  # results for the accuracy protocol, outside the timed steps
            acc = [accuracy(o["D_f"], o["C_f"], o["mask"], p.gt_disp, p.gt_occ, PRM["t_hi"]) for o, p in zip(res, pairs)]
            ms = sum(spans) / len(spans) / len(pairs)
            rows.append({"W": W, "H": H, "dmax": dmax, "iters": iters, "pairs": len(pairs), "ms_per_pair": ms,
                         "mpix_s": W * H / (ms * 1e-3) / 1e6,
                         "rounds_per_step": (s1.gpu_rounds - s0.gpu_rounds) / nsteps, "kernel_ms_per_step": kern,
                         **{k: float(np.mean([a[k] for a in acc])) for k in acc[0]}})
        ctx.close()
    out = {"metric": "ms per pair and error rates (sweep of the paper's runtime table)", "workload": "sweep",
           "unit": "ms/pair", "higher_is_better": False, "data": "synthetic",
           "config": {"workload": "polygon scenes (20 planes, noise sigma 2), 16x16 initial cells, 4 pairs per point "
                                  "submitted together; L2 flushed between steps",
                      "omega": "dense (t_grad 0)" if PRM["t_grad"] == 0 else f"semi-dense (t_grad {PRM['t_grad']})"},
           "rows": rows}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--window-us", type=int, default=0, help="batching window of the request scheduler")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", choices=("driving", "mixed", "serving", "large", "burst", "sweep", "kernel-validate",
                                           "kernel-raster"), default="driving")
    ap.add_argument("--dense", action="store_true", help="the dense variant: t_grad 0, every pixel evaluated")
    ap.add_argument("--host-threads", type=int, default=0, help="host triangulation workers (0: the core count)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default kernel work shapes")
    ap.add_argument("--host-mesh", action="store_true",
                    help="triangulate every pass on the host (the default re-tessellates on the device)")
    ap.add_argument("--config", choices=("driving_1242x375", "vga_polygons"), default="driving_1242x375",
                    help="scene configuration of the main workload (and of --impl reference)")
    ap.add_argument("--kernel-size", type=int, default=4096)
    ap.add_argument("--cell", type=int, default=8, help="kernel-validate: cell side of the resample records (0: none)")
    ap.add_argument("--plain-kernel", action="store_true", help="kernel-validate: the single-pass kernel")
    ap.add_argument("--mesh-step", type=int, default=6, help="kernel-raster: support-point spacing in pixels")
    ap.add_argument("--rate-hz", type=float, default=120.0)
    ap.add_argument("--duration-s", type=float, default=10.0)
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = args.config
    if args.dense:
        PRM["t_grad"] = 0
    if args.workload == "sweep":
        return run_sweep(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload.startswith("kernel-"):
        return run_kernel(args, args.workload.split("-", 1)[1])
    if args.workload in ("mixed", "large", "burst"):
        return run_batch_workload(args, args.workload)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
