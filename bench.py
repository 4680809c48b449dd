#!/usr/bin/env python
"""Benchmark of the watershed + waterfall hot path (arXiv 2410.08946) on GB300.

Workload (one "step"): the whole hierarchy -- watershed steps I-IV plus the
waterfall up to NL = 6 levels -- of a 928 x 928 x 928 (799,178,752 voxel)
uint16 gradient volume, 6-connectivity.  The volume is the seeded synthetic
stand-in for the paper's 800-megavoxel MicroCT image: distance to the nearest
of 50,000 random seed points scaled to [0, 65535], plus uniform noise
U{0..64}.  Inputs (1.6 GB) and outputs (19.2 GB) are far larger than L2, so
no cache flush is needed between steps.

Prints ONE JSON line (rank 0).  Keys:
  value / unit        Gvoxels processed per second, device-resident input
  e2e                 the same through ws_segment_host (pinned host buffers,
                      host<->device copies inside the timed region; median
                      of the per-step times, each step listed)
  roofline            the dominant kernel phase: algorithmic bytes per launch
                      / its CUDA-event time, against the measured HBM peak
  path_roofline       the whole step: (2 + 4 NL) bytes per voxel / step time
  path_dram           the whole step's measured DRAM bytes (ncu record of its
                      main kernels, while their source matches) / step time
  cpu_baseline        the CPU oracle (1 thread) on a bounded sample volume
  phases_ms           per-phase device time per step (CUDA events)
  gpu_launches        kernels libws enqueued per timed step
  clocks              nvidia-smi samples taken during the timed region
  small_configs       the other configurations (2D 256^2 and 4096^2, a 512^3
                      volume in 6- and 26-connectivity) and the NEXT-row
                      measurements (3D gradient, region-graph export, the
                      paper-literal waterfall); batch, serve: configs 3 and 4
--impl reference times the CPU oracle itself (the reference arm).
Multi-GPU (torchrun): replicas, one volume per rank, no collective on the
data path ("weak" scaling); value = voxels of all ranks / max rank time.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "watershed+waterfall Gvox/s & %HBM roofline; served p50/p99 ms vs per-image"
SIDE, SEEDS, NL, CONN = 928, 50000, 6, 6
SEED = 2410089460 + 2
FALLBACK_HBM_GBS = 6800.0

# Algorithmic bytes per voxel of each phase (minimal input + output of the
# function the phase computes; b = 2 bytes per uint16 sample).
PHASE_BYTES = {
    "step1": 2 + 2,              # k_init6: read G, write the 16-bit end slot (+ 8 B per path end, ~5% of voxels)
    "rag": 2 + 2,                # k_rag6: read end slots and G (per-basin and per-pair results only)
    "level_write": 2 + 4 * NL,   # k_write6: read end slots, write NL label planes
    "plateau": 2 + 4,            # k_plateau2 (plateau tiles only)
    "resolve_union": 2 + 4,      # k_resolve2 (plateau tiles only)
    "jump": 4 + 4,               # k_jump2 (plateau tiles only)
}
KERNEL_OF_PHASE = {"step1": "k_init6", "plateau": "k_plateau2", "resolve_union": "k_resolve2",
                   "jump": "k_jump2", "compact": "k_rank_*", "chase": "k_chase", "rag": "k_rag6",
                   "levels": "k_levels", "level_write": "k_write6", "cleanup": "k_edges_compact"}
# source file of each kernel (the traffic record is void once it changes)
KERNEL_SOURCE = {"k_init6": "ws_tiles.cuh", "k_rag6": "ws_tiles.cuh", "k_chase": "ws_tiles.cuh",
                 "k_write6": "ws_tiles.cuh", "k_levels": "ws_kernels.cuh"}


def workload_name(side):
    return (f"3D {side}x{side}x{side} uint16 distance-to-{SEEDS if side == SIDE else 'scaled'}-seeds + "
            f"U{{0..64}} noise, 6-connectivity, watershed + waterfall NL={NL}")


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def sample_seeds(side):
    return max(16, round(SEEDS * side ** 3 / SIDE ** 3))


class ClockSampler:
    """nvidia-smi clocks + throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _code_text(path):
    """The source without // comments, trailing blanks and empty lines: what the compiler sees, so that an
    edit of the comments alone keeps the traffic figures measured on that source."""
    out = []
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return "\n".join(out).encode()


def _source_sha(kernel):
    src = os.path.join(ROOT, "paper_2410_08946_gb300", "csrc", KERNEL_SOURCE.get(kernel, "ws_tiles.cuh"))
    return hashlib.sha256(_code_text(src)).hexdigest()[:16]


TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_short_name(full):
    """'void ws::<unnamed>::k_x<T, 1>(args)' -> 'k_x'."""
    n = full.replace("(anonymous namespace)::", "").replace("<unnamed>::", "").replace("void ", "")
    return n.split("<")[0].split("(")[0].strip().split("::")[-1]


def traffic_for(kernel, voxels, path=TRAFFIC_PATH):
    """DRAM bytes (read + write) per launch of `kernel` on `voxels` voxels,
    from the committed ncu record (bytes per voxel of a captured launch), if
    the kernel's source has not changed since it was captured."""
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    ent = rec.get(kernel)
    if not ent or ent.get("source_sha") != _source_sha(kernel):
        return None
    return ent["bytes_per_voxel"] * voxels


def path_dram(voxels, ms, peak, path=TRAFFIC_PATH):
    """Measured DRAM bytes of a whole step (read + write of the kernels that
    move nearly all of them, from the committed ncu record) over the step time;
    None unless every record matches the current source."""
    kerns = ("k_init6", "k_chase", "k_rag6", "k_write6")
    tr = {k: traffic_for(k, voxels, path) for k in kerns}
    if any(v is None for v in tr.values()):
        return None
    tot = sum(tr.values())
    ach = tot / (ms / 1e3) / 1e9
    return {"bytes_per_voxel": tot / voxels, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "kernels": list(kerns)}


def ingest_ncu(csv_path, voxels, out_path=TRAFFIC_PATH):
    """Writes profiles/traffic.json from an ncu --csv capture with the
    dram__bytes_read.sum / dram__bytes_write.sum metrics (one or more
    launches per kernel on a volume of `voxels` voxels)."""
    import csv
    per = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if len(r) > 10]
    hdr = rows[0]
    for r in rows[1:]:
        d = dict(zip(hdr, r))
        name = kernel_short_name(d["Kernel Name"])
        if d["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            v = float(d["Metric Value"].replace(",", ""))
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(d.get("Metric Unit", "byte"), 1)
            per.setdefault((name, d["ID"]), 0.0)
            per[(name, d["ID"])] += v * scale
    by = {}
    for (name, _), v in per.items():
        by.setdefault(name, []).append(v)
    out = {}
    for name, vs in by.items():
        if name in KERNEL_SOURCE:
            out[name] = {"bytes_per_voxel": statistics.median(vs) / voxels, "launches": len(vs),
                         "captured_voxels": voxels, "source_sha": _source_sha(name)}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out))
    return out


def host_link_gbs(torch, nbytes=4 << 30):
    """Host <-> device copy bandwidth of pinned memory (4 GiB each way)."""
    n = nbytes // 4
    dev = torch.empty(n, dtype=torch.int32, device="cuda")
    host = torch.empty(n, dtype=torch.int32).pin_memory()
    out = {}
    for name, dst, src in (("d2h", host, dev), ("h2d", dev, host)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        out[name] = 2 * nbytes / (time.perf_counter() - t0) / 1e9
    del dev, host
    return out


def cpu_baseline(side=320):
    """The oracle as it stands (one thread) on a bounded sample volume."""
    import oracle
    from paper_2410_08946_gb300 import synth
    n = sample_seeds(side)
    vol = synth.distance_volume(side, side, side, n, seed=SEED)
    t0 = time.perf_counter()
    oracle.segment(vol, CONN, NL)
    dt = time.perf_counter() - t0
    return {"value": side ** 3 / dt / 1e9, "unit": "Gvox/s", "cores": 1, "kind": "oracle",
            "sample": f"{side}^3 uint16 distance volume, {n} seeds (same density as 928^3 / 50,000), "
                      f"watershed + waterfall NL={NL}, one oracle run of {dt:.1f} s on 1 of "
                      f"{os.cpu_count()} host cores ({os.uname().machine})"}


def rank_env():
    """(world size, rank, local rank) of a torchrun launch; (1, 0, 0) otherwise."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group).  The
    timed region of every rank ends at the same barrier, so the slowest rank's
    time is the whole job's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units of all ranks (replicas: each rank does the same work) per second, in billions."""
    return units_per_rank * world / seconds / 1e9


def run_reference(args):
    """--impl reference: the CPU oracle on the host cores, bounded sample per step."""
    if rank_env()[1] != 0:   # under torchrun, rank 0 alone times the oracle
        return 0
    import oracle
    from paper_2410_08946_gb300 import synth
    side = args.ref_side
    n = sample_seeds(side)
    vol = synth.distance_volume(side, side, side, n, seed=SEED)
    for _ in range(args.warmup):
        oracle.segment(vol, CONN, NL)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.segment(vol, CONN, NL)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    value = side ** 3 / dt / 1e9
    sample = (f"{side}^3 uint16 distance volume, {n} seeds (same density as 928^3 / 50,000); "
              f"one oracle run per step on 1 of {os.cpu_count()} host cores ({os.uname().machine})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gvox/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": workload_name(SIDE), "sample_side": side, "l2": "not applicable (CPU)"},
            "cpu_baseline": {"value": value, "unit": "Gvox/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gvox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_small_configs(ctx, torch, reps=20):
    """Configs 0 and 1 (the 2D cases): 256^2 blob image, gradient + watershed +
    NL=3 (latency, us); 4096^2 blob gradient quantised to 16 levels, 4- and
    8-connectivity, NL=6 (Gpx/s and the algorithmic HBM fraction, b + 4 NL =
    25 B/px); a 512^3 volume in 6- and 26-connectivity; the region-graph export of
    two of its level planes; the paper-literal waterfall on it; its 3D gradient.  Device-resident
    inputs; median of `reps` CUDA-event timings."""
    import statistics
    from paper_2410_08946_gb300 import synth
    peak, _ = hbm_peak()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ctx.check()
        return statistics.median(ts), min(ts)

    out = {}
    img0 = torch.from_numpy(synth.blob_image(256, 256, 32, SEED - 2)).cuda()
    g0 = torch.empty_like(img0)
    lv0 = torch.empty((3, 256, 256), dtype=torch.int32, device="cuda")
    c0 = torch.empty(3, dtype=torch.int32, device="cuda")

    def cfg0():
        ctx.gradient(img0, 0, out=g0)
        ctx.segment(g0, 4, 3, lv0, c0)
    med, best = timed(cfg0)
    out["config0"] = {"workload": "2D 256x256 uint8 blob image: gradient + watershed + waterfall NL=3, "
                                  "4-connectivity", "us_median": med * 1e3, "us_min": best * 1e3}
    img1 = torch.from_numpy(synth.blob_image(4096, 4096, 2000, SEED - 1)).cuda()
    g1 = ctx.gradient(img1, 4)
    N1 = 4096 * 4096
    lv1 = torch.empty((6, 4096, 4096), dtype=torch.int32, device="cuda")
    c1 = torch.empty(6, dtype=torch.int32, device="cuda")
    for conn in (4, 8):
        med, best = timed(lambda: ctx.segment(g1, conn, 6, lv1, c1))
        out[f"config1_conn{conn}"] = {
            "workload": f"2D 4096x4096 uint8 blob gradient quantised to 16 levels, {conn}-connectivity, "
                        "watershed + waterfall NL=6", "ms_median": med, "gpx_s": N1 / med / 1e6,
            "alg_hbm_frac": 25 * N1 / (med / 1e3) / 1e9 / peak, "levels_counts": c1.cpu().tolist()}
    del lv1, g1, img1
    torch.cuda.empty_cache()
    # 26-connectivity (a NEXT row): 512^3 distance volume, same seed density as 928^3
    side = 512
    v = torch.from_numpy(synth.distance_volume(side, side, side, sample_seeds(side), seed=SEED)).cuda()
    lv2 = torch.empty((NL,) + tuple(v.shape), dtype=torch.int32, device="cuda")
    c2 = torch.empty(NL, dtype=torch.int32, device="cuda")
    # 3D gradient (blur + Sobel magnitude) of the same volume: 2 B in + 2 B out per voxel
    g3 = torch.empty_like(v)
    med, best = timed(lambda: ctx.gradient3d(v, 0, out=g3))
    out["gradient3d_512"] = {"workload": "3D gradient of the 512^3 uint16 volume: 5x5x5 binomial blur, 3x3x3 Sobel, "
                                         "exact isqrt, uint16 out", "ms_median": med,
                             "gvox_s": side ** 3 / med / 1e6, "alg_hbm_frac": 4 * side ** 3 / (med / 1e3) / 1e9 / peak}
    del g3
    for conn in (6, 26):
        med, best = timed(lambda: ctx.segment(v, conn, NL, lv2, c2))
        out[f"volume512_conn{conn}"] = {
            "workload": f"3D 512^3 uint16 distance volume, {conn}-connectivity, watershed + waterfall NL={NL}",
            "ms_median": med, "gvox_s": side ** 3 / med / 1e6,
            "alg_hbm_frac": (2 + 4 * NL) * side ** 3 / (med / 1e3) / 1e9 / peak, "levels_counts": c2.cpu().tolist()}
        if conn == 6:
            # region-graph export (the Sec. 6 graph) of level planes 0 and 3, the gradient as
            # the one value channel; algorithmic bytes: labels 4 + G 2 + values 2 per voxel
            for k in (0, 3):
                med, best = timed(lambda: ctx.region_graph(lv2[k], v, conn, values=v))
                G = ctx.region_graph(lv2[k], v, conn, values=v)
                out[f"region_graph512_level{k}"] = {
                    "workload": f"region graph of level {k} of the 512^3 6-connectivity segmentation: CSR with "
                                "pass values, sizes, sums and means of one uint16 channel",
                    "ms_median": med, "gvox_s": side ** 3 / med / 1e6, "regions": int(G["size"].numel()),
                    "edges": int(G["col"].numel()) // 2,
                    "alg_hbm_frac": 8 * side ** 3 / (med / 1e3) / 1e9 / peak}
                del G
        if conn == 6:
            # the paper-literal waterfall (Alg. 4 with Alg. 5's reconstruction) on the same volume,
            # and how far it strays from the graph form: per level, the share of voxels outside the
            # best-overlapping graph-form region of their literal region (a report, not the path)
            lv3 = torch.empty_like(lv2)
            c3 = torch.empty_like(c2)
            med, best = timed(lambda: ctx.waterfall_reconstruct(v, conn, NL, lv3, c3))
            ctx.segment(v, conn, NL, lv2, c2)
            ctx.check()
            ctx.phase_times()
            ctx.set_profiling(True)
            ctx.waterfall_reconstruct(v, conn, NL, lv3, c3)
            rphases = {k: round(t[0], 3) for k, t in ctx.phase_times().items() if t[1]}
            ctx.set_profiling(False)
            ctx.check()
            dis = []
            for k in range(NL):
                Kg = int(c2[k])
                key = lv3[k].reshape(-1).long() * Kg + lv2[k].reshape(-1).long()
                uniq, cnt = torch.unique(key, return_counts=True)
                bestov = torch.zeros(int(c3[k]), dtype=torch.long, device="cuda")
                bestov.scatter_reduce_(0, uniq // Kg, cnt, reduce="amax")
                dis.append(1.0 - float(bestov.sum()) / side ** 3)
                del key, uniq, cnt, bestov
            out["reconstruct512_conn6"] = {
                "workload": f"3D 512^3 uint16 distance volume, 6-connectivity, paper-literal waterfall (watershed "
                            f"of each reconstructed image) NL={NL}",
                "ms_median": med, "gvox_s": side ** 3 / med / 1e6, "levels_counts": c3.cpu().tolist(),
                "graph_form_counts": c2.cpu().tolist(), "voxels_off_graph_form": dis, "phases_ms": rphases}
            del lv3, c3
    del lv2, v
    torch.cuda.empty_cache()
    return out


def run_gradient3d(ctx, torch, vol_d, peak, reps=10):
    """The 3D gradient (5x5x5 binomial blur, 3x3x3 Sobel, exact isqrt) of the
    headline volume: 2 B in + 2 B out per voxel; median of `reps` CUDA-event
    timings after three warm-up runs (input and output larger than L2)."""
    import statistics
    out = torch.empty_like(vol_d)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        ctx.gradient3d(vol_d, 0, out=out)
    ts = []
    for _ in range(reps):
        e0.record(stream)
        ctx.gradient3d(vol_d, 0, out=out)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.check()
    n = vol_d.numel()
    med = statistics.median(ts)
    del out
    return {"workload": f"3D gradient of the {'x'.join(str(d) for d in reversed(vol_d.shape))} uint16 volume: "
                        "5x5x5 binomial blur, 3x3x3 Sobel, exact isqrt, uint16 out", "ms_median": med,
            "gvox_s": n / med / 1e6, "alg_hbm_frac": 4 * n / (med / 1e3) / 1e9 / peak}


def run_batch(ctx, binding, torch, n=512, NL=6, conn=4, reps=3):
    """Config 3: n 2D uint8 images, sides log-uniform in [64, 2048], as one
    CUDA-graph replay of the batched pipeline vs n per-image ws_segment calls,
    with the runtime parameters autotuned on the batch first."""
    from paper_2410_08946_gb300 import synth
    img = torch.from_numpy(synth.crop_pool_image(synth.BATCH_POOL_SEED)).cuda()
    pool = ctx.gradient(img)
    grads = [pool[y:y + h, x:x + w].contiguous() for y, x, h, w in synth.batch_windows(n)]
    npx = sum(g.numel() for g in grads)
    outs = [(torch.empty((NL,) + tuple(g.shape), dtype=torch.int32, device="cuda"),
             torch.empty(NL, dtype=torch.int32, device="cuda")) for g in grads]
    # the runtime parameters (jumps per round, CTAs per SM of the level kernel)
    # picked by measurement on this batch, before the graph captures them
    from paper_2410_08946_gb300 import autotune
    tuned = autotune.autotune(ctx, lambda: ctx.segment_batch(grads, conn, NL, [o[0] for o in outs],
                                                             [o[1] for o in outs]),
                              key=f"batch2d|u8|conn{conn}|NL{NL}|{autotune.size_bucket(npx)}", reps=3)
    default_ms = next((ms for prm, ms in tuned["table"] if prm == autotune.DEFAULTS), None)
    graph = ctx.graph(grads, conn, NL)
    ctx.check()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        graph.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        graph.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / reps
    for g, (lv, c) in zip(grads, outs):
        ctx.segment(g, conn, NL, lv, c)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for g, (lv, c) in zip(grads, outs):
            ctx.segment(g, conn, NL, lv, c)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1) / reps
    ctx.check()
    same = all(torch.equal(a, b[0]) for a, b in zip(graph.levels, outs))
    graph.close()
    ctx.phase_times()
    ctx.set_profiling(True)
    ctx.segment_batch(grads, conn, NL, [o[0] for o in outs], [o[1] for o in outs])
    ctx.check()
    phases = {k: round(v[0], 4) for k, v in ctx.phase_times().items() if v[1]}
    counts = ctx.counters()
    ctx.set_profiling(False)
    ctx.set_tuning()
    return {"workload": f"{n} 2D uint8 crops of a 4096^2 blob gradient, sides log-uniform [64, 2048], "
                        f"{npx} px, 4-connectivity, NL={NL}",
            "batched_graph_ms": ms_graph, "batched_gvox_s": npx / ms_graph / 1e6,
            "per_image_ms": ms_single, "per_image_gvox_s": npx / ms_single / 1e6,
            "speedup": ms_single / ms_graph, "identical": bool(same), "phases_ms_eager": phases,
            "device_counts": counts,
            "autotune": {"params": tuned["params"], "tile_shape": autotune.SHAPES[tuned["params"]["tile_shape"]],
                         "eager_ms": tuned["ms"], "eager_ms_defaults": default_ms,
                         "candidates": len(tuned["table"])}}


def run_batch_only(n=512, NL=6, conn=4, reps=5, cache_path=None):
    """The batch alone: tuned, recorded as a CUDA graph, replayed `reps` times
    between CUDA events, then replayed once more.  Prints the replay time and
    the kernels one replay launches, so that a launch list of this command's
    last replay (ncu) gives the kernels' own device time beside the replay's.
    With cache_path the tuning is read from (or stored in) that JSON file, so
    that a profiled run replays the configuration a plain run chose."""
    import torch
    from paper_2410_08946_gb300 import autotune, binding, synth
    binding.load()
    ctx = binding.Context(0)
    img = torch.from_numpy(synth.crop_pool_image(synth.BATCH_POOL_SEED)).cuda()
    pool = ctx.gradient(img)
    grads = [pool[y:y + h, x:x + w].contiguous() for y, x, h, w in synth.batch_windows(n)]
    npx = sum(g.numel() for g in grads)
    outs = [(torch.empty((NL,) + tuple(g.shape), dtype=torch.int32, device="cuda"),
             torch.empty(NL, dtype=torch.int32, device="cuda")) for g in grads]
    tuned = autotune.autotune(ctx, lambda: ctx.segment_batch(grads, conn, NL, [o[0] for o in outs],
                                                             [o[1] for o in outs]),
                              key=f"batch2d|u8|conn{conn}|NL{NL}|{autotune.size_bucket(npx)}", reps=3,
                              cache_path=cache_path)
    graph = ctx.graph(grads, conn, NL)
    ctx.check()
    for _ in range(3):
        graph.launch()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record(stream)
        graph.launch()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    before = ctx.launches()
    ctx.segment_batch(grads, conn, NL, [o[0] for o in outs], [o[1] for o in outs])
    per_call = ctx.launches() - before
    torch.cuda.synchronize()
    graph.launch()   # the replay a launch list of this command ends with
    torch.cuda.synchronize()
    ctx.check()
    graph.close()
    print(json.dumps({"workload": f"{n} 2D uint8 crops, {npx} px, 4-connectivity, NL={NL}",
                      "graph_replay_ms": statistics.median(ts), "graph_replay_ms_all": ts,
                      "kernels_per_replay": per_call, "autotune": tuned["params"]}), flush=True)
    ctx.close()
    return 0


def run_serve(ctx, binding, torch, seconds=10.0, rate=200.0, NL=4, budget=40 << 30, lanes=4):
    """Config 4: Poisson arrivals (rate/s for `seconds`), 80% 2D uint8 (sides
    log-uniform [256, 4096]) and 20% 3D uint16 (sides [64, 256]), device-resident
    requests, served by the continuous-batching loop vs one ws_segment per
    request on one stream.  Latency = arrival -> labels complete on the device."""
    import numpy as np
    from paper_2410_08946_gb300 import synth
    img = torch.from_numpy(synth.crop_pool_image(synth.SERVE_SEED)).cuda()
    pool2 = ctx.gradient(img)
    vs = synth.SERVE_VOLUME_SIDE
    pool3 = torch.from_numpy(synth.distance_volume(vs, vs, vs, synth.SERVE_VOLUME_SEEDS, seed=synth.SERVE_SEED)).cuda()
    reqs = synth.request_stream(rate, seconds, seed=synth.SERVE_SEED)
    inputs = []
    for i, r in enumerate(reqs):
        if r["kind"] == "2d":
            h, w = r["shape"]
            y, x = synth.request_window_2d(i, h, w)
            inputs.append((pool2[y:y + h, x:x + w].contiguous(), 4))
        else:
            d, h, w = r["shape"]
            inputs.append((pool3[:d, :h, :w].contiguous(), 6))
    npx = sum(g.numel() for g, _ in inputs)
    times = [r["t"] for r in reqs]

    def pct(v, q):
        return float(np.percentile(np.array(v) * 1e3, q))

    # served: submit at arrival times, poll completions
    srv = binding.Server(0, budget_bytes=budget, lanes=lanes, max_batch=64)
    for g, conn in inputs[:8]:                     # warm the lanes' workspaces
        srv.poll(srv.submit(g, conn, NL), 120_000_000)
    torch.cuda.synchronize()
    lat, pending = [], []
    failed = 0
    t0 = time.perf_counter()
    i = 0
    while i < len(inputs) or pending:
        now = time.perf_counter() - t0
        while i < len(inputs) and times[i] <= now:
            pending.append((srv.submit(inputs[i][0], inputs[i][1], NL), times[i]))
            i += 1
        still = []
        for tk, ta in pending:
            st, lv, c = srv.poll(tk, 0)
            if st == binding.WS_ERR_NOT_READY:
                still.append((tk, ta))
            elif st == binding.WS_OK:
                lat.append(time.perf_counter() - t0 - ta)
            else:
                failed += 1
        pending = still
        if i < len(inputs) and not pending:
            time.sleep(max(0.0, min(0.001, times[i] - (time.perf_counter() - t0))))
    wall_served = time.perf_counter() - t0
    # saturation: the first n_sat requests queued at once
    n_sat = min(len(inputs), 400)
    sat_px = sum(g.numel() for g, _ in inputs[:n_sat])
    t1 = time.perf_counter()
    tks = [srv.submit(g, conn, NL) for g, conn in inputs[:n_sat]]
    for tk in tks:
        if srv.poll(tk, 600_000_000)[0] != binding.WS_OK:
            failed += 1
    sat_served = time.perf_counter() - t1
    srv.close()
    # per-image: one ws_segment per request, in arrival order, one stream
    lat1 = []
    buf = torch.empty(NL * max(g.numel() for g, _ in inputs), dtype=torch.int32, device="cuda")
    cnt = torch.empty(NL, dtype=torch.int32, device="cuda")

    def single(g, conn):
        ctx.segment(g, conn, NL, buf[:NL * g.numel()].view((NL,) + tuple(g.shape)), cnt)

    t0 = time.perf_counter()
    for (g, conn), ta in zip(inputs, times):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        single(g, conn)
        torch.cuda.current_stream().synchronize()
        lat1.append(time.perf_counter() - t0 - ta)
    t1 = time.perf_counter()
    for g, conn in inputs[:n_sat]:
        single(g, conn)
    torch.cuda.synchronize()
    sat_single = time.perf_counter() - t1
    ctx.check()
    return {"workload": f"Poisson {rate:g} req/s for {seconds:g} s ({len(inputs)} requests, {npx} px): 80% 2D uint8 "
                        f"256..4096, 20% 3D uint16 64..256, NL={NL}, device-resident, budget {budget >> 30} GB, "
                        f"{lanes} lanes",
            "served_p50_ms": pct(lat, 50), "served_p99_ms": pct(lat, 99),
            "per_image_p50_ms": pct(lat1, 50), "per_image_p99_ms": pct(lat1, 99),
            "served_gvox_s_saturated": sat_px / sat_served / 1e9,
            "per_image_gvox_s_saturated": sat_px / sat_single / 1e9, "saturation_requests": n_sat,
            "offered_gvox_s": npx / seconds / 1e9, "served_wall_s": wall_served, "failed_requests": failed}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=SIDE, help="cube side (default 928)")
    ap.add_argument("--ref-side", type=int, default=192, help="sample side of the reference arm")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-image batch measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the smaller configurations and the NEXT-row "
                    "measurements (2D configs, 512^3 volume, gradient, region graph, literal waterfall)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--ingest-ncu", metavar="CSV", help="write profiles/traffic.json from an ncu DRAM capture "
                    "(dram__bytes_read.sum, dram__bytes_write.sum) of a --side S run, then exit")
    ap.add_argument("--batch-only", action="store_true", help="only the 512-image batch as a CUDA-graph replay "
                    "(tuned, then timed), ending with one more replay: for a launch list of one replay")
    ap.add_argument("--tune-cache", metavar="JSON", help="with --batch-only: read or store the batch's tuning here")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.ingest_ncu:
        ingest_ncu(args.ingest_ncu, args.side ** 3)
        return 0
    if args.batch_only:
        return run_batch_only(cache_path=args.tune_cache)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    from paper_2410_08946_gb300 import binding, synth
    if not os.path.exists(binding.LIB_PATH):
        __graft_entry__.build()

    side = args.side
    n_seeds = sample_seeds(side) if side != SIDE else SEEDS
    vol = synth.distance_volume(side, side, side, n_seeds, seed=SEED)
    N = vol.size
    grad_d = torch.from_numpy(vol).cuda()
    levels_d = torch.empty((NL,) + vol.shape, dtype=torch.int32, device="cuda")
    counts_d = torch.empty(NL, dtype=torch.int32, device="cuda")
    ctx = binding.Context(local)
    stream = torch.cuda.current_stream()

    def step():
        ctx.segment(grad_d, CONN, NL, levels_d, counts_d)

    for _ in range(args.warmup):
        step()
    ctx.check()
    ctx.phase_times()                      # discard
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else None)
    sampler.start()
    time.sleep(0.3)
    ctx.set_profiling(True)
    l0 = ctx.launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    launches = (ctx.launches() - l0) / args.steps
    ctx.check()
    phases = ctx.phase_times()
    ctx.set_profiling(False)
    clocks = sampler.stop()
    ms_total = max_over_ranks(ms_total, dist, "cuda")
    ms = ms_total / args.steps
    value = whole_job_rate(N, world, ms / 1e3)
    counts = counts_d.cpu().tolist()

    peak, peak_src = hbm_peak()
    per_step = {k: v[0] / args.steps for k, v in phases.items() if v[1]}
    dom = max((k for k in per_step if k in PHASE_BYTES), key=lambda k: per_step[k])
    dom_launches = phases[dom][1] / args.steps
    dom_ms = per_step[dom] / max(dom_launches, 1)
    alg = PHASE_BYTES[dom] * N
    achieved = alg / (dom_ms / 1e3) / 1e9
    kern = KERNEL_OF_PHASE.get(dom, dom)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_for(kern, N), "kernel": kern, "phase": dom,
                "alg_bytes_per_launch": alg, "peak_source": f"{peak_src} (copy, MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else "fallback 6.8 TB/s"}
    path_bytes = (2 + 4 * NL) * N
    path_achieved = path_bytes / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "Gvox/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": workload_name(side), "voxels": N, "NL": NL, "connectivity": CONN,
                       "levels_counts": counts, "l2": "inputs (1.6 GB) and outputs (19.2 GB) larger than L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "path_roofline": {"bytes_per_voxel": 2 + 4 * NL, "achieved": path_achieved, "peak": peak,
                              "unit": "GB/s", "frac": path_achieved / peak},
            "path_dram": path_dram(N, ms, peak),
            "phases_ms": {k: round(v, 4) for k, v in per_step.items()},
            "device_counts": ctx.counters(),
            "gpu_launches": launches, "clocks": clocks}

    if not args.no_e2e:
        grad_h = torch.from_numpy(vol).pin_memory()
        levels_h = torch.empty((NL,) + vol.shape, dtype=torch.int32).pin_memory()
        counts_h = torch.empty(NL, dtype=torch.int32)
        ctx.segment_host(grad_h, CONN, NL, levels_h, counts_h)       # warm the staging buffers
        if dist:
            dist.barrier()
        e2e_steps = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            ctx.segment_host(grad_h, CONN, NL, levels_h, counts_h)   # synchronises: copies in and out included
            e2e_steps.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.median(e2e_steps), dist, "cuda")
        line["e2e"] = {"value": whole_job_rate(N, world, e2e_s), "unit": "Gvox/s", "ms_per_step": e2e_s * 1e3,
                       "step_ms": [round(t * 1e3, 2) for t in e2e_steps],
                       "h2d_bytes_per_step": int(N * 2), "d2h_bytes_per_step": int(NL * N * 4 + NL * 4)}
        del grad_h, levels_h
        link = host_link_gbs(torch)
        line["e2e"]["host_link_gbs"] = link
        # the copies alone at the measured link speed: the end-to-end ceiling
        copy_s = N * 2 / (link["h2d"] * 1e9) + NL * N * 4 / (link["d2h"] * 1e9)
        line["e2e"]["copy_bound_gvox_s"] = N / copy_s / 1e9
    if world == 1 and not (args.no_small and args.no_batch):
        del levels_d
        torch.cuda.empty_cache()
        if not args.no_small:
            line["gradient3d_full"] = run_gradient3d(ctx, torch, grad_d, peak)
            line["small_configs"] = run_small_configs(ctx, torch)
        if not args.no_batch:
            line["batch"] = run_batch(ctx, binding, torch)
    if world == 1 and not args.no_serve:
        line["serve"] = run_serve(ctx, binding, torch, seconds=args.serve_seconds)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
