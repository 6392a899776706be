#!/usr/bin/env python
"""Benchmark of the quadric Gaussian rasterizer: forward + backward Mpix/s at 3M quadrics.

Workload: the unbounded 360-scene shape, 3,000,000 quadric primitives, one 1297x840
camera inside the unit ball (seeded synthetic scene; see paper_2411_16392_gb300/scenes.py).
A step = render_forward + render_backward (random N(0,1) upstream gradients on rgb,
alpha, depth and normal) through the C ABI, inputs resident in HBM. The scene (432 MB)
and the per-frame instance buffers (~1 GB) are larger than the 129 MB L2, so no flush is
needed between steps.

Prints ONE JSON line (rank 0). Beside the headline (value, e2e with every upstream plane
uploaded and every output plane read back, roofline of the dominant kernel, stages against
their roofs) it carries: fwd_only (the same frame forward only); configs (the 1,000-quadric
128x128 and 300k-quadric 1600x1200 workloads, forward and forward + backward, with the
oracle beside); cpu_baseline (the FP64 oracle on a stratified 32-tile sample of the
frame, extrapolated); parity (the benchmarked frame's per-output error against the oracle
on those tiles); variants and serving. `--impl reference` times the FP64 CPU oracle
instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s at 3M quadrics (1297x840)"
UNIT = "Mpix/s"
WORKLOAD = "unbounded_3m_1297x840"

# FP32 operations (FMA = 2, MUFU = 1) per pair class, counted from the kernel source
# (raster.cu, eval_pair and the two compositing loops) along the shortest path of each
# class: every evaluated pair forms its pixel offset and evaluates the screen conic of the
# chord ellipsoid (FLOP_EVAL); a pair inside it forms the local ray, the quadratic and its
# first root up to the E <= 9 test (FLOP_ISECT); a hit adds the chord test, F(u), l^2/sigma^2 and G
# (FLOP_HIT); a blended pair adds alpha, transmittance, colour, depth and the normal
# (FLOP_BLEND); a pair that produces a gradient in the backward adds the chain rule and
# its share of the warp reduction (FLOP_GRAD).
FLOP_EVAL = 13
FLOP_ISECT = 54
FLOP_HIT = 24
FLOP_BLEND = 46
FLOP_GRAD = 200

# Algorithmic HBM bytes of the memory-bound stages (minimal traffic of what each stage
# computes): per primitive read 144 B of parameters (mean 12, quaternion 16, scales 8,
# curvatures 8, opacity 4, bf16 SH 96) and write count, depth key, rectangle and flag
# (20 B); per visible primitive the 128-byte state record and the 80-byte tile-test bounds,
# written and read back by the tile-count pass. Binning per visible primitive:
# a 4-pass (key, index) sort (20 B per pass) and the state gather (256 B); per
# instance: the 4-byte emitted key, two stable tile passes (12 B each) and the range
# scan (4 B). Preprocess backward per visible primitive: the 80-byte gradient record,
# the parameters (144 B) and a read-modify-write of the float32 gradients (240 B x 2).
B_PRE_PRIM, B_PRE_VIS = 164, 128 + 2 * 80
# DRAM bytes (read + write) per launch of the compositing kernels at 3M / 1297x840 (mean over
# the launches of one ncu launch list of this benchmark, dram__bytes_read.sum +
# dram__bytes_write.sum), valid only while the kernels' sources hash to the recorded value.
TRAFFIC_SRC = ("paper_2411_16392_gb300/csrc/raster.cu", "paper_2411_16392_gb300/csrc/qgs_common.cuh")
TRAFFIC = {"hash": "cab7d0c979ceeed0", "k_raster_fwd": 13474889 + 814190, "k_raster_bwd": 56434790 + 10138}
B_BIN_VIS, B_BIN_INST = 4 * 20 + 256, 4 + 2 * 12 + 4
B_PREBWD_VIS = 80 + 144 + 480


def _traffic(kernel, n_prims):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SRC:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != TRAFFIC["hash"] or n_prims != 3_000_000:
        return None
    return TRAFFIC.get(kernel)


def reduce_step_time(ms_local, world, pixels, device="cpu"):
    """Whole-job timing over the ranks: the maximum of the ranks' per-step times (every rank
    takes part in the reduction) and the whole-job throughput in Mpix/s, world x pixels per
    step over that time. `device` holds the reduction's tensor (cuda under NCCL)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * pixels / (ms_max * 1e-3) / 1e6


def _rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons (every 20 ms, timestamped);
    started before the warm-up so that sampling is under way when the timed region begins,
    and summarised over the samples taken inside the timed region's wall-clock window."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self, window=None):
        """Summary of the samples whose timestamps fall in window = (t0, t1) (host
        time.time() seconds); with no sample inside, the samples within 0.25 s of it."""
        from datetime import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]),
                             {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}))
            except ValueError:
                continue
        os.unlink(self.path)
        where = "all samples"
        if window is not None:
            t0, t1 = window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            where = "timed region"
            if not inside:
                inside = [r for r in rows if t0 - 0.25 <= r[0] <= t1 + 0.25]
                where = "within 0.25 s of the timed region"
            rows = inside
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sms = sorted(r[1] for r in rows)
        reasons = set().union(*(r[3] for r in rows))
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": max(r[2] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "sampled": where, "interval_ms": 20}


def _json_default(o):
    """numpy scalars and arrays in the JSON line (counts and errors computed with numpy)."""
    if hasattr(o, "tolist"):
        return o.tolist()
    if hasattr(o, "item"):
        return o.item()
    raise TypeError(f"{type(o).__name__} is not JSON serializable")


def _dumps(line):
    return json.dumps(line, default=_json_default)


# ----------------------------------------------------------------------------- CPU oracle
def _stratified_tiles(tile_counts, n, seed):
    """One tile drawn from each of n strata of equal size, the frame's tiles ordered by
    their list length; returns the drawn tiles and the strata sizes."""
    import numpy as np
    order = np.argsort(tile_counts, kind="stable")
    strata = [st for st in np.array_split(order, min(n, order.size)) if st.size]
    rng = np.random.default_rng(seed)
    return [int(st[rng.integers(st.size)]) for st in strata], [int(st.size) for st in strata]


def _tile_mask(cam, tiles):
    import numpy as np
    TX = (cam.W + 15) // 16
    m = np.zeros((cam.H, cam.W), bool)
    for t in tiles:
        ty, tx = divmod(int(t), TX)
        m[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    return m


def oracle_sample(sc, cam, n_tiles=32, seed=0, keep=False):
    """Time the FP64 oracle (as it stands) on a bounded, stratified sample of one frame: the
    FP32 binning of every primitive, then forward + backward (N(0, 1) upstream gradients) of
    n_tiles 16x16 tiles, one drawn from each of n_tiles equal strata of the frame's tiles
    ordered by list length. Frame time = binning + per-call set-up + sum over strata of
    (tiles in the stratum) x (time of its drawn tile): a stratified estimate, extrapolated.
    keep: also return the oracle's outputs and gradients of those tiles (for the parity
    block)."""
    import numpy as np
    import torch
    import oracle.qgs_oracle as O
    t0 = time.perf_counter()
    binning = O.bin_fp32(sc, cam, emit=False)
    t_bin = time.perf_counter() - t0
    tiles, sizes = _stratified_tiles(binning.tile_counts, n_tiles, seed)
    rng = np.random.default_rng(seed + 17)
    mask = _tile_mask(cam, tiles).astype(np.float64)
    H, W = cam.H, cam.W
    g = {"rgb": rng.normal(size=(3, H, W)) * mask, "alpha": rng.normal(size=(H, W)) * mask,
         "depth": rng.normal(size=(H, W)) * mask, "normal": rng.normal(size=(3, H, W)) * mask}
    g = {k: v.astype(np.float32).astype(np.float64) for k, v in g.items()}
    times = {}
    t0 = time.perf_counter()
    ref = O.render(sc, cam, binning, tiles=tiles, grad_images=g, timings=times)
    t_tiles = time.perf_counter() - t0
    setup = t_tiles - sum(times.values())
    frame_s = t_bin + setup + sum(n * times.get(t, 0.0) for t, n in zip(tiles, sizes))
    res = {"value": W * H / frame_s / 1e6, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
           "extrapolated": True,
           "sample": (f"FP32 binning of all {sc.n} primitives ({t_bin:.2f} s) + FP64 forward+backward of "
                      f"{len(tiles)} 16x16 tiles, one per stratum of the {binning.tiles_x * binning.tiles_y} "
                      f"tiles ordered by list length ({t_tiles:.2f} s), extrapolated to the frame by stratum "
                      f"size"),
           "sample_wall_s": t_bin + t_tiles, "frame_s_extrapolated": frame_s}
    if keep:
        res["_keep"] = (binning, tiles, g, ref)
    return res


def oracle_full_frame(sc, cam, seed=0):
    """The FP64 oracle on a whole frame, forward + backward, timed (no extrapolation)."""
    import numpy as np
    import torch
    import oracle.qgs_oracle as O
    rng = np.random.default_rng(seed)
    H, W = cam.H, cam.W
    g = {"rgb": rng.normal(size=(3, H, W)), "alpha": rng.normal(size=(H, W)), "depth": rng.normal(size=(H, W)),
         "normal": rng.normal(size=(3, H, W))}
    t0 = time.perf_counter()
    O.render(sc, cam, grad_images=g)
    dt = time.perf_counter() - t0
    return {"value": W * H / dt / 1e6, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "extrapolated": False, "sample": f"whole {W}x{H} frame, FP32 binning + FP64 forward+backward",
            "sample_wall_s": dt}


def parity_block(sc, cam, ras, ds, kept, dev):
    """Per-output error of the benchmarked frame against the FP64 oracle on the CPU
    baseline's sampled tiles (spec precision pattern: the error against the oracle is
    stated for each output): the GPU's forward planes and, with the same upstream
    gradients (zero outside those tiles), its parameter gradients. Errors are in units of
    the bars and as plain maxima; near-threshold pixels are compared to their branches
    (tests/parity_util)."""
    import numpy as np
    import torch
    from tests.parity_util import TOL_ABS, TOL_DEPTH_REL, compare_grads, compare_images, near_pixels
    import oracle.qgs_oracle as O
    binning, tiles, g, ref = kept
    t0 = time.perf_counter()
    out = {k: v.detach().cpu().numpy().astype(np.float64) for k, v in ras.forward(ds, cam).items()}
    gd = {k: torch.from_numpy(v.astype(np.float32)).to(dev) for k, v in g.items()}
    gg = {k: v.cpu().numpy() for k, v in ras.backward(ds, cam, gd).items()}
    mask = _tile_mask(cam, tiles)
    st = compare_images(out, ref, sc, cam, binning, mask)
    far = mask & ~near_pixels(ref, mask)
    plain = {k: float(np.abs(out[k] - ref[k])[..., far].max(initial=0.0)) for k in ("rgb", "alpha", "normal")}
    plain["depth_rel"] = float((np.abs(out["depth"] - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-6))[far]
                               .max(initial=0.0))
    touched = np.unique(np.concatenate([O.tile_list(binning, t) for t in tiles])).astype(np.int64)
    gr, npix, unres = compare_grads(gg, ref, sc, cam, g, binning, mask, touched)
    grel = {}
    for k, v in ref["grads"].items():
        a = v[touched]
        scale = np.maximum(np.abs(a), 1e-3 * np.abs(a).max(initial=0.0))
        scale = np.where(scale > 0, scale, 1.0)
        grel[k] = float((np.abs(np.asarray(gg[k], np.float64).reshape(v.shape)[touched] - a) / scale).max(initial=0.0))
    return {"tiles": len(tiles), "pixels": int(mask.sum()), "primitives_compared": int(touched.size),
            "bars": {"rgb_alpha_normal_abs": TOL_ABS, "depth_rel": TOL_DEPTH_REL, "grad_rel": 1e-3},
            "max_err": plain, "max_err_of_bar": st["errors"], "near_threshold_pixel_frac": st["near_frac"],
            "near_threshold_worst_of_bar": st["near_worst"], "ambiguous_pixels": st["ambiguous"],
            "grad_max_rel_err": grel,
            "grad_of_bar": {k: v["ratio"] for k, v in gr.items()},
            "grad_plain_of_bar": {k: v["strict"] for k, v in gr.items()},
            "grad_widened_frac": {k: v["widened"] for k, v in gr.items()},
            "grad_banded_frac": {k: v["banded"] for k, v in gr.items()},
            "bracketed_pixels": npix, "wall_s": time.perf_counter() - t0}


def serving_parity(dev, n_req=4, n_pix=24, seed=3):
    """Per-output error of served requests against the FP64 oracle (the mixed-resolution
    serving workload): n_req forward requests of the 1M-quadric serving scene at the serving
    resolutions, submitted together so that they render as one batch, each checked at n_pix
    sampled pixels against the oracle's branches (tests/parity_util.check_pixels, without
    asserting)."""
    import numpy as np
    from tests.parity_util import _best_branch, _gpu_pixel, _graze_band, _pixel_errors
    import oracle.qgs_oracle as O
    from paper_2411_16392_gb300.render import DeviceScene
    from paper_2411_16392_gb300.scenes import orbit_camera, serving_scene
    from paper_2411_16392_gb300.serve import Server, host_planes
    t0 = time.perf_counter()
    sc = serving_scene(0, 1_000_000)
    ds = DeviceScene.from_host(sc, dev)
    rng = np.random.default_rng(seed)
    cams = [orbit_camera(rng) for _ in range(n_req)]
    srv = Server(dev.index, budget_bytes=64 << 30, slots=1, queue=64, batch=n_req)
    sid = srv.load_scene(ds)
    tickets = [srv.submit(sid, c) for c in cams]
    outs = [srv.wait(t, c, out=host_planes(c)) for t, c in zip(tickets, cams)]
    st = srv.stats()
    srv.close()
    worst, unmatched, per = {}, 0, []
    for cam, out in zip(cams, outs):
        binning = O.bin_fp32(sc, cam, emit=False)
        pix = [(int(x), int(y)) for x, y in zip(rng.integers(0, cam.W, n_pix), rng.integers(0, cam.H, n_pix))]
        br = O.bracket_pixels(sc, cam, pix, binning)
        e_req = 0.0
        for (x, y), it in zip(pix, br):
            gv = _gpu_pixel(out, x, y, False)
            best = _best_branch(gv, it, False)
            unmatched += best > 1.0
            e_req = max(e_req, best)
            band = _graze_band(it)
            leaf = min((l for g_, l in zip(it["groups"], it["leaves"]) if g_ == "d"),
                       key=lambda l: _pixel_errors(gv, l, False, band))
            for k, lim, rel in (("rgb", 1e-4, False), ("alpha", 1e-4, False), ("normal", 1e-4, False),
                                ("depth", 1e-4, True)):
                d = float(np.max(np.abs(np.asarray(gv[k], np.float64) - np.asarray(leaf[k]).reshape(np.shape(gv[k])))))
                if rel:
                    d /= max(abs(float(leaf[k][0])), 1e-6)
                worst[k] = max(worst.get(k, 0.0), d)
        per.append({"width": cam.W, "height": cam.H, "worst_of_bar": e_req})
    return {"workload": "serving_1m_mixed_res", "requests": n_req, "batched_together": int(st["max_batch"]),
            "pixels_per_request": n_pix, "max_err": {("depth_rel" if k == "depth" else k): v for k, v in worst.items()},
            "ambiguous_pixels": unmatched, "requests_detail": per, "wall_s": time.perf_counter() - t0}


def _config(sc, cam, world=1):
    return {"workload": WORKLOAD if sc.n == 3_000_000 else f"unbounded_{sc.n}_1297x840", "primitives": sc.n,
            "width": cam.W, "height": cam.H,
            "l2": "inputs larger than L2 (scene 432 MB, instances ~1 GB per frame)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    from paper_2411_16392_gb300.scenes import scene_unbounded
    sc, cam = scene_unbounded(0, args.prims)
    for w in range(args.warmup):
        oracle_sample(sc, cam, 4, seed=1000 + w)
    vals = []
    t0 = time.perf_counter()
    for k in range(args.steps):
        vals.append(oracle_sample(sc, cam, args.ref_tiles, seed=k))
    wall = time.perf_counter() - t0
    frame_s = sum(v["frame_s_extrapolated"] for v in vals) / len(vals)
    value = cam.W * cam.H / frame_s / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": frame_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(sc, cam, args.gpus),
            "extrapolated": True,
            "timed_wall_s": wall,
            "note": ("ms_per_step is the oracle's extrapolated time for one whole frame (a stratified "
                     "estimate from the sampled tiles of each step); the steps' own wall time is timed_wall_s"),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": vals[0]["cores"],
                             "extrapolated": True,
                             "sample": vals[0]["sample"] + f"; {args.steps} steps, wall {wall:.1f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(_dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU
def serve_measure(dev_index, scenes, jobs, gaps, slots, batch=1, budget=64 << 30, grad_sets=None):
    """Open-loop serving run: job k = (scene index, camera, backward?) is submitted at the
    cumulative time of gaps[:k+1] (Poisson arrivals); backward jobs carry one of the
    `grad_sets` upstream planes (pinned host tensors). Returns the server's latency
    statistics (submit -> result ready on the device)."""
    import threading
    from paper_2411_16392_gb300.serve import Server
    n_req = len(jobs)
    srv = Server(dev_index, budget_bytes=budget, slots=slots, queue=max(64, n_req), batch=batch)
    sids = [srv.load_scene(ds) for ds in scenes]

    def submit(k):
        si, cam, bwd = jobs[k]
        if bwd:
            return srv.submit(sids[si], cam, backward=True, grad_out=grad_sets[k % len(grad_sets)])
        return srv.submit(sids[si], cam)

    for k in range(min(4, n_req)):              # warm-up (buffers, kernels)
        srv.wait(submit(k))
    srv.reset_stats()
    tickets = []
    lock = threading.Lock()

    def waiter():
        k = 0
        while k < n_req:
            with lock:
                have = len(tickets)
            if k < have:
                srv.wait(tickets[k])
                k += 1
            else:
                time.sleep(0.0002)

    th = threading.Thread(target=waiter)
    th.start()
    t_next = time.perf_counter()
    for k, gap in enumerate(gaps):
        t_next += gap
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        t = submit(k)
        with lock:
            tickets.append(t)
    th.join()
    st = srv.stats()
    srv.close()
    return {k: st[k] for k in ("p50_ms", "p99_ms", "mean_ms", "frames_per_s", "completed", "max_in_flight",
                               "batches", "max_batch")}


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2411_16392_gb300 import _lib as L
    L.load()
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    from paper_2411_16392_gb300.scenes import scene_unbounded

    sc, cam = scene_unbounded(0, args.prims)
    ds = DeviceScene.from_host(sc, dev)
    ras = Rasterizer(dev)
    H, W = cam.H, cam.W
    P = H * W
    gen = torch.Generator(device=dev).manual_seed(1234 + rank)
    gout = {"rgb": torch.randn(3, H, W, device=dev, generator=gen),
            "alpha": torch.randn(H, W, device=dev, generator=gen),
            "depth": torch.randn(H, W, device=dev, generator=gen),
            "normal": torch.randn(3, H, W, device=dev, generator=gen)}
    grads = {k: torch.zeros(*s, device=dev) for k, s in
             (("mean", (sc.n, 3)), ("quat", (sc.n, 4)), ("scale", (sc.n, 2)), ("curv", (sc.n, 2)),
              ("opacity", (sc.n,)), ("sh", (sc.n, 48)))}
    out = {"rgb": torch.empty(3, H, W, device=dev), "alpha": torch.empty(H, W, device=dev),
           "depth": torch.empty(H, W, device=dev), "normal": torch.empty(3, H, W, device=dev)}

    def step():
        ras.forward(ds, cam, out)
        ras.backward(ds, cam, gout, grads)

    clocks = ClockSampler(local)
    clocks.start()                 # sampling under way before the timed region starts
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: device time of K steps (CUDA events on the launching stream). The
    # per-pair counters are compiled out of the compositing kernels here (they are collected
    # in an extra step below); stage events are recorded and the last step's are read after.
    lib = ras.lib
    L.check(lib.qgs_set_profiling(ras._ctx, 1), ras._ctx)
    ras.set_pair_counters(False)
    step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if world > 1:
        dist.barrier()
    clk = clocks.stop((t_wall0, t_wall1))
    st_timed = ras.stats()  # stage times of the last timed step
    ms = e0.elapsed_time(e1) / args.steps
    # forward alone (the same frame, rendered K times)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ras.forward(ds, cam, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1) / args.steps
    # stage times averaged over a few more steps (read after each one), then the pair
    # counters of one step
    stage = {"ms_raster_fwd": [], "ms_raster_bwd": [], "ms_preprocess": [], "ms_depth_sort": [], "ms_emit": [],
             "ms_tile_sort": [], "ms_preprocess_bwd": []}
    for _ in range(min(args.steps, 5)):
        step()
        stt = ras.stats()
        for k in stage:
            stage[k].append(stt[k])
    ras.set_pair_counters(True)
    step()
    st = ras.stats()
    ras.set_pair_counters(False)
    st["ms_raster_bwd_timed"] = st_timed["ms_raster_bwd"]
    st["ms_raster_fwd_timed"] = st_timed["ms_raster_fwd"]
    L.check(lib.qgs_set_profiling(ras._ctx, 0), ras._ctx)
    ms_max, value = reduce_step_time(ms, world, P, dev)

    # ---- end to end through the public API with host buffers
    if args.no_e2e:
        e2e_value, h2d, d2h = None, 0, 0
    else:
        e2e_value, h2d, d2h = _e2e(args, ras, ds, cam, gout, grads, out, dev, world, P)
    variants = None
    if rank == 0 and world == 1 and args.variant_steps > 0:
        variants = _variants(args, ds, cam, gout, grads, dev)
    legs = None
    if rank == 0 and world == 1 and args.config_steps > 0:
        legs = _config_legs(args, dev)
    return _report(args, rank, world, sc, cam, st, stage, clk, ms_max, value, e2e_value, h2d, d2h, variants,
                   ms_fwd=ms_fwd, ras=ras, ds=ds, dev=dev, legs=legs)


def fp32_peak_tflops(n_sm, sm_mhz):
    """FP32 FMA throughput: SMs x 128 FP32 lanes x 2 flop per FMA x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def _time_steps(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _config_legs(args, dev):
    """The two smaller workloads: 1,000 quadrics at 128x128 (the oracle renders it whole)
    and the 300k-quadric object scene at 1600x1200 (the oracle samples it): forward and
    forward + backward Mpix/s, pair evaluations/s, the compositing kernels against the FP32
    roof, and the oracle beside (cpu_baseline)."""
    import torch
    from paper_2411_16392_gb300 import _lib as L
    from paper_2411_16392_gb300.render import DeviceScene, Rasterizer
    from paper_2411_16392_gb300.scenes import scene_object, scene_small
    res = {}
    stream = torch.cuda.current_stream(dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    for name, (sc, cam), full in (("small_1k_128x128", scene_small(0, 1000), True),
                                  ("object_300k_1600x1200", scene_object(0), False)):
        ds = DeviceScene.from_host(sc, dev)
        ras = Rasterizer(dev)
        H, W = cam.H, cam.W
        gen = torch.Generator(device=dev).manual_seed(7)
        gout = {"rgb": torch.randn(3, H, W, device=dev, generator=gen),
                "alpha": torch.randn(H, W, device=dev, generator=gen),
                "depth": torch.randn(H, W, device=dev, generator=gen),
                "normal": torch.randn(3, H, W, device=dev, generator=gen)}
        out = ras.forward(ds, cam)
        grads = ras.backward(ds, cam, gout)
        ras.set_pair_counters(False)
        ms_fwd = _time_steps(lambda: ras.forward(ds, cam, out), args.config_steps, 3, stream)
        ms_step = _time_steps(lambda: (ras.forward(ds, cam, out), ras.backward(ds, cam, gout, grads)),
                              args.config_steps, 3, stream)
        L.check(ras.lib.qgs_set_profiling(ras._ctx, 1), ras._ctx)
        ras.forward(ds, cam, out)
        ras.backward(ds, cam, gout, grads)
        tim = ras.stats()
        ras.set_pair_counters(True)
        ras.forward(ds, cam, out)
        ras.backward(ds, cam, gout, grads)
        st = ras.stats()
        L.check(ras.lib.qgs_set_profiling(ras._ctx, 0), ras._ctx)
        flops_fwd = (st["pair_evals"] * FLOP_EVAL + st["pair_isect"] * FLOP_ISECT + st["pair_hits"] * FLOP_HIT
                     + st["pair_blended"] * FLOP_BLEND)
        isect_frac = st["pair_isect"] / max(1, st["pair_evals"])
        flops_bwd = (st["bwd_pairs"] * (FLOP_EVAL + isect_frac * FLOP_ISECT)
                     + st["bwd_contrib"] * (FLOP_HIT + FLOP_GRAD))
        peak = fp32_peak_tflops(n_sm, 2070.0)
        leg = {"primitives": sc.n, "width": W, "height": H, "visible": st["n_visible"],
               "instances": st["n_instances"],
               "fwd_mpix_per_s": H * W / (ms_fwd * 1e-3) / 1e6, "fwd_ms": ms_fwd,
               "fwd_bwd_mpix_per_s": H * W / (ms_step * 1e-3) / 1e6, "fwd_bwd_ms": ms_step,
               "pair_evals_per_s_fwd": st["pair_evals"] / (ms_fwd * 1e-3),
               "raster_fwd": {"ms": tim["ms_raster_fwd"], "frac_fp32_roof":
                              flops_fwd / (tim["ms_raster_fwd"] * 1e-3) / 1e12 / peak if tim["ms_raster_fwd"] > 0
                              else None},
               "raster_bwd": {"ms": tim["ms_raster_bwd"], "frac_fp32_roof":
                              flops_bwd / (tim["ms_raster_bwd"] * 1e-3) / 1e12 / peak if tim["ms_raster_bwd"] > 0
                              else None},
               "roof_note": f"FP32 roof at the maximum clock ({peak:.1f} TFLOP/s, {n_sm} SMs)"}
        if not args.no_cpu_baseline:
            if full:
                leg["cpu_baseline"] = oracle_full_frame(sc, cam)
            else:
                cb = oracle_sample(sc, cam, 16)
                cb.pop("frame_s_extrapolated", None)
                leg["cpu_baseline"] = cb
        res[name] = leg
        ras.close()
        del ds
    return res


def _variants(args, ds, cam, gout, grads, dev):
    """The same fwd+bwd step with each optional path of the renderer (not the headline):
    the extra channels (curvature, distortion, median depth with their gradients), the
    Euclidean density, and the StopThePop ordering."""
    import torch
    from paper_2411_16392_gb300.render import Rasterizer
    H, W = cam.H, cam.W
    res = {}
    gx = dict(gout)
    gx["curvature"] = torch.randn(H, W, device=dev)
    gx["distortion"] = torch.randn(H, W, device=dev)
    for name, kw, extras in (("extra_channels", {}, True), ("euclid", {"density": "euclid"}, False),
                             ("stopthepop", {"order": "stp"}, False)):
        ras = Rasterizer(dev, **kw)
        ras.set_pair_counters(False)   # timed steps as the headline's: counters compiled out
        g = gx if extras else gout

        def step():
            ras.forward(ds, cam, extras=extras)
            ras.backward(ds, cam, g, grads)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream(dev)
        e0.record(stream)
        for _ in range(args.variant_steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.variant_steps
        ras.lib.qgs_set_profiling(ras._ctx, 1)
        step()                         # stage times of a step like the timed ones
        st = ras.stats()
        ras.set_pair_counters(True)
        step()                         # blended-pair count from a step with the counters
        pb = ras.stats()["pair_blended"]
        res[name] = {"mpix_per_s": H * W / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                     "ms_raster_fwd": st["ms_raster_fwd"], "ms_raster_bwd": st["ms_raster_bwd"],
                     "pair_blended": pb}
        ras.close()
    return res


def _e2e(args, ras, ds, cam, gout, grads, out, dev, world, P):
    import torch
    import torch.distributed as dist
    H, W = cam.H, cam.W
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    host_g = {k: v.cpu().pin_memory() for k, v in gout.items()}
    host_out = {k: torch.empty(v.shape, pin_memory=True) for k, v in out.items()}
    dev_g = {k: torch.empty_like(v) for k, v in gout.items()}
    h2d = sum(v.numel() * 4 for v in host_g.values())
    d2h = sum(v.numel() * 4 for v in host_out.values())

    # the copies run on a side stream: this step's upstream gradients go up while the
    # forward renders, its four planes come down while the backward runs; the step (timed on
    # the main stream) ends when both copies are complete
    cs = torch.cuda.Stream(dev)
    ev_g = torch.cuda.Event()
    ev_f = torch.cuda.Event()
    ev_d = torch.cuda.Event()

    def e2e_step():
        cs.wait_stream(stream)  # the previous step is done with dev_g and host_out
        with torch.cuda.stream(cs):
            for k in dev_g:
                dev_g[k].copy_(host_g[k], non_blocking=True)
            ev_g.record(cs)
        ras.forward(ds, cam, out)
        ev_f.record(stream)
        stream.wait_event(ev_g)
        ras.backward(ds, cam, dev_g, grads)
        cs.wait_event(ev_f)
        with torch.cuda.stream(cs):
            for k in host_out:
                host_out[k].copy_(out[k], non_blocking=True)
            ev_d.record(cs)
        stream.wait_event(ev_d)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ne = max(3, args.steps // 2)
    e0.record(stream)
    for _ in range(ne):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / ne
    _, e2e_value = reduce_step_time(ms_e2e, world, P, dev)
    return e2e_value, h2d, d2h


def _report(args, rank, world, sc, cam, st, stage, clk, ms_max, value, e2e_value, h2d, d2h, variants=None,
            ms_fwd=None, ras=None, ds=None, dev=None, legs=None):
    import torch
    import torch.distributed as dist
    H, W = cam.H, cam.W
    # ---- roofline of the dominant kernel (FP32 ALU bound)
    peaks, peak_kind = _peaks()
    mean = {k: (sum(v) / len(v) if v and min(v) >= 0 else None) for k, v in stage.items()}
    # the compositing kernels' durations in the last timed step (CUDA events on their stream)
    bwd_ms = st["ms_raster_bwd_timed"] if st.get("ms_raster_bwd_timed", -1) >= 0 else mean["ms_raster_bwd"]
    fwd_ms = st["ms_raster_fwd_timed"] if st.get("ms_raster_fwd_timed", -1) >= 0 else mean["ms_raster_fwd"]
    flops_fwd = (st["pair_evals"] * FLOP_EVAL + st["pair_isect"] * FLOP_ISECT + st["pair_hits"] * FLOP_HIT
                 + st["pair_blended"] * FLOP_BLEND)
    # backward recomputes the pairs up to each pixel's last blended one
    isect_frac = st["pair_isect"] / max(1, st["pair_evals"])
    flops_bwd = (st["bwd_pairs"] * (FLOP_EVAL + isect_frac * FLOP_ISECT)
                 + st["bwd_contrib"] * (FLOP_HIT + FLOP_GRAD))
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count if dev is not None else 152
    peak_tflops = fp32_peak_tflops(n_sm, sm_mhz)
    if bwd_ms is not None and (fwd_ms is None or bwd_ms >= fwd_ms):
        dom, dom_ms, dom_flops = "k_raster_bwd", bwd_ms, flops_bwd
    else:
        dom, dom_ms, dom_flops = "k_raster_fwd", fwd_ms, flops_fwd
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": (achieved / peak_tflops) if achieved else None, "traffic": _traffic(dom, sc.n),
                "peak_note": f"FP32 FMA pipe: {n_sm} SMs (read from the device) x 128 lanes x 2 flop x "
                             f"{sm_mhz:.0f} MHz (median SM clock sampled during the timed region)",
                "ms_per_launch": dom_ms,
                "flops_per_launch": dom_flops}
    # ---- every stage against its own roof; the frame against the sum of the roofs
    hbm = peaks.get("hbm_gbs", 6800.0)
    V, I, N = st["n_visible"], st["n_instances"], sc.n
    work = {"ms_preprocess": ("hbm", N * B_PRE_PRIM + V * B_PRE_VIS),
            "ms_binning": ("hbm", V * B_BIN_VIS + I * B_BIN_INST),
            "ms_raster_fwd": ("alu", flops_fwd),
            "ms_raster_bwd": ("alu", flops_bwd),
            "ms_preprocess_bwd": ("hbm", V * B_PREBWD_VIS)}
    stage_t = dict(mean)
    if all(stage_t.get(k) is not None for k in ("ms_depth_sort", "ms_emit", "ms_tile_sort")):
        stage_t["ms_binning"] = stage_t["ms_depth_sort"] + stage_t["ms_emit"] + stage_t["ms_tile_sort"]
    stages, roof_sum = {}, 0.0
    for k, (bound, amount) in work.items():
        ms = stage_t.get(k)
        peak_v = hbm * 1e9 if bound == "hbm" else peak_tflops * 1e12
        roof_ms = amount / peak_v * 1e3
        roof_sum += roof_ms
        if ms:
            ach = amount / (ms * 1e-3)
            stages[k[3:]] = {"bound": bound, "ms": ms, "roof_ms": roof_ms,
                             "achieved": ach / (1e9 if bound == "hbm" else 1e12),
                             "unit": "GB/s" if bound == "hbm" else "TFLOP/s", "frac": ach / peak_v}
    frame_roof = {"ms_roof_sum": roof_sum, "ms_measured": ms_max, "frac": roof_sum / ms_max if ms_max else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(sc, cam, world),
            "frame": {"visible": st["n_visible"], "instances": st["n_instances"]},
            "fwd_only": ({"mpix_per_s": world * H * W / (ms_fwd * 1e-3) / 1e6, "ms": ms_fwd}
                         if ms_fwd else None),
            "pair_evals_per_s": world * st["pair_evals"] / (ms_max * 1e-3),
            "stage_ms": mean, "counters": {k: st[k] for k in ("pair_evals", "pair_isect", "pair_hits",
                                                               "pair_blended", "grazing_resolves",
                                                               "bwd_pairs", "bwd_contrib")},
            "roofline": roofline, "peak_source": peak_kind, "stage_roofline": stages, "frame_roofline": frame_roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int((st["launches_fwd"] + st["launches_bwd"]) * args.steps),
            "clocks": clk}
    if variants:
        line["variants"] = variants
    if rank == 0 and world == 1 and args.serve_requests > 0:
        line["serving"] = _serving_leg(args)
    if legs:
        line["configs"] = legs
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(sc, cam, args.cpu_tiles, keep=not args.no_parity)
        kept = cb.pop("_keep", None)
        cb.pop("frame_s_extrapolated", None)
        line["cpu_baseline"] = cb
        if kept is not None:
            line["parity"] = parity_block(sc, cam, ras, ds, kept, dev)
            if args.serve_requests > 0:
                line["parity"]["serving"] = serving_parity(dev)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(_dumps(line), flush=True)
    return 0


def _serving_leg(args):
    """Served p50/p99 latency and frames/s of the 1M-quadric serving workload at each
    arrival rate: plain one-at-a-time (1 slot, no batching), one slot that renders up to
    --serve-batch queued small views in shared launches, concurrent slots without batching,
    and the server with both (--serve-slots slots, batches of --serve-batch; with several
    slots the server's policy forms no batches, see csrc/serve.cu batch_pays); the same
    arrival process for all four."""
    import torch
    from paper_2411_16392_gb300.render import DeviceScene
    from paper_2411_16392_gb300.scenes import serving_scene
    import numpy as np
    from paper_2411_16392_gb300.scenes import orbit_camera
    dev = torch.device("cuda", torch.cuda.current_device())
    ds = DeviceScene.from_host(serving_scene(0, 1_000_000), dev)
    res = {"workload": "serving_1m_mixed_res", "requests": args.serve_requests, "rates": []}
    legs = (("one_at_a_time", 1, 1), ("one_slot_batched", 1, args.serve_batch),
            (f"slots{args.serve_slots}", args.serve_slots, 1), ("batched", args.serve_slots, args.serve_batch))
    n = args.serve_requests
    for rate in args.serve_rate:
        rng = np.random.default_rng(0)
        jobs = [(0, orbit_camera(rng), False) for _ in range(n)]
        gaps = rng.exponential(1.0 / rate, n)
        r = {"arrival_rate_per_s": rate}
        for name, slots, batch in legs:
            r[name] = serve_measure(dev.index, [ds], jobs, gaps, slots, batch)
        r["batched_config"] = {"slots": args.serve_slots, "max_batch": args.serve_batch}
        res["rates"].append(r)
    del ds
    rates = [r for r in args.serve_mixed_rate if r > 0]
    if rates:
        res["mixed"] = [_serving_mixed_leg(args, dev, r) for r in rates]
    return res


def _serving_mixed_leg(args, dev, rate):
    """Six resident scenes of 0.2/0.5/1/2/3/4 M quadrics; each request picks a scene
    uniformly; 80 % are forward views at the serving resolutions, 20 % forward + backward
    at 1297x840 with N(0, 1) upstream gradients; HBM-budget admission. Plain one-at-a-time
    against slots with batching, same arrivals."""
    import numpy as np
    import torch
    from paper_2411_16392_gb300.render import DeviceScene
    from paper_2411_16392_gb300.scenes import orbit_camera, serving_scene
    sizes = (200_000, 500_000, 1_000_000, 2_000_000, 3_000_000, 4_000_000)
    scenes = [DeviceScene.from_host(serving_scene(10 + k, m), dev) for k, m in enumerate(sizes)]
    n = args.serve_requests
    rng = np.random.default_rng(1)
    jobs = []
    for _ in range(n):
        si = int(rng.integers(len(sizes)))
        if rng.random() < 0.2:
            jobs.append((si, orbit_camera(rng, res=(1297, 840)), True))
        else:
            jobs.append((si, orbit_camera(rng), False))
    gaps = rng.exponential(1.0 / rate, n)
    gen = torch.Generator().manual_seed(2)
    grad_sets = []
    for _ in range(4):
        g = {"rgb": torch.randn(3, 840, 1297, generator=gen), "alpha": torch.randn(840, 1297, generator=gen),
             "depth": torch.randn(840, 1297, generator=gen), "normal": torch.randn(3, 840, 1297, generator=gen)}
        grad_sets.append({k: v.pin_memory() for k, v in g.items()})
    res = {"workload": "serving_6_scenes_0.2-4m_80fwd_20fwdbwd", "requests": n,
           "arrival_rate_per_s": rate, "backward_share": 0.2}
    for name, slots, batch in (("one_at_a_time", 1, 1), ("batched", args.serve_slots, args.serve_batch)):
        res[name] = serve_measure(dev.index, scenes, jobs, gaps, slots, batch, grad_sets=grad_sets)
    res["batched_config"] = {"slots": args.serve_slots, "max_batch": args.serve_batch}
    del scenes
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-tiles", type=int, default=32, help="stratified tiles of the oracle's CPU baseline")
    ap.add_argument("--ref-tiles", type=int, default=4, help="stratified tiles per step of the reference arm")
    ap.add_argument("--no-parity", action="store_true", help="skip the per-output error block")
    ap.add_argument("--config-steps", type=int, default=10,
                    help="timed steps of the 1k and 300k workloads (0: skip those legs)")
    ap.add_argument("--prims", type=int, default=3_000_000,
                    help="primitive count (the benchmark workload is 3,000,000; smaller counts are for profiling)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=600, help="requests per serving run (0: skip)")
    ap.add_argument("--serve-rate", type=lambda v: [float(x) for x in v.split(",")],
                    default=[200.0, 400.0, 500.0, 1000.0, 2000.0],
                    help="Poisson arrival rates, requests/s (comma-separated)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=8, help="most views per batch in the batched leg")
    ap.add_argument("--variant-steps", type=int, default=5,
                    help="timed steps of each optional renderer path (extra channels, Euclid, StopThePop; 0: skip)")
    ap.add_argument("--serve-mixed-rate", type=lambda v: [float(x) for x in v.split(",")], default=[100.0, 250.0],
                    help="arrival rates of the six-scene forward/backward serving leg (comma-separated; 0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
