#!/usr/bin/env python
"""Benchmark of the 2.7K virtual-stereo pair: remap -> 64-label BP -> JBU -> xyz.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step is a batch of P independent frame pairs of 2704 x 1520 RGB (P =
--pairs-in-flight, default 3) through the whole hot path: radial
undistort/rectify remap of both frames fused with the x4 downsample (Section
2.1, 2.2), hierarchical min-sum BP with 64 labels, 4 levels x 10 iterations
on 676 x 380 (Eq. 1), joint bilateral upsampling of the labels to 2704 x 1520
fused with the reprojection to an FP32 point cloud (Eq. 2, 3).  Each step is
one CUDA-graph replay in which the P pairs run on P streams, so one pair's
latency-bound coarse BP levels overlap another's bandwidth-bound kernels;
the line also reports the plain rate (one pair per replay).  Inputs are
seeded synthetic terrain pairs rendered on the host; eight distinct pairs
(197 MB, more than the 126 MB L2) are resident in HBM and rotated so no step
reads its inputs from L2.

Outside the timed region the line also carries the end-to-end rate through
the public API, the streaming flight, the batched BP and whole pairs, the
smoothed BP and its adjoint, and the pose step between two frames (Section
2.3), each with its own timing.

Prints ONE JSON line (rank 0).  Pairs are independent, so N GPUs run N
replicas ("scaling": "weak") and the value is all pairs over the slowest rank.
``--impl reference`` times the CPU oracle instead (rank 0 only), on bounded
crops of the same workload scaled to pairs/s.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2.7K pairs/s (BP 64 lbl + JBU)"
UNIT = "pairs/s"
W_FULL, H_FULL, SCALE = 2704, 1520, 4
WORKLOAD = ("2704x1520 RGB pair: remap+downsample x4 -> 676x380 min-sum BP 64 labels, "
            "4 levels x 10 iters -> JBU 5x5 (sigma_s 1, sigma_r 12) + reprojection B=0.5 m to FP32 xyz")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--pairs-in-flight", type=int, default=3)   # measured best of 2, 3, 4, 6, 8
    ap.add_argument("--plain-steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=40)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--stream-frames", type=int, default=1500)
    ap.add_argument("--batch-pairs", type=int, default=48)
    ap.add_argument("--smooth-reps", type=int, default=20)
    ap.add_argument("--pose-reps", type=int, default=20)
    ap.add_argument("--small-reps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def slowest_over_ranks(value, device):
    """The largest of every rank's `value` (a time), via all-reduce MAX; the
    value itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world, units_per_rank, slowest_s):
    """Whole-job rate of `world` independent replicas: every rank's units over
    the slowest rank's time."""
    return world * units_per_rank / slowest_s


def replica_seeds(rank):
    """Scene seeds of a rank: each replica renders its own two terrain pairs."""
    return (2 * rank, 2 * rank + 1)


# ---------------------------------------------------------------------------
# CPU oracle pipeline (the reference arm and the cpu_baseline leg only)


def oracle_pipeline(left, right, cam, baseline):
    import oracle
    dl = oracle.rectify_remap(left, cam)
    dr = oracle.rectify_remap(right, cam)
    lrl, lgl = oracle.downsample_luma(dl, SCALE)
    _, lgr = oracle.downsample_luma(dr, SCALE)
    lab = oracle.bp(lgl, lgr, 64, 4, 10, 20, 10, 40, mode=oracle.MSG_DT)
    disp = oracle.guided_upsample(lab, lrl, dl, SCALE, 2, 1.0, 12.0)
    return oracle.reproject(disp, cam, baseline)


def crop_pair(left, right, cam, wc, hc):
    """A centred wc x hc crop treated as its own frame (principal point moved)."""
    x0 = (W_FULL - wc) // 2 // 4 * 4
    y0 = (H_FULL - hc) // 2 // 4 * 4
    c = list(cam)
    c[2] -= x0
    c[3] -= y0
    return (np.ascontiguousarray(left[y0:y0 + hc, x0:x0 + wc]),
            np.ascontiguousarray(right[y0:y0 + hc, x0:x0 + wc]), tuple(c))


def time_oracle_sample(left, right, cam, frac_budget_s):
    """The largest centred crop (wc, hc) whose oracle run fits the budget."""
    wc, hc = 256, 128
    l, r, c = crop_pair(left, right, cam, wc, hc)
    t0 = time.perf_counter()
    oracle_pipeline(l, r, c, 0.5)
    t_small = time.perf_counter() - t0
    per_px = t_small / (wc * hc)
    area = min(W_FULL * H_FULL, max(64 * 32, frac_budget_s / per_px))
    if area >= W_FULL * H_FULL:
        wc, hc = W_FULL, H_FULL
    else:
        aspect = W_FULL / H_FULL
        hc = max(32, int(np.sqrt(area / aspect)) // 32 * 32)
        wc = max(64, int(hc * aspect) // 32 * 32)
    return wc, hc


def cpu_sample_run(left, right, cam, wc, hc):
    l, r, c = crop_pair(left, right, cam, wc, hc)
    t0 = time.perf_counter()
    oracle_pipeline(l, r, c, 0.5)
    return time.perf_counter() - t0, (wc * hc) / (W_FULL * H_FULL)


def cpu_model():
    """The host CPU's model name (/proc/cpuinfo), or the platform's description."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_threads(n):
    """Sets the oracle's row-loop threads; returns the count in use."""
    import oracle
    return oracle.set_threads(n)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1902_09733_b300 import synth
    oracle.build()
    cores = oracle_threads(os.cpu_count() or 1)
    left, right = synth.terrain_pair(0)
    cam = synth.TERRAIN_CAMERA
    budget = 150.0 / max(1, args.steps + args.warmup)
    wc, hc = time_oracle_sample(left, right, cam, budget)
    for _ in range(args.warmup):
        cpu_sample_run(left, right, cam, wc, hc)
    tot, frac = 0.0, 0.0
    for _ in range(args.steps):
        t, f = cpu_sample_run(left, right, cam, wc, hc)
        tot += t
        frac += f
    value = frac / tot
    sample = (f"centred {wc}x{hc} crop of the 2704x1520 pair per step, oracle pipeline (DT messages), scaled by "
              f"area; rows over {cores} OpenMP threads ({cpu_model()})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "oracle": f"plain C, rows over {cores} threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if re.match(r"^[0-9.]+$", r[1])]
        smax = [float(r[2]) for r in rows if re.match(r"^[0-9.]+$", r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm


def sweep_bytes_per_launch(w, h, L):
    """Algorithmic bytes of one level-0 sweep launch, averaged over the two
    colours: each active pixel reads its data term (L bytes) and its in-frame
    incoming messages (L bytes each) and writes one message (L bytes) to each
    in-frame neighbour."""
    yy, xx = np.mgrid[0:h, 0:w]
    deg = (xx > 0).astype(int) + (xx < w - 1) + (yy > 0) + (yy < h - 1)
    per = (1 + 2 * deg) * L
    col = (xx + yy) & 1
    return 0.5 * (per[col == 0].sum() + per[col == 1].sum())


def sweep_ops_per_launch(w, h, L):
    """Algorithmic integer operations of one level-0 sweep launch, averaged
    over the two colours: per active pixel and label, the belief sum of the
    data term and the in-frame incoming messages (one add each), and per
    outgoing message the exclusion of its own incoming message (1), the
    forward and backward passes of the lower envelope (an add and a minimum
    each, 4), the running minimum (1) and the cap and shift min(G - H, Ts)
    (2): 36 L per interior pixel."""
    yy, xx = np.mgrid[0:h, 0:w]
    deg = (xx > 0).astype(int) + (xx < w - 1) + (yy > 0) + (yy < h - 1)
    per = (deg + 8 * deg) * L
    col = (xx + yy) & 1
    return 0.5 * (per[col == 0].sum() + per[col == 1].sum())


def alu_peak_ops(dev, torch, sm_mhz):
    """Peak of the integer ALU pipe in 16-bit operations per second: 64 lanes
    per SM per clock (4 sub-partitions of 16), each lane one packed add-min
    on two 16-bit halves (4 operations: viaddmin_u16x2), at the maximum SM
    clock."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 64 * 4 * sm_mhz * 1e6


def code_sha256(path: str) -> str:
    """SHA-256 of a source file's code: comments and blank lines removed, so
    edits to comments do not retire a capture of the same kernels."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln.strip()).encode()).hexdigest()


def committed_traffic(kernel_src: str):
    """DRAM bytes per launch of the level-0 sweep from the committed ncu
    summary, if it was taken on the current kernel code."""
    path = os.path.join(ROOT, "profiles", "k_bp_sweep_level0_2704x1520.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    sh = re.search(r"kernel_code_sha256:\s*([0-9a-f]+)", text)
    if not m or not sh:
        return None
    return float(m.group(1)) if sh.group(1) == code_sha256(kernel_src) else None


def straight_leg_frames(synth, torch, dev, cam, seed, n):
    """n consecutive 2704x1520 frames, 0.05 m apart along +x at 100 m over a
    terrain with box buildings, drawn on the GPU (device tensors)."""
    from paper_1902_09733_b300.scene import GpuScene
    poses = np.array([(-0.025 * (n - 1) + 0.05 * i, 0.0, 0.0) for i in range(n)])
    scene = synth.FlightScene(seed, 2.0 * 100.0 * 1.4 + 0.05 * n + 8.0)
    gs = GpuScene(scene, dev)
    return [gs.render(p, synth.TERRAIN_CAMERA) for p in poses]


def run_batched(args, vs, synth, torch, dev, cam):
    """48 grey pairs: downsample factor 2/4/8 of 2704x1520 and 32/64/96/128
    labels drawn from a seed, frame offsets 1..5 along a 100 m flight leg."""
    g = np.random.default_rng(2024)
    n = args.batch_pairs
    frames = straight_leg_frames(synth, torch, dev, cam, 7, 6)
    grey = {}
    for s in (2, 4, 8):
        for i, f in enumerate(frames):
            _, _, lg = vs.rectify_remap(f, cam, scale=s, dst=None, low_rgb=None)
            grey[(s, i)] = lg
    torch.cuda.synchronize()
    pairs, shapes = [], []
    for _ in range(n):
        s = int(g.choice([2, 4, 8]))
        L = int(g.choice([32, 64, 96, 128]))
        off = int(g.integers(1, 6))
        pairs.append((grey[(s, 0)], grey[(s, off)], vs.BPParams(L, 4, 10, 20, 10, 40)))
        shapes.append((s, L))
    # autotune the sweep kernels once per (scale, labels) shape
    tuned = {}
    for (s, L) in sorted(set(shapes)):
        p = vs.BPParams(L, 4, 10, 20, 10, 40)
        tuned[f"s{s}_L{L}"] = vs.bp_autotune(grey[(s, 0)], grey[(s, 1)], p)
    labels = [torch.empty(tuple(p[0].shape), dtype=torch.uint8, device=dev) for p in pairs]
    ws_b = torch.empty(vs.bp_batch_workspace_size(pairs), dtype=torch.uint8, device=dev)
    ws_s = torch.empty(max(vs.bp_workspace_size(p[0].shape[1], p[0].shape[0], p[2]) for p in pairs),
                       dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream(device=dev)

    def batched():
        vs.bp_stereo_batch(pairs, labels=labels, workspace=ws_b)

    def sequential():
        for (l, r, p), lab in zip(pairs, labels):
            vs.bp_stereo(l, r, p, labels=lab, workspace=ws_s)

    def graph_ms(fn, reps=5):
        with torch.cuda.stream(st):
            fn()
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=st):
            fn()
        gr.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            for _ in range(reps):
                gr.replay()
            e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    n0 = vs.kernel_launches()
    sequential()
    torch.cuda.synchronize()
    seq_launches = vs.kernel_launches() - n0
    t_seq = graph_ms(sequential)
    res = {}
    for mode in ("streams", "lockstep"):
        vs.bp_batch_mode(mode)
        n0 = vs.kernel_launches()
        batched()
        torch.cuda.synchronize()
        launches = vs.kernel_launches() - n0
        res[mode] = (graph_ms(batched), launches)
    vs.bp_batch_mode("streams")
    vs.bp_autotune_reset()
    t_bat, bat_launches = res["streams"]
    px = sum(int(p[0].numel()) * p[2].labels for p in pairs)
    return {"pairs": n, "batched_ms": t_bat, "sequential_ms": t_seq, "speedup": t_seq / t_bat,
            "batched_pairs_per_s": n / (t_bat * 1e-3), "schedule": "streams (4 library streams, pairs balanced by size)",
            "launches_batched": bat_launches, "launches_sequential": seq_launches,
            "lockstep_ms": res["lockstep"][0], "launches_lockstep": res["lockstep"][1],
            "label_pixels_per_batch": px,
            "mix": {f"s{s}_L{L}": shapes.count((s, L)) for (s, L) in sorted(set(shapes))},
            "autotuned_variants": tuned}


def run_batched_pairs(args, vs, synth, torch, dev, cam):
    """48 whole pairs (remap of both frames, BP, upsample + reproject) with the
    same seeded mix as run_batched: downsample factor 2/4/8 of 2704x1520,
    32/64/96/128 labels, frame offsets 1..5 (baseline 0.05 m each) along a
    100 m flight leg; one vs_pair_run_batch against 48 vs_pair_run calls,
    both as CUDA-graph replays."""
    g = np.random.default_rng(2024)
    n = args.batch_pairs
    frames = straight_leg_frames(synth, torch, dev, cam, 7, 6)
    camv = vs.Camera(*synth.TERRAIN_CAMERA)
    jobs, mix = [], []
    for _ in range(n):
        s = int(g.choice([2, 4, 8]))
        L = int(g.choice([32, 64, 96, 128]))
        off = int(g.integers(1, 6))
        cfg = vs.PairConfig(W_FULL, H_FULL, camv, 0.05 * off, vs.BPParams(L, 4, 10, 20, 10, 40),
                            vs.JBUParams(s, 2, 1.0, 12.0))
        xyz = torch.empty((H_FULL, W_FULL, 3), dtype=torch.float32, device=dev)
        jobs.append((cfg, frames[0], frames[off], None, xyz))
        mix.append((s, L))
    ws_b = torch.empty(vs.pair_batch_workspace_size(jobs), dtype=torch.uint8, device=dev)
    ws_s = torch.empty(max(vs.pair_workspace_size(j[0]) for j in jobs), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream(device=dev)

    def batched():
        vs.pair_run_batch(jobs, workspace=ws_b, stream=st)

    def sequential():
        for cfg, l, r, _, xyz in jobs:
            vs.pair_run(cfg, l, r, xyz=xyz, workspace=ws_s, stream=st)

    def graph_ms(fn, reps=5):
        with torch.cuda.stream(st):
            fn()
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=st):
            fn()
        gr.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            for _ in range(reps):
                gr.replay()
            e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    t_seq = graph_ms(sequential)
    t_bat = graph_ms(batched)
    return {"pairs": n, "batched_ms": t_bat, "sequential_ms": t_seq, "speedup": t_seq / t_bat,
            "batched_pairs_per_s": n / (t_bat * 1e-3), "sequential_pairs_per_s": n / (t_seq * 1e-3),
            "api": "vs_pair_run_batch (pairs balanced over 4 library streams) vs vs_pair_run one after another",
            "steps": "remap x2 + BP (4 x 10) + JBU + xyz per pair",
            "mix": {f"s{s}_L{L}": mix.count((s, L)) for (s, L) in sorted(set(mix))}}


def sp_kernel_band(L, lam, T):
    """Band of the library's SIMT smoothed-BP kernels: the smallest of 4, 6, 8
    holding the labels closer than T / lambda, 0 (dense) beyond or at 16 labels."""
    b = 0
    while b < 64 and lam * b < T:
        b += 1
    if L < 32 or b > 8:
        return 0
    return 4 if b <= 4 else (6 if b <= 6 else 8)


def sp_flops(L, band):
    """FP32 flops of one forward and one adjoint message of the smoothed BP.

    band = 0: the dense Toeplitz products, L^2 FMAs per product (K u forward;
    K u, the correlation and K r in the adjoint).  band > 0: each product is
    kinf * sum + the band |d - d'| < band, L (2 band - 1) - band (band - 1)
    FMAs plus L - 1 adds for the sum; the adjoint's correlation covers the
    band and its tail two running-sum passes of L - band adds and FMAs."""
    if band == 0:
        return 2.0 * L * L, 6.0 * L * L
    prod = 2.0 * (L * (2 * band - 1) - band * (band - 1)) + (L - 1)
    corr = 2.0 * (L + 2 * sum(L - d for d in range(1, band)))
    tail = 2 * (L - band) * 3.0
    return prod, 2 * prod + corr + tail


def run_smooth(args, vs, synth, torch, dev):
    """Smoothed (sum-product) BP and its adjoint on a 338x190x48 FP32 cost
    volume (truncated absolute differences of a seeded noise pair with
    disparities up to 40 px), 8 synchronous iterations, checkpoint every 2.
    Times one forward call and one adjoint call (which recomputes 4 of the 8
    iterations) per kernel family, with CUDA events, and relates the SIMT
    kernels to the FP32 FMA peak by the flops they execute (sp_flops)."""
    W, H, L = 338, 190, 48
    left, right, _ = synth.noise_pair(11, w=W, h=H, max_disp=40.0)
    IL = torch.from_numpy(left.astype(np.float32)).to(dev)
    IR = torch.from_numpy(right.astype(np.float32)).to(dev)
    cost = torch.full((H, W, L), 20.0, device=dev)
    for d in range(L):
        cost[:, d:, d] = torch.clamp((IL[:, d:] - IR[:, :W - d]).abs(), max=20.0)
    cost = cost.contiguous()
    p = vs.SPParams(labels=L, iters=8, ckpt_every=2, lam=2.5, trunc=13.75, tau=2.0)
    g = torch.Generator(device=dev).manual_seed(5)
    gb = torch.randn((H, W, L), device=dev, generator=g)
    edges = 2 * (W - 1) * H + 2 * W * (H - 1)
    sm_mhz = 2032.0
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        sm_mhz = float(json.load(open(pk_path)).get("sm_max_mhz", sm_mhz))
    fp32_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s, FMA = 2 flops
    out = {"workload": f"{W}x{H}x{L} FP32 cost volume, 8 synchronous iterations, checkpoint every 2, "
                       "lambda 2.5, trunc 13.75, tau 2", "reps": args.smooth_reps}
    for fam in ("simt", "tensor"):
        vs.sp_select_kernels(fam)
        bel, ws = vs.sp_forward(cost, p)
        gc, gp = vs.sp_backward(cost, p, gb, ws)
        for _ in range(3):
            vs.sp_forward(cost, p, beliefs=bel, workspace=ws)
            vs.sp_backward(cost, p, gb, ws, grad_cost=gc, grad_params=gp)
        torch.cuda.synchronize()
        vs.profile_enable(4096)
        vs.profile_collect()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        for _ in range(args.smooth_reps):
            vs.sp_forward(cost, p, beliefs=bel, workspace=ws)
        e[1].record()
        for _ in range(args.smooth_reps):
            vs.sp_backward(cost, p, gb, ws, grad_cost=gc, grad_params=gp)
        e[2].record()
        torch.cuda.synchronize()
        vs.sp_status(ws, W, H, p)
        by = {}
        for tag, ms in vs.profile_collect():
            by.setdefault(tag, []).append(ms)
        vs.profile_enable(0)
        fwd_us = 1e3 * statistics.median(by["smooth_fwd"])
        adj_us = 1e3 * statistics.median(by["smooth_adj"])
        r = {"forward_ms": e[0].elapsed_time(e[1]) / args.smooth_reps,
             "adjoint_ms": e[1].elapsed_time(e[2]) / args.smooth_reps,
             "forward_iteration_us": fwd_us, "adjoint_iteration_us": adj_us}
        if fam == "simt":
            band = sp_kernel_band(L, p.lam, p.trunc)   # lambda 2.5, T 13.75: 6
            f_msg, a_msg = sp_flops(L, band)
            fl_f, fl_a = edges * f_msg, edges * a_msg
            d_f, d_a = sp_flops(L, 0)
            r["alu"] = {"bound": "alu", "unit": "TFLOP/s", "peak": fp32_peak,
                        "peak_source": f"148 SMs x 128 FP32 FMA lanes x 2 x {sm_mhz:.0f} MHz",
                        "kernels": f"banded (K constant beyond {band} labels): {f_msg:.0f} / {a_msg:.0f} "
                                   f"flops per forward / adjoint message, against {d_f:.0f} / {d_a:.0f} dense",
                        "forward_achieved": fl_f / (fwd_us * 1e-6) / 1e12,
                        "adjoint_achieved": fl_a / (adj_us * 1e-6) / 1e12}
            r["alu"]["forward_frac"] = r["alu"]["forward_achieved"] / fp32_peak
            r["alu"]["adjoint_frac"] = r["alu"]["adjoint_achieved"] / fp32_peak
            # algorithmic bytes per iteration: forward, per pixel, D and the four
            # incoming rows read and the four outgoing messages written (9 L
            # floats); adjoint, the four gradients of the messages it sent and D
            # plus the four rows it recomputes from read, the four slot
            # gradients written and dL/dD read and written (15 L floats)
            pix = W * H
            fb, ab = 9 * L * 4 * pix, 15 * L * 4 * pix
            hbm_peak = float(json.load(open(pk_path)).get("hbm_gbs", 6400.0)) if os.path.exists(pk_path) else 6400.0
            r["hbm"] = {"unit": "GB/s", "peak": hbm_peak, "forward_alg_bytes": fb, "adjoint_alg_bytes": ab,
                        "forward_achieved": fb / (fwd_us * 1e-6) / 1e9,
                        "adjoint_achieved": ab / (adj_us * 1e-6) / 1e9}
            r["hbm"]["forward_frac"] = r["hbm"]["forward_achieved"] / hbm_peak
            r["hbm"]["adjoint_frac"] = r["hbm"]["adjoint_achieved"] / hbm_peak
        out[fam] = r
    vs.sp_select_kernels("simt")
    out["default_kernels"] = "simt"
    return out


def run_small(args, vs, synth, torch, dev):
    """The small configuration: BP on a 160x120 grey noise pair, 16 labels,
    3 levels x 5 iterations (its state sits in L2; the call is latency- and
    launch-bound).  Per-call latency with CUDA events, 20 warm-up and `reps`
    timed calls, median and p99, launched eagerly and as one CUDA-graph
    replay; the oracle on the same pair (DT messages), median of 3, on one
    thread and on all cores."""
    left, right, _ = synth.noise_pair(0)
    p = vs.BPParams(16, 3, 5, 20, 10, 40)
    L_t, R_t = torch.from_numpy(left).to(dev), torch.from_numpy(right).to(dev)
    h, w = left.shape
    ws = torch.empty(vs.bp_workspace_size(w, h, p), dtype=torch.uint8, device=dev)
    lab = torch.empty((h, w), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream(device=dev)
    call = lambda: vs.bp_stereo(L_t, R_t, p, labels=lab, workspace=ws)
    with torch.cuda.stream(st):
        call()
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=st):
        call()
    out = {"workload": "BP 160x120 grey noise pair, 16 labels, 3 levels x 5 iterations", "unit": "us per call",
           "reps": args.small_reps}
    for mode, fn in (("eager", call), ("graph", gr.replay)):
        ts = []
        with torch.cuda.stream(st):
            for i in range(20 + args.small_reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                e1.synchronize()
                if i >= 20:
                    ts.append(1e3 * e0.elapsed_time(e1))
        ts.sort()
        out[mode] = {"median_us": ts[len(ts) // 2], "p99_us": ts[min(len(ts) - 1, int(0.99 * len(ts)))]}
    if not args.no_cpu_baseline:
        import oracle
        cpu = {}
        for n in (1, os.cpu_count() or 1):
            used = oracle_threads(n)
            tt = []
            for _ in range(3):
                t0 = time.perf_counter()
                oracle.bp(left, right, 16, 3, 5, 20, 10, 40, mode=oracle.MSG_DT)
                tt.append(time.perf_counter() - t0)
            cpu[str(used)] = 1e6 * statistics.median(tt)
        oracle_threads(os.cpu_count() or 1)
        out["cpu_oracle_us"] = cpu
    return out


def run_pose(args, vs, synth, torch, dev):
    """The pose step (Section 2.3, Eq. 4-7) between frames 300 and 320 of a
    seeded lawnmower flight at 100 m (2704x1520, rendered on the GPU without
    lens distortion, frame 1's cloud from its rendered depth): integer Harris
    response, one corner per cell of a 30x30 grid, ZSSD (radius 5, search
    +-32 px), EPnP with two inlier rounds; and the same with the later
    pair's right image too (frame 323), the two poses averaged.  GPU: CUDA
    events over `reps` calls of each stage and of the whole step
    (vs_pose_estimate, vs_pose_estimate_stereo); CPU: the oracle on the same
    frames, once (a bounded sample: one step)."""
    from paper_1902_09733_b300.scene import GpuScene
    W, H = W_FULL, H_FULL
    cam6 = synth.TERRAIN_CAMERA[:4] + (0.0, 0.0)
    poses = synth.lawnmower_path(8, 800)
    scene = synth.FlightScene(8, synth.lawnmower_extent(poses), n_buildings=80)
    gs = GpuScene(scene, dev)
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    f1 = gs.render(poses[300], cam6, depth=depth)
    f2 = gs.render(poses[320], cam6)
    r2 = gs.render(poses[323], cam6)   # the later pair's right image (k = 3, 0.15 m on)
    vv, uu = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float32),
                            torch.arange(W, device=dev, dtype=torch.float32), indexing="ij")
    xyz = torch.stack([(uu - cam6[2]) / cam6[0] * depth, (vv - cam6[3]) / cam6[1] * depth, depth], -1).contiguous()
    p = vs.PoseParams(grid=30, margin=40, threshold25=0, radius=5, search=32)
    cam = vs.Camera(*cam6[:4])
    ws = torch.empty(vs.pose_workspace_size(W, H, p), dtype=torch.uint8, device=dev)
    ws2 = torch.empty(vs.pose_stereo_workspace_size(W, H, p), dtype=torch.uint8, device=dev)
    corners = vs.harris_corners(f1, p, workspace=ws)
    stages = {
        "harris_response": lambda: vs.harris_response(f1),
        "harris_corners": lambda: vs.harris_corners(f1, p, workspace=ws),
        "zssd_match": lambda: vs.zssd_match(f1, f2, corners, p),
        "pose_estimate": lambda: vs.pose_estimate(f1, f2, xyz, cam, p, workspace=ws),
        "pose_estimate_stereo": lambda: vs.pose_estimate_stereo(f1, f2, r2, xyz, cam, 0.15, p, workspace=ws2),
    }
    times = {}
    for name, fn in stages.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.pose_reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / args.pose_reps
    est = vs.pose_estimate(f1, f2, xyz, cam, p, workspace=ws).cpu().numpy()
    est2 = stages["pose_estimate_stereo"]().cpu().numpy()
    Rt, Tt = synth.relative_pose(poses[300], poses[320])
    ang = float(np.degrees(np.arccos(np.clip((np.trace(est[:9].reshape(3, 3).T @ Rt) - 1) / 2, -1, 1))))
    res = {"workload": "pose step between two 2704x1520 lawnmower frames 20 apart (1 m at 100 m): Harris "
                       "25R, 30x30 grid corners (margin 40), ZSSD radius 5 search +-32, EPnP + 2 inlier rounds",
           "unit": "pose steps/s", "value": 1e3 / times["pose_estimate"], "reps": args.pose_reps,
           "stage_ms": times, "inliers": float(est[13]), "reprojection_px": float(est[12]),
           "rotation_error_deg": ang, "translation": est[9:12].tolist(), "true_translation": list(map(float, Tt)),
           "stereo": {"what": "left and right images of the later pair (frames 320, 323), poses averaged through "
                              "the virtual rig (vs_pose_estimate_stereo)",
                      "ms": times["pose_estimate_stereo"], "translation": est2[9:12].tolist(),
                      "rotation_error_deg": float(np.degrees(np.arccos(np.clip(
                          (np.trace(est2[:9].reshape(3, 3).T @ Rt) - 1) / 2, -1, 1))))}}
    if not args.no_cpu_baseline:
        from oracle import pose as opose
        h1, h2 = f1.cpu().numpy(), f2.cpu().numpy()
        P = xyz.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        r25 = opose.harris_response25(h1)
        c = opose.harris_corners(r25, 30, 40, 0)
        pos, _ = opose.zssd_match(h1, h2, c, radius=5, search=32)
        ok = (c[:, 0] >= 0) & ~np.isnan(pos).any(axis=1)
        pts = P[c[ok, 1], c[ok, 0]]
        ok2 = ~np.isnan(pts).any(axis=1)
        opose.epnp_inliers(pts[ok2], pos[ok][ok2], cam6[:4])
        tsec = time.perf_counter() - t0
        res["cpu_oracle"] = {"value": 1.0 / tsec, "unit": "pose steps/s", "s_per_step": tsec, "cores": 1,
                             "kind": "oracle", "sample": "one pose step on the same frames (numpy, int64 / FP64)"}
    return res


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1902_09733_b300 as vs
    from paper_1902_09733_b300 import build, synth
    build.build()
    dev = torch.device("cuda", local)

    cam = vs.Camera(*synth.TERRAIN_CAMERA)
    bp = vs.BPParams(labels=64, levels=4, iters=10, data_trunc=20, smooth_slope=10, smooth_trunc=40)
    jbu = vs.JBUParams(scale=SCALE, radius=2, sigma_s=1.0, sigma_r=12.0)
    cfg = vs.PairConfig(W_FULL, H_FULL, cam, 0.5, bp, jbu)

    # eight distinct resident pairs (197 MB > L2)
    host_pairs = []
    for seed in replica_seeds(rank):
        l, r = synth.terrain_pair(seed)
        host_pairs.extend(synth.pair_variants(l, r))
    pairs = [(torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev)) for l, r in host_pairs]
    P = max(1, args.pairs_in_flight)
    ws = [torch.empty(vs.pair_workspace_size(cfg), dtype=torch.uint8, device=dev) for _ in range(P)]
    xyz = [torch.empty((H_FULL, W_FULL, 3), dtype=torch.float32, device=dev) for _ in range(P)]

    stream = torch.cuda.Stream(device=dev)
    side = [torch.cuda.Stream(device=dev) for _ in range(P)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        vs.pair_run(cfg, *pairs[0], xyz=xyz[0], workspace=ws[0])   # load every kernel once
    torch.cuda.synchronize()

    def capture(first, n):
        """A graph that runs pairs first .. first+n-1 (mod 8) on n streams."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            if n == 1:
                vs.pair_run(cfg, *pairs[first % len(pairs)], xyz=xyz[0], workspace=ws[0], stream=stream)
            else:
                fork = torch.cuda.Event()
                fork.record(stream)
                joins = []
                for k in range(n):
                    side[k].wait_event(fork)
                    vs.pair_run(cfg, *pairs[(first + k) % len(pairs)], xyz=xyz[k], workspace=ws[k],
                                stream=side[k])
                    e = torch.cuda.Event()
                    e.record(side[k])
                    joins.append(e)
                for e in joins:
                    stream.wait_event(e)
        return g

    n0 = vs.kernel_launches()
    graphs = [capture(P * i, P) for i in range(len(pairs))]
    launches_per_step = (vs.kernel_launches() - n0) // len(pairs)
    plain_graphs = [capture(i, 1) for i in range(len(pairs))]
    # single-pair graphs whose launches are bracketed by CUDA events
    # (profiling stays on until these have been replayed and collected: the
    # graphs record into its events)
    vs.profile_enable(4096)
    prof_graphs = [capture(i, 1) for i in range(len(pairs))]
    torch.cuda.synchronize()

    def timed(gs, steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for k in range(steps):
                gs[k % len(gs)].replay()
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    # warm-up
    for k in range(args.warmup):
        graphs[k % len(graphs)].replay()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    K = args.steps
    elapsed_ms = timed(graphs, K)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    slowest_ms = slowest_over_ranks(elapsed_ms, dev)

    # plain rate (one pair per replay) and the per-kernel event times of
    # single-pair replays, right after the timed region
    plain = None
    if args.plain_steps > 0:
        for k in range(args.warmup):
            plain_graphs[k % len(plain_graphs)].replay()
        t_plain = timed(plain_graphs, args.plain_steps)
        plain = {"value": args.plain_steps / (t_plain * 1e-3), "unit": UNIT, "steps": args.plain_steps,
                 "ms_per_pair": t_plain / args.plain_steps}
    timed(prof_graphs, len(prof_graphs))
    recs = vs.profile_collect()
    n_prof_pairs = len(prof_graphs)
    del prof_graphs
    # the same events in the timed configuration: P pairs in flight
    recs_flight = []
    if P > 1:
        pf = capture(0, P)
        timed([pf], 1)
        recs_flight = vs.profile_collect()
        del pf
    vs.profile_enable(0)
    timing_src = "CUDA events around each launch in single-pair graph replays right after the timed region"

    # per-kernel durations from the event pairs of the last replays
    by_tag = {}
    for tag, ms in recs:
        by_tag.setdefault(tag, []).append(ms)
    sweep_ms = statistics.mean(by_tag["sweep_level0"]) if by_tag.get("sweep_level0") else None
    flight_l0 = [ms for tag, ms in recs_flight if tag == "sweep_level0"]
    sweep_ms_flight = statistics.mean(flight_l0) if flight_l0 else None
    w, h = W_FULL // SCALE, H_FULL // SCALE
    alg_bytes = sweep_bytes_per_launch(w, h, 64)
    alg_ops = sweep_ops_per_launch(w, h, 64)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6400.0
    achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9 if sweep_ms else None
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = alu_peak_ops(dev, torch, sm_max) / 1e9
    alu_achieved = alg_ops / (sweep_ms * 1e-3) / 1e9 if sweep_ms else None
    traffic = committed_traffic(os.path.join(ROOT, "paper_1902_09733_b300", "csrc", "vs_bp.cu"))
    kernel_share = None
    if recs:
        tot = sum(ms for _, ms in recs)
        kernel_share = {k: round(sum(v) / tot, 4) for k, v in by_tag.items()}
    # the other HBM-facing stages of the pair, by their own algorithmic bytes:
    # remap -- both frames read, the left written at full resolution with its
    # low-res RGB and both low-res greys (two launches per pair); upsample --
    # labels, low-res and full-res guides read, the FP32 cloud written, and
    # one ex2 per pixel and tap against the measured special-function rate
    # (30 per clock per SM on this GPU)
    stage_rooflines = None
    if by_tag.get("remap") and by_tag.get("upsample"):
        full, low = W_FULL * H_FULL * 3, w * h * 3
        remap_bytes = 2 * full + full + low + 2 * w * h
        # one launch per pair (both frames) or one per frame: the sum per pair
        remap_ms = sum(by_tag["remap"]) / n_prof_pairs
        up_bytes = w * h + low + full + W_FULL * H_FULL * 12
        up_ms = statistics.mean(by_tag["upsample"])
        ex2 = W_FULL * H_FULL * 25
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mufu_peak = nsm * 30 * sm_max * 1e6
        stage_rooflines = {
            "remap": {"alg_bytes_per_pair": remap_bytes, "ms_per_pair": remap_ms,
                      "achieved_gbs": remap_bytes / (remap_ms * 1e-3) / 1e9,
                      "frac": remap_bytes / (remap_ms * 1e-3) / 1e9 / peak, "bound": "instruction issue"},
            "upsample": {"alg_bytes": up_bytes, "ms": up_ms, "achieved_gbs": up_bytes / (up_ms * 1e-3) / 1e9,
                         "frac": up_bytes / (up_ms * 1e-3) / 1e9 / peak, "ex2_per_launch": ex2,
                         "mufu_frac": ex2 / (up_ms * 1e-3) / mufu_peak, "bound": "instruction issue"},
            "peak_gbs": peak, "timing": timing_src}

    # end to end through the public streaming API from pinned host memory:
    # every step copies both frames in and the point cloud out; consecutive
    # steps overlap their copies and compute on three streams
    e2e = None
    if args.e2e_steps > 0:
        pipe = vs.Pipeline(cfg, mode="pairs", depth=3)
        lh = [torch.from_numpy(host_pairs[i][0]).pin_memory() for i in range(2)]
        rh = [torch.from_numpy(host_pairs[i][1]).pin_memory() for i in range(2)]
        xh = [torch.empty((H_FULL, W_FULL, 3), dtype=torch.float32).pin_memory() for _ in range(3)]
        for i in range(6):
            pipe.submit_pair(lh[i % 2], rh[i % 2], xh[i % 3])
        pipe.flush()
        pipe.latencies()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            pipe.submit_pair(lh[i % 2], rh[i % 2], xh[i % 3])
        pipe.flush()
        t_e2e = time.perf_counter() - t0
        lat = sorted(pipe.latencies())
        pipe.close()
        t_e2e = slowest_over_ranks(t_e2e, dev)
        e2e = {"value": replica_rate(world, args.e2e_steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": 2 * W_FULL * H_FULL * 3, "d2h_bytes_per_step": W_FULL * H_FULL * 3 * 4,
               "steps": args.e2e_steps, "api": "vs_pipeline_submit_pair (3 streams, depth 3)",
               "latency_ms_p50": lat[len(lat) // 2] if lat else None}

    # streaming flight: 1500 distinct frames of a seeded lawnmower flight at
    # 100 m (legs of 25 m joined by half-circle turns, camera heading along
    # the track), rendered on the GPU into pinned host memory before the
    # timed run; one new frame per pair, each frame remapped once, pairs of
    # frames k = 3 apart
    streaming = None
    if args.stream_frames > 0 and rank == 0:
        from paper_1902_09733_b300.scene import GpuScene
        k = 3
        nf = args.stream_frames
        poses = synth.lawnmower_path(100 + rank, nf)
        scene = synth.FlightScene(100 + rank, synth.lawnmower_extent(poses), n_buildings=80)
        gs = GpuScene(scene, dev)
        distinct = nf
        host = None
        while host is None:
            try:
                host = torch.empty((distinct, H_FULL, W_FULL, 3), dtype=torch.uint8, pin_memory=True)
            except RuntimeError:
                distinct //= 2
                if distinct < 16:
                    raise
        buf = torch.empty((H_FULL, W_FULL, 3), dtype=torch.uint8, device=dev)
        t_r = time.perf_counter()
        for i in range(distinct):
            gs.render(poses[i], synth.TERRAIN_CAMERA, out=buf)
            host[i].copy_(buf)
        torch.cuda.synchronize()
        render_s = time.perf_counter() - t_r
        del gs
        fcfg = vs.PairConfig(W_FULL, H_FULL, cam, 0.05 * k, bp, jbu)
        xh = [torch.empty((H_FULL, W_FULL, 3), dtype=torch.float32).pin_memory() for _ in range(3)]
        pipe = vs.Pipeline(fcfg, mode="flight", depth=3, k=k)
        for f in range(8):
            pipe.submit_frame(host[f], xh[f % 3])
        pipe.flush()
        pipe.latencies()
        pipe.close()
        pipe = vs.Pipeline(fcfg, mode="flight", depth=3, k=k)
        t0 = time.perf_counter()
        for f in range(nf):
            pipe.submit_frame(host[f % distinct], xh[f % 3] if f >= k else None)
        pipe.flush()
        t_s = time.perf_counter() - t0
        lat = sorted(pipe.latencies())
        pipe.close()
        del host
        n_pairs = nf - k
        streaming = {"pairs_per_s": n_pairs / t_s, "frames": nf, "distinct_frames": distinct, "k": k,
                     "baseline_m": 0.05 * k, "latency_ms_p50": lat[len(lat) // 2],
                     "latency_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                     "h2d_bytes_per_pair": W_FULL * H_FULL * 3, "d2h_bytes_per_pair": W_FULL * H_FULL * 12,
                     "render_s": render_s,
                     "input": f"{distinct} distinct frames of a seeded lawnmower flight at 100 m (25 m legs, "
                              "8 m half-circle turns, 80 box buildings 5-30 m), rendered on the GPU into "
                              "pinned host memory before the timed run"}

    # batched BP: 48 pairs of uneven sizes and label counts in lockstep,
    # against the same 48 pairs as sequential single-pair calls (both as
    # CUDA-graph replays, after autotuning the sweep kernels on each shape)
    batched = None
    if args.batch_pairs > 0 and rank == 0:
        batched = run_batched(args, vs, synth, torch, dev, cam)
        batched["whole_pairs"] = run_batched_pairs(args, vs, synth, torch, dev, cam)

    # smoothed BP + adjoint (the differentiable relaxation of Eq. 1)
    small = None
    if args.small_reps > 0 and rank == 0:
        small = run_small(args, vs, synth, torch, dev)
    pose = None
    if args.pose_reps > 0 and rank == 0:
        pose = run_pose(args, vs, synth, torch, dev)
    smooth = None
    if args.smooth_reps > 0 and rank == 0:
        smooth = run_smooth(args, vs, synth, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on one full pair: all host cores (rows over OpenMP
        # threads) and one thread, median of 3 runs each
        cam_t = synth.TERRAIN_CAMERA
        rates = {}
        for n in (os.cpu_count() or 1, 1):
            used = oracle_threads(n)
            ts = []
            for _ in range(3):
                tsec, frac = cpu_sample_run(host_pairs[0][0], host_pairs[0][1], cam_t, W_FULL, H_FULL)
                ts.append(tsec)
            rates[used] = (frac / statistics.median(ts), statistics.median(ts))
        all_cores = max(rates)
        cpu = {"value": rates[all_cores][0], "unit": UNIT, "cores": all_cores, "kind": "oracle",
               "cpu_model": cpu_model(),
               "single_thread": {"value": rates[1][0], "unit": UNIT, "cores": 1,
                                 "s_per_pair": rates[1][1]},
               "sample": "one full 2704x1520 pair through the oracle pipeline (FP64 remap/JBU, int32 BP with "
                         f"DT messages), median of 3 runs: {rates[all_cores][1]:.2f} s on {all_cores} threads "
                         f"(rows of each stage over OpenMP), {rates[1][1]:.2f} s on one"}

    if rank == 0:
        value = replica_rate(world, K * P, slowest_ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": slowest_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}", "pairs_in_flight": P,
                       "l2": "8 distinct input pairs (197 MB) rotated per step, larger than L2",
                       "launch": f"one CUDA graph replay per step, {P} pairs on {P} streams"},
            "plain": plain,
            "roofline": {"bound": "alu", "kernel": "k_bp_sweep_staged / k_bp_sweep (the 10 level-0 sweeps)",
                         "achieved": alu_achieved, "peak": alu_peak, "unit": "Gop/s",
                         "frac": alu_achieved / alu_peak if alu_achieved else None, "traffic": traffic,
                         "alg_ops_per_launch": alg_ops, "avg_launch_ms": sweep_ms,
                         "avg_launch_ms_in_flight": sweep_ms_flight,
                         "peak_source": f"derived: SMs x 64 ALU lanes x 4 ops (packed add-min) x {sm_max:.0f} MHz",
                         "timing": timing_src,
                         "hbm": {"alg_bytes_per_launch": alg_bytes, "achieved_gbs": achieved, "peak_gbs": peak,
                                 "alg_frac": achieved / peak if achieved else None,
                                 "dram_frac": traffic / (sweep_ms * 1e-3) / 1e9 / peak if traffic and sweep_ms
                                 else None, "peak_source": f"{peak_src} hbm_gbs"},
                         "note": "ops: 16-bit integer adds and minima of the O(L) min-sum update, 36 L per "
                                 "interior active pixel; traffic: one-pass ncu DRAM bytes per launch with "
                                 "the default pairs in flight; the level's costs and messages mostly stay in L2, and "
                                 "the integer ALU pipe is the busiest unit"},
            "kernel_share": kernel_share,
            "stage_rooflines": stage_rooflines,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "streaming": streaming,
            "batched": batched,
            "smooth_bp": smooth,
            "pose": pose,
            "small_config": small,
            "gpu_launches": launches_per_step * K,
            "pairs_per_step": P,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
