#!/usr/bin/env python3
"""Benchmark of the GB300 mapping iteration (VIGS-SLAM Sec. 3.3, Eq. 6).

One step = one full mapping iteration of the plain single-view workload:
640x480 view (fx = fy = 525) inside a synthetic room of 200k Gaussians;
project -> bin/sort -> composite colour+depth -> L1 colour/depth + isotropic
loss -> backward to every parameter and the pose -> Adam.  The iteration is
replayed from a CUDA graph; inputs (map, target image and depth) are resident
in HBM when the timed region starts; before each timed iteration the map and
Adam state are restored to the same starting values and L2 is flushed (a
256 MiB write), both outside the per-step events.

Metric: mapping iterations/s (whole job; N GPUs run independent replicas,
weak scaling).  Also reported: Gpix-splats/s (sum over pixels of the splats a
pixel visits, divided by the forward-raster time), per-stage times, the
roofline of the dominant kernel, the end-to-end rate through the C ABI with
host buffers, and the FP64 oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mapping iters/sec (fwd+bwd, 1 GB300) and Gpix-splats/s vs plain form at oracle tolerance"
WORKLOAD = "plain single view, SLAM scale: 640x480, 200k Gaussians on a synthetic room (6 planes + 20 boxes)"
# The rasterisers' arithmetic per (pixel, splat) pair, two ways: FP32 operations
# with a fused multiply-add counted as one (against the lane peak: 152 SMs x
# 128 FP32 lanes x clock), and FP32 FLOPs of the method's arithmetic with a
# multiply-add counted as two (against the FLOP peak, twice the lane peak).
# Forward per visited pair: offset 2, exponent 9, opacity 1, cutoff test 2,
# weight and colour / depth accumulation 9 -> 23 FLOPs (+ 1 exp2).  Backward per
# pair: the forward's weight again 12, the transmittance before the splat 2,
# dL/dalpha 13, the colour behind 12, dL/dpower 3, the ten gradients 20 -> 62
# FLOPs (+ 1 exp2, 1 reciprocal).
FWD_OPS_PER_PAIR = 20
BWD_OPS_PER_PAIR = 45
FWD_FLOP_PER_PAIR = 23
BWD_FLOP_PER_PAIR = 62
L2_FLUSH_BYTES = 256 << 20
# Algorithmic bytes of the memory-bound stages: projection 56 B read per
# Gaussian (once for all views) + 64 B written per (view, Gaussian); binning 56 B per entry (rect and depth read by
# the count and scatter passes), 28 B per key (composite written, read and the
# key and value written by the per-tile sort) and 528 B per tile (32 stripe
# counters zeroed, counted, scanned; the total and the range); projection
# backward 56 B of parameters + 48 B of 2D gradients per view read and 56 B of
# gradients written per Gaussian; Adam 28 B per parameter element (14 per
# Gaussian).  For binning, the radix-sort reference count (12 B per key
# duplicated + 2 x 12 B per key per 8-bit pass over 31 depth bits and the tile
# bits) is reported beside it.
PROJECT_BYTES_PER_GAUSSIAN, PROJECT_BYTES_PER_ENTRY = 56, 64
BIN_BYTES_PER_ENTRY, BIN_BYTES_PER_KEY, BIN_BYTES_PER_TILE = 56, 28, 528
PROJECT_BWD_BYTES_PER_GAUSSIAN, PROJECT_BWD_BYTES_PER_ENTRY = 56 + 56, 48
ADAM_BYTES_PER_ELEMENT, ADAM_ELEMENTS_PER_GAUSSIAN = 28, 14
# From one ncu capture of one iteration of this workload (640x480, 200k
# Gaussians, tile 16): dram__bytes_read.sum + dram__bytes_write.sum per launch
# of each stage's kernels (cold cache), and the binding pipe of the rasterisers
# (their full-section captures).  None where the kernel changed after the
# capture.
# Keyed by (stage, tile, ring, block_masks) for the forward (its staging variant)
# and (stage, tile, None, block_masks) for the others; block_masks 1 is the
# build with the masks and the tile culling the autotuner pairs with them.
PROFILED_TRAFFIC = {("gs_project", 16, None, 0): 11.30e6, ("gs_render_fwd_loss", 16, False, 0): 14.25e6,
                    ("gs_project_bwd", 16, None, 0): 16.41e6, ("gs_adam_step", 16, None, 0): 44.83e6,
                    ("gs_project", 16, None, 1): 11.28e6, ("gs_bin_sort", 16, None, 1): 30.65e6,
                    ("gs_render_fwd_loss", 16, False, 1): 14.61e6,
                    ("gs_render_bwd_raster_loss", 16, None, 1): 27.59e6, ("gs_project_bwd", 16, None, 1): 16.42e6,
                    ("gs_adam_step", 16, None, 1): 44.82e6}
# L2 bytes (lts__t_bytes.sum) per launch of the binning stage's kernels, from
# the same kind of capture.
PROFILED_L2 = {("gs_bin_sort", 16, 1): 115.1e6}
PROFILED_PIPE = {
    ("gs_render_fwd_loss", 16, False, 0): "the deepest blocks' serial walks, then instruction issue: SMs active 64.5 % "
                                          "of the launch, 62.7 % of active cycles issue; pipes ALU 38.3 %, FMA 28.1 %, "
                                          "XU (ex2) 9.4 %",
    ("gs_render_fwd_loss", 16, False, 1): "the deepest blocks' serial walks, then instruction issue: SMs active 67.8 % "
                                          "of the launch, 65.0 % of active cycles issue; pipes ALU 46.0 %, LSU 28.0 %, "
                                          "FMA 22.4 %, XU (ex2) 6.8 %",
    ("gs_render_bwd_raster_loss", 16, None, 1): "instruction issue: 70.6 % of active cycles issue; pipes LSU 45.2 %, "
                                                "ALU 44.9 %, FMA 29.8 %, XU (ex2, rcp) 5.5 %; SMs active 93 % of the "
                                                "launch"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = threading.Event()
        self.start_at = 0
        self.after = False

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=5.0)          # nvidia-smi is up before the timed region starts
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def mark(self):
        """Start of the timed region: samples before it are dropped."""
        self.start_at = len(self.lines)

    def __exit__(self, *a):
        if self.proc is not None:
            if len(self.lines) <= self.start_at:
                # a timed region shorter than the sampling period: keep the first
                # sample taken right after it (noted in the summary)
                t0 = time.time()
                while len(self.lines) <= self.start_at and time.time() - t0 < 0.5:
                    time.sleep(0.005)
                self.after = True
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.start_at:]:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); mx = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}
        if self.after:
            out["note"] = "timed region shorter than the 20 ms sampling period: sample taken just after it"
        return out


def build_step(device, g, gt, cams, candidates=(8, 16, 32), stages=(2, 3), masks=(1, 0)):
    """Target images of the perturbed map (input preparation, not timed), then a
    mapping step on the map with the tile size, the forward's splat staging and
    the block masks autotuned over `candidates` x `stages` x `masks`."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep, autotune_tile
    params = G.RenderParams(tile=16)
    mp = MapParams()
    P = G.gs_total_pixels(cams)
    dummy_c = torch.zeros(3 * P, device=device); dummy_d = torch.zeros(P, device=device)
    tstep = MappingStep(G.Gaussians.from_numpy(gt, device), cams, dummy_c, dummy_d, params, mp)
    tstep.render()
    torch.cuda.synchronize()
    tc = tstep.img.color.clone(); td = tstep.img.depth.clone()
    del tstep
    gd = G.Gaussians.from_numpy(g, device)
    params, tune = autotune_tile(gd, cams, tc, td, params, mp, candidates=candidates, stages=stages, masks=masks)
    step = MappingStep(gd, cams, tc, td, params, mp)
    step.tune = tune
    return params, mp, step, tc, td


def timed_run(step, steps, warmup, flush, dist=None, clock_index=None):
    """Graph-replayed iterations, each from the same map and Adam state (restored
    before the step) after an L2 flush.  Two graphs of the same C-ABI calls
    are captured: a plain one, whose replays are timed by CUDA events recorded on
    the launch stream around each replay (the per-step times), and one with an
    event-record node before and after each call, replayed as many times again for
    the per-stage medians (the event nodes themselves add a few microseconds to a
    step, so they stay out of the per-step times).  Returns per-step ms, per-stage
    median ms, visited pairs and the clock summary."""
    import torch
    step.step()
    if step.ensure_capacity():
        step.step()
        assert not step.ensure_capacity()
    pairs = plain_visited_pairs(step)
    evs = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(len(step.stages) + 1)]
    staged_graph = step.capture(warmup=1, events=evs)
    step.capture(warmup=0)                          # the plain graph, replayed by step()
    for _ in range(warmup):
        step.step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    pristine = [t.clone() for t in step.g.tensors()]

    def restore():
        for t, p0 in zip(step.g.tensors(), pristine):
            t.copy_(p0)
        for t in step.m + step.v:
            t.zero_()
        step.d_step.zero_()

    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    per_stage = {k: [] for k in step.stages}
    times = []
    clk = ClockSampler(clock_index) if clock_index is not None else None
    if clk:
        clk.__enter__()
    try:
        torch.cuda.synchronize()
        if clk:
            clk.mark()
        for _ in range(steps):
            restore()
            flush()
            ev[0].record(s); step.step(); ev[1].record(s)
            torch.cuda.synchronize()
            times.append(ev[0].elapsed_time(ev[1]))
    finally:
        if clk:
            clk.__exit__()
    for _ in range(steps):
        restore()
        flush()
        staged_graph.replay()
        torch.cuda.synchronize()
        for j, nm in enumerate(step.stages):
            per_stage[nm].append(evs[j].elapsed_time(evs[j + 1]))
    if dist is not None:
        dist.barrier()
    status = step.check()
    if status != 0:
        raise RuntimeError(f"device status {status} after the timed region")
    st = {k: statistics.median(v) for k, v in per_stage.items()}
    return times, st, pairs, (clk.summary() if clk else None)


def bwd_ctas_per_sm(step, tile) -> int:
    """The backward rasteriser's occupancy variant the library picks: 2 CTAs per
    SM up to 256 pixel blocks per SM, else 3."""
    items = step.total_tiles * (tile // 8) * (tile // 4)
    return 2 if items <= 256 * 152 else 3


def launches_per_step(step) -> int:
    """Kernels of ours per iteration: project 1; bin/sort 6 (count zeroing, striped
    tile counts, stripe prefixes, tile offsets and work lists, scatter, per-tile
    sort) + 1 for the block masks; render 1 (with the fused loss); loss (unfused
    only): accumulator zeroing 1 + 2; backward: gradient zeroing 1 (the block
    order's launch when the fused backward orders its blocks, few blocks per SM)
    + raster 1, pose/iso zeroing 1 + projection backward 1; Adam 1."""
    return 1 + 6 + int(step.params.block_masks) + 1 + (0 if step.fused_loss else 3) + 4 + 1


def raster_stages(step):
    """Names of the forward and backward raster stages of this step's calls."""
    if step.fused_loss:
        return "gs_render_fwd_loss", "gs_render_bwd_raster_loss"
    return "gs_render_fwd", "gs_render_bwd_raster"


def _oracle_prm(params):
    return dict(tile=params.tile, near=params.near_plane, alpha_min=params.alpha_min, alpha_max=params.alpha_max,
                T_cut=params.T_cut, dilation=params.dilation, radius_sigma=params.radius_sigma,
                bg=tuple(params.bg), sh_degree=params.sh_degree)


def _oracle_workloads():
    """The three workloads the oracle is timed on: the 64x48 / 256-Gaussian case,
    the 640x480 / 200k-Gaussian room (the benchmark's workload) and the
    4k-Gaussian sub-sample of the 1M SH-3 room over its 16 keyframes at 160x128."""
    import numpy as np
    from paper_2512_02293_gb300 import synth
    g1, gt1, c1 = synth.cfg1_problem(0)
    g2, gt2, c2 = synth.cfg2_problem()
    g4f, _, cams4 = synth.cfg4_problem()
    cs4 = [synth.Camera(c.fx / 8, c.fy / 8, c.cx / 8, c.cy / 8, 160, 128, c.R_wc, c.t_wc) for c in cams4]
    idx = np.sort(np.random.default_rng(3).choice(g4f.n, 4000, replace=False))
    g4 = g4f.subset(idx)
    return [("64x48 / 256 Gaussians", g1, gt1, [c1], 0),
            ("640x480 / 200k Gaussians", g2, gt2, [c2], 0),
            ("4k-Gaussian sub-sample of the 1M SH-3 room, 16 views at 160x128", g4, synth.perturb_map(g4, 7), cs4, 3)]


def _oracle_iteration_fn(g, gt, cams, params, mp, sh_degree):
    """A closure that runs one full FP64 mapping iteration (render, Eq. 6 loss,
    gradients, Adam) from the same starting state every call."""
    import oracle
    prm = dict(_oracle_prm(params), sh_degree=sh_degree)
    targets = []
    for c in cams:
        img = oracle.render_fwd(oracle.project(gt, c, prm), c, prm)
        targets.append((img["color"], img["depth"]))
    lambdas = (mp.lambda_c, mp.lambda_d, mp.lambda_iso)

    def one():
        st = oracle.adam_state(g)                  # fresh state (outside the timed call)
        t0 = time.perf_counter()
        oracle.mapping_iteration(g, cams, targets, prm, lambdas, mp.lr, st, mp.beta1, mp.beta2, mp.eps)
        return time.perf_counter() - t0
    return one


L2_PEAK = {}     # measured once per run by measure_l2_peak


def measure_l2_peak(device, total_gib=2.0):
    """Read bandwidth of a buffer that stays in L2 (129 MB), by the library's
    gs_l2_read_probe: one launch reads the buffer over and over (about
    `total_gib` GiB in all) with 16-byte loads cached in L2 only; bytes read over
    the launch's device time, for buffers of 8 to 96 MiB, the best of
    the sizes.  This is the denominator of the binning stage's L2 roofline (its
    keys, counters and ranges live in L2 between the stage's six launches)."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    best, per = 0.0, {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = torch.zeros(1, device=device)
    for mib in (8, 16, 32, 48, 64, 96):
        n = mib * (1 << 20) // 4
        reps = max(1, int(total_gib * (1 << 30)) // (n * 4))
        buf = torch.ones(n, device=device)
        for _ in range(2):
            G.gs_l2_read_probe(buf, reps, out)
        torch.cuda.synchronize()
        times = []
        for _ in range(5):
            ev[0].record(); G.gs_l2_read_probe(buf, reps, out); ev[1].record(); torch.cuda.synchronize()
            times.append(ev[0].elapsed_time(ev[1]))
        gbs = reps * n * 4 / (min(times) * 1e-3) / 1e9
        per[f"{mib}MiB"] = round(gbs, 1)
        best = max(best, gbs)
        del buf
    L2_PEAK.update({"gbs": best, "per_size": per,
                    "method": f"gs_l2_read_probe: one launch reading an L2-resident buffer over and over (about "
                              f"{total_gib:g} GiB), best of 8 / 16 / 32 / 48 / 64 / 96 MiB buffers"})
    return L2_PEAK


def plain_visited_pairs(step) -> int:
    """Sum of n_contrib over the step's views on the plain lists (every tile of
    each rectangle): the method's count of visited (pixel, splat) pairs.  With
    tile culling the step's own n_contrib counts positions in the shorter lists,
    so one uncaptured render without it gives the count (the image is the same)."""
    import dataclasses
    import torch
    from paper_2512_02293_gb300.mapping import MappingStep
    if not step.params.cull_tiles:
        return int(step.img.n_contrib.to(torch.int64).sum().item())
    plain = MappingStep(step.g, step.cams, step.target_color, step.target_depth,
                        dataclasses.replace(step.params, cull_tiles=0), step.mp, fused_loss=step.fused_loss)
    plain.render()
    if plain.ensure_capacity():
        plain.render()
    n = int(plain.img.n_contrib.to(torch.int64).sum().item())
    del plain
    torch.cuda.empty_cache()
    return n


def evaluated_pairs(step, alpha_min=None) -> int:
    """(pixel, splat) pairs the rasterisers evaluate, counted independently of
    their kernels: for every 8 x 4 pixel block of every tile, the splats of the
    tile's list before the block's deepest n_contrib whose weight can reach
    0.99 alpha_min somewhere in the block's box of pixel centres (the culling test,
    here in FP64 from the projected splats: the maximum of the concave power over
    the box edges that face the mean), times the block's 32 lanes.  A lower bound
    of the kernels' per-lane work: a walk also passes the positions it culls, and
    a batch of 32 positions may run past the deepest n_contrib."""
    import torch
    T = step.params.tile
    bw, bh = T // 8, T // 4
    nb = bw * bh
    amin = step.params.alpha_min if alpha_min is None else alpha_min
    dev = step.device
    M = min(step.num_keys(), step.bins.capacity)
    if M == 0:
        return 0
    tile = step.bins.keys[:M] >> 32
    ent = step.bins.vals[:M].to(torch.int64)
    ranges = step.bins.ranges.to(torch.int64)
    pos = torch.arange(M, device=dev) - ranges[tile, 0]
    # per view: tiles across, first global tile, first pixel
    tx_v = [(int(c.width) + T - 1) // T for c in step.cams]
    ty_v = [(int(c.height) + T - 1) // T for c in step.cams]
    tbase = [0]
    pbase = [0]
    for c, a, b in zip(step.cams, tx_v, ty_v):
        tbase.append(tbase[-1] + a * b)
        pbase.append(pbase[-1] + int(c.width) * int(c.height))
    # deepest n_contrib of every block: [total_tiles, nb]
    nc = step.img.n_contrib.to(torch.int64)
    maxnc = torch.zeros(tbase[-1], nb, device=dev, dtype=torch.int64)
    for v, c in enumerate(step.cams):
        W, H = int(c.width), int(c.height)
        img = torch.zeros(ty_v[v] * T, tx_v[v] * T, device=dev, dtype=torch.int64)
        img[:H, :W] = nc[pbase[v]:pbase[v] + W * H].view(H, W)
        blk = img.view(ty_v[v], bh, 4, tx_v[v], bw, 8).amax(dim=(2, 5))          # [ty, bh, tx, bw]
        maxnc[tbase[v]:tbase[v + 1]] = blk.permute(0, 2, 1, 3).reshape(-1, nb)
    tb = torch.tensor(tbase[:-1], device=dev)
    txs = torch.tensor(tx_v, device=dev)
    v = torch.searchsorted(tb, tile, right=True) - 1
    lt = tile - tb[v]
    gx, gy = (lt % txs[v]).double() * T, (lt // txs[v]).double() * T
    xy = step.proj.xy[ent].double()
    co = step.proj.conic_o[ent].double()
    A, B, C, o = co[:, 0], co[:, 1], co[:, 2], co[:, 3]
    qa, qb, qc = -0.5 * A, -B, -0.5 * C                   # power = qa dx^2 + qb dx dy + qc dy^2
    L = torch.log(torch.clamp(0.99 * amin / o, min=1e-300))
    ox, oy = gx + 0.5 - xy[:, 0], gy + 0.5 - xy[:, 1]
    count = 0
    for b in range(nb):
        dx0 = ox + (b % bw) * 8
        dx1 = dx0 + 7.0
        dy0 = oy + (b // bw) * 4
        dy1 = dy0 + 3.0
        vx = torch.minimum(torch.clamp(dx0, min=0.0), dx1)
        vy = torch.minimum(torch.clamp(dy0, min=0.0), dy1)
        ty = torch.minimum(torch.maximum(-qb * vx / (2 * qc), dy0), dy1)
        tx = torch.minimum(torch.maximum(-qb * vy / (2 * qa), dx0), dx1)
        pv = qa * vx * vx + qb * vx * ty + qc * ty * ty
        ph = qa * tx * tx + qb * tx * vy + qc * vy * vy
        reach = (torch.maximum(pv, ph) >= L) & (o >= 0.99 * amin)
        count += int((reach & (pos < maxnc[tile, b])).sum().item())
    return 32 * count


def stage_rooflines(step, st, pairs, params, bwd_label=None, profiled=True):
    """Roofline of every stage of one iteration from its CUDA-event time in the
    instrumented graph replays: the rasterisers against the FP32 lane peak
    (operations, a multiply-add as one) and the FP32 FLOP peak (a multiply-add as
    two), the other stages against the measured HBM copy bandwidth."""
    peaks, peak_kind = _peaks()
    # the ncu figures belong to the 640x480 / 200k workload they were captured on
    prof = (lambda table, key: table.get(key)) if profiled else (lambda table, key: None)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    lane_peak = 152 * 128 * sm_mhz * 1e6 / 1e12          # T lane-ops/s
    flop_peak = 2.0 * lane_peak                          # T FLOP/s FP32
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {}
    if not st:
        return out
    fwd_st, bwd_st = raster_stages(step)
    few = step.total_tiles * (params.tile // 8) * (params.tile // 4) <= 256 * 152
    ring = params.splat_stages == 3 or (params.splat_stages == 0 and few)
    fl = str(step.fused_loss).lower()
    kern = {fwd_st: f"k_render_fwd<{params.tile}, {fl}, ring={ring}> ({3 if ring else 2} batches of 32 splats staged "
                    f"per warp)",
            bwd_st: f"k_render_bwd<{params.tile}, {bwd_ctas_per_sm(step, params.tile)}, {fl}> (+ its 2D-gradient "
                    f"zero-fill{' and block ordering' if few and step.fused_loss else ''})"}
    evald = evaluated_pairs(step)
    for stage, ops, flop in ((fwd_st, FWD_OPS_PER_PAIR, FWD_FLOP_PER_PAIR), (bwd_st, BWD_OPS_PER_PAIR,
                                                                            BWD_FLOP_PER_PAIR)):
        sec = st[stage] * 1e-3
        ach = pairs * ops / sec / 1e12
        ach_f = pairs * flop / sec / 1e12
        ach_e = evald * ops / sec / 1e12
        out[stage] = {"bound": "alu", "kernel": kern[stage], "achieved": ach, "peak": lane_peak,
                      "unit": "T FP32 lane-ops/s", "frac": ach / lane_peak,
                      "work": f"{pairs} visited (pixel, splat) pairs x {ops} FP32 ops (a multiply-add as one)",
                      "flop": {"achieved": ach_f, "peak": flop_peak, "unit": "TFLOP/s FP32", "frac": ach_f / flop_peak,
                               "work": f"{pairs} pairs x {flop} FLOPs (a multiply-add as two)"},
                      "evaluated_pairs": {
                          "pairs": evald, "achieved": ach_e, "frac": ach_e / lane_peak,
                          "work": f"{evald} evaluated (pixel, splat) pairs x {ops} FP32 ops",
                          "note": "the pairs the culling keeps: each 8x4 block's list positions before its deepest "
                                  "n_contrib whose splat can reach 0.99 alpha_min in the block, x 32 lanes, counted "
                                  "in FP64 from the projected splats; the visited count above (sum of n_contrib) "
                                  "includes the pairs the culling proves weightless and skips"},
                      "binding_pipe": prof(PROFILED_PIPE, (stage, params.tile, ring if stage == fwd_st else None,
                                                           params.block_masks)),
                      "traffic": prof(PROFILED_TRAFFIC, (stage, params.tile, ring if stage == fwd_st else None,
                                                         params.block_masks)),
                      "ms": st[stage],
                      "peak_basis": f"152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({peak_kind} sm_max_mhz)"}
    E = step.n * step.V
    M = step.num_keys()
    T = step.total_tiles
    tile_bits = max(1, (T - 1).bit_length())
    lsd_passes = -(-(31 + tile_bits) // 8)
    hbm_stages = {
        "gs_project": (step.n * PROJECT_BYTES_PER_GAUSSIAN + E * PROJECT_BYTES_PER_ENTRY,
                       f"{step.n} Gaussians x {PROJECT_BYTES_PER_GAUSSIAN} B + {E} entries x {PROJECT_BYTES_PER_ENTRY} B"),
        "gs_bin_sort": (E * BIN_BYTES_PER_ENTRY + M * BIN_BYTES_PER_KEY + T * BIN_BYTES_PER_TILE,
                        f"{E} entries x {BIN_BYTES_PER_ENTRY} B + {M} keys x {BIN_BYTES_PER_KEY} B + {T} tiles x "
                        f"{BIN_BYTES_PER_TILE} B"),
        "gs_project_bwd": (step.n * (PROJECT_BWD_BYTES_PER_GAUSSIAN + step.V * PROJECT_BWD_BYTES_PER_ENTRY),
                           f"{step.n} Gaussians x ({PROJECT_BWD_BYTES_PER_GAUSSIAN} + {step.V} views x "
                           f"{PROJECT_BWD_BYTES_PER_ENTRY}) B"),
        "gs_adam_step": (step.n * ADAM_ELEMENTS_PER_GAUSSIAN * ADAM_BYTES_PER_ELEMENT,
                         f"{step.n * ADAM_ELEMENTS_PER_GAUSSIAN} elements x {ADAM_BYTES_PER_ELEMENT} B"),
    }
    for stage, (nbytes, work) in hbm_stages.items():
        if stage not in st:
            continue
        gbs = nbytes / (st[stage] * 1e-3) / 1e9
        out[stage] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                      "work": work, "ms": st[stage],
                      "traffic": prof(PROFILED_TRAFFIC, (stage, params.tile, None, params.block_masks)),
                      "peak_basis": f"hbm_gbs ({peak_kind})"}
    if "gs_bin_sort" in out:
        lsd = M * (12 + 24 * lsd_passes)
        out["gs_bin_sort"]["radix_reference"] = {
            "bytes": lsd, "achieved": lsd / (st["gs_bin_sort"] * 1e-3) / 1e9,
            "frac": lsd / (st["gs_bin_sort"] * 1e-3) / 1e9 / hbm,
            "work": f"{M} keys x (12 + 24 x {lsd_passes} passes) B: an 8-bit LSD radix sort's traffic"}
        if L2_PEAK.get("gbs"):
            b = out["gs_bin_sort"]
            alg = b["achieved"] * b["ms"] * 1e-3 * 1e9             # algorithmic bytes
            l2 = {"achieved": b["achieved"], "peak": L2_PEAK["gbs"], "unit": "GB/s",
                  "frac": b["achieved"] / L2_PEAK["gbs"], "work": b["work"],
                  "peak_basis": "L2 read bandwidth measured in this run (" + L2_PEAK["method"] + ")",
                  "peak_per_size": L2_PEAK["per_size"]}
            t = prof(PROFILED_L2, ("gs_bin_sort", params.tile, params.block_masks))
            if t is not None:
                l2["traffic"] = t
                l2["traffic_frac"] = t / (b["ms"] * 1e-3) / 1e9 / L2_PEAK["gbs"]
            l2["algorithmic_bytes"] = alg
            b["l2"] = l2
    return out


def cpu_baseline(params, mp, reps=3):
    """The FP64 oracle, as it stands, on the host cores: the median of `reps`
    full mapping iterations (render, loss, gradients and the Adam update) on
    one thread and on every processor, for each workload of _oracle_workloads.
    The headline value is the 640x480 / 200k workload on all processors."""
    import oracle
    procs = oracle.num_procs()
    rows = {}
    for name, g, gt, cams, sh in _oracle_workloads():
        fn = _oracle_iteration_fn(g, gt, cams, params, mp, sh)
        row = {}
        for threads in (1, procs):
            prev = oracle.set_threads(threads)
            try:
                t = statistics.median(fn() for _ in range(reps))
            finally:
                oracle.set_threads(prev)
            row[f"{threads}_thread{'s' if threads > 1 else ''}_s"] = round(t, 4)
        rows[name] = row
    head = rows["640x480 / 200k Gaussians"][f"{procs}_thread{'s' if procs > 1 else ''}_s"]
    return {"value": 1.0 / head, "unit": "iters/s", "cores": procs, "kind": "oracle",
            "sample": f"median of {reps} full FP64 mapping iterations (forward, Eq. 6 loss, gradients, Adam) of "
                      f"the benchmark's 640x480 / 200k-Gaussian workload on {procs} host threads (OpenMP)",
            "single_thread_value": 1.0 / rows["640x480 / 200k Gaussians"]["1_thread_s"],
            "seconds_per_iteration": rows}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores (all processors,
    OpenMP).  Each step is one full mapping iteration of the benchmark's
    workload (640x480 view, 200k Gaussians: project, composite, Eq. 6 loss,
    backward to every parameter and the pose, Adam), from the same starting
    map and Adam state every step, as the GPU arm's steps are."""
    if rank != 0:
        return 0
    import oracle
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import synth
    from paper_2512_02293_gb300.mapping import MapParams
    procs = oracle.num_procs()
    oracle.set_threads(procs)
    g, gt, cam = synth.cfg2_problem()
    mp = MapParams()
    one = _oracle_iteration_fn(g, gt, [cam], G.RenderParams(tile=16), mp, 0)
    for _ in range(args.warmup):
        one()
    total = sum(one() for _ in range(args.steps))
    value = args.steps / total
    sample = (f"each step one full FP64 mapping iteration of the 640x480 / 200k-Gaussian workload (projection, "
              f"compositing, Eq. 6 loss, backward incl. pose, Adam) on {procs} host threads (OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def whole_job_rate(local_ms: float, steps: int, world: int, dist=None, device=None):
    """Replicas: every rank ran `steps` iterations; the job's time is the
    slowest rank's (max over ranks), its rate = all ranks' iterations / time."""
    total_ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1000.0), total_ms


def window_run(device, args, flush, plain_rate, dist=None, world=1):
    """The batched mapping window: 8 keyframes of uneven size (4x 640x480,
    2x 752x480, 2x 1280x1024) on a 5 m trajectory through a 500k-Gaussian room,
    every stage one launch over all views (persistent rasterisers), the whole
    iteration one CUDA graph, tile size autotuned."""
    from paper_2512_02293_gb300 import synth
    g, gt, cams = synth.cfg3_problem()
    params, mp, step, tc, td = build_step(device, g, gt, cams, args.tiles, args.stages, args.masks)
    steps = max(10, args.steps // 4)
    times, st, pairs, _ = timed_run(step, steps, args.warmup, flush, dist)
    rate, total_ms = whole_job_rate(sum(times), steps, world, dist, device)
    views = len(cams)
    roof = stage_rooflines(step, st, pairs, params, profiled=False) if st else None
    return {"workload": "batched window: 8 keyframes (4x 640x480, 2x 752x480, 2x 1280x1024), 500k Gaussians",
            "roofline": roof,
            "value": rate, "unit": "iters/s", "steps": steps, "ms_per_step": total_ms / steps,
            "views_per_s": rate * views, "views_per_s_vs_plain_iters_per_s": rate * views / plain_rate,
            "tile": params.tile, "splat_stages": params.splat_stages, "block_masks": params.block_masks,
            "cull_tiles": params.cull_tiles,
            "autotune_ms": {str(k): round(v, 4) for k, v in step.tune.items()},
            "pixels_per_iter": step.total_pixels, "pairs_per_iter": pairs, "keys_per_iter": step.num_keys(),
            "gpix_splats_per_s": pairs / (st[raster_stages(step)[0]] * 1e-3) / 1e9 if st else None,
            "stages_ms": st, "graph": True, "persistent_raster": True}


MLP_FWD_FLOP = 2 * (196 * 128 + 128 * 128 + 128 * 8)            # per sample, the network's own MACs x 2
MLP_BWD_FLOP = 2 * (128 * 128 + 128 * 128 + 196 * 128 + 2 * 8 * 128)  # dH1, dW2, dW1, dW3, dH2
MLP_FWD_BYTES = 208 * 2 + 8 * 4                                   # BF16 input row + FP32 output


def learned_init_run(device, args):
    """The learned initialiser: training pairs from 50 seeded rooms (the plain
    mapper, 100 iterations from the heuristic insertion of ~49k Gaussians per
    640x480 keyframe), tensor-core training, inference / backward throughput,
    and iterations to the heuristic's PSNR at 100 mapper iterations on 5
    held-out rooms."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import learned_init as L
    cfg = L.InitConfig()
    t0 = time.perf_counter()
    Xs, Ts = [], []
    for r in range(args.li_rooms):
        X, T = L.training_pairs(100 + r, cfg, device)
        Xs.append(X); Ts.append(T)
    X = torch.cat(Xs); T = torch.cat(Ts)
    del Xs, Ts
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).to(device)
    X = X.index_select(0, perm).contiguous(); T = T.index_select(0, perm).contiguous()
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n = X.shape[0]
    net = L.LearnedInit(0, device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    losses = net.train(X, T, epochs=args.li_epochs, batch=8192, lr=1e-3)
    ev[1].record(); torch.cuda.synchronize()
    train_ms = ev[0].elapsed_time(ev[1])
    # kernel throughput over the whole dataset (inputs larger than L2)
    Y = torch.empty(n, 8, device=device)
    Z1 = torch.empty(n, 128, device=device, dtype=torch.bfloat16); Z2 = torch.empty_like(Z1)
    dY = torch.empty(n, 8, device=device); loss = torch.zeros(1, device=device)
    for _ in range(2):
        G.gs_mlp_fwd(net.packed, X, Y=Y)
    ms_f = []
    for _ in range(5):
        ev[0].record(); G.gs_mlp_fwd(net.packed, X, Y=Y); ev[1].record(); torch.cuda.synchronize()
        ms_f.append(ev[0].elapsed_time(ev[1]))
    G.gs_mlp_fwd(net.packed, X, Z1=Z1, Z2=Z2, T=T, dY=dY, loss=loss, loss_scale=1.0 / (8 * n))
    ms_b = []
    for _ in range(5):
        ev[0].record(); G.gs_mlp_bwd(net.packed, X, Z1, Z2, dY, net.grads); ev[1].record(); torch.cuda.synchronize()
        ms_b.append(ev[0].elapsed_time(ev[1]))
    fwd_ms, bwd_ms = statistics.median(ms_f), statistics.median(ms_b)
    peaks, kind = _peaks()
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fwd_tf = n * MLP_FWD_FLOP / (fwd_ms * 1e-3) / 1e12
    fwd_gbs = n * MLP_FWD_BYTES / (fwd_ms * 1e-3) / 1e9
    bwd_tf = n * MLP_BWD_FLOP / (bwd_ms * 1e-3) / 1e12
    rooms = []
    for seed in range(900, 900 + args.li_eval_rooms):
        kf = L.Keyframe(seed, cfg, device)
        heur, dh = L.mapping_curve(kf, None, 150)
        lrn, dl = L.mapping_curve(kf, net.predict(kf.X), 150)
        rooms.append({"seed": seed, "iters_to_heuristic_psnr100": L.iterations_to_reach(lrn, float(heur[99])),
                      "psnr_heuristic": [round(float(heur[i]), 2) for i in (0, 9, 49, 99, 149)],
                      "psnr_learned": [round(float(lrn[i]), 2) for i in (0, 9, 49, 99, 149)],
                      "depth_l1_m_at150": [round(dh, 4), round(dl, 4)]})
    its = [r["iters_to_heuristic_psnr100"] for r in rooms]
    return {"workload": f"{args.li_rooms} rooms x ~49k inserted Gaussians per 640x480 keyframe (3-view window), "
                        f"{n} pairs; MLP 196-128-128-8 GELU, BF16 weights/activations, FP32 accumulate",
            "pairs": n, "pair_generation_s": round(gen_s, 2), "epochs": args.li_epochs,
            "train_ms": round(train_ms, 1), "train_pairs_per_s": args.li_epochs * n / (train_ms * 1e-3),
            "loss_first_last": [round(losses[0], 4), round(losses[-1], 4)],
            "mlp_fwd": {"ms": round(fwd_ms, 4), "samples_per_s": n / (fwd_ms * 1e-3),
                        "roofline": {"bound": "hbm", "achieved": fwd_gbs, "peak": hbm_peak, "unit": "GB/s",
                                     "frac": fwd_gbs / hbm_peak,
                                     "tensor_tflops": fwd_tf, "tensor_frac": fwd_tf / bf16_peak,
                                     "work": f"{MLP_FWD_BYTES} B and {MLP_FWD_FLOP} FLOP per sample",
                                     "peak_basis": f"{kind} hbm_gbs / bf16_tflops"}},
            "mlp_bwd": {"ms": round(bwd_ms, 4), "samples_per_s": n / (bwd_ms * 1e-3), "tensor_tflops": bwd_tf,
                        "tensor_frac": bwd_tf / bf16_peak},
            "eval_rooms": rooms,
            "iters_to_heuristic_psnr100_mean": float(np.mean([i if i is not None else 151 for i in its]))}


def differentiation_run(device, steps=10, warmup=3):
    """The differentiation workload through the autograd binding: 16 keyframes
    at 1280x1024 over 1M Gaussians with degree-3 SH colour; forward render,
    an L1 colour + depth loss against the perturbed map's images, and the
    backward to every parameter and each keyframe's pose tangent.  Wall clock
    per iteration issued eagerly, and the device time per replay of the same
    iteration captured once in a CUDA graph (the binding synchronises nowhere
    in forward or backward; the key buffers' overflow flag is checked after)."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import synth
    from paper_2512_02293_gb300.autograd import Rasterizer, render
    g, gt, cams = synth.cfg4_problem()
    params = G.RenderParams(sh_degree=3, tile=16)
    rast = Rasterizer(cams, g.n, params)
    leaf = lambda m: [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device).requires_grad_(True)
                      for a in m.arrays()]
    with torch.no_grad():
        tcol, tdep = render(*leaf(gt), torch.zeros(len(cams), 6, device=device), rast)
        tcol, tdep = tcol.clone(), tdep.clone()
    leaves = leaf(g)
    xi = torch.zeros(len(cams), 6, device=device, requires_grad=True)

    def one():
        col, dep = render(*leaves, xi, rast)
        loss = 0.9 * (col - tcol).abs().mean() + 0.1 * (dep - tdep).abs().mean()
        loss.backward()
        return loss

    for _ in range(warmup):
        one()
    if rast.ensure_capacity():
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1000.0 / steps
    # the same iteration captured once and replayed
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            one()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        one()
    cs = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ts = []
    for _ in range(steps):
        ev[0].record(cs); graph.replay(); ev[1].record(cs)
        torch.cuda.synchronize()
        ts.append(ev[0].elapsed_time(ev[1]))
    status = rast.check()
    ts.sort()
    gms = ts[len(ts) // 2]
    nc = rast.img.n_contrib.to(torch.int64).sum().item()
    return {"workload": "16 keyframes 1280x1024, 1M Gaussians, degree-3 SH (48 coefficients), gradients to all "
                        "parameters and 16 pose tangents, via torch.autograd", "ms_per_iter": round(ms, 3),
            "iters_per_s": 1000.0 / ms, "views_per_s": 16 * 1000.0 / ms,
            "graph_ms_per_iter": round(gms, 3), "graph_iters_per_s": 1000.0 / gms, "status_after": status,
            "pixels_per_iter": rast.total_pixels, "pairs_per_iter": int(nc),
            "gpix_splats_per_s_fwd_bwd": int(nc) / (gms * 1e-3) / 1e9,
            "keys_per_iter": int(rast.bins.num_keys.item()) & 0xFFFFFFFF,
            "timing": "ms_per_iter: wall clock of eagerly issued iterations (loss terms are torch ops); "
                      "graph_ms_per_iter: CUDA events around replays of one captured iteration (median)"}


def tracking_run(device, seeds=(0, 1, 2)):
    """Pose refinement through the re-rendering loss.  (1) The 640x480 / 200k
    view: the keyframe pose perturbed by up to 3 cm and ~1.1 deg, recovered by
    250 gradient steps on the pose tangent with the map fixed (wall clock; each
    step reads the 6 gradient components back).  (2) The 8 keyframes of the 5 m
    path through the 500k-Gaussian room, tracked in sequence, each from the
    previous estimate's error carried along the path plus fresh noise: the
    absolute trajectory error before and after."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import synth
    from paper_2512_02293_gb300.autograd import se3_left_update
    from paper_2512_02293_gb300.mapping import MapParams, MappingStep
    from paper_2512_02293_gb300.tracking import PoseTracker, TrajectoryTracker, pose_error
    g, _, cam = synth.cfg2_problem()
    gd = G.Gaussians.from_numpy(g, device)
    P = cam.n_pixels
    r = MappingStep(gd, [cam], torch.zeros(3 * P, device=device), torch.zeros(P, device=device),
                    G.RenderParams(tile=16), MapParams())
    r.render()
    tc, td = r.img.color.clone(), r.img.depth.clone()
    out = []
    total_ms, total_it = 0.0, 0
    for seed in seeds:
        rng = np.random.default_rng(seed)
        start = se3_left_update(cam, np.concatenate([rng.uniform(-1, 1, 3) * 0.03, rng.uniform(-1, 1, 3) * 0.02]))
        tr = PoseTracker(gd, start, tc, td, G.RenderParams(tile=16))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr.run()
        total_ms += (time.perf_counter() - t0) * 1000.0
        total_it += tr.iters
        e0, e1 = pose_error(start, cam), pose_error(tr.cam, cam)
        out.append({"seed": seed, "start_err_m_rad": [round(e0[0], 5), round(e0[1], 5)],
                    "final_err_m_rad": [round(e1[0], 6), round(e1[1], 6)]})
    g3, _, cams = synth.cfg3_problem()
    gd3 = G.Gaussians.from_numpy(g3, device)
    targets = []
    for c in cams:
        P3 = c.n_pixels
        r3 = MappingStep(gd3, [c], torch.zeros(3 * P3, device=device), torch.zeros(P3, device=device),
                         G.RenderParams(tile=16), MapParams())
        r3.render()
        targets.append((r3.img.color.clone(), r3.img.depth.clone()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    traj = TrajectoryTracker(gd3, cams, targets, G.RenderParams(tile=16), seed=5).run()
    traj_s = time.perf_counter() - t0
    return {"workload": "640x480 keyframe, 200k-Gaussian map fixed, pose perturbed by <= 3 cm / ~1.1 deg",
            "iterations": tr.iters, "ms_per_iteration": round(total_ms / total_it, 4), "runs": out,
            "trajectory": {"workload": "8 keyframes (4x 640x480, 2x 752x480, 2x 1280x1024) along a 5 m path, "
                                       "500k-Gaussian map fixed; each keyframe from the previous estimate's error "
                                       "carried along the path plus <= 3 cm / ~1.1 deg of noise, 250 steps each",
                           "start_ate_rmse_m": round(traj["start_ate_rmse_m"], 5),
                           "ate_rmse_m": round(traj["ate_rmse_m"], 6),
                           "start_rot_rmse_rad": round(traj["start_rot_rmse_rad"], 5),
                           "rot_rmse_rad": round(traj["rot_rmse_rad"], 6), "wall_s": round(traj_s, 2)}}


def ba_run(device, K=16, h=60, w=80, window=3, steps=10):
    """One Levenberg-Marquardt step of the dense visual bundle adjustment
    (Eq. 2 / Eq. 4) on a 16-keyframe window at the tracker's 1/8 resolution of
    640x480 (60 x 80 inverse depths per keyframe), every pair of keyframes at
    most 3 apart as an edge; device time of gs_ba_step by graph replay.  Also
    the same window with the inertial factor of Eq. 3 between consecutive
    keyframes and one keyframe fixed (225 pose, velocity and bias unknowns)."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import synth
    R, t, disp, intr, edges, wts, vel, bias, bh, g, imu = synth.vi_scene(21, K=K, h=h, w=w, f=70.0, window=window)
    rng = np.random.default_rng(22)
    targets = rng.normal(0.0, 0.5, (len(edges), h, w, 2)) + np.stack(np.meshgrid(np.arange(w) + 0.5,
                                                                             np.arange(h) + 0.5), -1)
    win = G.BAWindow(R, t, disp, intr, edges, targets, wts, 2, device)
    m = graph_time_ms(lambda: G.gs_ba_step(win, 1e-3, 1e-3), steps=steps)
    win_vi = G.BAWindow(R, t, disp, intr, edges, targets, wts, 1, device, imu=imu, vel=vel, bias=bias, bias_hat=bh,
                        gravity=g)
    m_vi = graph_time_ms(lambda: G.gs_ba_step(win_vi, 1e-3, 1e-3), steps=steps)
    n_res = len(edges) * h * w
    # algorithmic bytes: every residual's target and weight pair read once, every
    # inverse depth read and written once (the poses are negligible)
    nbytes = n_res * BA_BYTES_PER_RESIDUAL + K * h * w * BA_BYTES_PER_DEPTH
    peaks, kind = _peaks()
    gbs = nbytes / (m * 1e-3) / 1e9
    return {"workload": f"{K} keyframes, {h}x{w} inverse depths each, {len(edges)} edges (|i - j| <= {window}), "
                        f"{n_res} residual pixels, 2 poses fixed", "ms_per_step": round(m, 4),
            "residual_pixels_per_s": n_res / (m * 1e-3), "status": int(win.status[0].item()),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                         "frac": gbs / peaks.get("hbm_gbs", 6800.0),
                         "work": f"{BA_BYTES_PER_RESIDUAL} B per residual pixel + {BA_BYTES_PER_DEPTH} B per "
                                 f"inverse depth ({nbytes} B per step)",
                         "peak_basis": f"{kind} hbm_gbs",
                         "note": "four dependent launches and a one-CTA solve of the 84 x 84 reduced system: "
                                 "the step is latency bound at this size"},
            "visual_inertial": {"workload": f"the same window with the inertial factor between the {K - 1} "
                                            f"consecutive pairs, 1 keyframe fixed (225 x 225 reduced system)",
                                "ms_per_step": round(m_vi, 4), "status": int(win_vi.status[0].item())}}


def mlp_kernels_run(device, n=2_457_600, steps=5):
    """The initialiser network's kernels alone on a synthetic batch of the
    training set's size (seeded weights, inputs U(-1, 1) in BF16, targets N(0, 1)):
    inference forward, training forward (Z1, Z2, loss and dY stored) and backward."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import synth
    gen = torch.Generator(device=device).manual_seed(5)
    X = (torch.rand(n, G.MLP_IN_STRIDE, device=device, generator=gen) * 2 - 1).to(torch.bfloat16)
    T = torch.randn(n, G.MLP_OUT, device=device, generator=gen)
    params = {k: torch.from_numpy(v).to(device) for k, v in synth.mlp_params(0).items()}
    packed = G.MlpPacked(device)
    G.gs_mlp_pack(params, packed)
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    Y = torch.empty(n, G.MLP_OUT, device=device)
    Z1 = torch.empty(n, 128, device=device, dtype=torch.bfloat16); Z2 = torch.empty_like(Z1)
    dY = torch.empty(n, G.MLP_OUT, device=device); loss = torch.zeros(1, device=device)
    calls = {"fwd": lambda: G.gs_mlp_fwd(packed, X, Y=Y),
             "fwd_train": lambda: G.gs_mlp_fwd(packed, X, Z1=Z1, Z2=Z2, T=T, dY=dY, loss=loss,
                                               loss_scale=1.0 / (8 * n)),
             "bwd": lambda: G.gs_mlp_bwd(packed, X, Z1, Z2, dY, grads)}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {}
    for name, fn in calls.items():
        for _ in range(2):
            fn()
        ms = []
        for _ in range(steps):
            ev[0].record(); fn(); ev[1].record(); torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        out[name] = round(statistics.median(ms), 4)
    peaks, kind = _peaks()
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    return {"workload": f"{n} synthetic samples, MLP 196-128-128-8 GELU, BF16 operands, FP32 accumulation",
            "ms": out,
            "fwd_tensor_frac": n * MLP_FWD_FLOP / (out["fwd"] * 1e-3) / 1e12 / bf16_peak,
            "bwd_tensor_frac": n * MLP_BWD_FLOP / (out["bwd"] * 1e-3) / 1e12 / bf16_peak,
            "peak_basis": f"{kind} bf16_tflops"}


def refinement_run(device, views=16, iters=400):
    """Final colour refinement (Sec. 3.3): 16 keyframes at 640x480 along a 5 m
    path through a 200k-Gaussian room, one random keyframe per iteration, one
    captured graph per keyframe; CUDA-event time of the iterations (replayed
    back to back) and the mean PSNR over all keyframes before and after."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import synth
    from paper_2512_02293_gb300.mapping import MappingStep
    from paper_2512_02293_gb300.refinement import ColourRefiner
    g, gt, cams = synth.refinement_problem(0, views=views)
    P = cams[0].n_pixels
    tc, td = [], []
    for c in cams:
        r = MappingStep(G.Gaussians.from_numpy(gt, device), [c], torch.zeros(3 * P, device=device),
                        torch.zeros(P, device=device), G.RenderParams(tile=16))
        r.render()
        tc.append(r.img.color.clone()); td.append(r.img.depth.clone())
        del r
    ref = ColourRefiner(G.Gaussians.from_numpy(g, device), cams, tc, td, G.RenderParams(tile=16), seed=0)
    before = ref.mean_psnr()
    ref.run(20)                                     # warm-up
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    ref.run(iters, check_every=iters + 1)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    grown = ref.check()
    after = ref.mean_psnr()
    return {"workload": f"{views} keyframes 640x480, 200k-Gaussian room, one random keyframe per iteration, "
                        "one CUDA graph per keyframe",
            "iterations": iters, "ms_per_iteration": round(ms / iters, 4), "iterations_per_s": iters / (ms * 1e-3),
            "timing": "CUDA events around the whole loop, iterations back to back as the refinement runs them "
                      "(no L2 flush between them: the 11 MB map stays resident)",
            "mean_psnr_db_before_after": [round(before, 2), round(after, 2)],
            "draws_per_keyframe": ref.draws.tolist(), "buffers_regrown": bool(grown)}


def graph_time_ms(fn, reps=10, steps=10):
    """Median device time of one call of fn: the call is captured reps times into
    a CUDA graph and the replays are timed with CUDA events, so that the host's
    argument marshalling of a short C-ABI call is not counted."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        for _ in range(reps):
            fn()
    graph.replay()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ms = []
    for _ in range(steps):
        ev[0].record(); graph.replay(); ev[1].record()
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]) / reps)
    return statistics.median(ms)


def insertion_run(device, steps=20):
    """Keyframe insertion (Sec. 3.3): the 7 x 7 RGB-D patches of ~49k pixels of a
    640x480 keyframe (2.5 px grid), the initialiser network's forward, and the
    learned and heuristic insertion of the new Gaussians; CUDA-event times of
    each call, inputs resident on the device."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    from paper_2512_02293_gb300 import learned_init as LI
    cfg = LI.InitConfig()
    kf = LI.Keyframe(900, cfg, device)
    net = LI.LearnedInit(0, device)
    n = kf.n
    Y = torch.empty(n, G.MLP_OUT, device=device)
    g = kf.new_map()
    cam = kf.cams[0]
    calls = {
        "gs_extract_patches": lambda: G.gs_extract_patches(kf.color0, kf.depth0, cam, kf.uv, kf.X),
        "gs_mlp_fwd": lambda: G.gs_mlp_fwd(net.packed, kf.X, Y=Y, status=net.status),
        "gs_insert_gaussians (learned)": lambda: G.gs_insert_gaussians(kf.color0, kf.depth0, cam, kf.uv, cfg.stride,
                                                                       g, 0, Y=Y),
        "gs_insert_gaussians (heuristic)": lambda: G.gs_insert_gaussians(kf.color0, kf.depth0, cam, kf.uv,
                                                                         cfg.stride, g, 0),
    }
    # each call is tens of microseconds of GPU work, less than the host's ctypes
    # marshalling: timed by graph replay
    out = {name: round(graph_time_ms(fn, steps=steps), 4) for name, fn in calls.items()}
    peaks, kind = _peaks()
    image_bytes = cam.n_pixels * 16                       # RGB + depth, read once
    ext_bytes = n * INSERT_PATCH_BYTES + image_bytes
    ins_bytes = n * INSERT_GAUSSIAN_BYTES
    ms_ext, ms_ins = out["gs_extract_patches"], out["gs_insert_gaussians (learned)"]
    gbs = (ext_bytes + ins_bytes) / ((ms_ext + ms_ins) * 1e-3) / 1e9
    return {"workload": f"{n} samples of one 640x480 keyframe (2.5 px grid), room of {cfg.room_gaussians} Gaussians",
            "ms": out, "samples_per_s": n / ((ms_ext + out["gs_mlp_fwd"] + ms_ins) * 1e-3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                         "frac": gbs / peaks.get("hbm_gbs", 6800.0),
                         "kernels": "k_extract_patches + k_insert (learned)",
                         "work": f"{INSERT_PATCH_BYTES} B per patch row + the image once; "
                                 f"{INSERT_GAUSSIAN_BYTES} B per inserted Gaussian",
                         "peak_basis": f"{kind} hbm_gbs"}}


INSERT_PATCH_BYTES = 8 + 2 * 208                # uv read, BF16 row written
INSERT_GAUSSIAN_BYTES = 8 + 16 + 32 + 4 * (3 + 4 + 3 + 1 + 3)   # uv, pixel RGB-D, Y read; the Gaussian written
BA_BYTES_PER_RESIDUAL = 8 + 8                # target u* and weight pair
BA_BYTES_PER_DEPTH = 4 + 4                   # inverse depth read and written
LOOP_CLOSURE_BYTES = 12 + 16 + 12 + 4 + 12 + 16 + 12   # read mean, quat, log-scale, anchor; write the first three


def loop_closure_run(device, n=4_000_000, K=1000):
    """The loop-closure Gaussian update (Eq. 7, Eq. 8) over a 4M-Gaussian map
    anchored to 1000 keyframes, 4000 consecutive Gaussians per keyframe as
    insertion lays them out (336 MB moved, more than L2), device time by graph
    replay; the roofline is HBM."""
    import torch
    from paper_2512_02293_gb300 import gs as G
    rng = np.random.default_rng(11)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
    g = G.Gaussians(t(rng.uniform(-3, 3, (n, 3))), t(rng.standard_normal((n, 4))), t(rng.normal(-4, 0.3, (n, 3))),
                    t(rng.standard_normal(n)), t(rng.uniform(0, 1, (n, 3))))
    # insertion appends each keyframe's Gaussians as one run, so anchors are sorted
    anchor = torch.from_numpy((np.arange(n, dtype=np.int64) * K // n).astype(np.int32)).to(device)
    from scipy.spatial.transform import Rotation
    pose = lambda seed: t(np.concatenate([Rotation.random(K, random_state=seed).as_matrix().reshape(K, 9),
                                          rng.uniform(-3, 3, (K, 3))], 1))
    pb, pa = pose(1), pose(2)
    ds = t(rng.uniform(0.9, 1.1, K))
    m = graph_time_ms(lambda: G.gs_loop_closure_update(g, anchor, pb, pa, ds))
    peaks, kind = _peaks()
    gbs = n * LOOP_CLOSURE_BYTES / (m * 1e-3) / 1e9
    return {"workload": f"{n} Gaussians anchored to {K} keyframes ({n // K} consecutive per keyframe)",
            "ms": round(m, 4),
            "gaussians_per_s": n / (m * 1e-3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                         "frac": gbs / peaks.get("hbm_gbs", 6800.0),
                         "work": f"{LOOP_CLOSURE_BYTES} B per Gaussian", "peak_basis": f"{kind} hbm_gbs"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-window", action="store_true")
    ap.add_argument("--no-learned-init", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the loop-closure, pose-refinement and bundle-adjustment lines")
    ap.add_argument("--li-rooms", type=int, default=50)
    ap.add_argument("--li-epochs", type=int, default=40)
    ap.add_argument("--li-eval-rooms", type=int, default=5)
    ap.add_argument("--tile", type=int, choices=[8, 16, 32], default=None,
                    help="fix the tile size instead of autotuning over {8, 16, 32}")
    ap.add_argument("--splat-stages", type=int, choices=[2, 3], default=None,
                    help="fix the forward rasteriser's splat staging instead of autotuning over {2, 3}")
    ap.add_argument("--block-masks", type=int, choices=[0, 1], default=None,
                    help="fix the binning's pixel-block masks (1) or the rasterisers' own test (0) instead of "
                         "autotuning")
    ap.add_argument("--only", choices=["loop_closure", "pose_refinement", "bundle_adjustment", "keyframe_insertion",
                                       "mlp_kernels", "final_colour_refinement"],
                    default=None, help="run one extra section alone and print its line (for profiling runs)")
    ap.add_argument("--mlp-samples", type=int, default=2_457_600, help="batch of the mlp_kernels section")
    args = ap.parse_args()
    args.tiles = (args.tile,) if args.tile else (8, 16, 32)
    args.stages = (args.splat_stages,) if args.splat_stages else (2, 3)
    args.masks = (args.block_masks,) if args.block_masks is not None else (1, 0)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    args.warmup = max(args.warmup, 3)

    import torch
    from paper_2512_02293_gb300 import build as B
    from paper_2512_02293_gb300 import gs as G
    B.build()
    G.load_library()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    if args.only is not None:
        runs = {"loop_closure": loop_closure_run, "pose_refinement": tracking_run,
                "bundle_adjustment": ba_run, "keyframe_insertion": insertion_run,
                "final_colour_refinement": refinement_run,
                "mlp_kernels": lambda d: mlp_kernels_run(d, n=args.mlp_samples)}
        print(json.dumps({"section": args.only, args.only: runs[args.only](device)}), flush=True)
        return 0

    from paper_2512_02293_gb300 import synth
    g, gt, cam = synth.cfg2_problem()
    params, mp, step, tc, td = build_step(device, g, gt, [cam], args.tiles, args.stages, args.masks)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, device=device, dtype=torch.float32)
    flush = lambda: flush_buf.fill_(1.0)
    times, st, pairs, clocks = timed_run(step, args.steps, args.warmup, flush, dist, local)
    value, total_ms = whole_job_rate(sum(times), args.steps, world, dist, device)

    # end to end through the C ABI with host buffers: H2D of the target image and
    # depth from pinned memory each step, D2H of the loss
    from paper_2512_02293_gb300.mapping import MappingStep
    e2e_step = MappingStep(step.g, step.cams, torch.empty_like(tc), torch.empty_like(td), params, mp,
                           key_capacity=step.bins.capacity)
    h_tc = tc.cpu().pin_memory(); h_td = td.cpu().pin_memory()
    h_loss = torch.empty(e2e_step.loss_terms.shape, dtype=torch.float32).pin_memory()
    h_iso = torch.empty(1, dtype=torch.float32).pin_memory()
    e2e_pristine = [t.clone() for t in e2e_step.g.tensors()]

    def e2e_restore():
        # the same map and Adam state before every step (identical work per step, as in the timed run)
        for t, p0 in zip(e2e_step.g.tensors(), e2e_pristine):
            t.copy_(p0)
        for t in e2e_step.m + e2e_step.v:
            t.zero_()
        e2e_step.d_step.zero_()

    def e2e_loop(io_in_graph=False):
        def one():
            if io_in_graph:
                e2e_step.step()                      # the graph holds the copies
            else:
                e2e_step.target_color.copy_(h_tc, non_blocking=True)
                e2e_step.target_depth.copy_(h_td, non_blocking=True)
                e2e_step.step()
                h_loss.copy_(e2e_step.loss_terms, non_blocking=True)
                h_iso.copy_(e2e_step.iso, non_blocking=True)
        for _ in range(args.warmup):
            one()
        total = 0.0
        for _ in range(args.steps):
            e2e_restore()                            # outside the timed span, like the L2 flush
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            one()
            torch.cuda.current_stream().synchronize()
            total += time.perf_counter() - t0
        return total

    # eager: the C-ABI calls issued from Python every step
    eager_rate, _ = whole_job_rate(e2e_loop() * 1000.0, args.steps, world, dist, device)
    # captured: MappingStep.capture() once, then every step() replays the graph,
    # the per-step host copies (targets in, loss out) included in it as memcpy nodes
    e2e_step.capture(warmup=1, host_io=(h_tc, h_td, h_loss, h_iso))
    e2e_rate, _ = whole_job_rate(e2e_loop(io_in_graph=True) * 1000.0, args.steps, world, dist, device)
    e2e = {"value": e2e_rate, "unit": "iters/s",
           "h2d_bytes_per_step": int(h_tc.numel() * 4 + h_td.numel() * 4),
           "d2h_bytes_per_step": int(h_loss.numel() * 4 + h_iso.numel() * 4),
           "eager_value": eager_rate,
           "note": "MappingStep API, wall clock per step (map and Adam state restored and L2 flushed between "
                   "steps, outside the timed span): "
                   "pinned-host target image and depth copied in, the step, the loss terms read back, stream "
                   "synchronised; value with the step captured once together with its host copies "
                   "(MappingStep.capture(host_io=...): memcpy nodes of the same graph) and replayed, "
                   "eager_value with the two copies in, the C-ABI calls and the two copies out issued "
                   "each step"}

    measure_l2_peak(device)               # after the timed region: the L2 roofline's denominator
    stages_roof = stage_rooflines(step, st, pairs, params)
    roofline = None
    if st:
        dominant = max(st, key=st.get)
        roofline = dict(stages_roof[dominant])
        roofline["dominant_stage"] = dominant
        fwd_st, bwd_st = raster_stages(step)
        for tag, stg in (("fwd", fwd_st), ("bwd", bwd_st)):     # both rasterisers, each with its own work and time
            roofline[tag] = dict(stages_roof[stg], stage=stg)
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "views": 1, "gaussians": g.n, "resolution": "640x480",
                       "tile": params.tile, "splat_stages": params.splat_stages,
                       "block_masks": params.block_masks, "cull_tiles": params.cull_tiles,
                       "autotune_ms": {str(k): round(v, 4) for k, v in step.tune.items()},
                       "lambdas": [mp.lambda_c, mp.lambda_d, mp.lambda_iso], "graph": True,
                       "l2": "flushed between timed iterations (256 MiB write, outside the step events)",
                       "per_step_state": "map and Adam state restored before every timed step (identical work per step)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "gpix_splats_per_s": pairs / (st[raster_stages(step)[0]] * 1e-3) / 1e9 if st else None,
            "pairs_per_iter": pairs, "keys_per_iter": step.num_keys(),
            "stages_ms": st, "roofline": roofline, "roofline_stages": stages_roof, "e2e": e2e,
            "gpu_launches": launches_per_step(step) * args.steps, "clocks": clocks}
    if not args.no_window:
        line["window"] = window_run(device, args, flush, value, dist, world)
    if not args.no_learned_init:
        line["learned_init"] = learned_init_run(device, args)
    if not args.no_extras:
        line["loop_closure_update"] = loop_closure_run(device)
        line["pose_refinement"] = tracking_run(device)
        line["bundle_adjustment"] = ba_run(device)
        line["keyframe_insertion"] = insertion_run(device)
        line["final_colour_refinement"] = refinement_run(device)
    if not args.no_window:
        line["differentiation"] = differentiation_run(device)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(params, mp)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
