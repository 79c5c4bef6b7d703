#!/usr/bin/env python3
"""Benchmark of the GB300 render path of 4D Gaussian Splatting (arXiv 2412.20720).

Headline workload (one step): 300,000 synthetic 4D Gaussians (spatial SH
degree 3 x temporal order 2) over [-3,3]^3 x [0,1], rendered at 1352x1014 from
an orbit camera of radius 6 for the 300 timestamps t_k = k/299 of a sweep,
one view per call (plain form): preprocess -> bin_sort -> render_image (the
forward compositor without the state a backward pass needs) through the C
ABI for every view, with --inflight frames in flight (FramePipeline: one
workspace and one stream per slot, frame k on slot k % inflight).  value =
rendered frames/s over all ranks.

Also reported ("train"): fwd+bwd iterations/s of the training step on the same
scene -- 4 timestamps x 1 camera at 1352x1014 in one batched call, L1 loss
against target images rendered by the CUDA path from a second seeded scene,
backward to every parameter, and an Adam step.

Timing: W untimed warm-up steps, then K steps between a barrier +
synchronize on both sides, CUDA events on the launching stream, max over
ranks.  The scene's parameters (193 MB) exceed the 129 MB L2, so no flush is
inserted between frames.  `--impl reference` times the FP64 CPU oracle on the
host cores on the same workload (one full view per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "4dgs-orbit-sweep-300k"
METRIC = "rendered frames/s (300k 4D Gaussians, 1352x1014, 300-timestamp sweep, one view per call)"
UNIT = "frames/s"
SWEEP = 300
N_GAUSS = 300_000
W_IMG, H_IMG = 1352, 1014
# Algorithmic FP32 flops of the compositor: an alpha evaluation is 2 subtractions,
# 3 products and 3 multiply-adds of the conic form (8), a*G and the 0.99 clamp
# (2) and the skip test (1) = 11; a composited entry adds T*(1-alpha) (2),
# alpha*T (1), three colour multiply-adds (6) = 9.  The ex2 goes to the SFU.
FLOPS_PER_EVAL = 11
FLOPS_PER_COMP = 9
# DRAM bytes (read + write) of one image-mode compositor launch on this
# workload, per block shape: the mean over the frames of a 4-view orbit sweep captured by
# ncu (profiles/launches_orbit_300k_1352x1014.md, traffic section); emptied
# whenever the kernel changes.
# keyed by (tile, pixels per thread, shared batch)
RENDER_FWD_TRAFFIC = {(16, 4, 128): 6.979e6, (16, 4, 256): 6.986e6, (16, 2, 128): 6.969e6,
                      (16, 2, 256): 6.963e6}


def parse():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--n", type=int, default=N_GAUSS, help="Gaussians (default: the headline 300k)")
    p.add_argument("--views", type=int, default=SWEEP, help="views per sweep step (default 300)")
    p.add_argument("--train-iters", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the batched multi-view measurements")
    p.add_argument("--inflight", type=int, default=8, help="headline frames in flight (one stream and workspace each)")
    p.add_argument("--stage-blocks", type=int, default=1,
                   help="resident blocks per SM of the latency-bound stages (0 = full-GPU grids)")
    p.add_argument("--shape", default=None, help="compositor shape tile/pixels_per_thread/shared_batch (e.g. 16/4/128) "
                                                 "instead of the autotune (for profiling a fixed kernel)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value over the ranks (a job's time is its slowest rank's);
    one all-reduce of a float64 on `device` when world > 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank processes units_per_rank)."""
    return units_per_rank * world / (ms_max / 1000.0)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_query_id(torch, dev) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:  # pragma: no cover
        return str(dev.index or 0)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------ CPU oracle

def oracle_frames(n: int, ks, seconds_budget: float = 30.0):
    """Full views rendered by the FP64 oracle on the host cores.  Returns
    (frames/s, threads, frames done)."""
    import numpy as np

    import oracle
    from paper_2412_20720_gb300 import synthetic as sy
    scene = sy.orbit_scene(n)
    params = scene.as_dict()
    st = oracle.Settings(sh_degree=3, t_order=2, tile=16, period=1.0, near_plane=float(np.float32(0.2)),
                         dilation=float(np.float32(0.3)), p_t_min=float(np.float32(0.05)))
    t0 = time.perf_counter()
    done = 0
    for k in ks:
        v = sy.orbit_view(k, SWEEP, W_IMG, H_IMG)
        pr = oracle.preprocess(params, v, st)
        oracle.render(pr, v, st)
        done += 1
        if time.perf_counter() - t0 > seconds_budget:
            break
    dt = time.perf_counter() - t0
    return done / dt, oracle.num_threads(), done


# ----------------------------------------------------------------- ours

def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import PARAM_KEYS, FramePipeline, RenderConfig, autotune

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    scene = sy.orbit_scene(args.n)
    host = scene.as_dict()
    params = {k: torch.from_numpy(host[k]).to(dev) for k in PARAM_KEYS}
    nviews = args.views
    views = [sy.orbit_view(k, nviews, W_IMG, H_IMG) for k in range(nviews)]
    # Lean grids for the latency-bound stages (one resident preprocess and
    # radix block per SM, two emission blocks): the frames in flight share
    # the SMs.
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 24, stage_blocks_per_sm=args.stage_blocks)
    # One view per call; args.inflight frames in flight (one workspace and one
    # stream per slot), frame k on slot k % inflight.
    pipe = FramePipeline(scene.n, views[0], cfg, depth=args.inflight, device=dev)
    r = pipe.slots[0]
    vv = [fgs4d.make_views([v]) for v in views]
    # Visible-pair capacity sized to the sweep's own views (largest count +
    # 10%): the depth sort and pair scan size their grids by it.
    vis_cap = pipe.fit_visible_capacity(params, view_sets=vv)
    # Compositor shape and tile edge timed as the sweep runs: every 10th view
    # of the sweep submitted through the pipeline.
    if args.shape:
        st_, sp_, sb_ = (int(x) for x in args.shape.split("/"))
        pipe.set_tile(st_, sp_, sb_)
        tuned = {"tile": st_, "pixels_per_thread": sp_, "shared_batch": sb_, "ms": {}, "timed": "fixed by --shape"}
    else:
        tuned = autotune(r, params, view_sets=vv[::10], tiles=(16, 8), batches=(256, 128), pipeline=pipe)
    g = r.gaussians(params)
    ws, wsb, s = r.ws.data_ptr(), r.ws_bytes, r.settings
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    npx = W_IMG * H_IMG
    imgs = [torch.empty(3 * npx, dtype=torch.float32, device=dev) for _ in range(pipe.depth)]
    # preprocess; bin_sort (as the library reports it); render.
    launches_per_frame = 1 + fgs4d.bin_sort_kernels(scene.n, vv[0][0], vv[0][1], s) + 1

    # Capacity and work counts over the whole sweep (outside the timed region).
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    vis, inst, evals, comps = [], [], [], []
    for k in range(nviews):
        v, n1 = vv[k]
        fgs4d.preprocess(g, v, n1, s, ws, wsb, st)
        fgs4d.bin_sort(scene.n, v, n1, s, ws, wsb, st)
        stats.zero_()
        fgs4d.render_stats(scene.n, v, n1, s, ws, wsb, imgs[0].data_ptr(), stats.data_ptr(), st)
        code, counts = r.status()
        if code != fgs4d.OK:
            raise RuntimeError("view %d: %s (counts %s)" % (k, fgs4d.status_string(code), counts))
        vis.append(counts[0])
        inst.append(counts[1])
        e, c = stats.tolist()
        evals.append(e)
        comps.append(c)

    def sweep(comp_ev=None, after=None):
        pipe.begin()
        for k in range(nviews):
            j = pipe.slot_of_next()
            pipe.submit(g, vv[k][0], vv[k][1], imgs[j].data_ptr(), events=None if comp_ev is None else comp_ev[k],
                        after=None if after is None else (lambda sst, k=k, j=j: after(sst, k, j)))
        pipe.end()

    # Warm-up, then the timed sweep steps.
    for _ in range(args.warmup):
        sweep()
    torch.cuda.synchronize()
    K = args.steps
    comp_evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nviews)] for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_query_id(torch, dev))
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    start.record(stream)
    for step in range(K):
        sweep(comp_evs[step])
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    pipe.check()
    ms = start.elapsed_time(end)
    comp_ms_timed = float(np.mean([e[0].elapsed_time(e[1]) for step in comp_evs for e in step]))
    ms_max = max_over_ranks(ms, world, dev)
    value = job_rate(K * nviews, world, ms_max)

    # Per-stage durations with one frame in flight (separate, untimed passes
    # over the sweep on one stream, events between the stages): with the
    # timed configuration, and with full-GPU grids for the latency-bound
    # stages (the same workspace layout), from which the kernels' rooflines
    # are taken.
    def stage_pass(settings):
        acc = np.zeros(3)
        ev4 = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nviews)]
        for k in range(nviews):
            v, n1 = vv[k]
            ev4[k][0].record(stream)
            fgs4d.preprocess(g, v, n1, settings, ws, wsb, st)
            ev4[k][1].record(stream)
            fgs4d.bin_sort(scene.n, v, n1, settings, ws, wsb, st)
            ev4[k][2].record(stream)
            fgs4d.render_image(scene.n, v, n1, settings, ws, wsb, imgs[0].data_ptr(), None, st)
            ev4[k][3].record(stream)
        torch.cuda.synchronize()
        for e4 in ev4:
            acc += [e4[0].elapsed_time(e4[1]), e4[1].elapsed_time(e4[2]), e4[2].elapsed_time(e4[3])]
        return acc / nviews

    stage_ms = stage_pass(s)
    s_full = fgs4d.Settings.from_buffer_copy(s)
    s_full.stage_blocks_per_sm = 0
    stage_full = stage_pass(s_full)
    code, _ = r.status()
    if code != fgs4d.OK:
        raise RuntimeError("per-stage passes: %s" % fgs4d.status_string(code))

    # Roofline of the dominant kernel (the compositor): FP32-ALU bound.
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    mean_flops = FLOPS_PER_EVAL * np.mean(evals) + FLOPS_PER_COMP * np.mean(comps)
    achieved_timed = mean_flops / (comp_ms_timed * 1e-3) / 1e12
    achieved_iso = mean_flops / (stage_full[2] * 1e-3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    pre_bytes = 68.0 * scene.n + (576.0 + 56.0) * np.mean(vis)
    pre_gbs = pre_bytes / (stage_full[0] * 1e-3) / 1e9

    # ---------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(host[k]).pin_memory() for k in PARAM_KEYS}
        host_imgs = [torch.empty(3 * npx, dtype=torch.float32).pin_memory() for _ in range(pipe.depth)]
        h2d = sum(int(p.numel() * p.element_size()) for p in pinned.values())
        d2h = nviews * 3 * npx * 4

        def copy_back(sst, k, j):
            with torch.cuda.stream(sst):
                host_imgs[j].copy_(imgs[j], non_blocking=True)

        def e2e_step():
            for kk in PARAM_KEYS:
                params[kk].copy_(pinned[kk], non_blocking=True)
            sweep(after=copy_back)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        e_ms = (time.perf_counter() - t0) * 1000.0
        e2e = {"value": job_rate(K * nviews, world, max_over_ranks(e_ms, world, dev)), "unit": UNIT,
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h,
               "path": "parameters copied from pinned host memory each step, then the sweep through the C ABI "
                       "(%d frames in flight); each image copied to pinned host memory on its frame's stream"
                       % pipe.depth}

    # ---------------------------------------------------------- train step
    train = run_train(args, dev, scene, params, world, barrier)

    # ---------------------------------------------------------- batched views
    batched = None
    if not args.no_batched:
        batched = [run_batched(dev, sy.sphere_scene(), sy.sphere_views(64), "sphere-1M-64views-mixed-res", 2, 8,
                               tiles=(16, 8)),
                   run_batched(dev, sy.urban_scene(), sy.urban_views(), "urban-3M-6cams-x-2t-1920x1080", 2, 6,
                               plain=False)]

    # ---------------------------------------------------------- CPU oracle
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps, cores, nfr = oracle_frames(args.n, [SWEEP // 2], 60.0)
        cpu = {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d full view(s) (view k=%d of the sweep: %d Gaussians, %dx%d) rendered by the FP64 "
                         "oracle with OpenMP over pixel rows" % (nfr, SWEEP // 2, args.n, W_IMG, H_IMG)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded; shapes and distributions of the paper's workloads)",
            "config": {"workload": WORKLOAD, "gaussians": args.n, "sh_degree": 3, "t_order": 2,
                       "resolution": [W_IMG, H_IMG], "views_per_step": nviews, "views_per_call": 1,
                       "vis_capacity": vis_cap, "frames_in_flight": pipe.depth,
                       "stage_blocks_per_sm": args.stage_blocks,
                       "l2": "inputs larger than L2 (193 MB of parameters vs 129 MB L2); no flush",
                       "parallelism": "views replicated per GPU" if world > 1 else "single GPU"},
            "gpu_launches": launches_per_frame * nviews * K,
            "frames_in_flight": pipe.depth,
            "autotune": tuned,
            "stages_ms_per_frame": {"preprocess": stage_ms[0], "bin_sort": stage_ms[1], "render_fwd": stage_ms[2],
                                    "basis": "one frame in flight, the timed configuration: a separate untimed "
                                             "pass over the sweep"},
            "stages_ms_per_frame_full_grids": {"preprocess": stage_full[0], "bin_sort": stage_full[1],
                                               "render_fwd": stage_full[2],
                                               "basis": "one frame in flight, stage_blocks_per_sm = 0 (full-GPU "
                                                        "grids for preprocess, sorting and emission)"},
            "work_per_frame": {"visible": float(np.mean(vis)), "instances": float(np.mean(inst)),
                               "alpha_evals": float(np.mean(evals)), "composited": float(np.mean(comps))},
            "roofline": {"kernel": "render_fwd_kernel (image mode, fgs4d_render_image)", "bound": "alu",
                         "achieved": achieved_timed, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": achieved_timed / fp32_peak,
                         "traffic": RENDER_FWD_TRAFFIC.get((tuned["tile"], tuned["pixels_per_thread"],
                                                            tuned["shared_batch"])),
                         "peak_basis": "SMs x 128 FP32 lanes x 2 (FMA) x max SM clock %.0f MHz (derived)" % sm_max,
                         "flops_per_launch": mean_flops, "launch_ms": comp_ms_timed,
                         "duration_basis": "CUDA events around each compositor launch on its slot stream in the "
                                           "timed region (other frames' kernels share the GPU meanwhile)"},
            "roofline_throughput": {"kernel": "render_fwd_kernel (image mode, fgs4d_render_image)", "bound": "alu",
                                    "achieved": mean_flops * value / world / 1e12, "peak": fp32_peak,
                                    "unit": "TFLOP/s", "frac": mean_flops * value / world / 1e12 / fp32_peak,
                                    "duration_basis": "the compositor's flops of every frame over the timed "
                                                      "region's wall time (one GPU; the other stages share it)"},
            "roofline_isolated": {"kernel": "render_fwd_kernel (image mode, fgs4d_render_image)", "bound": "alu",
                                  "achieved": achieved_iso,
                                  "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved_iso / fp32_peak,
                                  "launch_ms": float(stage_full[2]),
                                  "duration_basis": "one frame in flight (the full-grid per-stage pass)"},
            "preprocess_roofline": {"bound": "hbm", "achieved": pre_gbs, "peak": hbm, "unit": "GB/s",
                                    "frac": pre_gbs / hbm, "bytes_per_launch": pre_bytes,
                                    "duration_basis": "one frame in flight, full-GPU grid",
                                    "peak_basis": "measured hbm_gbs"},
            "clocks": clk,
            "e2e": e2e,
            "train": train,
            "batched": batched,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_train(args, dev, scene, params, world, barrier):
    """Training step: 4 timestamps x 1 camera, L1 loss, backward, Adam.  Two
    forms of the same step: the 4 views in one batched call, and the 4 views
    as single-view calls on 4 streams (ViewParallel; gradients accumulate in
    the same buffers).  value = the faster one, each replayed as one CUDA
    graph."""
    import torch

    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import (PARAM_KEYS, Adam, RenderConfig, Renderer, ViewParallel, autotune,
                                               l1_loss)

    views = sy.train_views(4, W_IMG, H_IMG)
    # The 4-view call runs alone on the GPU: full-GPU grids.  The view-parallel
    # form runs four calls at once: lean grids for their latency-bound stages.
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 25)
    tgt_scene = sy.orbit_scene(args.n, seed=sy.TARGET_SEED)
    tparams = {k: torch.from_numpy(v).to(dev) for k, v in tgt_scene.as_dict().items()}
    rt = Renderer(tgt_scene.n, views, cfg, device=dev)
    target = rt.forward(tparams).clone()
    rt.check()
    targets = [t.reshape(-1).clone() for t in rt.split(target)]
    del rt, tparams
    leaf = {k: params[k].clone().requires_grad_(True) for k in PARAM_KEYS}
    r = Renderer(scene.n, views, cfg, device=dev)
    tuned = autotune(r, {k: leaf[k].detach() for k in PARAM_KEYS}, backward=True, tiles=(16, 8), batches=(256, 128))
    vp = ViewParallel(scene.n, [[v] for v in views],
                      RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 24,
                                   stage_blocks_per_sm=args.stage_blocks),
                      device=dev)
    vp.set_tile(tuned["tile"], tuned["pixels_per_thread"], tuned["shared_batch"])
    grads = {k: torch.zeros_like(leaf[k]) for k in PARAM_KEYS}
    # Adam with the library's kernel; its step count lives on the device, so
    # the whole step can be replayed as one CUDA graph.
    pr = {k: leaf[k].detach() for k in PARAM_KEYS}
    opt = Adam(pr, lr=1e-4)
    total = int(target.numel())
    vp_loss = torch.zeros(1, dtype=torch.float32, device=dev)

    # The gradients start at zero and Adam clears each one after reading it
    # (zero_grad), so every step accumulates into zeros without a fill.
    def it_batched():
        img = r.forward(pr)
        loss, dimg = l1_loss(img, target)
        r.backward(pr, dimg, grads)
        opt.step(grads, zero_grad=True)
        return loss

    def it_parallel():
        vp_loss.zero_()
        vp.step(pr, lambda j, img: l1_loss(img, targets[j], mean_count=total, loss=vp_loss)[1], grads)
        opt.step(grads, zero_grad=True)
        return vp_loss

    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        barrier()
        a.record(stream)
        for _ in range(args.train_iters):
            out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        return a.elapsed_time(b) / args.train_iters, out

    def graph_of(it):
        # The step as one CUDA graph (what a training loop replays), after the
        # warm-up the capture needs on a side stream.
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                it()
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            out = it()
        graph.replay()
        return graph, out

    res = {}
    for name, it in (("batched_call", it_batched), ("view_parallel", it_parallel)):
        graph, g_loss = graph_of(it)
        ms, _ = timed(lambda: graph.replay())
        loss = float(g_loss.item())
        plain_ms, _ = timed(it)  # the same step launched call by call from Python
        del graph
        res[name] = {"ms_per_iter": max_over_ranks(ms, world, dev), "loss": loss,
                     "plain_launches_ms_per_iter": max_over_ranks(plain_ms, world, dev)}
    codes = [r.status()[0]] + [g.status()[0] for g in vp.groups]
    best = min(res, key=lambda k: res[k]["ms_per_iter"])
    ms = res[best]["ms_per_iter"]
    return {"metric": "fwd+bwd iters/s", "value": job_rate(1, world, ms), "unit": "iters/s", "ms_per_iter": ms,
            "form": best,
            "workload": "4 timestamps x 1 camera at 1352x1014, %d Gaussians, L1 loss (mean over the 4 images), "
                        "backward to all parameters, Adam step (fgs4d kernel); the step replayed as one CUDA graph"
                        % scene.n,
            "forms": res,
            "status": fgs4d.status_string(min(codes)), "autotune": tuned,
            "targets": "rendered by the CUDA path from a second seeded scene"}


def run_batched(dev, scene, views, label, steps, group, plain=True, tiles=(16,)):
    """Forward + backward of many (camera, t) views of mixed resolution: one
    multi-view call per group of ``group`` views, all groups of a step
    captured in one CUDA graph, against one plain single-view call per view.
    The upstream image gradient is a fixed random tensor (the loss does not
    change the kernel work)."""
    import torch

    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer, autotune

    params = {k: torch.from_numpy(v).to(dev) for k, v in scene.as_dict().items()}
    n = scene.n
    groups = [views[i:i + group] for i in range(0, len(views), group)]
    rs, tuned, vis_tot, inst_tot, max_inst = [], None, 0, 0, 0
    for gv in groups:
        # Size each group's capacities on one forward per tile edge with
        # generous ones.
        probe = Renderer(n, gv, RenderConfig(sh_degree=3, t_order=2, vis_capacity=min(n * len(gv), 1 << 29),
                                             inst_capacity=(1 << 30) - 1), device=dev)
        counts = None
        for t in tiles:
            probe.set_tile(t)
            probe.forward(params)
            c = probe.check()
            counts = c if counts is None else [max(a, b) for a, b in zip(counts, c)]
        del probe
        torch.cuda.empty_cache()
        cfg = RenderConfig(sh_degree=3, t_order=2, vis_capacity=int(counts[0] * 1.1) + 1024,
                           inst_capacity=min(int(counts[1] * 1.1) + 1024, (1 << 30) - 1))
        r = Renderer(n, gv, cfg, device=dev)
        if tuned is None:
            tuned = autotune(r, params, backward=True, reps=2, tiles=tiles, batches=(256, 128))
        r.set_tile(tuned["tile"], tuned["pixels_per_thread"], tuned["shared_batch"])
        rs.append(r)
        vis_tot += counts[0]
        inst_tot += counts[1]
        max_inst = max(max_inst, counts[1])
    gen = torch.Generator(device=dev).manual_seed(3)
    dLs = [torch.randn(3 * r.total_pixels, device=dev, generator=gen) * 1e-3 for r in rs]
    grads = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS}

    def step():
        for gk in grads.values():
            gk.zero_()
        for r, dL in zip(rs, dLs):
            r.forward(params)
            r.backward(params, dL, grads)

    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream(dev).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        graph.replay()
    b.record(stream)
    torch.cuda.synchronize()
    codes = [r.status()[0] for r in rs]
    code = next((c for c in codes if c != fgs4d.OK), fgs4d.OK)
    graph_ms = a.elapsed_time(b) / steps
    out = {"workload": label, "gaussians": n, "views": len(views), "views_per_call": group,
           "resolutions": sorted({"%dx%d" % (v["width"], v["height"]) for v in views}),
           "visible_pairs": vis_tot, "instances": inst_tot, "status": fgs4d.status_string(code),
           "autotune": tuned,
           "graph_batched": {"ms_per_step": graph_ms, "views_per_s": len(views) * 1000.0 / graph_ms,
                             "fwd_bwd_iters_per_s": 1000.0 / graph_ms}}
    del graph
    # The same groups as calls on parallel streams (lean grids for their
    # latency-bound stages; the same workspace layout), one graph.
    nstreams = min(4, len(rs))
    streams = [torch.cuda.Stream(dev) for _ in range(nstreams)]
    lean = []
    for r in rs:
        sl = fgs4d.Settings.from_buffer_copy(r.settings)
        sl.stage_blocks_per_sm = 1
        lean.append(sl)
    full = [r.settings for r in rs]

    def step_parallel():
        for gk in grads.values():
            gk.zero_()
        cur = torch.cuda.current_stream(dev)
        ev = torch.cuda.Event()
        ev.record(cur)
        for i, (r, dL) in enumerate(zip(rs, dLs)):
            st = streams[i % nstreams]
            st.wait_event(ev)
            with torch.cuda.stream(st):
                r.forward(params)
                r.backward(params, dL, grads)
        for st in streams:
            cur.wait_stream(st)

    for r, sl in zip(rs, lean):
        r.settings = sl
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(2):
            step_parallel()
    torch.cuda.current_stream(dev).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_parallel()
    graph.replay()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        graph.replay()
    b.record(stream)
    torch.cuda.synchronize()
    par_ms = a.elapsed_time(b) / steps
    codes = [r.status()[0] for r in rs]
    for r, sf in zip(rs, full):
        r.settings = sf
    del graph
    out["graph_parallel_streams"] = {"streams": nstreams, "ms_per_step": par_ms,
                                     "views_per_s": len(views) * 1000.0 / par_ms,
                                     "fwd_bwd_iters_per_s": 1000.0 / par_ms,
                                     "status": fgs4d.status_string(next((c for c in codes if c != fgs4d.OK),
                                                                        fgs4d.OK))}
    if plain:
        # One single-view renderer per resolution; each view is its own call.
        per_res = {}
        singles = []
        for v in views:
            key = (v["width"], v["height"])
            if key not in per_res:
                c1 = RenderConfig(sh_degree=3, t_order=2, vis_capacity=n, inst_capacity=max_inst + 1024,
                                  pixels_per_thread=tuned["pixels_per_thread"], tile=tuned["tile"],
                                  shared_batch=tuned["shared_batch"])
                per_res[key] = Renderer(n, [v], c1, device=dev)
            rr = per_res[key]
            singles.append((rr, fgs4d.make_views([v]), torch.randn(3 * v["width"] * v["height"], device=dev,
                                                                   generator=gen) * 1e-3))
        g_ = {k: params[k] for k in PARAM_KEYS}

        def plain_step():
            for gk in grads.values():
                gk.zero_()
            for rr, (vv, nv), dl in singles:
                st = rr.stream()
                ws = rr.ws.data_ptr()
                gg = rr.gaussians(g_)
                fgs4d.preprocess(gg, vv, nv, rr.settings, ws, rr.ws_bytes, st)
                fgs4d.bin_sort(n, vv, nv, rr.settings, ws, rr.ws_bytes, st)
                img = torch.empty_like(dl)
                fgs4d.render_fwd(n, vv, nv, rr.settings, ws, rr.ws_bytes, img.data_ptr(), None, st)
                fgs4d.render_bwd(gg, vv, nv, rr.settings, ws, rr.ws_bytes, dl.data_ptr(),
                                 fgs4d.make_grads({k: grads[k].data_ptr() for k in PARAM_KEYS}), st)

        plain_step()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            plain_step()
        b.record(stream)
        torch.cuda.synchronize()
        for rr in per_res.values():
            code2, _ = rr.status()
            if code2 != fgs4d.OK:
                out["plain_status"] = fgs4d.status_string(code2)
        plain_ms = a.elapsed_time(b) / steps
        out["plain_per_view"] = {"ms_per_step": plain_ms, "views_per_s": len(views) * 1000.0 / plain_ms,
                                 "fwd_bwd_iters_per_s": 1000.0 / plain_ms}
        out["graph_speedup"] = plain_ms / graph_ms
        del per_res, singles
    del rs
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------ reference

def run_reference(args, rank, world):
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    ks = list(range(0, SWEEP, max(1, SWEEP // max(1, K + W))))[:K + W]
    oracle_frames(args.n, ks[:W], 1e9) if W else None
    fps, cores, nfr = oracle_frames(args.n, ks[W:W + K], 1e9)
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": 1000.0 / fps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD, "gaussians": args.n, "sh_degree": 3, "t_order": 2,
                       "resolution": [W_IMG, H_IMG], "views_per_step": 1},
            "cpu_baseline": {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full view of the sweep per step (FP64 oracle, OpenMP)"},
            "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
