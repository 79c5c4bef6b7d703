#!/usr/bin/env python3
"""Benchmark of the GB300 render path of 4D Gaussian Splatting (arXiv 2412.20720).

Headline workload (one step): 300,000 synthetic 4D Gaussians (spatial SH
degree 3 x temporal order 2) over [-3,3]^3 x [0,1], rendered at 1352x1014 from
an orbit camera of radius 6 for the 300 timestamps t_k = k/299 of a sweep,
one view per call (plain form): preprocess -> bin_sort -> render_image (the
forward compositor without the state a backward pass needs) through the C
ABI for every view, with --inflight frames in flight (FramePipeline: one
workspace and one stream per slot, frame k on slot k % inflight).  value =
rendered frames/s over all ranks; with N ranks the sweep has 300 N views and
rank r renders the views k = r (mod N).

Also reported ("train"): fwd+bwd iterations/s of the training step on the same
scene -- 4 timestamps x 1 camera at 1352x1014, L1 loss against target images
rendered by the FP64 oracle from a second seeded scene (rendered in the CPU
baseline leg; the CUDA path renders them when that leg does not run),
backward to every parameter; the same step with an Adam update is reported
beside it.  Per-stage times and the rooflines of the forward and backward
compositors come from an untimed pass with one step alone.  "batched": the
1M-Gaussian 64-view mixed-resolution workload and the 3M-Gaussian urban rig,
with per-stage times.  "c0": the 2k-Gaussian 128x96 configuration.
"extensions": the rows built beyond the render path (auxiliary channels,
densification statistics and the 4D split, the Compact-4DGS mask, scale-gated
features), each timed on the headline scene with its roofline.

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
# The compositor adjoint repeats the alpha evaluation (11) at every list
# position up to a pixel's last composited entry; a composited entry then
# costs 1 - alpha (1), T / (1 - alpha) (1, with an SFU reciprocal), w =
# alpha T (1), three colour-gradient multiply-adds (6), dL/dC . c (5),
# dL/dalpha = T Dc - Dr / (1 - alpha) (3), Dr += w Dc (2), gp = g_alpha
# alpha (1), gp dy (1) and the three moment sums (4) = 25.
FLOPS_PER_BWD_COMP = 25
# Issue slots of one SM per clock: four schedulers, one warp instruction each.
ISSUE_PER_SM_CLK = 4
# One ncu capture of the image-mode compositor (render_fwd_kernel, mode 3) on
# this workload: DRAM bytes (read + write) and warp instructions per launch,
# averaged over the captured launches (the first three of the timed sweep,
# views 0-2).  Valid only for the compositor sources it was taken from
# (sha256 prefix of csrc/render.cu + csrc/fgs4d_internal.cuh) and block
# shape; any other build reports null.
NCU_RENDER_FWD = {"render_cu_sha256": "eb51d3ae1b99e20c", "shape": "16/4/128", "dram_bytes": 5.02e6, "warp_insts": 125.43e6,
                  "views": [0, 1, 2], "capture": "ncu --set full --clock-control none --nvtx --nvtx-include timed/ "
                                                 "-k regex:render_fwd_kernel -c 3 on python bench.py --steps 1 "
                                                 "--warmup 1 --shape 16/4/128 (no other legs)"}


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
    p.add_argument("--batched", choices=("all", "sphere", "urban"), default="all",
                   help="which batched workloads to run (default both)")
    p.add_argument("--urban-views", type=int, default=12,
                   help="views of the urban rig used (default all 12; fewer for profiling a small case)")
    p.add_argument("--urban-group", type=int, default=6, help="urban views per call (default 6)")
    p.add_argument("--inflight", type=int, default=8, help="headline frames in flight (one stream and workspace each)")
    p.add_argument("--stage-blocks", type=int, default=1,
                   help="resident blocks per SM of the latency-bound stages (0 = full-GPU grids)")
    p.add_argument("--shape", default=None, help="compositor shape tile/pixels_per_thread/shared_batch (e.g. 16/4/128) "
                                                 "instead of the autotune (for profiling a fixed kernel)")
    p.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    p.add_argument("--no-c0", action="store_true", help="skip the 2k-Gaussian configuration")
    p.add_argument("--no-ext", action="store_true",
                   help="skip the rows beyond the render path (aux channels, densification, mask, features)")
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


def shard_views(views_per_rank: int, rank: int, world: int):
    """Indices of the sweep views rank `rank` renders.  The job's sweep has
    views_per_rank * world distinct (camera, t) views; rank r takes the views
    k = r (mod world), so every view is rendered exactly once and the work
    per GPU stays fixed as world grows (weak scaling, no exchange)."""
    return list(range(rank, views_per_rank * world, world))


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

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_settings():
    import numpy as np

    import oracle
    return oracle.Settings(sh_degree=3, t_order=2, tile=16, period=1.0, near_plane=float(np.float32(0.2)),
                           dilation=float(np.float32(0.3)), p_t_min=float(np.float32(0.05)))


def row_window(view, y0: int, h: int) -> dict:
    """Rows [y0, y0 + h) of a view, as a view of its own (principal point
    shifted; same pixels, same samples)."""
    import numpy as np
    v = dict(view)
    v.update(height=h, cy=np.float32(float(view["cy"]) - y0))
    return v


def oracle_frames(n: int, ks, seconds_budget: float = 30.0):
    """Full views rendered by the FP64 oracle on the host cores.  Returns
    (frames/s, threads, frames done)."""
    import oracle
    from paper_2412_20720_gb300 import synthetic as sy
    params = sy.orbit_scene(n).as_dict()
    st = oracle_settings()
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


def oracle_window_seconds(params, view, rows: int, backward: bool = False, threads: int = 1):
    """Seconds of the oracle's forward (and adjoint) of the middle ``rows``
    rows of ``view`` on ``threads`` host threads, and the share of the view's
    pixels they are."""
    import numpy as np

    import oracle
    H = int(view["height"])
    v = row_window(view, (H - rows) // 2, rows)
    st = oracle_settings()
    before = oracle.num_threads()
    oracle.set_num_threads(threads)
    try:
        t0 = time.perf_counter()
        pr = oracle.preprocess(params, v, st)
        img, _, _, _ = oracle.render(pr, v, st)
        if backward:
            oracle.render_backward(params, pr, v, st, np.sign(img - 0.5))
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(before)
    return dt, rows / H


def cpu_leg(args, scene, tgt_scene, train_views):
    """The oracle on the host cores (rank 0, N = 1): the headline frame rate
    (one full view, all cores; a row window on one core), the C2 targets
    (the oracle renders the training views of the target scene), and the
    training step's rate (one view's forward + adjoint, all cores and one
    core on a row window).  Returns (headline cpu_baseline, train
    cpu_baseline, targets as [3, H, W] float32 arrays)."""
    import numpy as np

    import oracle
    model = cpu_model()
    cores = os.cpu_count()
    fps, threads, nfr = oracle_frames(args.n, [SWEEP // 2], 60.0)
    params = scene.as_dict()
    rows = 64
    t1, share = oracle_window_seconds(params, sy_orbit_view(SWEEP // 2), rows, threads=1)
    head = {"value": fps, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": model, "host_cpus": cores,
            "sample": "%d full view(s) (view k=%d of the sweep: %d Gaussians, %dx%d) rendered by the FP64 oracle "
                      "with OpenMP over pixel rows" % (nfr, SWEEP // 2, args.n, W_IMG, H_IMG),
            "one_core": {"value": share / t1, "unit": UNIT, "cores": 1,
                         "sample": "the middle %d rows of the same view on one thread, scaled to a full view"
                                   % rows}}
    # C2 targets: the oracle's render of the target scene at the training views.
    st = oracle_settings()
    tparams = tgt_scene.as_dict()
    t0 = time.perf_counter()
    targets = []
    for v in train_views:
        img, _, _, _ = oracle.render(oracle.preprocess(tparams, v, st), v, st)
        targets.append(img.astype(np.float32))
    t_targets = time.perf_counter() - t0
    # One view of the training step: forward + adjoint of the L1 loss.
    v = train_views[0]
    t0 = time.perf_counter()
    pr = oracle.preprocess(params, v, st)
    img, _, _, _ = oracle.render(pr, v, st)
    npx = img.size * len(train_views)
    oracle.render_backward(params, pr, v, st, np.sign(img - targets[0]) / npx)
    t_view = time.perf_counter() - t0
    t1b, share_b = oracle_window_seconds(params, v, rows, backward=True, threads=1)
    train = {"value": 1.0 / (len(train_views) * t_view), "unit": "iters/s", "cores": threads, "kind": "oracle",
             "cpu_model": model, "host_cpus": cores,
             "sample": "one view of the 4-view step (%d Gaussians, %dx%d): forward + adjoint of the L1 loss by the "
                       "FP64 oracle with OpenMP over pixel rows, scaled to 4 views" % (scene.n, W_IMG, H_IMG),
             "one_core": {"value": share_b / (len(train_views) * t1b), "unit": "iters/s", "cores": 1,
                          "sample": "the middle %d rows of the view on one thread, scaled to 4 full views" % rows},
             "targets": {"views": len(train_views), "seconds": t_targets,
                         "frames_per_s": len(train_views) / t_targets}}
    return head, train, targets


def sy_orbit_view(k: int):
    from paper_2412_20720_gb300 import synthetic as sy
    return sy.orbit_view(k, SWEEP, W_IMG, H_IMG)


def render_cu_sha256() -> str:
    """sha256 prefix of the compositor's sources (render.cu and the shared
    alpha evaluation in fgs4d_internal.cuh)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("render.cu", "fgs4d_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2412_20720_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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
    # This rank's share of the job's sweep (views_per_rank x world views).
    views = [sy.orbit_view(k, nviews * world, W_IMG, H_IMG) for k in shard_views(nviews, rank, world)]
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
    stats = torch.zeros(3, dtype=torch.int64, device=dev)  # fgs4d_render_stats adds three counters
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
        e, c, _ = stats.tolist()
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
    torch.cuda.nvtx.range_push("timed")  # lets a profiler restrict itself to the timed sweep
    for step in range(K):
        sweep(comp_evs[step])
    torch.cuda.nvtx.range_pop()
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

    # Roofline of the dominant kernel (the compositor): FP32-ALU bound.  Its
    # duration is taken with one frame in flight (events around each launch
    # in the per-stage pass), so no other frame's kernels share the SMs.
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = props.multi_processor_count
    fp32_peak = nsm * 128 * 2 * sm_max * 1e6 / 1e12
    mean_flops = FLOPS_PER_EVAL * np.mean(evals) + FLOPS_PER_COMP * np.mean(comps)
    comp_ms = float(stage_ms[2])
    achieved = mean_flops / (comp_ms * 1e-3) / 1e12
    achieved_timed = mean_flops / (comp_ms_timed * 1e-3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    pre_bytes = 68.0 * scene.n + (576.0 + 56.0) * np.mean(vis)
    pre_gbs = pre_bytes / (stage_full[0] * 1e-3) / 1e9
    shape = "%d/%d/%d" % (tuned["tile"], tuned["pixels_per_thread"], tuned["shared_batch"])
    ncu_ok = NCU_RENDER_FWD["render_cu_sha256"] == render_cu_sha256() and NCU_RENDER_FWD["shape"] == shape
    issue = None
    if ncu_ok and NCU_RENDER_FWD["warp_insts"] and len(evals) >= 3:
        # The issue-slot ceiling: the captured views' warp instructions per
        # alpha evaluation, times this sweep's mean evaluations, at one warp
        # instruction per scheduler per clock on every SM.
        per_eval = NCU_RENDER_FWD["warp_insts"] / float(np.mean([evals[v] for v in NCU_RENDER_FWD["views"]]))
        floor_ms = per_eval * np.mean(evals) / (nsm * ISSUE_PER_SM_CLK * sm_max * 1e6) * 1e3
        issue = {"warp_insts_per_alpha_eval": per_eval, "issue_limited_ms": floor_ms, "frac": floor_ms / comp_ms,
                 "basis": "ncu warp instructions per alpha evaluation of this build x the sweep's mean evaluations "
                          "/ (SMs x 4 schedulers x max SM clock)"}

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

    # ---------------------------------------------------------- CPU oracle
    # (rank 0 at N = 1 only; it also renders the training step's targets)
    cpu = cpu_train = targets = None
    train_views = sy.train_views(4, W_IMG, H_IMG)
    tgt_scene = sy.orbit_scene(args.n, seed=sy.TARGET_SEED)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, cpu_train, targets = cpu_leg(args, scene, tgt_scene, train_views)

    # ---------------------------------------------------------- train step
    train = None
    if not args.no_train:
        train = run_train(args, dev, scene, params, world, barrier, train_views, tgt_scene, targets, fp32_peak)
        if train is not None:
            train["cpu_baseline"] = cpu_train

    # ---------------------------------------------------------- batched views
    # (rank 0 only: the other ranks' lines are not printed, and no collective follows)
    batched = None
    if not args.no_batched and rank == 0:
        batched = []
        if args.batched in ("all", "sphere"):
            batched.append(run_batched(dev, sy.sphere_scene(), sy.sphere_views(64), "sphere-1M-64views-mixed-res", 2, 8,
                                       tiles=(16, 8), hbm=hbm))
        if args.batched in ("all", "urban"):
            uv = sy.urban_views()[:args.urban_views]
            label = "urban-3M-6cams-x-2t-1920x1080" if len(uv) == 12 and args.urban_group == 6 else \
                "urban-3M-%dviews-1920x1080-%d-per-call" % (len(uv), args.urban_group)
            batched.append(run_batched(dev, sy.urban_scene(), uv, label, 2, args.urban_group, plain=False, hbm=hbm))

    # ---------------------------------------------------------- rows beyond the render path
    ext = None
    if not args.no_ext and rank == 0:
        ext = run_extensions(dev, scene.n, params, [sy.orbit_view(k, nviews, W_IMG, H_IMG)
                                                    for k in range(0, nviews, max(1, nviews // 8))][:8],
                             fp32_peak, hbm)

    # ---------------------------------------------------------- C0
    c0 = None if args.no_c0 or rank != 0 else run_tiny(dev)

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
                       "parallelism": ("views sharded: rank r renders views k = r mod %d of a %d-view sweep"
                                       % (world, nviews * world)) if world > 1 else "single GPU"},
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
                         "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": NCU_RENDER_FWD["dram_bytes"] if ncu_ok else None,
                         "peak_basis": "SMs x 128 FP32 lanes x 2 (FMA) x max SM clock %.0f MHz (derived; no FP32 "
                                       "peak is measured)" % sm_max,
                         "flops_per_launch": mean_flops, "launch_ms": comp_ms,
                         "duration_basis": "CUDA events around each compositor launch with one frame in flight "
                                           "(the per-stage pass over the sweep, timed configuration)",
                         "issue": issue,
                         "in_timed_region": {"launch_ms": comp_ms_timed, "achieved": achieved_timed,
                                             "frac": achieved_timed / fp32_peak,
                                             "basis": "events around each launch inside the timed region, %d "
                                                      "frames sharing the GPU" % pipe.depth}},
            "roofline_throughput": {"kernel": "render_fwd_kernel (image mode, fgs4d_render_image)", "bound": "alu",
                                    "achieved": mean_flops * value / world / 1e12, "peak": fp32_peak,
                                    "unit": "TFLOP/s", "frac": mean_flops * value / world / 1e12 / fp32_peak,
                                    "duration_basis": "the compositor's flops of every frame over the timed "
                                                      "region's wall time (one GPU; the other stages share it)"},
            "preprocess_roofline": {"bound": "hbm", "achieved": pre_gbs, "peak": hbm, "unit": "GB/s",
                                    "frac": pre_gbs / hbm, "bytes_per_launch": pre_bytes,
                                    "duration_basis": "one frame in flight, full-GPU grid",
                                    "peak_basis": "measured hbm_gbs"},
            "clocks": clk,
            "e2e": e2e,
            "train": train,
            "batched": batched,
            "c0": c0,
            "extensions": ext,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def compositor_counts(r, params, views_nv=None):
    """(alpha evaluations, composited entries, evaluations up to each
    pixel's last composited entry) of one forward of renderer r."""
    import torch

    from paper_2412_20720_gb300 import fgs4d
    stats = torch.zeros(3, dtype=torch.int64, device=r.device)
    out = torch.empty(3 * r.total_pixels, dtype=torch.float32, device=r.device)
    g = r.gaussians(params)
    st = r.stream()
    fgs4d.preprocess(g, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, st)
    fgs4d.bin_sort(r.n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, st)
    fgs4d.render_stats(r.n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, out.data_ptr(),
                       stats.data_ptr(), st)
    r.check()
    return [int(x) for x in stats.tolist()]


def fwd_bwd_stage_ms(r, params, dL, grads, reps: int = 3, loss=None):
    """Per-stage milliseconds of one forward + backward call of renderer r
    alone on the GPU (events between the stages; mean of ``reps``):
    preprocess, bin_sort, render_fwd, [loss,] render_bwd_composite,
    render_bwd_preprocess.  ``loss(img)`` (optional) returns dL/dimg."""
    import numpy as np
    import torch

    from paper_2412_20720_gb300 import fgs4d
    stream = torch.cuda.current_stream(r.device)
    st = stream.cuda_stream
    g = r.gaussians(params)
    gg = r._grads(grads, None)
    ws, wsb = r.ws.data_ptr(), r.ws_bytes
    img = torch.empty(3 * r.total_pixels, dtype=torch.float32, device=r.device)
    names = ["preprocess", "bin_sort", "render_fwd"] + (["l1_loss"] if loss else []) + \
        ["render_bwd_composite", "render_bwd_preprocess"]
    acc = np.zeros(len(names))
    for _ in range(reps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(stream)
        fgs4d.preprocess(g, r.views, r.nviews, r.settings, ws, wsb, st)
        ev[1].record(stream)
        fgs4d.bin_sort(r.n, r.views, r.nviews, r.settings, ws, wsb, st)
        ev[2].record(stream)
        fgs4d.render_fwd(r.n, r.views, r.nviews, r.settings, ws, wsb, img.data_ptr(), None, st)
        k = 3
        ev[k].record(stream)
        d = dL
        if loss:
            d = loss(img)
            k += 1
            ev[k].record(stream)
        fgs4d.render_bwd_composite(r.n, r.views, r.nviews, r.settings, ws, wsb, d.data_ptr(), st)
        ev[k + 1].record(stream)
        fgs4d.render_bwd_preprocess(g, r.views, r.nviews, r.settings, ws, wsb, gg, st)
        ev[k + 2].record(stream)
        torch.cuda.synchronize()
        if _ > 0:  # the first pass warms up
            acc += [ev[i].elapsed_time(ev[i + 1]) for i in range(len(names))]
    r.check()
    return dict(zip(names, (acc / reps).tolist()))


def run_train(args, dev, scene, params, world, barrier, views, tgt_scene, targets_np, fp32_peak):
    """Training step (C2): 4 timestamps x 1 camera, L1 loss, backward to every
    parameter (gradients cleared at the start of each step).  Two forms of
    the same step: the 4 views in one batched call, and the 4 views as
    single-view calls on 4 streams (ViewParallel; gradients accumulate in
    the same buffers); value = the faster one, replayed as one CUDA graph.
    The same step followed by an Adam update is reported beside it."""
    import numpy as np
    import torch

    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300.render import (PARAM_KEYS, Adam, RenderConfig, Renderer, ViewParallel, autotune,
                                               l1_loss)

    # The 4-view call runs alone on the GPU: full-GPU grids.  The view-parallel
    # form runs four calls at once: lean grids for their latency-bound stages.
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 25)
    if targets_np is not None:
        targets = [torch.from_numpy(np.ascontiguousarray(t).reshape(-1)).to(dev) for t in targets_np]
        target_src = "rendered by the FP64 oracle from a second seeded scene (seed %d)" % tgt_scene_seed()
    else:
        tparams = {k: torch.from_numpy(v).to(dev) for k, v in tgt_scene.as_dict().items()}
        rt = Renderer(tgt_scene.n, views, cfg, device=dev)
        tflat = rt.forward(tparams).clone()
        rt.check()
        targets = [t.reshape(-1).clone() for t in rt.split(tflat)]
        del rt, tparams
        target_src = "rendered by the CUDA path from a second seeded scene (the CPU leg did not run)"
    target = torch.cat(targets)
    pr = {k: params[k].clone() for k in PARAM_KEYS}
    r = Renderer(scene.n, views, cfg, device=dev)
    tuned = autotune(r, pr, backward=True, tiles=(16, 8), batches=(256, 128))
    vp = ViewParallel(scene.n, [[v] for v in views],
                      RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 24,
                                   stage_blocks_per_sm=args.stage_blocks),
                      device=dev)
    vp.set_tile(tuned["tile"], tuned["pixels_per_thread"], tuned["shared_batch"])
    grads = {k: torch.zeros_like(pr[k]) for k in PARAM_KEYS}
    opt = Adam(pr, lr=1e-4)
    total = int(target.numel())
    vp_loss = torch.zeros(1, dtype=torch.float32, device=dev)

    def it_batched():
        for gk in grads.values():
            gk.zero_()
        img = r.forward(pr)
        loss, dimg = l1_loss(img, target)
        r.backward(pr, dimg, grads)
        return loss

    def it_parallel():
        for gk in grads.values():
            gk.zero_()
        vp_loss.zero_()
        vp.step(pr, lambda j, img: l1_loss(img, targets[j], mean_count=total, loss=vp_loss)[1], grads)
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
    best = min(res, key=lambda k: res[k]["ms_per_iter"])
    ms = res[best]["ms_per_iter"]
    step = it_batched if best == "batched_call" else it_parallel

    def it_adam():
        loss = step()
        opt.step(grads)
        return loss

    graph, _ = graph_of(it_adam)
    ms_adam, _ = timed(lambda: graph.replay())
    del graph
    ms_adam = max_over_ranks(ms_adam, world, dev)
    codes = [r.status()[0]] + [g.status()[0] for g in vp.groups]

    # Stages of the 4-view call alone, and the compositors' work counts.
    torch.cuda.nvtx.range_push("train-stages")
    stages = fwd_bwd_stage_ms(r, pr, None, grads, loss=lambda img: l1_loss(img, target)[1])
    torch.cuda.nvtx.range_pop()
    ev, co, evb = compositor_counts(r, pr)
    flops_fwd = FLOPS_PER_EVAL * ev + FLOPS_PER_COMP * co
    flops_bwd = FLOPS_PER_EVAL * evb + FLOPS_PER_BWD_COMP * co
    ach_b = flops_bwd / (stages["render_bwd_composite"] * 1e-3) / 1e12
    ach_f = flops_fwd / (stages["render_fwd"] * 1e-3) / 1e12
    return {"metric": "fwd+bwd iters/s", "value": job_rate(1, world, ms), "unit": "iters/s", "ms_per_iter": ms,
            "form": best,
            "workload": "4 timestamps x 1 camera at 1352x1014, %d Gaussians, L1 loss (mean over the 4 images), "
                        "backward to all parameters; the step replayed as one CUDA graph" % scene.n,
            "targets": target_src,
            "forms": res,
            "with_adam": {"ms_per_iter": ms_adam, "iters_per_s": job_rate(1, world, ms_adam),
                          "step": "the same step followed by fgs4d_adam_update_set (Adam, one launch)"},
            "stages_ms": stages,
            "stages_basis": "the 4-view call alone on the GPU, events between the stages (full-GPU grids)",
            "work": {"alpha_evals": ev, "composited": co, "bwd_alpha_evals": evb},
            "roofline": {"kernel": "render_bwd_kernel (fgs4d_render_bwd_composite)", "bound": "alu",
                         "achieved": ach_b, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach_b / fp32_peak,
                         "traffic": None, "flops_per_launch": flops_bwd,
                         "launch_ms": stages["render_bwd_composite"],
                         "flops_basis": "%d per alpha evaluation up to each pixel's last composited entry + %d per "
                                        "composited (pixel, entry)" % (FLOPS_PER_EVAL, FLOPS_PER_BWD_COMP),
                         "duration_basis": "CUDA events around fgs4d_render_bwd_composite (slot-gradient clear + "
                                           "render_bwd_kernel), the 4-view call alone"},
            "roofline_fwd": {"kernel": "render_fwd_kernel (mode with backward state)", "bound": "alu",
                             "achieved": ach_f, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach_f / fp32_peak,
                             "launch_ms": stages["render_fwd"]},
            "status": fgs4d.status_string(min(codes)), "autotune": tuned}


def tgt_scene_seed() -> int:
    from paper_2412_20720_gb300 import synthetic as sy
    return sy.TARGET_SEED


def bin_sort_bytes(vis: int, inst: int, total_tiles: int) -> float:
    """Algorithmic DRAM bytes of fgs4d_bin_sort: the depth sort's four 8-bit
    passes over the visible pairs (key and value read and written, 16 B), the
    pair scan (52 B read and 52 B written per pair), the emission (8 B per
    instance) and the tile sort's ceil(bits / 8) passes (16 B per instance),
    plus the ranges (8 B per tile)."""
    import math
    passes = max(1, math.ceil(max(1, math.ceil(math.log2(max(total_tiles, 2)))) / 8))
    return vis * (4 * 16 + 104) + inst * (8 + 16 * passes) + 8 * total_tiles


def run_batched(dev, scene, views, label, steps, group, plain=True, tiles=(16,), hbm=6800.0):
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
    # Per-stage times: each group's call alone on the GPU, events between the
    # stages, summed over the groups of a step.
    stages = {}
    torch.cuda.nvtx.range_push("batched-stages")
    for r, dL in zip(rs, dLs):
        for k, v in fwd_bwd_stage_ms(r, params, dL, grads, reps=2).items():
            stages[k] = stages.get(k, 0.0) + v
    torch.cuda.nvtx.range_pop()
    tiles_tot = sum(int(r.layout.total_tiles) for r in rs)
    bs_bytes = bin_sort_bytes(vis_tot, inst_tot, tiles_tot // len(rs)) if rs else 0.0
    bs_gbs = bs_bytes / (stages["bin_sort"] * 1e-3) / 1e9
    out = {"workload": label, "gaussians": n, "views": len(views), "views_per_call": group,
           "resolutions": sorted({"%dx%d" % (v["width"], v["height"]) for v in views}),
           "visible_pairs": vis_tot, "instances": inst_tot, "status": fgs4d.status_string(code),
           "autotune": tuned,
           "graph_batched": {"ms_per_step": graph_ms, "views_per_s": len(views) * 1000.0 / graph_ms,
                             "fwd_bwd_iters_per_s": 1000.0 / graph_ms},
           "stages_ms_per_step": stages,
           "stages_basis": "each call alone on the GPU (full-GPU grids), events between the stages, summed over "
                           "the %d calls of a step" % len(rs),
           "bin_sort_roofline": {"bound": "hbm", "achieved": bs_gbs, "peak": hbm, "unit": "GB/s",
                                 "frac": bs_gbs / hbm, "bytes_per_step": bs_bytes,
                                 "bytes_basis": "bin_sort_bytes(): depth sort, pair scan, emission, tile-sort "
                                                "passes and ranges",
                                 "peak_basis": "measured hbm_gbs"}}
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


def run_extensions(dev, scene_n: int, params: dict, views, fp32_peak: float, hbm: float, reps: int = 3):
    """The rows built beyond the render path, each on the headline scene (one
    1352x1014 view per call, ``views`` of the sweep), timed with CUDA events
    around the launches after the view's preprocess and bin_sort (mean of
    ``reps`` after a warm-up, averaged over the views):

    - auxiliary channels (depth, opacity, flow): fgs4d_render_aux and
      fgs4d_render_aux_bwd against fgs4d_render_fwd / fgs4d_render_bwd;
    - densification statistics: fgs4d_render_bwd with and without them, and
      the 4D split of every Gaussian into 2 children;
    - the Compact-4DGS mask: preprocess with and without the mask, and the
      mask loss over 32M logits;
    - scale-gated features, D = 8 / 16 / 32: the feature compositor and its
      adjoint.

    Compositor rooflines count FP32 flops (FMA = 2) per alpha evaluation and
    per composited (pixel, entry) as the headline does, with the extra
    channels' multiply-adds; the split and the mask loss count their bytes."""
    import numpy as np
    import torch

    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 24)
    r = Renderer(scene_n, views[:1], cfg, device=dev)
    vv = [fgs4d.make_views([v]) for v in views]
    ws, wsb = r.ws.data_ptr(), r.ws_bytes
    g = r.gaussians(params)
    gen = torch.Generator(device="cpu").manual_seed(7)
    mask_logit = (torch.randn(scene_n, generator=gen) + 2.0).to(dev)
    gm = r.gaussians({**params, "mask_logit": mask_logit})
    grads = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS}
    gg = r._grads(grads, None)
    dens = torch.zeros(scene_n, 4, dtype=torch.float32, device=dev)
    ggd = r._grads(grads, dens)
    npx = r.total_pixels
    rgb = torch.empty(3 * npx, dtype=torch.float32, device=dev)
    aux = torch.empty(4 * npx, dtype=torch.float32, device=dev)
    dL = torch.randn(3 * npx, generator=gen).to(dev) * 1e-3
    dA = torch.cat([torch.randn(2 * npx, generator=gen), torch.zeros(2 * npx)]).to(dev) * 1e-3
    feats = {D: torch.randn(scene_n, D, generator=gen).to(dev) for D in (8, 16, 32)}
    gates = {D: torch.rand(D, generator=gen).to(dev) for D in (8, 16, 32)}
    fout = {D: torch.empty(D * npx, dtype=torch.float32, device=dev) for D in (8, 16, 32)}
    fdl = {D: (torch.randn(D * npx, generator=gen) * 1e-3).to(dev) for D in (8, 16, 32)}
    fgrad = {D: torch.zeros(scene_n, D, dtype=torch.float32, device=dev) for D in (8, 16, 32)}
    ggate = {D: torch.zeros(D, dtype=torch.float32, device=dev) for D in (8, 16, 32)}

    def t_ms(fn):
        fn()
        acc = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            acc += a.elapsed_time(b)
        return acc / reps

    names = ["fwd", "bwd", "aux", "aux_bwd", "bwd_densify", "pre", "pre_mask"] + \
        ["feat%d" % D for D in (8, 16, 32)] + ["feat%d_bwd" % D for D in (8, 16, 32)]
    ms = {k: [] for k in names}
    work = {"evals": [], "comps": [], "evals_bwd": []}
    for v, n1 in vv:
        def prep(gx=g):
            fgs4d.preprocess(gx, v, n1, r.settings, ws, wsb, st)
        def sort():
            fgs4d.bin_sort(r.n, v, n1, r.settings, ws, wsb, st)
        stats = torch.zeros(3, dtype=torch.int64, device=dev)
        prep()
        sort()
        fgs4d.render_stats(r.n, v, n1, r.settings, ws, wsb, rgb.data_ptr(), stats.data_ptr(), st)
        ev, co, evb = (int(x) for x in stats.tolist())
        work["evals"].append(ev)
        work["comps"].append(co)
        work["evals_bwd"].append(evb)
        ms["pre"].append(t_ms(prep))
        ms["pre_mask"].append(t_ms(lambda: prep(gm)))
        prep()
        sort()
        ms["aux"].append(t_ms(lambda: fgs4d.render_aux(g, v, n1, r.settings, ws, wsb, 0.01, rgb.data_ptr(), None,
                                                       aux.data_ptr(), st)))
        ms["aux_bwd"].append(t_ms(lambda: fgs4d.render_aux_bwd(g, v, n1, r.settings, ws, wsb, dL.data_ptr(),
                                                               dA.data_ptr(), gg, st)))
        ms["fwd"].append(t_ms(lambda: fgs4d.render_fwd(r.n, v, n1, r.settings, ws, wsb, rgb.data_ptr(), None, st)))
        ms["bwd"].append(t_ms(lambda: fgs4d.render_bwd(g, v, n1, r.settings, ws, wsb, dL.data_ptr(), gg, st)))
        ms["bwd_densify"].append(t_ms(lambda: fgs4d.render_bwd(g, v, n1, r.settings, ws, wsb, dL.data_ptr(), ggd,
                                                               st)))
        for D in (8, 16, 32):
            ms["feat%d" % D].append(t_ms(lambda: fgs4d.render_features(
                r.n, v, n1, r.settings, ws, wsb, feats[D].data_ptr(), D, gates[D].data_ptr(), fout[D].data_ptr(),
                st)))
            ms["feat%d_bwd" % D].append(t_ms(lambda: fgs4d.render_features_bwd(
                r.n, v, n1, r.settings, ws, wsb, feats[D].data_ptr(), D, gates[D].data_ptr(), fdl[D].data_ptr(),
                fgrad[D].data_ptr(), ggate[D].data_ptr(), st)))
    code, _ = r.status()
    m = {k: float(np.mean(x)) for k, x in ms.items()}
    ev, co, evb = (float(np.mean(work[k])) for k in ("evals", "comps", "evals_bwd"))

    def alu(flops, t):
        return {"bound": "alu", "achieved": flops / t / 1e9, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": flops / t / 1e9 / fp32_peak, "flops_per_launch": flops, "launch_ms": t}

    # Split: every Gaussian into 2 children (0.59 GB moved); mask loss over
    # 32M logits (384 MB: larger than L2, as at the paper's largest scenes
    # with several times their Gaussians between prunings).
    nsplit, kids = scene_n, 2
    idx = torch.randperm(scene_n, generator=gen)[:nsplit].to(torch.int32).to(dev)
    eps = torch.randn(nsplit, kids, 4, generator=gen).to(dev)
    src = fgs4d.make_gaussians({k: params[k].data_ptr() for k in PARAM_KEYS}, scene_n)
    outs = {k: torch.empty((nsplit * kids,) + tuple(params[k].shape[1:]), dtype=torch.float32, device=dev)
            for k in PARAM_KEYS}
    dst = fgs4d.GaussiansOut(*(outs[k].data_ptr() for k in PARAM_KEYS), nsplit * kids)
    split_ms = t_ms(lambda: fgs4d.split_gaussians(src, idx.data_ptr(), nsplit, kids, eps.data_ptr(), 1.6,
                                                  r.settings, dst, st))
    row = sum(int(np.prod(params[k].shape[1:])) * 4 for k in PARAM_KEYS)  # bytes of one Gaussian's parameters
    split_bytes = nsplit * (4 + row) + nsplit * kids * (16 + row)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    n_mask = 32 << 20
    big_logit = torch.randn(n_mask, generator=gen).to(dev)
    mgrad = torch.zeros(n_mask, dtype=torch.float32, device=dev)
    mloss_ms = t_ms(lambda: fgs4d.mask_loss(big_logit.data_ptr(), n_mask, loss.data_ptr(), mgrad.data_ptr(), st))
    mloss_bytes = 12.0 * n_mask

    def hbm_line(b, t):
        return {"bound": "hbm", "achieved": b / t / 1e6, "peak": hbm, "unit": "GB/s", "frac": b / t / 1e6 / hbm,
                "bytes_per_launch": b, "launch_ms": t}

    aux_extra = 6  # depth and the two flow channels: three multiply-adds per composited entry
    out = {
        "workload": "%s, %d views of the sweep, one view per call" % (WORKLOAD, len(views)),
        "status": fgs4d.status_string(code),
        "basis": "CUDA events around each launch after the view's preprocess and bin_sort, mean of %d runs after a "
                 "warm-up, averaged over the views" % reps,
        "work_per_view": {"alpha_evals": ev, "composited": co, "alpha_evals_bwd": evb},
        "aux_channels": {
            "render_aux_ms": m["aux"], "render_fwd_ms": m["fwd"], "render_aux_bwd_ms": m["aux_bwd"],
            "render_bwd_ms": m["bwd"],
            "roofline": alu(FLOPS_PER_EVAL * ev + (FLOPS_PER_COMP + aux_extra) * co, m["aux"]),
            "roofline_bwd": alu(FLOPS_PER_EVAL * evb + (FLOPS_PER_BWD_COMP + 6) * co, m["aux_bwd"]),
            "flops_basis": "forward: %d per evaluation, %d per composited entry (colour + depth + flow); backward: "
                           "%d per evaluation up to the last composited entry, %d per composited entry"
                           % (FLOPS_PER_EVAL, FLOPS_PER_COMP + aux_extra, FLOPS_PER_EVAL, FLOPS_PER_BWD_COMP + 6)},
        "densify": {
            "render_bwd_ms": m["bwd"], "render_bwd_with_stats_ms": m["bwd_densify"],
            "overhead": m["bwd_densify"] / m["bwd"] - 1.0,
            "split": {"parents": nsplit, "children_per_parent": kids, "ms": split_ms,
                      "roofline": hbm_line(split_bytes, split_ms),
                      "bytes_basis": "index and parameter row of each parent read, one 4D draw read and one "
                                     "parameter row written per child (%d B a row)" % row}},
        "mask": {
            "preprocess_ms": m["pre"], "preprocess_with_mask_ms": m["pre_mask"],
            "overhead": m["pre_mask"] / m["pre"] - 1.0,
            "mask_loss": {"gaussians": n_mask, "ms": mloss_ms, "roofline": hbm_line(mloss_bytes, mloss_ms),
                          "bytes_basis": "mask logit read, gradient read and written (12 B per Gaussian)"}},
        "features": {},
    }
    for D in (8, 16, 32):
        out["features"]["D%d" % D] = {
            "render_features_ms": m["feat%d" % D], "render_features_bwd_ms": m["feat%d_bwd" % D],
            "roofline": alu(FLOPS_PER_EVAL * ev + (4 + 2 * D) * co, m["feat%d" % D]),
            "roofline_bwd": alu(FLOPS_PER_EVAL * ev + (4 + 2 * D) * co, m["feat%d_bwd" % D]),
            "flops_basis": "%d per evaluation, 4 + 2 D per composited entry (T alpha, T - T alpha, D multiply-adds; "
                           "the adjoint: D multiply-adds into the per-entry sums)" % FLOPS_PER_EVAL}
    return out


def run_tiny(dev, frames: int = 400):
    """C0: 2,000 Gaussians (degree 1 x order 1), one 128x96 view per call,
    preprocess + bin_sort + render_image; frames/s over ``frames`` calls
    (one frame in flight), after a warm-up."""
    import torch

    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer
    sc = sy.tiny_scene()
    params = {k: torch.from_numpy(v).to(dev) for k, v in sc.as_dict().items()}
    views = [sy.tiny_view(128, 96, t=k / (frames - 1)) for k in range(frames)]
    r = Renderer(sc.n, views[:1], RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 18), device=dev)
    vv = [fgs4d.make_views([v]) for v in views]
    g = r.gaussians({k: params[k] for k in PARAM_KEYS})
    out = torch.empty(3 * 128 * 96, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream

    def sweep():
        for v, n1 in vv:
            fgs4d.preprocess(g, v, n1, r.settings, r.ws.data_ptr(), r.ws_bytes, st)
            fgs4d.bin_sort(sc.n, v, n1, r.settings, r.ws.data_ptr(), r.ws_bytes, st)
            fgs4d.render_image(sc.n, v, n1, r.settings, r.ws.data_ptr(), r.ws_bytes, out.data_ptr(), None, st)

    sweep()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sweep()
    b.record(stream)
    torch.cuda.synchronize()
    code, _ = r.status()
    ms = a.elapsed_time(b)
    return {"workload": "tiny-2k-128x96 (2,000 Gaussians, SH degree 1 x order 1)", "frames_per_s": frames / ms * 1e3,
            "ms_per_frame": ms / frames, "frames": frames, "status": fgs4d.status_string(code),
            "basis": "one view per call, one frame in flight, CUDA events around %d calls" % frames}


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
            "cpu_baseline": {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                             "host_cpus": os.cpu_count(),
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
