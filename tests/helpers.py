"""Shared helpers of the parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded FP32 inputs.

Discrete decisions (cull flags, the integer radius, tile-rect edges) are taken
in FP32 by the kernels and in FP64 by the oracle.  Gaussians whose decision
lies within a relative 1e-5 of its threshold in the oracle are removed from
the input before BOTH sides run, so both sides take the same decisions on the
rest.  Per-pixel decisions (alpha skip, clamp, transmittance stop, depth
order within 2 ulp) are flagged by the oracle's pixel margin; pixels with a
margin below 1e-3 are left out of element-wise comparisons (and their loss
gradient is set to zero), and their share is bounded by each test.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer

GAUSS_MARGIN = 1e-5
PIXEL_MARGIN = 1e-3


def f32(x: float) -> float:
    return float(np.float32(x))


def oracle_settings(cfg: RenderConfig) -> oracle.Settings:
    """The oracle sees the FP32 values of the settings the GPU gets."""
    return oracle.Settings(sh_degree=cfg.sh_degree, t_order=cfg.t_order, tile=cfg.tile, period=f32(cfg.period),
                           near_plane=f32(cfg.near_plane), dilation=f32(cfg.dilation), p_t_min=f32(cfg.p_t_min),
                           bg=tuple(f32(b) for b in cfg.bg))


def keep_clear_of_boundaries(params: dict, views, cfg: RenderConfig) -> np.ndarray:
    """Boolean mask of the Gaussians whose discrete decisions are clear of
    their thresholds in every view."""
    st = oracle_settings(cfg)
    keep = np.ones(params["mean"].shape[0], dtype=bool)
    for v in views:
        pr = oracle.preprocess(params, v, st)
        keep &= pr["margin"] >= GAUSS_MARGIN
    return keep


def subset(params: dict, mask) -> dict:
    return {k: np.ascontiguousarray(v[mask]) for k, v in params.items()}


def to_device(params: dict):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(params[k], dtype=np.float32)).cuda() for k in PARAM_KEYS}


class GpuRun:
    """One forward through the C ABI, with the documented workspace regions
    read back."""

    def __init__(self, params: dict, views, cfg: RenderConfig):
        import torch
        self.params = to_device(params)
        self.n = params["mean"].shape[0]
        self.renderer = Renderer(self.n, views, cfg)
        self.flat = self.renderer.forward(self.params)
        self.counts = self.renderer.check()
        torch.cuda.synchronize()
        r = self.renderer
        self.images = [x.cpu().numpy() for x in r.split(self.flat)]
        tp = r.total_pixels
        self.T = r.workspace_view(r.layout.pix_T, torch.float32, tp).cpu().numpy()
        self.last = r.workspace_view(r.layout.pix_last, torch.int32, tp).cpu().numpy()
        nv = self.counts[0]
        self.geom = r.workspace_view(r.layout.rec_geom, torch.float32, 4 * nv).cpu().numpy().reshape(nv, 4)
        self.color = r.workspace_view(r.layout.rec_color, torch.float32, 4 * nv).cpu().numpy().reshape(nv, 4)
        self.blue = r.workspace_view(r.layout.rec_blue, torch.float32, nv).cpu().numpy()
        self.tau = r.workspace_view(r.layout.rec_tau, torch.float32, nv).cpu().numpy()
        self.meta = r.workspace_view(r.layout.rec_meta, torch.int32, 4 * nv).cpu().numpy().reshape(nv, 4)
        self.depth_bits = r.workspace_view(r.layout.depth_key, torch.int32, nv).cpu().numpy().view(np.uint32)

    def pixel_planes(self, view_index: int):
        """Per-pixel T and last for one view as [H, W] arrays."""
        off = 0
        for k, (h, w) in enumerate(self.renderer.sizes):
            if k == view_index:
                return self.T[off:off + h * w].reshape(h, w), self.last[off:off + h * w].reshape(h, w)
            off += h * w
        raise IndexError(view_index)

    def backward(self, dimgs):
        """dimgs: list of [3, H, W] per view.  Returns (param grads, slot grads)."""
        import torch
        flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dimgs]).astype(np.float32)).cuda()
        grads = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.renderer.backward(self.params, flat, grads)
        self.renderer.check()
        r = self.renderer
        nv = self.counts[0]
        slot = r.workspace_view(r.layout.slot_grad, torch.float32, 12 * nv).cpu().numpy().reshape(nv, 12)
        return {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}, slot


def records_from_gpu(run: GpuRun):
    """Decode the GPU's per-slot records into oracle units."""
    L2E = 1.4426950408889634
    g, c = run.geom.astype(np.float64), run.color.astype(np.float64)
    conic = np.stack([2 * g[:, 2] / L2E, g[:, 3] / L2E, 2 * c[:, 0] / L2E], axis=1)
    rect = np.stack([run.meta[:, 2] & 0xFFFF, run.meta[:, 2] >> 16, run.meta[:, 3] & 0xFFFF, run.meta[:, 3] >> 16],
                    axis=1)
    rgb = np.stack([c[:, 2], c[:, 3], run.blue.astype(np.float64)], axis=1)
    return {"index": run.meta[:, 0], "view": run.meta[:, 1], "uv": g[:, :2], "conic": conic, "a": np.exp2(c[:, 1]),
            "rgb": rgb, "rect": rect, "depth_bits": run.depth_bits, "tau": run.tau.astype(np.float64)}


def compare_group(name, gpu, ref, rtol, floor_frac):
    """|gpu - ref| <= rtol |ref| + floor_frac max|ref| element-wise; returns the
    worst ratio error / bound (must be <= 1)."""
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    bound = rtol * np.abs(ref) + floor_frac * max(np.abs(ref).max(), 1e-30)
    ratio = np.abs(gpu - ref) / bound
    worst = int(np.argmax(ratio))
    assert ratio[worst] <= 1.0, "%s: gpu %r vs oracle %r at %d (ratio %.3g)" % (name, gpu[worst], ref[worst], worst,
                                                                               ratio[worst])
    return float(ratio.max())


def canonical_ranges(gr):
    """Tile ranges as [start, end) with empty tiles as (0, 0): the library may
    leave any start >= end in a tile without instances."""
    import numpy as np
    gr = np.array(gr, dtype=np.int64).reshape(-1, 2) & 0xFFFFFFFF
    out = gr.copy()
    out[gr[:, 0] >= gr[:, 1]] = 0
    return out
