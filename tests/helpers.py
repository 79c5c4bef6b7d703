"""Shared helpers of the parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded FP32 inputs.

Discrete decisions (cull flags, the integer radius, tile-rect edges, the
1/255 skip, the 1e-4 stop, the depth order) are taken in FP32 by the kernels
and in FP64 by the oracle.  No input is removed and no pixel is left out:

- Per Gaussian, the oracle marks every decision within RELAX (relative) of
  its threshold (orc_preprocess_relaxed); the GPU may take either outcome
  there, and its records must lie within the bounds both outcomes allow.
- Per pixel, the oracle returns every result an FP32 renderer may produce
  whose per-pixel inputs lie within TOL of the FP64 values
  (orc_render_pixels_admissible); the bounds in TOL are the record
  tolerances that check_records verifies on the same run.  Every pixel must
  match one of its admissible results within IMAGE_ATOL.
- Gradients are compared for a loss whose image gradient is zero at the
  pixels where some decision (or the derivative of the 0.99 clamp or of the
  colour clamp) has more than one admissible outcome; there both sides
  differentiate the same discrete structure.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer

IMAGE_ATOL = 2e-4
# Per-Gaussian decisions: relative window of the cull thresholds, the radius
# and the rect edges (the FP32 error of those quantities is ~1e-6 relative).
RELAX = 2e-5
# Per-pixel inputs: the record tolerances of check_records (the conic's
# factors u11, u22 to 3e-5 relative and u12 to 3e-5 (|u12| + sqrt(Q11)),
# centre 1e-6 relative + 2e-7 of the largest coordinate, opacity 1e-5
# relative), ex2.approx and rounding (1e-6), depth keys within 2 ulp.
UV_TOL = (1e-6, 2e-7)
TOL = oracle.Tolerance(eps_conic=3e-5, eps_uv=UV_TOL[0], eps_a=1e-5, eps_alpha=1e-6, depth_ulps=2)


def pixel_tolerance(pr) -> oracle.Tolerance:
    """TOL with the centre's absolute floor of this projection: 2e-7 of the
    largest |u|, |v| among the Gaussians the oracle keeps or may keep."""
    alive = (pr["status"] == 0) | ((pr["uncertain"] & 1) > 0)
    big = float(np.abs(pr["uv"][alive]).max()) if alive.any() else 0.0
    return oracle.Tolerance(**{**TOL.__dict__, "eps_uv_abs": UV_TOL[1] * big})


def f32(x: float) -> float:
    return float(np.float32(x))


def oracle_settings(cfg: RenderConfig) -> oracle.Settings:
    """The oracle sees the FP32 values of the settings the GPU gets."""
    return oracle.Settings(sh_degree=cfg.sh_degree, t_order=cfg.t_order, tile=cfg.tile, period=f32(cfg.period),
                           near_plane=f32(cfg.near_plane), dilation=f32(cfg.dilation), p_t_min=f32(cfg.p_t_min),
                           bg=tuple(f32(b) for b in cfg.bg))


def subset(params: dict, mask) -> dict:
    return {k: np.ascontiguousarray(v[mask]) for k, v in params.items()}


def to_device(params: dict):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(params[k], dtype=np.float32)).cuda() for k in PARAM_KEYS}


class CudaRender:
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


def records_from_gpu(run: CudaRender):
    """Decode the GPU's per-slot records into oracle units.  The record
    holds the base-2 exponent's factors (a1, b1, b2): q2 = (a1 dx)^2 + (b1 dx
    + b2 dy)^2 = (1/2) log2(e) d^T Q d; "factor" is (u11, u12, u22) of the
    natural-log conic Q = U U^T, "conic" is Q = (A, B, C)."""
    L2E = 1.4426950408889634
    g, c = run.geom.astype(np.float64), run.color.astype(np.float64)
    sk = np.sqrt(0.5 * L2E)
    factor = np.stack([g[:, 2] / sk, g[:, 3] / sk, c[:, 0] / sk], axis=1)
    conic = np.stack([factor[:, 0] ** 2 + factor[:, 1] ** 2, factor[:, 1] * factor[:, 2], factor[:, 2] ** 2], axis=1)
    rect = np.stack([run.meta[:, 2] & 0xFFFF, run.meta[:, 2] >> 16, run.meta[:, 3] & 0xFFFF, run.meta[:, 3] >> 16],
                    axis=1)
    rgb = np.stack([c[:, 2], c[:, 3], run.blue.astype(np.float64)], axis=1)
    return {"index": run.meta[:, 0], "view": run.meta[:, 1], "uv": g[:, :2], "conic": conic, "factor": factor,
            "a": np.exp2(c[:, 1]),
            "rgb": rgb, "rect": rect, "depth_bits": run.depth_bits, "tau": run.tau.astype(np.float64)}


# Gradients of two runs that differ only in the order of the FP32 atomic sums:
# such sums differ by up to n eps sum|term|, far above eps |sum| where the
# terms cancel (a log-scale gradient at 3% of the largest one was seen 5.5e-5
# apart in relative terms).
ORDER_RTOL, ORDER_FLOOR = 1e-4, 1e-5


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


def oracle_factor(conic):
    """(u11, u12, u22) of the conic Q = U U^T (U upper triangular), and the
    floor sqrt(Q11) of u12's error."""
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    u22 = np.sqrt(C)
    return np.stack([np.sqrt(np.maximum(A * C - B * B, 0) / C), B / u22, u22], axis=1), np.sqrt(A)


def oracle_proj(params, view, cfg: RenderConfig):
    """The oracle's per-Gaussian chain with its decisions relaxed by RELAX."""
    return oracle.preprocess(params, view, oracle_settings(cfg), relax=RELAX)


def view_records(run, k: int):
    """The GPU records of view k (slots are in (view, Gaussian) order)."""
    rec = records_from_gpu(run)
    sel = rec["view"] == k
    return {key: val[sel] for key, val in rec.items()}


def check_records(run, params, view, cfg, k: int = 0, sample=None):
    """Per-slot records of view k against the relaxed oracle: the GPU's
    visible set holds every Gaussian the oracle keeps for certain and only
    Gaussians it keeps or may keep; each rect lies between rect_lo and
    rect_hi; values within the record tolerances (those of TOL).  Returns
    the oracle projection."""
    pr = oracle_proj(params, view, cfg)
    unc = (pr["uncertain"] & 1) > 0
    certain = np.flatnonzero((pr["status"] == 0) & ~unc)
    allowed = (pr["status"] == 0) | unc
    rec = view_records(run, k)
    idx = rec["index"]
    assert np.all(np.diff(idx) > 0)
    assert np.all(allowed[idx]), "GPU keeps Gaussians the oracle culls for certain: %s" % idx[~allowed[idx]][:10]
    missing = np.setdiff1d(certain, idx)
    assert missing.size == 0, "GPU culls Gaussians the oracle keeps for certain: %s" % missing[:10]
    sel = np.arange(idx.size) if sample is None else sample
    i = idx[sel]
    r = rec["rect"][sel]
    hi, lo = pr["rect_hi"][i], pr["rect_lo"][i]
    assert np.all(hi[:, :2] <= r[:, :2]) and np.all(r[:, 2:] <= hi[:, 2:])
    cert = ~unc[i]
    assert np.all(r[cert, :2] <= lo[cert, :2]) and np.all(lo[cert, 2:] <= r[cert, 2:])
    compare_group("uv", rec["uv"][sel], pr["uv"][i], *UV_TOL)
    fac, floor = oracle_factor(pr["conic"][i])
    gf = rec["factor"][sel]
    for j, bound in ((0, fac[:, 0]), (1, np.abs(fac[:, 1]) + floor), (2, fac[:, 2])):
        ratio = np.abs(gf[:, j] - fac[:, j]) / (TOL.eps_conic * bound)
        w = int(np.argmax(ratio))
        assert ratio[w] <= 1.0, "factor %d of Gaussian %d: gpu %r oracle %r (%.3g of the bound)" % (
            j, i[w], gf[w, j], fac[w, j], ratio[w])
    compare_group("a", rec["a"][sel], pr["a_eff"][i], TOL.eps_a, 1e-7)
    compare_group("rgb", rec["rgb"][sel], pr["rgb"][i], 1e-5, 1e-6)
    compare_group("tau", rec["tau"][sel], np.log2(255.0 * pr["a_eff"][i]) + 4e-3, 1e-5, 1e-6)
    db = rec["depth_bits"][sel].astype(np.int64) - pr["depth_f32"][i].view(np.uint32).astype(np.int64)
    # The FP32 depth comes out of a longer rounded chain than the FP64
    # oracle's rounded depth: within depth_ulps, mostly equal.
    assert np.abs(db).max() <= TOL.depth_ulps
    assert (db == 0).mean() >= 0.8
    return pr


def match_admissible(cands, rgb, T):
    """Index of the admissible result closest to the GPU's (rgb [P, 3], T [P])
    and the distance max(|rgb - c|, |T - c_T|) to it, per pixel."""
    P = len(cands)
    kmax = max(c.shape[0] for c in cands)
    pad = np.full((P, kmax, 4), np.nan)
    for q, c in enumerate(cands):
        pad[q, :c.shape[0]] = c[:, :4]
    got = np.concatenate([rgb, T[:, None]], axis=1)
    d = np.nanmax(np.abs(pad - got[:, None, :]), axis=2)
    d = np.where(np.isnan(d), np.inf, d)
    best = np.argmin(d, axis=1)
    return best, d[np.arange(P), best]


def check_pixels(pr, view, cfg, pix, rgb, T, last=None, extra=None):
    """GPU values at pixels ``pix`` (rgb [P, 3], T [P], optional contributor
    positions [P]) against the oracle's admissible results.  Returns the
    oracle's flags [P] (see render_pixels_admissible) and the matched
    candidates [P, 5 + E]."""
    cands, flags = oracle.render_pixels_admissible(pr, view, oracle_settings(cfg), pix, pixel_tolerance(pr),
                                                   extra=extra)
    assert not (flags & 4).any(), "admissible walk ran out of budget at %d pixels" % int((flags & 4).sum())
    best, dist = match_admissible(cands, np.asarray(rgb, np.float64), np.asarray(T, np.float64))
    worst = int(np.argmax(dist))
    assert dist[worst] <= IMAGE_ATOL, ("pixel %d: gpu rgb %s T %r, admissible %s" %
                                       (int(pix[worst]), rgb[worst], T[worst], cands[worst][:, :4]))
    chosen = np.stack([cands[q][best[q]] for q in range(len(cands))])
    if last is not None:
        # the GPU counts positions in its own (shortened) lists: compare
        # whether anything was composited
        assert np.all((np.asarray(last) == 0) == (chosen[:, 4] == 0))
    return flags, chosen


def check_image(run, params, view, cfg, k: int = 0, pr=None):
    """Every pixel of view k against the oracle's admissible results.
    Returns (oracle projection, flags [H, W])."""
    if pr is None:
        pr = oracle_proj(params, view, cfg)
    H, W = int(view["height"]), int(view["width"])
    Tg, lastg = run.pixel_planes(k)
    pix = np.arange(W * H)
    flags, _ = check_pixels(pr, view, cfg, pix, run.images[k].reshape(3, -1).T, Tg.reshape(-1), lastg.reshape(-1))
    return pr, flags.reshape(H, W)


def oracle_flags(pr, view, cfg, pix=None):
    """The oracle's admissibility flags (render_pixels_admissible) at pixels
    ``pix`` (default: every pixel, returned as [H, W])."""
    H, W = int(view["height"]), int(view["width"])
    allpix = pix is None
    pix = np.arange(W * H) if allpix else pix
    _, flags = oracle.render_pixels_admissible(pr, view, oracle_settings(cfg), pix, pixel_tolerance(pr))
    assert not (flags & 4).any()
    return flags.reshape(H, W) if allpix else flags


def loss_gradient_at_settled_pixels(rng, flags, shape):
    """A random image gradient that is zero where a decision or a derivative
    is unsettled (flags & 3): the loss both sides differentiate."""
    return rng.standard_normal(shape) * ((flags & 3) == 0)


def canonical_ranges(gr):
    """Tile ranges as [start, end) with empty tiles as (0, 0): the library may
    leave any start >= end in a tile without instances."""
    import numpy as np
    gr = np.array(gr, dtype=np.int64).reshape(-1, 2) & 0xFFFFFFFF
    out = gr.copy()
    out[gr[:, 0] >= gr[:, 1]] = 0
    return out
