"""PyTorch glue over the fgs4d C ABI: device memory, streams and autograd.

Every step of the render path (preprocess, binning, sort, compositing and
their adjoints) runs in libfgs4d.so; this module only allocates buffers,
passes pointers and the current CUDA stream, and wires the backward pass
into ``torch.autograd``.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import fgs4d

PARAM_KEYS = ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")


@dataclass
class RenderConfig:
    sh_degree: int = 3
    t_order: int = 2
    period: float = 1.0
    near_plane: float = 0.2
    dilation: float = 0.3
    p_t_min: float = 0.05
    bg: tuple = (0.0, 0.0, 0.0)
    vis_capacity: int = 0
    inst_capacity: int = 1 << 22
    pixels_per_thread: int = 0  # compositor block shape (0 = library default); see autotune()
    tile: int = 16  # tile edge in pixels, 16 or 8; see autotune()
    shared_batch: int = 0  # records staged per shared-memory batch, 128 or 256 (0 = 256); see autotune()
    mask_threshold: float = 0.03  # epsilon of the Compact-4DGS mask (Sec. 8.3.2 runs it at 0.03); used with "mask_logit"
    # Grids of the latency-bound stages: 0 = full-GPU grids (lowest latency for one frame alone);
    # k = at most k resident blocks per SM, which leaves SMs to frames or views rendered concurrently
    # (FramePipeline, ViewParallel).  Results are identical.
    stage_blocks_per_sm: int = 0

    def settings(self) -> fgs4d.Settings:
        return fgs4d.make_settings(self.sh_degree, self.t_order, self.period, self.near_plane, self.dilation,
                                   self.p_t_min, self.bg, self.vis_capacity, self.inst_capacity,
                                   self.pixels_per_thread, self.tile, self.shared_batch, self.stage_blocks_per_sm)


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _check_param(name, t, n, device):
    if not isinstance(t, torch.Tensor) or t.device != device or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float32 tensor on %s" % (name, device))
    if t.shape[0] != n:
        raise ValueError("%s has %d rows, expected %d" % (name, t.shape[0], n))


class Renderer:
    """Renders N Gaussians into a fixed set of views.  One workspace carries a
    forward to its backward, so keep one forward/backward pair in flight per
    renderer (use separate renderers for overlapping work)."""

    def __init__(self, n: int, views, config: RenderConfig, device=None):
        fgs4d.load()
        dev = torch.device(device if device is not None else "cuda")
        if dev.type != "cuda":
            raise ValueError("the fgs4d render path runs on CUDA devices only")
        self.device = torch.device("cuda", dev.index if dev.index is not None else torch.cuda.current_device())
        self.n = int(n)
        self.config = config
        self.settings = config.settings()
        self.view_dicts = list(views)
        self.views, self.nviews = fgs4d.make_views(self.view_dicts)
        self.sizes = [(int(v["height"]), int(v["width"])) for v in self.view_dicts]
        self._allocate()

    def _allocate(self):
        self.ws_bytes = fgs4d.workspace_size(self.settings, self.n, self.views, self.nviews)
        self.layout = fgs4d.workspace_layout(self.settings, self.n, self.views, self.nviews)
        # 256-byte aligned device workspace.
        self._ws_raw = None
        self._ws_raw = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self._ws_raw.data_ptr()) % 256
        self.ws = self._ws_raw[off:off + self.ws_bytes]
        self.total_pixels = int(self.layout.total_pixels)

    def set_tile(self, tile: int, pixels_per_thread: int = 0, shared_batch: int = 0):
        """Switches the tile edge (16 or 8), the compositor block shape and its
        shared-memory batch size; a new tile edge re-lays out (and
        reallocates) the workspace."""
        self.settings.pixels_per_thread = int(pixels_per_thread)
        self.settings.shared_batch = int(shared_batch)
        if int(tile) != int(self.settings.tile):
            self.settings.tile = int(tile)
            self._allocate()

    def fit_visible_capacity(self, params: dict, view_sets=None, margin: float = 1.1) -> int:
        """Sizes the visible-pair capacity to the caller's own views: runs
        preprocess for every (views, nviews) set of ``view_sets`` (default:
        the renderer's views), takes the largest visible count, adds
        ``margin`` and rounds up to a multiple of 1024, then re-lays out the
        workspace (the depth sort and pair scan size their grids by the
        capacity).  A later view with more visible pairs reports a capacity
        overflow (status) and needs a larger capacity.  Returns the
        capacity."""
        g = self.gaussians(params)
        st = self.stream()
        view_sets = view_sets or [(self.views, self.nviews)]
        need = 0
        for views, nv in view_sets:
            fgs4d.preprocess(g, views, nv, self.settings, _ptr(self.ws), self.ws_bytes, st)
            code, counts = self.status()
            if code not in (fgs4d.OK, fgs4d.ERR_CAPACITY):
                raise fgs4d.Fgs4dError(code, "fit_visible_capacity")
            need = max(need, int(counts[0]), int(counts[2]))
        cap = max(1024, -(-int(need * margin) // 1024) * 1024)
        self.settings.vis_capacity = cap
        self.config.vis_capacity = cap
        self._allocate()
        return cap

    # ---------------------------------------------------------------- plumbing
    def stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def gaussians(self, params: dict) -> fgs4d.Gaussians:
        for k in PARAM_KEYS:
            _check_param(k, params[k], self.n, self.device)
        mask = params.get("mask_logit")
        if mask is not None:
            _check_param("mask_logit", mask, self.n, self.device)
        return fgs4d.make_gaussians({k: _ptr(params[k]) for k in PARAM_KEYS}, self.n,
                                    _ptr(mask) if mask is not None else 0, self.config.mask_threshold)

    def split(self, flat: torch.Tensor, channels: int = 3) -> list:
        """Flat [sum C H W] planar buffer -> list of [C, H, W] views."""
        out, off = [], 0
        for h, w in self.sizes:
            out.append(flat[off:off + channels * h * w].view(channels, h, w))
            off += channels * h * w
        return out

    # ------------------------------------------------------------------ calls
    def forward(self, params: dict, out_rgb: torch.Tensor | None = None, out_T: torch.Tensor | None = None):
        """Runs preprocess, bin_sort and render_fwd; returns the flat RGB buffer."""
        g = self.gaussians(params)
        if out_rgb is None:
            out_rgb = torch.empty(3 * self.total_pixels, dtype=torch.float32, device=self.device)
        st = self.stream()
        ws = _ptr(self.ws)
        fgs4d.preprocess(g, self.views, self.nviews, self.settings, ws, self.ws_bytes, st)
        fgs4d.bin_sort(self.n, self.views, self.nviews, self.settings, ws, self.ws_bytes, st)
        fgs4d.render_fwd(self.n, self.views, self.nviews, self.settings, ws, self.ws_bytes, _ptr(out_rgb),
                         _ptr(out_T) if out_T is not None else None, st)
        return out_rgb

    def forward_aux(self, params: dict, flow_dt: float, out_rgb: torch.Tensor | None = None,
                    out_aux: torch.Tensor | None = None):
        """Like forward, plus the auxiliary planes: returns (rgb, aux) with aux
        flat [sum_v 4 H W], per view (depth, opacity, flow_u, flow_v)."""
        g = self.gaussians(params)
        if out_rgb is None:
            out_rgb = torch.empty(3 * self.total_pixels, dtype=torch.float32, device=self.device)
        if out_aux is None:
            out_aux = torch.empty(4 * self.total_pixels, dtype=torch.float32, device=self.device)
        st = self.stream()
        ws = _ptr(self.ws)
        fgs4d.preprocess(g, self.views, self.nviews, self.settings, ws, self.ws_bytes, st)
        fgs4d.bin_sort(self.n, self.views, self.nviews, self.settings, ws, self.ws_bytes, st)
        fgs4d.render_aux(g, self.views, self.nviews, self.settings, ws, self.ws_bytes, flow_dt, _ptr(out_rgb), None,
                         _ptr(out_aux), st)
        return out_rgb, out_aux

    def _grads(self, grads: dict, densify_stats):
        for k in PARAM_KEYS:
            _check_param("grad " + k, grads[k], self.n, self.device)
        ptrs = {k: _ptr(grads[k]) for k in PARAM_KEYS}
        if grads.get("mask_logit") is not None:
            _check_param("grad mask_logit", grads["mask_logit"], self.n, self.device)
            ptrs["mask_logit"] = _ptr(grads["mask_logit"])
        if densify_stats is not None:
            if (densify_stats.dtype != torch.float32 or tuple(densify_stats.shape) != (self.n, 4)
                    or not densify_stats.is_contiguous() or densify_stats.device != self.device):
                raise ValueError("densify_stats must be a contiguous float32 [n, 4] tensor on the render device")
            ptrs["densify_stats"] = _ptr(densify_stats)
        return fgs4d.make_grads(ptrs)

    def _check_features(self, features: torch.Tensor, gate):
        if (features.dim() != 2 or features.shape[0] != self.n or features.dtype != torch.float32
                or not features.is_contiguous() or features.device != self.device):
            raise ValueError("features must be a contiguous float32 [n, D] tensor on the render device")
        D = int(features.shape[1])
        if gate is not None and (tuple(gate.shape) != (D,) or gate.dtype != torch.float32 or gate.device != self.device):
            raise ValueError("gate must be a float32 [D] tensor on the render device")
        return D

    def forward_features(self, params: dict, features: torch.Tensor, gate: torch.Tensor | None = None):
        """Feature map of the normalised scale-gated features (Sec. 7):
        preprocess, bin_sort, then the feature compositor; returns the flat
        buffer [sum_v D H W] (per view planar [D, H, W])."""
        g = self.gaussians(params)
        D = self._check_features(features, gate)
        out = torch.empty(D * self.total_pixels, dtype=torch.float32, device=self.device)
        st = self.stream()
        ws = _ptr(self.ws)
        fgs4d.preprocess(g, self.views, self.nviews, self.settings, ws, self.ws_bytes, st)
        fgs4d.bin_sort(self.n, self.views, self.nviews, self.settings, ws, self.ws_bytes, st)
        fgs4d.render_features(self.n, self.views, self.nviews, self.settings, ws, self.ws_bytes, _ptr(features), D,
                              _ptr(gate) if gate is not None else None, _ptr(out), st)
        return out

    def backward_features(self, features: torch.Tensor, gate, dL_dF: torch.Tensor, grad_features: torch.Tensor,
                          grad_gate: torch.Tensor | None = None):
        """Adds dL/dfeatures (and dL/dgate) for the last forward_features;
        the geometry is held fixed."""
        D = self._check_features(features, gate)
        if grad_features.shape != features.shape or not grad_features.is_contiguous():
            raise ValueError("grad_features must match features")
        dL = dL_dF.contiguous()
        fgs4d.render_features_bwd(self.n, self.views, self.nviews, self.settings, _ptr(self.ws), self.ws_bytes,
                                  _ptr(features), D, _ptr(gate) if gate is not None else None, _ptr(dL),
                                  _ptr(grad_features), _ptr(grad_gate) if grad_gate is not None else None,
                                  self.stream())

    def backward(self, params: dict, dL_drgb: torch.Tensor, grads: dict, densify_stats: torch.Tensor | None = None):
        """Adds dL/dparams into ``grads`` for the last forward of this renderer;
        with ``densify_stats`` ([n, 4]) also accumulates, per visible (view,
        Gaussian), (|dL/dmu_2d|, |dL/dmu_t|, 1, 0)."""
        g = self.gaussians(params)
        gg = self._grads(grads, densify_stats)
        dL = dL_drgb.contiguous()
        fgs4d.render_bwd(g, self.views, self.nviews, self.settings, _ptr(self.ws), self.ws_bytes, _ptr(dL), gg,
                         self.stream())

    def backward_aux(self, params: dict, dL_drgb: torch.Tensor, dL_daux: torch.Tensor, grads: dict):
        """Adds dL/dparams into ``grads`` for a loss on the image and the depth
        and opacity planes of the last forward_aux (flow planes ignored)."""
        g = self.gaussians(params)
        gg = self._grads(grads, None)
        dL = dL_drgb.contiguous()
        dA = dL_daux.contiguous()
        fgs4d.render_aux_bwd(g, self.views, self.nviews, self.settings, _ptr(self.ws), self.ws_bytes, _ptr(dL),
                             _ptr(dA), gg, self.stream())

    def status(self):
        """Synchronises and returns (code, [visible, instances, visible needed, instances needed])."""
        return fgs4d.get_status(_ptr(self.ws), self.ws_bytes, self.stream())

    def check(self):
        code, counts = self.status()
        if code != fgs4d.OK:
            raise fgs4d.Fgs4dError(code, "render (counts %s)" % counts)
        return counts

    def workspace_view(self, offset: int, dtype: torch.dtype, count: int) -> torch.Tensor:
        """A typed view of a documented workspace region (see fgs4d_layout)."""
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return self.ws[offset:offset + nbytes].view(dtype)


PPT_CANDIDATES = {16: (2, 4, 8), 8: (1, 2)}


def autotune(renderer: Renderer, params: dict, view_sets=None, tiles=(16,), candidates=None, batches=(256,),
             reps: int = 3, backward: bool = False, cache_path: str | None = None, pipeline=None) -> dict:
    """Picks the tile edge (among ``tiles``: 16, 8), the compositor block
    shape (pixels per thread, ``candidates`` or all valid ones per tile) and
    its shared-memory batch size (among ``batches``: 256, 128) that run the
    caller's own workload fastest, and sets them on ``renderer`` (a new tile
    edge reallocates its workspace).

    Each (tile, shape) is timed with CUDA events on the current stream over
    ``reps`` runs of preprocess + bin_sort + render_fwd (+ render_bwd if
    ``backward``) for every view set in ``view_sets`` (default: the renderer's
    views) -- the tile edge changes the sort's work as well as the
    compositor's.  With ``cache_path``, the choice is stored in a JSON file
    keyed by (GPU, resolutions, views, N rounded to a power of two) and
    reused.  With ``pipeline`` (a FramePipeline holding ``renderer`` as a
    slot; forward only, one view per set), each shape is applied to every
    slot and timed with the view sets submitted through the pipeline, frames
    in flight as they will run.  Returns {"tile": t, "pixels_per_thread": p,
    "shared_batch": b, "ms": {"t/p/b": ms}}."""
    import json
    import os

    dev_name = torch.cuda.get_device_name(renderer.device)
    bucket = 1 << max(0, int(renderer.n - 1).bit_length())
    res = "+".join("%dx%d" % (w, h) for h, w in sorted(set(renderer.sizes)))
    key = "%s|%s|v%d|n%d|%s|t%s|b%s" % (dev_name, res, renderer.nviews, bucket, "fb" if backward else "f",
                                        ",".join(str(t) for t in tiles), ",".join(str(b) for b in batches))
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            c = cache[key]
            renderer.set_tile(int(c["tile"]), int(c["pixels_per_thread"]), int(c["shared_batch"]))
            return c
    view_sets = view_sets or [(renderer.views, renderer.nviews)]
    g = renderer.gaussians(params)
    st = renderer.stream()
    out = torch.empty(3 * renderer.total_pixels, dtype=torch.float32, device=renderer.device)
    dL = torch.ones_like(out) if backward else None
    grads = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS} if backward else None
    stream = torch.cuda.current_stream(renderer.device)
    ms = {}
    shapes = [(t, p, b) for t in tiles
              for p in (candidates if candidates is not None and t == 16 else PPT_CANDIDATES[int(t)])
              for b in batches]
    if pipeline is not None:
        if backward:
            raise ValueError("autotune: a pipeline times forward frames only")
        for tile, p, bsz in shapes:
            pipeline.set_tile(tile, p, bsz)
            outs = [torch.empty(3 * r.total_pixels, dtype=torch.float32, device=renderer.device)
                    for r in pipeline.slots]

            def sweep():
                pipeline.begin()
                for views, nv in view_sets:
                    j = pipeline.slot_of_next()
                    pipeline.submit(g, views, nv, outs[j].data_ptr())
                pipeline.end()
            sweep()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                sweep()
            b.record(stream)
            b.synchronize()
            if all(r.status()[0] == fgs4d.OK for r in pipeline.slots):
                ms["%d/%d/%d" % (tile, p, bsz)] = a.elapsed_time(b) / reps
        if not ms:
            raise RuntimeError("autotune: every candidate overflowed a capacity")
        best = min(ms, key=ms.get)
        bt, bp, bb = (int(x) for x in best.split("/"))
        pipeline.set_tile(bt, bp, bb)
        return {"tile": bt, "pixels_per_thread": bp, "shared_batch": bb, "ms": ms, "timed": "pipeline"}
    for tile, p, bsz in shapes:
        renderer.set_tile(tile, p, bsz)
        ws, wsb = renderer.ws.data_ptr(), renderer.ws_bytes
        total = 0.0
        for views, nv in view_sets:
            def run():
                fgs4d.preprocess(g, views, nv, renderer.settings, ws, wsb, st)
                fgs4d.bin_sort(renderer.n, views, nv, renderer.settings, ws, wsb, st)
                fgs4d.render_fwd(renderer.n, views, nv, renderer.settings, ws, wsb, out.data_ptr(), None, st)
                if backward:
                    fgs4d.render_bwd(g, views, nv, renderer.settings, ws, wsb, dL.data_ptr(),
                                     fgs4d.make_grads({k: grads[k].data_ptr() for k in PARAM_KEYS}), st)
            run()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                run()
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b) / reps
        code, _ = renderer.status()
        if code == fgs4d.OK:  # a shape whose run overflowed a capacity is not a candidate
            ms["%d/%d/%d" % (tile, p, bsz)] = total
    if not ms:
        raise RuntimeError("autotune: every candidate overflowed a capacity")
    best = min(ms, key=ms.get)
    bt, bp, bb = (int(x) for x in best.split("/"))
    renderer.set_tile(bt, bp, bb)
    result = {"tile": bt, "pixels_per_thread": bp, "shared_batch": bb, "ms": ms}
    if cache_path:
        cache[key] = result
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return result


class FramePipeline:
    """Independent single views rendered with ``depth`` frames in flight.

    Each in-flight slot owns a Renderer (its own workspace) and a CUDA
    stream; the k-th frame submitted after ``begin`` runs preprocess,
    bin_sort and the compositor on slot k % depth.  Frames on different
    slots share only the parameters (which must not change while frames are
    in flight), so the latency-bound binning and sorting of one frame run
    beside the ALU-bound compositing of another; frames on one slot run in
    submission order, so a slot's output buffer may be reused by its next
    frame.  ``end`` makes the caller's current stream wait for every slot.
    A config with ``stage_blocks_per_sm`` = 1 keeps the latency-bound stages
    of one frame from filling the SMs the other frames' compositors use.
    """

    def __init__(self, n: int, view: dict, config: RenderConfig, depth: int = 3, device=None):
        import dataclasses
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.depth = int(depth)
        self.slots = [Renderer(n, [view], dataclasses.replace(config), device=device) for _ in range(self.depth)]
        self.device = self.slots[0].device
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.depth)]
        self._next = 0

    def fit_visible_capacity(self, params: dict, view_sets, margin: float = 1.1) -> int:
        """Renderer.fit_visible_capacity on the first slot, applied to all."""
        cap = self.slots[0].fit_visible_capacity(params, view_sets=view_sets, margin=margin)
        for r in self.slots[1:]:
            r.settings.vis_capacity = cap
            r.config.vis_capacity = cap
            r._allocate()
        return cap

    def set_tile(self, tile: int, pixels_per_thread: int = 0, shared_batch: int = 0):
        for r in self.slots:
            r.set_tile(tile, pixels_per_thread, shared_batch)

    def begin(self):
        """Every slot stream waits for the work already on the current stream."""
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream(self.device))
        for st in self.streams:
            st.wait_event(ev)
        self._next = 0

    def slot_of_next(self) -> int:
        return self._next % self.depth

    def submit(self, g: fgs4d.Gaussians, views, nviews: int, out_rgb: int, out_T: int | None = None,
               events=None, after=None, image_only: bool = True) -> int:
        """Launches one frame (views, nviews from fgs4d.make_views) on the
        next slot; ``g`` from any slot's gaussians().  ``events`` = (e0, e1)
        are recorded around the compositor launch, ``after(stream)`` is
        called on the slot stream after it (e.g. to enqueue a copy of the
        output).  ``image_only`` (default) renders with fgs4d_render_image
        (no state for a backward pass is kept); False uses fgs4d_render_fwd.
        Returns the slot index."""
        j = self._next % self.depth
        self._next += 1
        r, st = self.slots[j], self.streams[j]
        ws, wsb, s, sp = r.ws.data_ptr(), r.ws_bytes, r.settings, st.cuda_stream
        fgs4d.preprocess(g, views, nviews, s, ws, wsb, sp)
        fgs4d.bin_sort(r.n, views, nviews, s, ws, wsb, sp)
        if events is not None:
            events[0].record(st)
        (fgs4d.render_image if image_only else fgs4d.render_fwd)(r.n, views, nviews, s, ws, wsb, out_rgb, out_T, sp)
        if events is not None:
            events[1].record(st)
        if after is not None:
            after(st)
        return j

    def end(self):
        cur = torch.cuda.current_stream(self.device)
        for st in self.streams:
            cur.wait_stream(st)

    def check(self):
        """Synchronises; raises if any slot's workspace reports an error."""
        return [r.check() for r in self.slots]


class ViewParallel:
    """A batch of views rendered as independent calls on parallel streams.

    Each group of views gets its own Renderer (workspace) and CUDA stream.
    ``step`` forks from the current stream, runs forward, the caller's loss
    and backward of every group on that group's stream, and joins back.  The
    backward passes add into the same gradient buffers (the preprocess
    adjoint accumulates with atomics, so groups may overlap); the
    latency-bound binning and sorting of one group run beside the
    compositing of another."""

    def __init__(self, n: int, view_groups, config: RenderConfig, device=None):
        import dataclasses
        self.groups = [Renderer(n, list(g), dataclasses.replace(config), device=device) for g in view_groups]
        self.device = self.groups[0].device
        self.streams = [torch.cuda.Stream(self.device) for _ in self.groups]

    def set_tile(self, tile: int, pixels_per_thread: int = 0, shared_batch: int = 0):
        for r in self.groups:
            r.set_tile(tile, pixels_per_thread, shared_batch)

    def step(self, params: dict, loss_fn, grads: dict, densify_stats: torch.Tensor | None = None):
        """For every group j (on its stream): img = forward, dL/dimg =
        loss_fn(j, img), backward into ``grads``.  Returns the images."""
        cur = torch.cuda.current_stream(self.device)
        ev = torch.cuda.Event()
        ev.record(cur)
        imgs = []
        for j, (r, st) in enumerate(zip(self.groups, self.streams)):
            st.wait_event(ev)
            with torch.cuda.stream(st):
                img = r.forward(params)
                r.backward(params, loss_fn(j, img), grads, densify_stats)
                imgs.append(img)
        for st in self.streams:
            cur.wait_stream(st)
        for img in imgs:
            img.record_stream(cur)  # the caller's stream reads them after the join
        return imgs

    def check(self):
        return [r.check() for r in self.groups]


class Render4DGS(torch.autograd.Function):
    """Differentiable render: (renderer, *params) -> flat RGB [sum 3HW]."""

    @staticmethod
    def forward(ctx, renderer: Renderer, mean, log_scale, q_l, q_r, opacity_logit, sh):
        params = dict(zip(PARAM_KEYS, (mean, log_scale, q_l, q_r, opacity_logit, sh)))
        out = renderer.forward(params)
        ctx.renderer = renderer
        ctx.save_for_backward(mean, log_scale, q_l, q_r, opacity_logit, sh)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        saved = ctx.saved_tensors
        params = dict(zip(PARAM_KEYS, saved))
        grads = {k: torch.zeros_like(v) for k, v in params.items()}
        ctx.renderer.backward(params, grad_out, grads)
        return (None,) + tuple(grads[k] for k in PARAM_KEYS)


def render(renderer: Renderer, params: dict) -> torch.Tensor:
    return Render4DGS.apply(renderer, *(params[k] for k in PARAM_KEYS))


def split_gaussians(params: dict, idx: torch.Tensor, eps: torch.Tensor, shrink: float, config: RenderConfig) -> dict:
    """Children of the Gaussians ``idx`` ([m] int32) sampled from their full
    4D Gaussians: ``eps`` ([m, K, 4] standard normal draws) gives K children
    each; returns the children's parameter tensors (m K rows)."""
    device = params["mean"].device
    n = params["mean"].shape[0]
    for k in PARAM_KEYS:
        _check_param(k, params[k], n, device)
    m, K = int(idx.shape[0]), int(eps.shape[1]) if eps.dim() == 3 else 0
    if idx.dtype != torch.int32 or eps.dtype != torch.float32 or tuple(eps.shape) != (m, K, 4):
        raise ValueError("idx must be int32 [m] and eps float32 [m, K, 4]")
    idx, eps = idx.contiguous(), eps.contiguous()
    out = {k: torch.empty((m * K,) + tuple(params[k].shape[1:]), dtype=torch.float32, device=device)
           for k in PARAM_KEYS}
    src = fgs4d.make_gaussians({k: _ptr(params[k]) for k in PARAM_KEYS}, n)
    dst = fgs4d.GaussiansOut(*(_ptr(out[k]) for k in PARAM_KEYS), m * K)
    fgs4d.split_gaussians(src, _ptr(idx), m, K, _ptr(eps), shrink, config.settings(), dst,
                          torch.cuda.current_stream(device).cuda_stream)
    return out


def mask_loss(mask_logit: torch.Tensor, grad: torch.Tensor | None = None):
    """Mask compression loss of Compact-4DGS, mean sigmoid(m) (Sec. 4.3);
    adds its gradient into ``grad`` (allocated when None).  Returns (loss, grad)."""
    device = mask_logit.device
    n = mask_logit.shape[0]
    _check_param("mask_logit", mask_logit, n, device)
    if grad is None:
        grad = torch.zeros_like(mask_logit)
    _check_param("mask grad", grad, n, device)
    loss = torch.zeros(1, dtype=torch.float32, device=device)
    fgs4d.mask_loss(_ptr(mask_logit), n, _ptr(loss), _ptr(grad), torch.cuda.current_stream(device).cuda_stream)
    return loss, grad


class Adam:
    """Adam over the parameter tensors with the fgs4d kernel (one streaming
    pass over all tensors); the step count lives on the device, so ``step``
    can be captured in a CUDA graph.  ``lr`` may be one float or a dict per
    key."""

    def __init__(self, params: dict, lr=1e-4, betas=(0.9, 0.999), eps=1e-8):
        self.params = params
        device = next(iter(params.values())).device
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.t = torch.zeros(1, dtype=torch.int32, device=device)
        self.lr = lr if isinstance(lr, dict) else {k: float(lr) for k in params}
        self.betas, self.eps = betas, eps

    def step(self, grads: dict, zero_grad: bool = False):
        """One Adam step from ``grads``; with ``zero_grad`` the gradients are
        cleared in the same pass (each after it is read), ready for the next
        step's accumulation."""
        st = torch.cuda.current_stream(self.t.device).cuda_stream
        fgs4d.adam_tick(_ptr(self.t), st)
        keys = list(self.params)
        for i in range(0, len(keys), fgs4d.ADAM_MAX_TENSORS):
            fgs4d.adam_update_set([(_ptr(self.params[k]), _ptr(grads[k]), _ptr(self.m[k]), _ptr(self.v[k]),
                                    self.params[k].numel(), self.lr[k]) for k in keys[i:i + fgs4d.ADAM_MAX_TENSORS]],
                                  self.betas[0], self.betas[1], self.eps, _ptr(self.t), zero_grad, st)


def l1_loss(img: torch.Tensor, target: torch.Tensor, mean_count: int | None = None,
            loss: torch.Tensor | None = None):
    """L1 loss and its gradient with the fgs4d kernel: returns (loss[1], dL/dimg).

    With ``mean_count`` the call is one part of a loss averaged over
    ``mean_count`` elements (images rendered by separate calls): the part's
    sum |img - target| / mean_count is ADDED to ``loss`` (a zeroed float32
    [1] tensor, created when None) and dL/dimg = sign / mean_count."""
    img = img.contiguous()
    target = target.contiguous()
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=img.device)
    grad = torch.empty_like(img)
    st = torch.cuda.current_stream(img.device).cuda_stream
    if mean_count is None:
        fgs4d.l1_loss(_ptr(img), _ptr(target), img.numel(), _ptr(loss), _ptr(grad), st)
    else:
        fgs4d.l1_loss_part(_ptr(img), _ptr(target), img.numel(), int(mean_count), _ptr(loss), _ptr(grad), st)
    return loss, grad
