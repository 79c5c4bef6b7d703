"""ctypes binding of the fgs4d C ABI (include/fgs4d.h).

Argument marshalling only: every step of the render path runs in the CUDA
kernels of libfgs4d.so.  The functions keep the C names without the prefix
(``preprocess`` -> ``fgs4d_preprocess``) and take device pointers as ints.
Loading fails loudly when the library is missing and cannot be built: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK = 0
ERR_ARG = -1
ERR_CUDA = -2
ERR_WORKSPACE = -3
ERR_CAPACITY = -4
ERR_TIMEOUT = -5
ERR_INTERNAL = -6
ERR_UNSUPPORTED = -7
MAX_VIEWS = 128
MAX_SH_DEGREE = 3
MAX_T_ORDER = 4
TILE = 16  # default tile edge; 8 is the other supported size

EXPORTED = ("fgs4d_workspace_size", "fgs4d_workspace_layout", "fgs4d_preprocess", "fgs4d_bin_sort",
            "fgs4d_bin_sort_kernels", "fgs4d_render_fwd", "fgs4d_render_image", "fgs4d_render_aux",
            "fgs4d_render_stats", "fgs4d_render_bwd", "fgs4d_render_bwd_composite",
            "fgs4d_render_bwd_preprocess", "fgs4d_render_aux_bwd", "fgs4d_split_gaussians",
            "fgs4d_mask_loss", "fgs4d_adam_tick", "fgs4d_adam_update", "fgs4d_adam_update_set",
            "fgs4d_render_features",
            "fgs4d_render_features_bwd", "fgs4d_l1_loss", "fgs4d_l1_loss_part", "fgs4d_sort_depth_static",
            "fgs4d_sort_depth_static_status", "fgs4d_wait_selftest", "fgs4d_get_status", "fgs4d_status_string")
STATIC_SORT_MAX = 1 << 20
ADAM_MAX_TENSORS = 16


class AdamTensor(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("exp_avg", C.c_void_p), ("exp_avg_sq", C.c_void_p),
                ("count", C.c_int64), ("lr", C.c_float)]


class View(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("viewmat", C.c_float * 12), ("campos", C.c_float * 3),
                ("t", C.c_float)]


class Settings(C.Structure):
    _fields_ = [("sh_degree", C.c_int32), ("t_order", C.c_int32), ("period", C.c_float), ("tile", C.c_int32),
                ("near_plane", C.c_float), ("dilation", C.c_float), ("p_t_min", C.c_float), ("bg", C.c_float * 3),
                ("vis_capacity", C.c_int64), ("inst_capacity", C.c_int64), ("pixels_per_thread", C.c_int32),
                ("shared_batch", C.c_int32), ("stage_blocks_per_sm", C.c_int32)]


class Gaussians(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("q_l", C.c_void_p), ("q_r", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64), ("mask_logit", C.c_void_p),
                ("mask_threshold", C.c_float)]


class GaussiansGrad(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("q_l", C.c_void_p), ("q_r", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("densify_stats", C.c_void_p),
                ("mask_logit", C.c_void_p)]


class GaussiansOut(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("q_l", C.c_void_p), ("q_r", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64)]


class Layout(C.Structure):
    _fields_ = [(k, C.c_size_t) for k in ("bytes", "counters", "rec_geom", "rec_color", "rec_blue", "rec_tau",
                                          "rec_meta",
                                          "depth_key", "sorted_slots", "inst_tile", "inst_slot", "tile_ranges",
                                          "pix_T", "pix_last", "slot_grad")] + \
               [(k, C.c_int64) for k in ("vis_capacity", "inst_capacity", "total_tiles", "total_pixels")]


_lib = None


class Fgs4dError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, status_string(code), code))
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Load libfgs4d.so, building it first if it is missing or stale and
    nvcc is available.  Raises if the CUDA library cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    if not _build.up_to_date():
        _build.build()
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libfgs4d.so is missing; build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.POINTER
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.fgs4d_workspace_size.argtypes = [P(Settings), i64, P(View), i32, P(C.c_size_t)]
    lib.fgs4d_workspace_layout.argtypes = [P(Settings), i64, P(View), i32, P(Layout)]
    lib.fgs4d_preprocess.argtypes = [P(Gaussians), P(View), i32, P(Settings), vp, C.c_size_t, vp]
    lib.fgs4d_bin_sort.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp]
    lib.fgs4d_bin_sort_kernels.argtypes = [i64, P(View), i32, P(Settings), P(C.c_int32)]
    lib.fgs4d_render_fwd.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp, vp, vp]
    lib.fgs4d_render_image.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp, vp, vp]
    lib.fgs4d_render_aux.argtypes = [P(Gaussians), P(View), i32, P(Settings), vp, C.c_size_t, C.c_float, vp, vp,
                                     vp, vp]
    lib.fgs4d_render_stats.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp, vp, vp]
    lib.fgs4d_render_bwd.argtypes = [P(Gaussians), P(View), i32, P(Settings), vp, C.c_size_t, vp, P(GaussiansGrad),
                                     vp]
    lib.fgs4d_render_aux_bwd.argtypes = [P(Gaussians), P(View), i32, P(Settings), vp, C.c_size_t, vp, vp,
                                         P(GaussiansGrad), vp]
    lib.fgs4d_render_bwd_composite.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp, vp]
    lib.fgs4d_render_bwd_preprocess.argtypes = [P(Gaussians), P(View), i32, P(Settings), vp, C.c_size_t,
                                                P(GaussiansGrad), vp]
    lib.fgs4d_split_gaussians.argtypes = [P(Gaussians), vp, i64, i32, vp, C.c_float, P(Settings), P(GaussiansOut), vp]
    lib.fgs4d_mask_loss.argtypes = [vp, i64, vp, vp, vp]
    lib.fgs4d_render_features.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp, i32, vp, vp, vp]
    lib.fgs4d_render_features_bwd.argtypes = [i64, P(View), i32, P(Settings), vp, C.c_size_t, vp, i32, vp, vp, vp, vp,
                                              vp]
    lib.fgs4d_adam_tick.argtypes = [vp, vp]
    lib.fgs4d_adam_update.argtypes = [vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float, vp, vp]
    lib.fgs4d_adam_update_set.argtypes = [P(AdamTensor), i32, C.c_float, C.c_float, C.c_float, vp, i32, vp]
    lib.fgs4d_l1_loss.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.fgs4d_l1_loss_part.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    lib.fgs4d_sort_depth_static.argtypes = [vp, i64, vp, vp]
    lib.fgs4d_sort_depth_static_status.argtypes = [vp]
    lib.fgs4d_wait_selftest.argtypes = [vp, C.c_size_t, vp]
    lib.fgs4d_get_status.argtypes = [vp, C.c_size_t, vp, P(C.c_int64)]
    lib.fgs4d_status_string.argtypes = [C.c_int]
    lib.fgs4d_status_string.restype = C.c_char_p
    for name in EXPORTED[:-1]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().fgs4d_status_string(int(code)).decode()


def _check(code: int, what: str):
    if code != OK:
        raise Fgs4dError(code, what)


# ------------------------------------------------------------ struct helpers

def make_view(d) -> View:
    """From a mapping with width, height, fx, fy, cx, cy, viewmat (3x4),
    campos (3), t."""
    v = View()
    v.width, v.height = int(d["width"]), int(d["height"])
    v.fx, v.fy, v.cx, v.cy = (float(d[k]) for k in ("fx", "fy", "cx", "cy"))
    vm = np.asarray(d["viewmat"], dtype=np.float32).reshape(12)
    for k in range(12):
        v.viewmat[k] = float(vm[k])
    cp = np.asarray(d["campos"], dtype=np.float32).reshape(3)
    for k in range(3):
        v.campos[k] = float(cp[k])
    v.t = float(d["t"])
    return v


def make_views(views) -> tuple:
    arr = (View * len(views))(*[make_view(v) for v in views])
    return arr, len(views)


def make_settings(sh_degree=3, t_order=2, period=1.0, near_plane=0.2, dilation=0.3, p_t_min=0.05,
                  bg=(0.0, 0.0, 0.0), vis_capacity=0, inst_capacity=1 << 22, pixels_per_thread=0,
                  tile=TILE, shared_batch=0, stage_blocks_per_sm=0) -> Settings:
    s = Settings()
    s.sh_degree, s.t_order, s.period, s.tile = int(sh_degree), int(t_order), float(period), int(tile)
    s.near_plane, s.dilation, s.p_t_min = float(near_plane), float(dilation), float(p_t_min)
    for k in range(3):
        s.bg[k] = float(bg[k])
    s.vis_capacity, s.inst_capacity = int(vis_capacity), int(inst_capacity)
    s.pixels_per_thread, s.shared_batch = int(pixels_per_thread), int(shared_batch)
    s.stage_blocks_per_sm = int(stage_blocks_per_sm)
    return s


def make_gaussians(ptrs: dict, n: int, mask_logit: int = 0, mask_threshold: float = 0.0) -> Gaussians:
    """Parameter pointers; ``mask_logit`` is the optional significance mask (0 = none)."""
    return Gaussians(*(ptrs[k] for k in ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")), int(n),
                     mask_logit or None, float(mask_threshold))


def make_grads(ptrs: dict) -> GaussiansGrad:
    """Gradient pointers; ``densify_stats`` is optional (0 = off)."""
    return GaussiansGrad(*(ptrs[k] for k in ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")),
                         ptrs.get("densify_stats", 0) or None, ptrs.get("mask_logit", 0) or None)


# ---------------------------------------------------------- entry points

def workspace_size(settings: Settings, n: int, views, nviews: int) -> int:
    out = C.c_size_t(0)
    _check(load().fgs4d_workspace_size(C.byref(settings), int(n), views, int(nviews), C.byref(out)),
           "fgs4d_workspace_size")
    return int(out.value)


def workspace_layout(settings: Settings, n: int, views, nviews: int) -> Layout:
    lay = Layout()
    _check(load().fgs4d_workspace_layout(C.byref(settings), int(n), views, int(nviews), C.byref(lay)),
           "fgs4d_workspace_layout")
    return lay


def preprocess(gaussians: Gaussians, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, stream: int):
    _check(load().fgs4d_preprocess(C.byref(gaussians), views, int(nviews), C.byref(settings), ws, ws_bytes, stream),
           "fgs4d_preprocess")


def bin_sort_kernels(n: int, views, nviews: int, settings: Settings) -> int:
    """Kernels fgs4d_bin_sort launches for these arguments on the current device."""
    out = C.c_int32(0)
    _check(load().fgs4d_bin_sort_kernels(int(n), views, int(nviews), C.byref(settings), C.byref(out)),
           "fgs4d_bin_sort_kernels")
    return int(out.value)


def bin_sort(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, stream: int):
    _check(load().fgs4d_bin_sort(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, stream),
           "fgs4d_bin_sort")


def render_fwd(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, out_rgb: int, out_T, stream):
    _check(load().fgs4d_render_fwd(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, out_rgb, out_T,
                                   stream), "fgs4d_render_fwd")


def render_image(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, out_rgb: int, out_T,
                 stream):
    _check(load().fgs4d_render_image(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, out_rgb, out_T,
                                     stream), "fgs4d_render_image")


def render_aux(gaussians: Gaussians, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, flow_dt: float,
               out_rgb: int, out_T, out_aux: int, stream):
    _check(load().fgs4d_render_aux(C.byref(gaussians), views, int(nviews), C.byref(settings), ws, ws_bytes,
                                   float(flow_dt), out_rgb, out_T, out_aux, stream), "fgs4d_render_aux")


def render_stats(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, out_rgb: int,
                 stats_out: int, stream):
    _check(load().fgs4d_render_stats(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, out_rgb,
                                     stats_out, stream), "fgs4d_render_stats")


def render_bwd(gaussians: Gaussians, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, dL_drgb: int,
               grads: GaussiansGrad, stream: int):
    _check(load().fgs4d_render_bwd(C.byref(gaussians), views, int(nviews), C.byref(settings), ws, ws_bytes, dL_drgb,
                                   C.byref(grads), stream), "fgs4d_render_bwd")


def render_bwd_composite(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, dL_drgb: int,
                         stream: int):
    _check(load().fgs4d_render_bwd_composite(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, dL_drgb,
                                             stream), "fgs4d_render_bwd_composite")


def render_bwd_preprocess(gaussians: Gaussians, views, nviews: int, settings: Settings, ws: int, ws_bytes: int,
                          grads: GaussiansGrad, stream: int):
    _check(load().fgs4d_render_bwd_preprocess(C.byref(gaussians), views, int(nviews), C.byref(settings), ws, ws_bytes,
                                              C.byref(grads), stream), "fgs4d_render_bwd_preprocess")


def render_aux_bwd(gaussians: Gaussians, views, nviews: int, settings: Settings, ws: int, ws_bytes: int,
                   dL_drgb: int, dL_daux: int, grads: GaussiansGrad, stream: int):
    _check(load().fgs4d_render_aux_bwd(C.byref(gaussians), views, int(nviews), C.byref(settings), ws, ws_bytes,
                                       dL_drgb, dL_daux, C.byref(grads), stream), "fgs4d_render_aux_bwd")


def split_gaussians(src: Gaussians, idx: int, m: int, k_children: int, eps: int, shrink: float, settings: Settings,
                    dst: GaussiansOut, stream: int):
    _check(load().fgs4d_split_gaussians(C.byref(src), idx, int(m), int(k_children), eps, float(shrink),
                                        C.byref(settings), C.byref(dst), stream), "fgs4d_split_gaussians")


def mask_loss(mask_logit: int, n: int, loss_out: int, grad_out: int, stream: int):
    _check(load().fgs4d_mask_loss(mask_logit, int(n), loss_out, grad_out, stream), "fgs4d_mask_loss")


def render_features(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, feat: int, D: int,
                    gate, out: int, stream):
    _check(load().fgs4d_render_features(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, feat, int(D),
                                        gate, out, stream), "fgs4d_render_features")


def render_features_bwd(n: int, views, nviews: int, settings: Settings, ws: int, ws_bytes: int, feat: int, D: int,
                        gate, dL_dF: int, g_feat: int, g_gate, stream):
    _check(load().fgs4d_render_features_bwd(int(n), views, int(nviews), C.byref(settings), ws, ws_bytes, feat,
                                            int(D), gate, dL_dF, g_feat, g_gate, stream), "fgs4d_render_features_bwd")


def adam_tick(step: int, stream: int):
    _check(load().fgs4d_adam_tick(step, stream), "fgs4d_adam_tick")


def adam_update(param: int, grad: int, exp_avg: int, exp_avg_sq: int, count: int, lr: float, beta1: float,
                beta2: float, eps: float, step: int, stream: int):
    _check(load().fgs4d_adam_update(param, grad, exp_avg, exp_avg_sq, int(count), float(lr), float(beta1),
                                    float(beta2), float(eps), step, stream), "fgs4d_adam_update")


def adam_update_set(tensors, beta1: float, beta2: float, eps: float, step: int, zero_grad: bool, stream: int):
    """tensors: sequence of (param, grad, exp_avg, exp_avg_sq, count, lr) with device pointers."""
    arr = (AdamTensor * max(1, len(tensors)))()
    for k, (p, g, m, v, count, lr) in enumerate(tensors):
        arr[k] = AdamTensor(p, g, m, v, int(count), float(lr))
    _check(load().fgs4d_adam_update_set(arr, len(tensors), float(beta1), float(beta2), float(eps), step,
                                        1 if zero_grad else 0, stream), "fgs4d_adam_update_set")


def l1_loss(img: int, target: int, count: int, loss_out: int, dL_dimg: int, stream: int):
    _check(load().fgs4d_l1_loss(img, target, int(count), loss_out, dL_dimg, stream), "fgs4d_l1_loss")


def l1_loss_part(img: int, target: int, count: int, mean_count: int, loss_out: int, dL_dimg: int, stream: int):
    _check(load().fgs4d_l1_loss_part(img, target, int(count), int(mean_count), loss_out, dL_dimg, stream),
           "fgs4d_l1_loss_part")


WAIT_SELFTEST_BYTES = 4096


def wait_selftest(scratch: int, scratch_bytes: int, stream: int) -> int:
    """Runs the bounded-wait self-test; returns the status code (ERR_TIMEOUT
    is the expected result)."""
    return int(load().fgs4d_wait_selftest(scratch, int(scratch_bytes), stream))


def sort_depth_static(depth_keys: int, n: int, sorted_slots: int, stream: int):
    """Depth sort with the library's own device scratch (no allocation);
    see fgs4d_sort_depth_static in include/fgs4d.h for who needs it."""
    _check(load().fgs4d_sort_depth_static(depth_keys, int(n), sorted_slots, stream), "fgs4d_sort_depth_static")


def sort_depth_static_status(stream: int) -> int:
    """Synchronises the stream and returns the device-side outcome of the last
    sort_depth_static call on the current device (OK, ERR_TIMEOUT or
    ERR_INTERNAL)."""
    return int(load().fgs4d_sort_depth_static_status(stream))


def get_status(ws: int, ws_bytes: int, stream: int):
    """Returns (status code, [visible, instances, visible needed, instances needed])."""
    counts = (C.c_int64 * 4)()
    code = load().fgs4d_get_status(ws, ws_bytes, stream, counts)
    return int(code), [int(c) for c in counts]
