"""FP64 CPU oracle of the 4D Gaussian Splatting render path (arXiv 2412.20720).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2412_20720_gb300``) never imports it, and this package
never imports the product path: the two share no code.  The only thing both
sides consume is the seeded synthetic input (plain FP32 arrays).

This module is argument marshalling over ``fgs4d_oracle.c``; every formula
lives in the C file, each function citing the passage it follows.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import build_oracle, build_oracle_sanitized, library_path

_lib = None


def _load():
    global _lib
    if _lib is None:
        # no-op when the library is newer than its source
        path = build_oracle_sanitized() if os.environ.get("FGS4D_ORACLE_SANITIZED") == "1" else build_oracle()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class _Params(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("q_l", C.c_void_p),
                ("q_r", C.c_void_p), ("opacity_logit", C.c_void_p), ("sh", C.c_void_p),
                ("n", C.c_int64), ("mask_logit", C.c_void_p), ("mask_threshold", C.c_double)]


class _View(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("pad0", C.c_int32), ("pad1", C.c_int32),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("viewmat", C.c_double * 12), ("campos", C.c_double * 3), ("t", C.c_double)]


class _Settings(C.Structure):
    _fields_ = [("sh_degree", C.c_int32), ("t_order", C.c_int32), ("tile", C.c_int32), ("pad", C.c_int32),
                ("period", C.c_double), ("near_plane", C.c_double), ("dilation", C.c_double),
                ("p_t_min", C.c_double), ("bg", C.c_double * 3)]


_PROJ_FIELDS = [("status", np.int32, 1), ("rect", np.int32, 4), ("p_t", np.float64, 1),
                ("a_eff", np.float64, 1), ("mu3", np.float64, 3), ("cov3", np.float64, 9),
                ("pc", np.float64, 3), ("cov2d", np.float64, 3), ("conic", np.float64, 3),
                ("uv", np.float64, 2), ("radius", np.float64, 1), ("depth", np.float64, 1),
                ("rgb", np.float64, 3), ("margin", np.float64, 1), ("depth_f32", np.float32, 1),
                ("uncertain", np.int32, 1), ("rect_lo", np.int32, 4), ("rect_hi", np.int32, 4)]


class _Proj(C.Structure):
    _fields_ = [(name, C.c_void_p) for name, _, _ in _PROJ_FIELDS]


_GRAD_FIELDS = ["mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh", "g_uv", "g_conic", "g_a", "g_rgb", "g_z",
                "mask_logit"]


class _Tol(C.Structure):
    _fields_ = [("eps_conic", C.c_double), ("eps_uv", C.c_double), ("eps_uv_abs", C.c_double), ("eps_a", C.c_double),
                ("eps_alpha", C.c_double), ("depth_ulps", C.c_int32), ("max_leaves", C.c_int32)]


@dataclass
class Tolerance:
    """Error bounds of an FP32 renderer's per-pixel inputs, relative to the
    FP64 values (see orc_render_pixels_admissible): the factors of the conic
    Q = U U^T (u11, u22 relative, u12 relative to |u12| + sqrt(Q11)),
    projected centre (eps_uv |u| + eps_uv_abs pixels), effective opacity, the
    exponential; depth keys within depth_ulps units in the last place."""
    eps_conic: float = 0.0
    eps_uv: float = 0.0
    eps_uv_abs: float = 0.0
    eps_a: float = 0.0
    eps_alpha: float = 0.0
    depth_ulps: int = 0
    max_leaves: int = 4096

    def _c(self) -> _Tol:
        return _Tol(self.eps_conic, self.eps_uv, self.eps_uv_abs, self.eps_a, self.eps_alpha, self.depth_ulps,
                    self.max_leaves)


class _Grads(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in _GRAD_FIELDS]


def _declare(lib):
    P = C.POINTER
    lib.orc_preprocess.argtypes = [P(_Params), P(_View), P(_Settings), P(_Proj)]
    lib.orc_preprocess.restype = C.c_int
    lib.orc_preprocess_relaxed.argtypes = [P(_Params), P(_View), P(_Settings), C.c_double, P(_Proj)]
    lib.orc_preprocess_relaxed.restype = C.c_int
    lib.orc_render_pixels_admissible.argtypes = [P(_View), P(_Settings), C.c_int64, P(_Proj), P(_Tol), C.c_void_p,
                                                 C.c_int32, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                                 C.c_void_p, C.c_void_p]
    lib.orc_render_pixels_admissible.restype = C.c_int
    lib.orc_alpha_bounds.argtypes = [P(_View), P(_Proj), P(_Tol), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]
    lib.orc_alpha_bounds.restype = None
    lib.orc_render.argtypes = [P(_View), P(_Settings), C.c_int64, P(_Proj), C.c_void_p, C.c_void_p,
                               C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_render.restype = C.c_int
    lib.orc_render_pixels.argtypes = [P(_View), P(_Settings), C.c_int64, P(_Proj), C.c_int64, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_render_pixels.restype = C.c_int
    lib.orc_render_backward.argtypes = [P(_Params), P(_View), P(_Settings), P(_Proj), C.c_void_p, P(_Grads)]
    lib.orc_render_backward.restype = C.c_int
    lib.orc_preprocess_backward.argtypes = [P(_Params), P(_View), P(_Settings), C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, P(_Grads)]
    lib.orc_preprocess_backward.restype = C.c_int
    lib.orc_aux.argtypes = [P(_Params), P(_View), P(_Settings), C.c_double, C.c_double, P(_Proj), C.c_void_p]
    lib.orc_aux.restype = C.c_int
    lib.orc_render_aux.argtypes = [P(_View), P(_Settings), C.c_int64, P(_Proj), C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_render_aux.restype = C.c_int
    lib.orc_render_aux_backward.argtypes = [P(_Params), P(_View), P(_Settings), P(_Proj), C.c_void_p, C.c_void_p,
                                            P(_Grads)]
    lib.orc_render_aux_backward.restype = C.c_int
    lib.orc_split_sample.argtypes = [P(_Params), C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_double, C.c_int64,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_split_sample.restype = C.c_int
    lib.orc_render_features.argtypes = [P(_View), P(_Settings), C.c_int64, P(_Proj), C.c_void_p, C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
    lib.orc_render_features.restype = C.c_int
    lib.orc_render_features_backward.argtypes = [P(_View), P(_Settings), C.c_int64, P(_Proj), C.c_void_p, C.c_int,
                                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_render_features_backward.restype = C.c_int
    lib.orc_gated_features.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]
    lib.orc_gated_features.restype = None
    lib.orc_rotation.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_rotation.restype = None
    lib.orc_real_sh.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
    lib.orc_real_sh.restype = None
    lib.orc_sort_instances.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int64,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_sort_instances.restype = C.c_int64
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = C.c_int
    lib.orc_set_num_threads.argtypes = [C.c_int]
    lib.orc_set_num_threads.restype = None


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Settings:
    """Render settings (the readings where the paper is silent)."""
    sh_degree: int = 3
    t_order: int = 2
    tile: int = 16
    period: float = 1.0
    near_plane: float = 0.2
    dilation: float = 0.3
    p_t_min: float = 0.05
    bg: tuple = (0.0, 0.0, 0.0)

    def _c(self) -> _Settings:
        s = _Settings()
        s.sh_degree, s.t_order, s.tile = self.sh_degree, self.t_order, self.tile
        s.period, s.near_plane, s.dilation, s.p_t_min = self.period, self.near_plane, self.dilation, self.p_t_min
        for k in range(3):
            s.bg[k] = self.bg[k]
        return s


def _view_c(view) -> _View:
    """``view``: mapping with width, height, fx, fy, cx, cy, viewmat (3x4),
    campos (3), t.  Values are taken as given (the FP32 values the GPU sees
    should be passed to compare like with like)."""
    v = _View()
    v.width, v.height = int(view["width"]), int(view["height"])
    v.fx, v.fy, v.cx, v.cy = (float(view[k]) for k in ("fx", "fy", "cx", "cy"))
    vm = np.asarray(view["viewmat"], dtype=np.float64).reshape(12)
    for k in range(12):
        v.viewmat[k] = vm[k]
    cp = np.asarray(view["campos"], dtype=np.float64).reshape(3)
    for k in range(3):
        v.campos[k] = cp[k]
    v.t = float(view["t"])
    return v


class _ParamsHold:
    def __init__(self, params, settings=None):
        # FP32 inputs are upcast exactly; FP64 inputs (finite differences) pass through.
        self.arrs = {k: np.ascontiguousarray(params[k], dtype=np.float64)
                     for k in ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")}
        n = self.arrs["mean"].shape[0]
        # The C side reads n rows of each array and (L+1)^2 (N_t+1) SH rows
        # per Gaussian: refuse anything shorter instead of reading past it.
        want = {"mean": (n, 4), "log_scale": (n, 4), "q_l": (n, 4), "q_r": (n, 4), "opacity_logit": (n,)}
        for k, shp in want.items():
            if self.arrs[k].shape != shp:
                raise ValueError("oracle parameter %s has shape %s, expected %s" % (k, self.arrs[k].shape, shp))
        sh = self.arrs["sh"]
        if sh.ndim != 3 or sh.shape[0] != n or sh.shape[2] != 3:
            raise ValueError("oracle parameter sh has shape %s, expected (%d, K, 3)" % (sh.shape, n))
        if settings is not None:
            K = (settings.sh_degree + 1) ** 2 * (settings.t_order + 1)
            if sh.shape[1] != K:
                raise ValueError("oracle parameter sh has %d rows per Gaussian; SH degree %d and temporal order %d "
                                 "take %d" % (sh.shape[1], settings.sh_degree, settings.t_order, K))
        mask = params.get("mask_logit")
        if mask is not None:  # optional Compact-4DGS significance mask
            self.arrs["mask_logit"] = np.ascontiguousarray(mask, dtype=np.float64)
        self.c = _Params(*(_ptr(self.arrs[k]) for k in ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")),
                         n, _ptr(self.arrs["mask_logit"]) if mask is not None else None,
                         float(params.get("mask_threshold", 0.0)))
        self.n = n


def preprocess(params, view, settings: Settings, relax: float = 0.0):
    """Per-Gaussian forward chain (FP64).  Returns a dict of arrays.  With
    relax > 0, decisions within that relative distance of their thresholds
    are marked ("uncertain", "rect_lo", "rect_hi"; orc_preprocess_relaxed);
    the FP64 decisions and values are the same either way."""
    lib = _load()
    ph = _ParamsHold(params, settings)
    n = ph.n
    out = {}
    for name, dt, w in _PROJ_FIELDS:
        out[name] = np.zeros((n, w) if w > 1 else (n,), dtype=dt)
    pc = _Proj(*(_ptr(out[name]) for name, _, _ in _PROJ_FIELDS))
    if relax > 0.0:
        rc = lib.orc_preprocess_relaxed(C.byref(ph.c), C.byref(_view_c(view)), C.byref(settings._c()), float(relax),
                                        C.byref(pc))
    else:
        rc = lib.orc_preprocess(C.byref(ph.c), C.byref(_view_c(view)), C.byref(settings._c()), C.byref(pc))
    if rc != 0:
        raise ValueError("oracle preprocess rejected the settings")
    return out


def _proj_c(proj):
    arrs = [np.ascontiguousarray(proj[name]) for name, _, _ in _PROJ_FIELDS]
    return _Proj(*(_ptr(a) for a in arrs)), arrs


def render(proj, view, settings: Settings, signature: bool = False):
    """Full image (FP64): returns img [3,H,W], T [H,W], ncontrib [H,W], margin [H,W]
    (and, if asked, the per-pixel signature: contributors + 65536 * clamped)."""
    lib = _load()
    W, H = int(view["width"]), int(view["height"])
    n = proj["status"].shape[0]
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), dtype=np.int32)
    mg = np.zeros((H, W))
    sig = np.zeros((H, W), dtype=np.int32)
    pc, keep = _proj_c(proj)
    rc = lib.orc_render(C.byref(_view_c(view)), C.byref(settings._c()), n, C.byref(pc), _ptr(img), _ptr(T),
                        _ptr(nc), _ptr(mg), _ptr(sig))
    if rc != 0:
        raise MemoryError("oracle render failed")
    if signature:
        return img, T, nc, mg, sig
    return img, T, nc, mg


def render_pixels(proj, view, settings: Settings, pix: np.ndarray):
    """Selected pixels (linear ids py*W+px): rgb [P,3], T [P], ncontrib [P], margin [P]."""
    lib = _load()
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    n = proj["status"].shape[0]
    rgb = np.zeros((pix.shape[0], 3))
    T = np.zeros(pix.shape[0])
    nc = np.zeros(pix.shape[0], dtype=np.int32)
    mg = np.zeros(pix.shape[0])
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_pixels(C.byref(_view_c(view)), C.byref(settings._c()), n, C.byref(pc), pix.shape[0],
                               _ptr(pix), _ptr(rgb), _ptr(T), _ptr(nc), _ptr(mg))
    if rc != 0:
        raise MemoryError("oracle render_pixels failed")
    return rgb, T, nc, mg


def render_pixels_admissible(proj, view, settings: Settings, pix: np.ndarray, tol: Tolerance, extra=None,
                             max_cands: int = 64):
    """Every result an FP32 renderer within ``tol`` may produce at the given
    pixels (linear ids py*W+px): a list of [k, 5 + E] arrays (r, g, b, T,
    contributors, extra channels), one per pixel, and flags [P] (bit 1 two
    outcomes were admissible somewhere, bit 2 a composited entry's derivative
    is uncertain, bit 4 the walk ran out of budget)."""
    lib = _load()
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    n = proj["status"].shape[0]
    ne = 0 if extra is None else int(np.asarray(extra).reshape(n, -1).shape[1])
    ex = None if extra is None else np.ascontiguousarray(np.asarray(extra, dtype=np.float64).reshape(n, ne))
    P = pix.shape[0]
    cands = np.zeros((P, max_cands, 5 + ne))
    ncands = np.zeros(P, dtype=np.int32)
    flags = np.zeros(P, dtype=np.int32)
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_pixels_admissible(C.byref(_view_c(view)), C.byref(settings._c()), n, C.byref(pc),
                                          C.byref(tol._c()), _ptr(ex) if ex is not None else None, ne, P, _ptr(pix),
                                          max_cands, _ptr(cands), _ptr(ncands), _ptr(flags))
    if rc != 0:
        raise MemoryError("oracle render_pixels_admissible failed")
    return [cands[q, :ncands[q]] for q in range(P)], flags


def alpha_bounds(proj, view, tol: Tolerance, idx, pix):
    """FP64 alpha = min(0.99, a exp(power)) of Gaussians idx at pixels pix
    (linear ids py*W+px, sample at the centre), and the relative error bound
    of an FP32 renderer's alpha there (render_pixels_admissible's model)."""
    lib = _load()
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    alpha = np.zeros(idx.shape[0])
    err = np.zeros(idx.shape[0])
    pc, keep = _proj_c(proj)
    lib.orc_alpha_bounds(C.byref(_view_c(view)), C.byref(pc), C.byref(tol._c()), idx.shape[0], _ptr(idx), _ptr(pix),
                         _ptr(alpha), _ptr(err))
    return alpha, err


def aux_records(params, proj, view, settings: Settings, flow_dt: float, relax: float = 0.0) -> np.ndarray:
    """Per Gaussian (z, flow_u, flow_v): camera depth of the sliced mean and
    its projected displacement over flow_dt (zeros for culled Gaussians; with
    relax > 0 and a projection from preprocess(..., relax), also filled for
    the Gaussians it marks as possibly present)."""
    lib = _load()
    ph = _ParamsHold(params, settings)
    aux = np.zeros((ph.n, 3))
    pc, keep = _proj_c(proj)
    lib.orc_aux(C.byref(ph.c), C.byref(_view_c(view)), C.byref(settings._c()), float(flow_dt), float(relax),
                C.byref(pc), _ptr(aux))
    return aux


def gated_features(features: np.ndarray, gate=None) -> np.ndarray:
    """Normalised scale-gated features S (.) f / |S (.) f| (FP64, [n, D])."""
    lib = _load()
    f = np.ascontiguousarray(features, dtype=np.float64)
    n, D = f.shape
    g = None if gate is None else np.ascontiguousarray(gate, dtype=np.float64)
    out = np.zeros((n, D))
    lib.orc_gated_features(_ptr(f), n, D, _ptr(g) if g is not None else None, _ptr(out))
    return out


def render_aux(proj, aux: np.ndarray, view, settings: Settings):
    """Image with auxiliary channels (FP64): img [3,H,W], T [H,W],
    aux [4,H,W] = (depth, opacity 1 - T, flow_u, flow_v), margin [H,W]."""
    lib = _load()
    W, H = int(view["width"]), int(view["height"])
    n = proj["status"].shape[0]
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    out = np.zeros((4, H, W))
    mg = np.zeros((H, W))
    aux = np.ascontiguousarray(aux, dtype=np.float64)
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_aux(C.byref(_view_c(view)), C.byref(settings._c()), n, C.byref(pc), _ptr(aux), _ptr(img),
                            _ptr(T), _ptr(out), _ptr(mg))
    if rc != 0:
        raise MemoryError("oracle render_aux failed")
    return img, T, out, mg


def render_features(proj, view, settings: Settings, features: np.ndarray, gate=None):
    """Feature map (FP64) [D, H, W] of the normalised scale-gated features,
    composited with the colour weights; also the pixel margin [H, W]."""
    lib = _load()
    W, H = int(view["width"]), int(view["height"])
    n = proj["status"].shape[0]
    f = np.ascontiguousarray(features, dtype=np.float64)
    D = f.shape[1]
    g = None if gate is None else np.ascontiguousarray(gate, dtype=np.float64)
    out = np.zeros((D, H, W))
    mg = np.zeros((H, W))
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_features(C.byref(_view_c(view)), C.byref(settings._c()), n, C.byref(pc), _ptr(f), D,
                                 _ptr(g) if g is not None else None, _ptr(out), _ptr(mg))
    if rc != 0:
        raise MemoryError("oracle render_features failed")
    return out, mg


def render_features_backward(proj, view, settings: Settings, features: np.ndarray, gate, dF: np.ndarray):
    """dL/dfeatures [n, D] and dL/dgate [D] (FP64) for a loss with feature-map
    gradient dF [D, H, W], geometry held fixed."""
    lib = _load()
    n = proj["status"].shape[0]
    f = np.ascontiguousarray(features, dtype=np.float64)
    D = f.shape[1]
    g = None if gate is None else np.ascontiguousarray(gate, dtype=np.float64)
    dF = np.ascontiguousarray(dF, dtype=np.float64)
    gf = np.zeros((n, D))
    gg = np.zeros(D)
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_features_backward(C.byref(_view_c(view)), C.byref(settings._c()), n, C.byref(pc), _ptr(f),
                                          D, _ptr(g) if g is not None else None, _ptr(dF), _ptr(gf), _ptr(gg))
    if rc != 0:
        raise MemoryError("oracle render_features_backward failed")
    return gf, gg


def _alloc_grads(n, K):
    shapes = {"mean": (n, 4), "log_scale": (n, 4), "q_l": (n, 4), "q_r": (n, 4), "opacity_logit": (n,),
              "sh": (n, K, 3), "g_uv": (n, 2), "g_conic": (n, 3), "g_a": (n,), "g_rgb": (n, 3), "g_z": (n,), "mask_logit": (n,)}
    g = {k: np.zeros(s) for k, s in shapes.items()}
    return g, _Grads(*(_ptr(g[k]) for k in _GRAD_FIELDS))


def render_backward(params, proj, view, settings: Settings, dimg: np.ndarray):
    """Exact reverse-mode gradient (FP64) of <dimg, image> w.r.t. the
    parameters; also returns the per-Gaussian 2D gradients."""
    lib = _load()
    ph = _ParamsHold(params, settings)
    K = ph.arrs["sh"].shape[1]
    g, gc = _alloc_grads(ph.n, K)
    dimg = np.ascontiguousarray(dimg, dtype=np.float64)
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_backward(C.byref(ph.c), C.byref(_view_c(view)), C.byref(settings._c()), C.byref(pc),
                                 _ptr(dimg), C.byref(gc))
    if rc != 0:
        raise MemoryError("oracle backward failed")
    return g


def render_aux_backward(params, proj, view, settings: Settings, dimg: np.ndarray, daux: np.ndarray):
    """Exact reverse-mode gradient (FP64) of <dimg, image> + <daux, aux> with
    aux = (depth, opacity, flow_u, flow_v) of render_aux; the flow planes of
    daux must be zero (flow is not differentiated)."""
    lib = _load()
    ph = _ParamsHold(params, settings)
    K = ph.arrs["sh"].shape[1]
    g, gc = _alloc_grads(ph.n, K)
    dimg = np.ascontiguousarray(dimg, dtype=np.float64)
    daux = np.ascontiguousarray(daux, dtype=np.float64)
    pc, keep = _proj_c(proj)
    rc = lib.orc_render_aux_backward(C.byref(ph.c), C.byref(_view_c(view)), C.byref(settings._c()), C.byref(pc),
                                     _ptr(dimg), _ptr(daux), C.byref(gc))
    if rc == -2:
        raise ValueError("flow planes of daux must be zero")
    if rc != 0:
        raise MemoryError("oracle aux backward failed")
    return g


def split_sample(params, idx, eps, shrink: float) -> dict:
    """Children drawn from the parents' full 4D Gaussians (FP64): eps
    [m, K, 4] standard normal draws; returns parameter arrays of m K rows."""
    lib = _load()
    ph = _ParamsHold(params)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    m, K = idx.shape[0], eps.shape[1]
    K3 = int(np.prod(ph.arrs["sh"].shape[1:]))
    out = {"mean": np.zeros((m * K, 4)), "log_scale": np.zeros((m * K, 4)), "q_l": np.zeros((m * K, 4)),
           "q_r": np.zeros((m * K, 4)), "opacity_logit": np.zeros(m * K),
           "sh": np.zeros((m * K,) + ph.arrs["sh"].shape[1:])}
    rc = lib.orc_split_sample(C.byref(ph.c), _ptr(idx), m, K, _ptr(eps), float(shrink), K3, _ptr(out["mean"]),
                              _ptr(out["log_scale"]), _ptr(out["q_l"]), _ptr(out["q_r"]),
                              _ptr(out["opacity_logit"]), _ptr(out["sh"]))
    if rc != 0:
        raise ValueError("index out of range")
    return out


def densify_stats(params, proj, view, settings: Settings, dimg: np.ndarray) -> np.ndarray:
    """Densification indicators of one view (Sec. 3.3, densification in
    spacetime) for a loss with image gradient dimg: per Gaussian
    (|dL/d(u, v)|, |dL/dmu_t|, 1 if visible else 0, 0), from the adjoint."""
    g = render_backward(params, proj, view, settings, dimg)
    vis = proj["status"] == 0
    out = np.zeros((vis.shape[0], 4))
    out[:, 0] = np.sqrt(g["g_uv"][:, 0] ** 2 + g["g_uv"][:, 1] ** 2)
    out[:, 1] = np.abs(g["mean"][:, 3])
    out[:, 2] = 1.0
    out[~vis] = 0.0
    return out


def preprocess_backward(params, view, settings: Settings, g_uv, g_conic, g_a, g_rgb):
    """Adjoint of the per-Gaussian chain alone, from given 2D gradients."""
    lib = _load()
    ph = _ParamsHold(params, settings)
    K = ph.arrs["sh"].shape[1]
    g, gc = _alloc_grads(ph.n, K)
    ins = [np.ascontiguousarray(a, dtype=np.float64) for a in (g_uv, g_conic, g_a, g_rgb)]
    lib.orc_preprocess_backward(C.byref(ph.c), C.byref(_view_c(view)), C.byref(settings._c()),
                                *(_ptr(a) for a in ins), C.byref(gc))
    return g


def rotation(q_l, q_r) -> np.ndarray:
    """R = L(q_l) R(q_r) for the normalised quaternions (4x4)."""
    lib = _load()
    a = np.ascontiguousarray(q_l, dtype=np.float64)
    b = np.ascontiguousarray(q_r, dtype=np.float64)
    R = np.zeros((4, 4))
    lib.orc_rotation(_ptr(a), _ptr(b), _ptr(R))
    return R


def real_sh(L: int, direction) -> np.ndarray:
    """Real orthonormal SH values Y_lm (index l*l+l+m) at a unit direction."""
    lib = _load()
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros((L + 1) ** 2)
    lib.orc_real_sh(L, _ptr(d), _ptr(Y))
    return Y


def sort_instances(rect, depth_f32, grid_w: int, grid_h: int, cap: int | None = None):
    """Tile-binned instance list of the tile rasterizer: one instance per tile
    of each rect, sorted by (tile, FP32 depth, index).
    Returns (keys u64 [M], vals i64 [M], ranges i64 [tiles, 2])."""
    lib = _load()
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    depth_f32 = np.ascontiguousarray(depth_f32, dtype=np.float32)
    n = rect.shape[0]
    w = np.clip(rect[:, 2] - rect[:, 0], 0, None).astype(np.int64)
    h = np.clip(rect[:, 3] - rect[:, 1], 0, None).astype(np.int64)
    m = int((w * h).sum())
    cap = m if cap is None else cap
    keys = np.zeros(max(m, 1), dtype=np.uint64)
    vals = np.zeros(max(m, 1), dtype=np.int64)
    ranges = np.zeros((grid_w * grid_h, 2), dtype=np.int64)
    got = lib.orc_sort_instances(n, _ptr(rect), _ptr(depth_f32), grid_w, grid_h, cap, _ptr(keys), _ptr(vals),
                                 _ptr(ranges))
    if got < 0:
        raise ValueError("instance count exceeds capacity")
    return keys[:got], vals[:got], ranges


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads the oracle's parallel loops use from now on."""
    _load().orc_set_num_threads(int(n))
