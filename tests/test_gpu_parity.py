"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element
by element on the same seeded inputs: per-Gaussian records, sort order (bit
exact), images, transmittance, contributor counts and gradients; plus the
edge cases of the method (empty scene, all culled, non-finite parameters,
capacity overflow) and the batched form."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig

from helpers import (PIXEL_MARGIN, GpuRun, canonical_ranges, compare_group, keep_clear_of_boundaries, oracle_settings,
                     records_from_gpu, subset)

pytestmark = pytest.mark.gpu

IMAGE_ATOL = 2e-4


def tiny_case(width=128, height=96, L=1, NT=1, bg=(0.0, 0.0, 0.0), seed=0, n=2000, t=0.5, tile=16):
    sc = sy.make_scene(n, seed, (-1, -1, -1), (1, 1, 1), sh_degree=L, t_order=NT)
    view = sy.tiny_view(width, height, t=t)
    cfg = RenderConfig(sh_degree=L, t_order=NT, bg=bg, inst_capacity=1 << 18, tile=tile)
    params = sc.as_dict()
    return subset(params, keep_clear_of_boundaries(params, [view], cfg)), view, cfg


def check_records(run, params, view, cfg, sample=None):
    pr = oracle.preprocess(params, view, oracle_settings(cfg))
    vis = np.flatnonzero(pr["status"] == 0)
    rec = records_from_gpu(run)
    np.testing.assert_array_equal(rec["index"], vis)
    sel = np.arange(vis.size) if sample is None else sample
    i = vis[sel]
    np.testing.assert_array_equal(rec["rect"][sel], pr["rect"][i])
    compare_group("uv", rec["uv"][sel], pr["uv"][i], 1e-6, 2e-7)
    compare_group("conic", rec["conic"][sel], pr["conic"][i], 2e-4, 1e-6)
    compare_group("a", rec["a"][sel], pr["a_eff"][i], 1e-5, 1e-7)
    compare_group("rgb", rec["rgb"][sel], pr["rgb"][i], 1e-5, 1e-6)
    compare_group("tau", rec["tau"][sel], np.log2(255.0 * pr["a_eff"][i]) + 4e-3, 1e-5, 1e-6)
    db = rec["depth_bits"][sel].astype(np.int64) - pr["depth_f32"][i].view(np.uint32).astype(np.int64)
    # The FP32 depth comes out of a longer rounded chain than the FP64 oracle's
    # rounded depth: within 2 ulp, mostly equal.
    assert np.abs(db).max() <= 2
    assert (db == 0).mean() >= 0.8
    return pr


def check_image(run, params, view, cfg, k=0):
    ost = oracle_settings(cfg)
    pr = oracle.preprocess(params, view, ost)
    img, T, nc, mg = oracle.render(pr, view, ost)
    ok = mg >= PIXEL_MARGIN
    assert ok.mean() >= 0.97, ok.mean()
    err = np.abs(run.images[k] - img)[:, ok]
    assert err.max() <= IMAGE_ATOL, err.max()
    # List positions differ from the oracle's (tiles a Gaussian cannot reach
    # at 1/255 are not in the GPU's lists), the transmittance does not.
    Tg, lastg = run.pixel_planes(k)
    assert np.abs(Tg - T)[ok].max() <= IMAGE_ATOL
    assert np.all((lastg == 0) == (nc == 0))
    return img, mg


# ------------------------------------------------------------- forward

def test_preprocess_records_match_oracle():
    params, view, cfg = tiny_case()
    run = GpuRun(params, [view], cfg)
    check_records(run, params, view, cfg)


@pytest.mark.parametrize("w,h,L,NT,bg", [(128, 96, 1, 1, (0.0, 0.0, 0.0)),
                                         (131, 77, 3, 2, (0.2, 0.5, 0.7)),
                                         (40, 200, 2, 0, (1.0, 1.0, 1.0)),
                                         (17, 33, 0, 4, (0.0, 0.3, 0.0))])
def test_image_matches_oracle(w, h, L, NT, bg):
    params, view, cfg = tiny_case(w, h, L, NT, bg)
    run = GpuRun(params, [view], cfg)
    check_records(run, params, view, cfg)
    check_image(run, params, view, cfg)


def _opaque_case():
    """A tenth of the Gaussians opaque (a = sigmoid(6) > 0.99) and centred at
    the view's timestamp (p(t) = 1): the 0.99 clamp acts near their centres."""
    sc = sy.make_scene(2000, 21, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    view = sy.tiny_view(112, 90, t=0.5)
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 18)
    params = sc.as_dict()
    params["opacity_logit"][::10] = 6.0
    params["mean"][::10, 3] = 0.5
    return subset(params, keep_clear_of_boundaries(params, [view], cfg)), view, cfg


def test_opaque_gaussians_reach_the_clamp():
    """Image and gradients with entries that reach min(0.99, a G): both the
    forward's per-batch clamp selection and the backward's constant clamp."""
    params, view, cfg = _opaque_case()
    pr = oracle.preprocess(params, view, oracle_settings(cfg))
    assert (pr["a_eff"][pr["status"] == 0] > 0.99).sum() >= 20
    run = GpuRun(params, [view], cfg)
    check_image(run, params, view, cfg)
    check_gradients(*_grad_case(params, view, cfg))


def test_full_size_orbit_view_sampled():
    """The benchmark's launch configuration (300k Gaussians, SH degree 3 x
    temporal order 2, 1352x1014, one view per call): sampled records and
    pixels against the oracle, which gathers each sampled pixel's list by a
    scan over all Gaussians."""
    sc = sy.orbit_scene()
    view = sy.orbit_view(37)
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 23)
    params = sc.as_dict()
    params = subset(params, keep_clear_of_boundaries(params, [view], cfg))
    run = GpuRun(params, [view], cfg)
    rng = np.random.default_rng(7)
    nv = run.counts[0]
    assert nv > 50_000
    check_records(run, params, view, cfg, sample=rng.choice(nv, 20_000, replace=False))
    W, H = view["width"], view["height"]
    pix = rng.choice(W * H, 3000, replace=False)
    ty, tx = 31, 40  # plus every pixel of one full tile
    tile_pix = np.array([(ty * 16 + y) * W + tx * 16 + x for y in range(16) for x in range(16)])
    pix = np.concatenate([pix, tile_pix])
    ost = oracle_settings(cfg)
    pr = oracle.preprocess(params, view, ost)
    rgb, T, nc, mg = oracle.render_pixels(pr, view, ost, pix)
    ok = mg >= PIXEL_MARGIN
    # ~180 alpha evaluations per pixel at this size: about one pixel in eight
    # has some decision within 1e-3 of its threshold.
    assert ok.mean() >= 0.8
    gimg = run.images[0].reshape(3, -1)[:, pix].T
    assert np.abs(gimg - rgb)[ok].max() <= IMAGE_ATOL
    Tg, lastg = run.pixel_planes(0)
    assert np.abs(Tg.reshape(-1)[pix] - T)[ok].max() <= IMAGE_ATOL


def test_batched_views_equal_single_views():
    sc = sy.make_scene(3000, 4, (-1, -1, -1), (1, 1, 1), sh_degree=3, t_order=2)
    views = [sy.tiny_view(128, 96, t=0.4),
             sy.look_at((1.5, -0.5, -2.5), (0, 0, 0), (0, -1, 0), 100, 70, 0.6),
             sy.look_at((-2.0, 0.3, 2.0), (0, 0, 0), (0, -1, 0), 64, 64, 0.55)]
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 19, bg=(0.1, 0.0, 0.2))
    params = sc.as_dict()
    params = subset(params, keep_clear_of_boundaries(params, views, cfg))
    batch = GpuRun(params, views, cfg)
    for k, v in enumerate(views):
        single = GpuRun(params, [v], cfg)
        np.testing.assert_array_equal(batch.images[k], single.images[0])
        check_image(batch, params, v, cfg, k)


def _check_views_against_oracle(run, params, views, cfg, min_clear=0.95):
    """Every view of one call against the oracle; the share of pixels clear
    of a per-pixel decision is bounded over all views together (a view of a
    handful of pixels can be wholly flagged)."""
    ost = oracle_settings(cfg)
    n_clear = n_all = 0
    for k, v in enumerate(views):
        pr = oracle.preprocess(params, v, ost)
        img, T, nc, mg = oracle.render(pr, v, ost)
        ok = mg >= PIXEL_MARGIN
        n_clear += int(ok.sum())
        n_all += ok.size
        assert run.images[k].shape == (3, v["height"], v["width"])
        Tg, lastg = run.pixel_planes(k)
        assert np.all((lastg == 0) == (nc == 0))
        if ok.any():
            assert np.abs(run.images[k] - img)[:, ok].max() <= IMAGE_ATOL
            assert np.abs(Tg - T)[ok].max() <= IMAGE_ATOL
    assert n_clear / n_all >= min_clear


def _crop(view, x0, y0, w, h):
    """The w x h window at (x0, y0) of a view's image, as a view of its own
    (same focal length, principal point shifted)."""
    v = dict(view)
    v.update(width=w, height=h, cx=np.float32(view["cx"] - x0), cy=np.float32(view["cy"] - y0))
    return v


@pytest.mark.parametrize("tile", [16, 8])
def test_single_pixel_and_one_pixel_wide_views(tile):
    """Windows of a 128x96 view smaller than one tile and one pixel wide or
    high, batched with windows one pixel past a tile edge: every tile is
    ragged."""
    sc = sy.make_scene(2000, 9, (-1, -1, -1), (1, 1, 1), sh_degree=2, t_order=1)
    full = sy.tiny_view(128, 96, t=0.5)
    views = [_crop(full, 64, 48, 1, 1), _crop(full, 70, 20, 1, 40), _crop(full, 40, 50, 37, 1),
             _crop(full, 50, 30, tile, tile), _crop(full, 30, 25, tile + 1, 2 * tile + 1),
             _crop(sy.tiny_view(128, 96, t=0.3), 0, 0, 128, 96)]
    cfg = RenderConfig(sh_degree=2, t_order=1, inst_capacity=1 << 18, bg=(0.3, 0.2, 0.1), tile=tile)
    params = sc.as_dict()
    params = subset(params, keep_clear_of_boundaries(params, views, cfg))
    run = GpuRun(params, views, cfg)
    _check_views_against_oracle(run, params, views, cfg)


def test_maximum_view_count_in_one_call():
    """FGS4D_MAX_VIEWS (camera, t) views of four sizes in one call: each
    matches the oracle, and the first and last equal their single-view
    renders bit for bit."""
    sc = sy.make_scene(2000, 10, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    sizes = ((24, 20), (33, 17), (16, 16), (9, 40))
    views = []
    for k in range(fgs4d.MAX_VIEWS):
        th = 2.0 * math.pi * k / fgs4d.MAX_VIEWS
        w, h = sizes[k % 4]
        views.append(sy.look_at((3.0 * math.sin(th), 0.4 * math.cos(3 * th), -3.0 * math.cos(th)), (0, 0, 0),
                                (0, -1, 0), w, h, k / (fgs4d.MAX_VIEWS - 1), hfov_deg=15.0))
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 20, bg=(0.0, 0.1, 0.0))
    params = sc.as_dict()
    params = subset(params, keep_clear_of_boundaries(params, views, cfg))
    run = GpuRun(params, views, cfg)
    _check_views_against_oracle(run, params, views, cfg)
    for k in (0, fgs4d.MAX_VIEWS - 1):
        np.testing.assert_array_equal(run.images[k], GpuRun(params, [views[k]], cfg).images[0])


def test_block_shapes_render_identically():
    """The autotuned compositor block shape (pixels per thread) changes the
    work split, not the arithmetic: bit-identical images, gradients equal up
    to the order of the atomic sums."""
    params, view, cfg = tiny_case(131, 77, 3, 2, (0.2, 0.1, 0.0))
    rng = np.random.default_rng(12)
    dimg = rng.standard_normal((3, 77, 131))
    runs = []
    for p, b in ((2, 256), (4, 256), (8, 256), (4, 128), (2, 128)):  # shapes and shared batch sizes
        c = RenderConfig(**{**cfg.__dict__, "pixels_per_thread": p, "shared_batch": b})
        run = GpuRun(params, [view], c)
        runs.append((run, run.backward([dimg])[0]))
    for run, g in runs[1:]:
        np.testing.assert_array_equal(run.images[0], runs[0][0].images[0])
        np.testing.assert_array_equal(run.T, runs[0][0].T)
        np.testing.assert_array_equal(run.last, runs[0][0].last)
        for k in PARAM_KEYS:
            compare_group(k, g[k], runs[0][1][k], 1e-4, 1e-5)


def test_autotune_picks_a_candidate_and_keeps_the_image():
    import torch
    from paper_2412_20720_gb300.render import Renderer, autotune
    from helpers import to_device
    params, view, cfg = tiny_case()
    r = Renderer(params["mean"].shape[0], [view], cfg)
    dev = to_device(params)
    ref = r.forward(dev).clone()
    res = autotune(r, dev, reps=2)
    assert res["pixels_per_thread"] in (2, 4, 8) and set(res["ms"]) == {"16/2/256", "16/4/256", "16/8/256"}
    assert r.settings.pixels_per_thread == res["pixels_per_thread"]
    assert torch.equal(r.forward(dev), ref)


# ------------------------------------------------------------- sort

def _write_records(r, rec, view_of_slot):
    """Writes synthetic per-slot records straight into the workspace."""
    import torch
    n = rec["rect"].shape[0]
    rect = rec["rect"]
    meta = np.zeros((n, 4), dtype=np.int32)
    meta[:, 0] = np.arange(n)
    meta[:, 1] = view_of_slot
    meta[:, 2] = rect[:, 0] | (rect[:, 1] << 16)
    meta[:, 3] = rect[:, 2] | (rect[:, 3] << 16)
    geom = np.concatenate([rec["uv"], rec["conic2"][:, :2]], axis=1).astype(np.float32)
    color = np.zeros((n, 4), dtype=np.float32)
    color[:, 0] = rec["conic2"][:, 2]
    color[:, 1] = -1.0  # log2 of the opacity 0.5
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    r.workspace_view(r.layout.counters, torch.int32, 64).zero_()
    r.workspace_view(r.layout.counters, torch.int32, 1).fill_(n)
    r.workspace_view(r.layout.rec_meta, torch.int32, 4 * n).copy_(dev(meta))
    r.workspace_view(r.layout.rec_geom, torch.float32, 4 * n).copy_(dev(geom))
    r.workspace_view(r.layout.rec_color, torch.float32, 4 * n).copy_(dev(color))
    r.workspace_view(r.layout.rec_tau, torch.float32, n).copy_(dev(rec["tau"].astype(np.float32)))
    r.workspace_view(r.layout.depth_key, torch.int32, n).copy_(dev(rec["depth"].astype(np.float32).view(np.int32)))


def _synthetic_records(rng, n, W, H, max_extent, tile=16):
    """Random tile rects, FP32 depths with exact ties, and 1/255 ellipses
    (u, v, A', B', C', tau) around centres near the rects."""
    gw, gh = (W + tile - 1) // tile, (H + tile - 1) // tile
    x0 = rng.integers(0, gw, n)
    y0 = rng.integers(0, gh, n)
    rect = np.stack([x0, y0, np.minimum(gw, x0 + rng.integers(0, max_extent, n)),
                     np.minimum(gh, y0 + rng.integers(0, max_extent, n))], axis=1).astype(np.int32)
    depth = rng.uniform(0.3, 40.0, n).astype(np.float32)
    depth[rng.integers(0, n, n // 10)] = depth[0]  # exact ties: order by slot
    depth[::97] = np.float32(0.2) + np.float32(1e-7)
    cx = (rect[:, 0] + rect[:, 2]) * (tile / 2) + rng.uniform(-tile / 2, tile / 2, n)
    cy = (rect[:, 1] + rect[:, 3]) * (tile / 2) + rng.uniform(-tile / 2, tile / 2, n)
    ang = rng.uniform(0, np.pi, n)
    s1 = np.exp(rng.uniform(np.log(0.5), np.log(30.0), n))
    s2 = np.exp(rng.uniform(np.log(0.5), np.log(30.0), n))
    c, s = np.cos(ang), np.sin(ang)
    k = 0.5 * np.log2(np.e)
    A = k * (c * c / s1 ** 2 + s * s / s2 ** 2)
    B = k * 2 * c * s * (1 / s1 ** 2 - 1 / s2 ** 2)
    C = k * (s * s / s1 ** 2 + c * c / s2 ** 2)
    return {"rect": rect, "depth": depth, "uv": np.stack([cx, cy], 1).astype(np.float32),
            "conic2": np.stack([A, B, C], 1).astype(np.float32), "tau": rng.uniform(0.0, 8.0, n).astype(np.float32)}


def _oracle_sorted(rec, W, H, tile=16):
    gw, gh = (W + tile - 1) // tile, (H + tile - 1) // tile
    return oracle.sort_instances(rec["rect"], rec["depth"], gw, gh, uv=rec["uv"], conic2=rec["conic2"],
                                 tau=rec["tau"], width=W, height=H, tile=tile)


# Visible capacities equal to the slot count and well above it (the pair scan
# and depth sort size their grids and look-back rows by the capacity).
@pytest.mark.parametrize("n,W,H,vis_cap", [(1, 16, 16, 0), (2047, 144, 112, 0), (70_001, 1352, 1014, 0),
                                           (70_001, 1352, 1014, 400_000), (150_001, 1352, 1014, 0)])
def test_bin_sort_bit_exact_on_synthetic_records(n, W, H, vis_cap):
    """Sorted instance list and tile ranges equal the oracle's bit for bit:
    the tiles of each rect that the FP32 ellipse test keeps, ordered by (tile,
    FP32 depth, slot), on records written straight into the workspace
    (ragged counts, exact depth ties, empty rects)."""
    import torch
    from paper_2412_20720_gb300.render import Renderer
    rng = np.random.default_rng(n)
    gw, gh = (W + 15) // 16, (H + 15) // 16
    rec = _synthetic_records(rng, n, W, H, 6)
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=40 * n + 16, vis_capacity=vis_cap)
    r = Renderer(n, [sy.tiny_view(W, H)], cfg)
    _write_records(r, rec, 0)
    fgs4d.bin_sort(n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, r.stream())
    counts = r.check()
    keys, vals, ranges = _oracle_sorted(rec, W, H)
    m = keys.shape[0]
    assert counts[1] == m
    full, _, _ = oracle.sort_instances(rec["rect"], rec["depth"], gw, gh)
    assert n < 10 or m < full.shape[0]  # the ellipse test drops tiles
    tiles = r.workspace_view(r.layout.inst_tile, torch.int32, m).cpu().numpy()
    slots = r.workspace_view(r.layout.inst_slot, torch.int32, m).cpu().numpy()
    gr = r.workspace_view(r.layout.tile_ranges, torch.int32, 2 * gw * gh).cpu().numpy().reshape(-1, 2)
    np.testing.assert_array_equal(tiles, (keys >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(slots, vals)
    np.testing.assert_array_equal(rec["depth"][slots].view(np.uint32),
                                  (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32))
    np.testing.assert_array_equal(canonical_ranges(gr), ranges)
    sorted_slots = r.workspace_view(r.layout.sorted_slots, torch.int32, n).cpu().numpy()
    np.testing.assert_array_equal(sorted_slots, np.argsort(rec["depth"], kind="stable"))


def test_bin_sort_bit_exact_multi_view():
    import torch
    from paper_2412_20720_gb300.render import Renderer
    rng = np.random.default_rng(99)
    sizes = [(200, 150), (64, 48), (1014, 1352)]
    ns = [3000, 500, 9000]
    views = [sy.tiny_view(w, h) for w, h in sizes]
    recs = [_synthetic_records(rng, n, w, h, 5) for n, (w, h) in zip(ns, sizes)]
    rec = {k: np.concatenate([x[k] for x in recs]) for k in recs[0]}
    vo = np.concatenate([np.full(n, k) for k, n in enumerate(ns)])
    total = rec["rect"].shape[0]
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=30 * total, vis_capacity=total)
    r = Renderer(total, views, cfg)
    _write_records(r, rec, vo)
    fgs4d.bin_sort(total, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, r.stream())
    counts = r.check()
    exp_tiles, exp_slots, exp_ranges = [], [], []
    tile_base = slot_base = inst_base = 0
    for k, (n, (w, h)) in enumerate(zip(ns, sizes)):
        keys, vals, ranges = _oracle_sorted(recs[k], w, h)
        exp_tiles.append((keys >> np.uint64(32)).astype(np.int64) + tile_base)
        exp_slots.append(vals + slot_base)
        rr = ranges.copy()
        nz = rr[:, 1] > rr[:, 0]
        rr[nz] += inst_base
        exp_ranges.append(rr)
        tile_base += ((w + 15) // 16) * ((h + 15) // 16)
        slot_base += n
        inst_base += keys.shape[0]
    m = inst_base
    assert counts[1] == m
    tiles = r.workspace_view(r.layout.inst_tile, torch.int32, m).cpu().numpy()
    slots = r.workspace_view(r.layout.inst_slot, torch.int32, m).cpu().numpy()
    gr = r.workspace_view(r.layout.tile_ranges, torch.int32, 2 * tile_base).cpu().numpy().reshape(-1, 2)
    np.testing.assert_array_equal(tiles, np.concatenate(exp_tiles))
    np.testing.assert_array_equal(slots, np.concatenate(exp_slots))
    np.testing.assert_array_equal(canonical_ranges(gr), np.concatenate(exp_ranges))


# ------------------------------------------------------------- edge cases

def test_empty_scene_renders_background():
    view = sy.tiny_view(50, 30)
    cfg = RenderConfig(sh_degree=1, t_order=1, bg=(0.25, 0.5, 0.75), inst_capacity=1024)
    empty = {k: v[:0] for k, v in sy.tiny_scene().as_dict().items()}
    run = GpuRun(empty, [view], cfg)
    assert run.counts[:2] == [0, 0]
    for ch, b in enumerate(cfg.bg):
        assert np.all(run.images[0][ch] == np.float32(b))
    assert np.all(run.T == 1.0) and np.all(run.last == 0)


def test_all_temporally_culled_renders_background():
    sc = sy.tiny_scene().as_dict()
    sc["mean"][:, 3] = 50.0  # far from t = 0.5 for every temporal scale
    view = sy.tiny_view(64, 48)
    cfg = RenderConfig(sh_degree=1, t_order=1, bg=(0.3, 0.3, 0.3), inst_capacity=1024)
    run = GpuRun(sc, [view], cfg)
    assert run.counts[0] == 0
    assert np.all(run.images[0] == np.float32(0.3))


def test_non_finite_parameters_are_culled_not_propagated():
    params, view, cfg = tiny_case(n=1500)
    clean = GpuRun(params, [view], cfg)
    bad = {k: v.copy() for k, v in params.items()}
    n = bad["mean"].shape[0]
    rng = np.random.default_rng(3)
    idx = rng.choice(n, 40, replace=False)
    for j, i in enumerate(idx):
        key = ("mean", "log_scale", "q_l", "q_r", "opacity_logit")[j % 5]
        val = (np.nan, np.inf, -np.inf)[j % 3]
        if key == "opacity_logit":
            bad[key][i] = val
        else:
            bad[key][i, j % 4] = val
    bad["q_l"][idx[0]] = 0.0  # zero quaternion: invalid
    keep = np.ones(n, bool)
    keep[idx] = False
    poisoned = GpuRun(bad, [view], cfg)
    removed = GpuRun(subset(params, keep), [view], cfg)
    assert np.isfinite(poisoned.images[0]).all()
    np.testing.assert_array_equal(poisoned.images[0], removed.images[0])


def test_instance_capacity_overflow_is_reported_and_recoverable():
    params, view, cfg = tiny_case()
    full = GpuRun(params, [view], cfg)
    need = full.counts[1]
    small = RenderConfig(sh_degree=1, t_order=1, inst_capacity=max(1, need // 3))
    from paper_2412_20720_gb300.render import Renderer
    from helpers import to_device
    r = Renderer(params["mean"].shape[0], [view], small)
    r.forward(to_device(params))
    code, counts = r.status()
    assert code == fgs4d.ERR_CAPACITY
    assert counts[1] == need // 3 and counts[3] == need
    again = GpuRun(params, [view], RenderConfig(sh_degree=1, t_order=1, inst_capacity=counts[3]))
    np.testing.assert_array_equal(again.images[0], full.images[0])


def test_visible_capacity_overflow_is_reported():
    params, view, cfg = tiny_case()
    from paper_2412_20720_gb300.render import Renderer
    from helpers import to_device
    r = Renderer(params["mean"].shape[0], [view], RenderConfig(sh_degree=1, t_order=1, vis_capacity=10,
                                                               inst_capacity=1 << 16))
    r.forward(to_device(params))
    code, counts = r.status()
    assert code == fgs4d.ERR_CAPACITY
    assert counts[0] == 10 and counts[2] > 10


# ------------------------------------------------------------- gradients

def _grad_case(params, view, cfg, seed=5):
    run = GpuRun(params, [view], cfg)
    ost = oracle_settings(cfg)
    pr = oracle.preprocess(params, view, ost)
    img, T, nc, mg = oracle.render(pr, view, ost)
    ok = mg >= PIXEL_MARGIN
    rng = np.random.default_rng(seed)
    dimg = rng.standard_normal(img.shape) * ok
    g_orc = oracle.render_backward(params, pr, view, ost, dimg)
    g_gpu, slot = run.backward([dimg])
    vis = records_from_gpu(run)["index"]
    return g_gpu, slot, g_orc, vis


def check_gradients(g_gpu, slot, g_orc, vis, rtol=1e-3, floor=1e-4):
    compare_group("g_uv", slot[:, 0:2], g_orc["g_uv"][vis], rtol, floor)
    compare_group("g_conic", slot[:, 2:5], g_orc["g_conic"][vis], rtol, floor)
    compare_group("g_a", slot[:, 5], g_orc["g_a"][vis], rtol, floor)
    compare_group("g_rgb", slot[:, 6:9], g_orc["g_rgb"][vis], rtol, floor)
    for k in PARAM_KEYS:
        compare_group(k, g_gpu[k], g_orc[k], rtol, floor)


@pytest.mark.parametrize("L,NT,bg", [(1, 1, (0.0, 0.0, 0.0)), (3, 2, (0.1, 0.2, 0.3))])
def test_gradients_match_oracle(L, NT, bg):
    params, view, cfg = tiny_case(96, 80, L, NT, bg)
    check_gradients(*_grad_case(params, view, cfg))


def test_gradients_match_oracle_on_fd_subset():
    """The 64-Gaussian 32x32 subset at degree 3 x order 2 whose oracle
    adjoint is pinned to FP64 finite differences on the CPU."""
    sc = sy.make_scene(64, 33, (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5),
                       spatial_log_scale=(math.log(0.03), math.log(0.12)), sh_degree=3, t_order=2)
    view = sy.tiny_view(32, 32, t=0.45)
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 12)
    params = sc.as_dict()
    params = subset(params, keep_clear_of_boundaries(params, [view], cfg))
    check_gradients(*_grad_case(params, view, cfg))


def test_l1_loss_kernel():
    import torch
    from paper_2412_20720_gb300.render import l1_loss
    rng = np.random.default_rng(8)
    a = rng.standard_normal(100_003).astype(np.float32)
    b = rng.standard_normal(100_003).astype(np.float32)
    b[:10] = a[:10]
    loss, grad = l1_loss(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    ref = np.abs(a.astype(np.float64) - b).mean()
    assert abs(float(loss.item()) - ref) <= 1e-5 * ref
    g = grad.cpu().numpy()
    np.testing.assert_array_equal(g, np.sign(a - b).astype(np.float32) / np.float32(a.size))
