"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element
by element on the same seeded inputs: per-Gaussian records, sort order (bit
exact), instance lists against the tile rasterizer's rect membership,
images, transmittance and gradients; plus the edge cases of the method
(empty scene, all culled, non-finite parameters, capacity overflow) and the
batched form.  No Gaussian is removed from the inputs and every pixel is
checked: where FP32 may take a decision either way, the GPU must match one
of the oracle's admissible results (helpers.py)."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig

from helpers import (CudaRender, canonical_ranges, check_image, check_pixels, check_records, compare_group,
                     loss_gradient_at_settled_pixels, oracle_proj, oracle_settings, pixel_tolerance, records_from_gpu,
                     subset)

pytestmark = pytest.mark.gpu


def tiny_case(width=128, height=96, L=1, NT=1, bg=(0.0, 0.0, 0.0), seed=0, n=2000, t=0.5, tile=16):
    sc = sy.make_scene(n, seed, (-1, -1, -1), (1, 1, 1), sh_degree=L, t_order=NT)
    view = sy.tiny_view(width, height, t=t)
    cfg = RenderConfig(sh_degree=L, t_order=NT, bg=bg, inst_capacity=1 << 18, tile=tile)
    return sc.as_dict(), view, cfg


# ------------------------------------------------------------- forward

def test_preprocess_records_match_oracle():
    params, view, cfg = tiny_case()
    run = CudaRender(params, [view], cfg)
    check_records(run, params, view, cfg)


@pytest.mark.parametrize("w,h,L,NT,bg", [(128, 96, 1, 1, (0.0, 0.0, 0.0)),
                                         (131, 77, 3, 2, (0.2, 0.5, 0.7)),
                                         (40, 200, 2, 0, (1.0, 1.0, 1.0)),
                                         (17, 33, 0, 4, (0.0, 0.3, 0.0))])
def test_image_matches_oracle(w, h, L, NT, bg):
    params, view, cfg = tiny_case(w, h, L, NT, bg)
    run = CudaRender(params, [view], cfg)
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
    return params, view, cfg


def test_opaque_gaussians_reach_the_clamp():
    """Image and gradients with entries that reach min(0.99, a G): both the
    forward's per-batch clamp selection and the backward's constant clamp."""
    params, view, cfg = _opaque_case()
    pr = oracle.preprocess(params, view, oracle_settings(cfg))
    assert (pr["a_eff"][pr["status"] == 0] > 0.99).sum() >= 20
    run = CudaRender(params, [view], cfg)
    check_image(run, params, view, cfg)
    check_gradients(*_grad_case(params, view, cfg))


def test_full_size_orbit_view_sampled():
    """The benchmark's launch configuration (300k Gaussians, SH degree 3 x
    temporal order 2, 1352x1014, one view per call): sampled records and
    pixels (plus every pixel of one tile) against the oracle, which gathers
    each sampled pixel's list by a scan over all Gaussians."""
    sc = sy.orbit_scene()
    view = sy.orbit_view(37)
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 23)
    params = sc.as_dict()
    run = CudaRender(params, [view], cfg)
    rng = np.random.default_rng(7)
    nv = run.counts[0]
    assert nv > 50_000
    pr = check_records(run, params, view, cfg, sample=rng.choice(nv, 20_000, replace=False))
    W, H = view["width"], view["height"]
    pix = rng.choice(W * H, 3000, replace=False)
    ty, tx = 31, 40  # plus every pixel of one full tile
    tile_pix = np.array([(ty * 16 + y) * W + tx * 16 + x for y in range(16) for x in range(16)])
    pix = np.concatenate([pix, tile_pix])
    Tg, lastg = run.pixel_planes(0)
    flags, _ = check_pixels(pr, view, cfg, pix, run.images[0].reshape(3, -1)[:, pix].T, Tg.reshape(-1)[pix],
                            lastg.reshape(-1)[pix])
    assert (flags & 1).mean() < 0.2  # most pixels have one admissible result


def test_batched_views_equal_single_views():
    sc = sy.make_scene(3000, 4, (-1, -1, -1), (1, 1, 1), sh_degree=3, t_order=2)
    views = [sy.tiny_view(128, 96, t=0.4),
             sy.look_at((1.5, -0.5, -2.5), (0, 0, 0), (0, -1, 0), 100, 70, 0.6),
             sy.look_at((-2.0, 0.3, 2.0), (0, 0, 0), (0, -1, 0), 64, 64, 0.55)]
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 19, bg=(0.1, 0.0, 0.2))
    params = sc.as_dict()
    batch = CudaRender(params, views, cfg)
    for k, v in enumerate(views):
        single = CudaRender(params, [v], cfg)
        np.testing.assert_array_equal(batch.images[k], single.images[0])
        check_records(batch, params, v, cfg, k)
        check_image(batch, params, v, cfg, k)


def _check_views_against_oracle(run, params, views, cfg):
    """Every pixel of every view of one call against the oracle."""
    for k, v in enumerate(views):
        assert run.images[k].shape == (3, v["height"], v["width"])
        check_records(run, params, v, cfg, k)
        check_image(run, params, v, cfg, k)


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
    run = CudaRender(params, views, cfg)
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
    run = CudaRender(params, views, cfg)
    _check_views_against_oracle(run, params, views, cfg)
    for k in (0, fgs4d.MAX_VIEWS - 1):
        np.testing.assert_array_equal(run.images[k], CudaRender(params, [views[k]], cfg).images[0])


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
        run = CudaRender(params, [view], c)
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
    # the record's factors of the base-2 form A' dx^2 + B' dx dy + C' dy^2 =
    # (a1 dx)^2 + (b1 dx + b2 dy)^2
    A, B, C = (rec["conic2"][:, j].astype(np.float64) for j in range(3))
    b2 = np.sqrt(C)
    b1 = B / (2 * b2)
    a1 = np.sqrt(A - b1 * b1)
    geom = np.stack([rec["uv"][:, 0], rec["uv"][:, 1], a1, b1], axis=1).astype(np.float32)
    color = np.zeros((n, 4), dtype=np.float32)
    color[:, 0] = b2
    color[:, 1] = -1.0  # log2 of the opacity 0.5
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    r.workspace_view(r.layout.counters, torch.int32, 64).zero_()
    r.workspace_view(r.layout.counters, torch.int32, 1).fill_(n)
    r.workspace_view(r.layout.rec_meta, torch.int32, 4 * n).copy_(dev(meta))
    r.workspace_view(r.layout.rec_geom, torch.float32, 4 * n).copy_(dev(geom))
    r.workspace_view(r.layout.rec_color, torch.float32, 4 * n).copy_(dev(color))
    r.workspace_view(r.layout.rec_tau, torch.float32, n).copy_(dev(rec["tau"].astype(np.float32)))
    r.workspace_view(r.layout.depth_key, torch.int32, n).copy_(dev(rec["depth"].astype(np.float32).view(np.int32)))


# An ellipse threshold no tile misses: q <= 1e30 holds for every record.
KEEP_ALL = np.float32(1e30)


def _synthetic_records(rng, n, W, H, max_extent, tile=16, tau=None):
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
    t = rng.uniform(0.0, 8.0, n).astype(np.float32) if tau is None else np.full(n, tau, np.float32)
    return {"rect": rect, "depth": depth, "uv": np.stack([cx, cy], 1).astype(np.float32),
            "conic2": np.stack([A, B, C], 1).astype(np.float32), "tau": t}


def _read_instances(r, m, ntiles):
    import torch
    tiles = r.workspace_view(r.layout.inst_tile, torch.int32, m).cpu().numpy().astype(np.int64)
    slots = r.workspace_view(r.layout.inst_slot, torch.int32, m).cpu().numpy().astype(np.int64)
    gr = r.workspace_view(r.layout.tile_ranges, torch.int32, 2 * ntiles).cpu().numpy().reshape(-1, 2)
    return tiles, slots, gr


# Visible capacities equal to the slot count and well above it (the pair scan
# and depth sort size their grids and look-back rows by the capacity); an
# instance capacity of 2^26 takes the instance sort with three sub-tiles per
# ticket; stage_blocks_per_sm > 0 takes the lean (one or two blocks per SM)
# persistent grids.
@pytest.mark.parametrize("n,W,H,vis_cap,inst_cap,stage_blocks", [
    (1, 16, 16, 0, 0, 0), (2047, 144, 112, 0, 0, 0), (70_001, 1352, 1014, 0, 0, 0),
    (70_001, 1352, 1014, 400_000, 0, 0), (150_001, 1352, 1014, 0, 0, 0), (2047, 144, 112, 0, 1 << 26, 0),
    (150_001, 1352, 1014, 0, 1 << 26, 0), (150_001, 1352, 1014, 0, 1 << 26, 1), (70_001, 1352, 1014, 0, 0, 2)])
def test_bin_sort_bit_exact_on_synthetic_records(n, W, H, vis_cap, inst_cap, stage_blocks):
    """With ellipses that meet every tile, the sorted instance list and tile
    ranges equal the oracle's bit for bit: one instance per tile of each
    rect, ordered by (tile, FP32 depth, slot), on records written straight
    into the workspace (ragged counts, exact depth ties, empty rects)."""
    import torch
    from paper_2412_20720_gb300.render import Renderer
    rng = np.random.default_rng(n)
    gw, gh = (W + 15) // 16, (H + 15) // 16
    rec = _synthetic_records(rng, n, W, H, 6, tau=KEEP_ALL)
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=inst_cap or 40 * n + 16, vis_capacity=vis_cap,
                       stage_blocks_per_sm=stage_blocks)
    r = Renderer(n, [sy.tiny_view(W, H)], cfg)
    _write_records(r, rec, 0)
    fgs4d.bin_sort(n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, r.stream())
    counts = r.check()
    keys, vals, ranges = oracle.sort_instances(rec["rect"], rec["depth"], gw, gh)
    m = keys.shape[0]
    assert counts[1] == m
    tiles, slots, gr = _read_instances(r, m, gw * gh)
    np.testing.assert_array_equal(tiles, (keys >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(slots, vals)
    np.testing.assert_array_equal(rec["depth"][slots].view(np.uint32),
                                  (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32))
    np.testing.assert_array_equal(canonical_ranges(gr), ranges)
    sorted_slots = r.workspace_view(r.layout.sorted_slots, torch.int32, n).cpu().numpy()
    np.testing.assert_array_equal(sorted_slots, np.argsort(rec["depth"], kind="stable"))


def _min_q_over_tile(rec, i, tx, ty, W, H, tile):
    """FP64 minimum of q = A' dx^2 + B' dx dy + C' dy^2 over the pixel centres
    of tile (tx, ty) inside the image."""
    xs = np.arange(tx * tile, min(tx * tile + tile, W)) + 0.5
    ys = np.arange(ty * tile, min(ty * tile + tile, H)) + 0.5
    dx = xs[None, :] - float(rec["uv"][i, 0])
    dy = ys[:, None] - float(rec["uv"][i, 1])
    A, B, C = (float(x) for x in rec["conic2"][i])
    return float((A * dx * dx + B * dx * dy + C * dy * dy).min())


@pytest.mark.parametrize("n,W,H,tile", [(3001, 300, 200, 16), (2001, 150, 110, 8)])
def test_tile_cull_drops_only_tiles_every_pixel_skips(n, W, H, tile):
    """With finite 1/255 ellipses (q <= tau, tau carrying the 4e-3 margin of
    the records) the instance list is the full rect membership of the tile
    rasterizer in the same (tile, depth, slot) order with some pairs left
    out, and every left-out pair has, in FP64, q > tau - 4e-3 at every pixel
    centre of its tile: alpha < 1/255 there, so every pixel skips it."""
    from paper_2412_20720_gb300.render import Renderer
    rng = np.random.default_rng(n + tile)
    gw, gh = (W + tile - 1) // tile, (H + tile - 1) // tile
    rec = _synthetic_records(rng, n, W, H, 6, tile=tile)
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=40 * n + 16, tile=tile)
    r = Renderer(n, [sy.tiny_view(W, H)], cfg)
    _write_records(r, rec, 0)
    fgs4d.bin_sort(n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, r.stream())
    counts = r.check()
    keys, vals, ranges = oracle.sort_instances(rec["rect"], rec["depth"], gw, gh)
    m = counts[1]
    tiles, slots, gr = _read_instances(r, m, gw * gh)
    full = list(zip((keys >> np.uint64(32)).astype(np.int64).tolist(), vals.tolist()))
    got = list(zip(tiles.tolist(), slots.tolist()))
    # an order-preserving subsequence of the full list
    pos = {p: j for j, p in enumerate(full)}
    jj = np.array([pos[p] for p in got])
    assert np.all(np.diff(jj) > 0)
    dropped = sorted(set(full) - set(got))
    assert 0.2 * len(full) < len(dropped) < len(full)
    for t, i in dropped:
        assert _min_q_over_tile(rec, i, t % gw, t // gw, W, H, tile) > float(rec["tau"][i]) - 4e-3, (t, i)
    # the ranges describe the kept list
    exp = np.zeros((gw * gh, 2), dtype=np.int64)
    for j, (t, _) in enumerate(got):
        if j == 0 or got[j - 1][0] != t:
            exp[t, 0] = j
        exp[t, 1] = j + 1
    np.testing.assert_array_equal(canonical_ranges(gr), exp)


def test_bin_sort_bit_exact_multi_view():
    from paper_2412_20720_gb300.render import Renderer
    rng = np.random.default_rng(99)
    sizes = [(200, 150), (64, 48), (1014, 1352)]
    ns = [3000, 500, 9000]
    views = [sy.tiny_view(w, h) for w, h in sizes]
    recs = [_synthetic_records(rng, n, w, h, 5, tau=KEEP_ALL) for n, (w, h) in zip(ns, sizes)]
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
        gw, gh = (w + 15) // 16, (h + 15) // 16
        keys, vals, ranges = oracle.sort_instances(recs[k]["rect"], recs[k]["depth"], gw, gh)
        exp_tiles.append((keys >> np.uint64(32)).astype(np.int64) + tile_base)
        exp_slots.append(vals + slot_base)
        rr = ranges.copy()
        nz = rr[:, 1] > rr[:, 0]
        rr[nz] += inst_base
        exp_ranges.append(rr)
        tile_base += gw * gh
        slot_base += n
        inst_base += keys.shape[0]
    m = inst_base
    assert counts[1] == m
    tiles, slots, gr = _read_instances(r, m, tile_base)
    np.testing.assert_array_equal(tiles, np.concatenate(exp_tiles))
    np.testing.assert_array_equal(slots, np.concatenate(exp_slots))
    np.testing.assert_array_equal(canonical_ranges(gr), np.concatenate(exp_ranges))


def check_instance_list(run, params, view, cfg, k=0, tiles_to_check=None):
    """The instance list of view k against the tile rasterizer the paper
    adapts (Sec. 3.2), computed from the oracle's FP64 records:
    - every listed (tile, Gaussian) pair is in the full rect membership
      (rect_hi: some admissible rect of a Gaussian the oracle keeps or may
      keep), and each tile's list is ordered by the oracle's FP32 depth keys
      and index, up to swaps of keys within 2 depth_ulps;
    - every pair of the certain membership that is not listed has, at every
      pixel centre of its tile, an FP64 alpha that may round below 1/255
      (alpha (1 - e) < 1/255 with the alpha error bound e of the admissible
      layer), so no pixel would composite it."""
    import torch
    r = run.renderer
    st = oracle_settings(cfg)
    pr = oracle_proj(params, view, cfg)
    tol = pixel_tolerance(pr)
    B = cfg.tile
    W, H = int(view["width"]), int(view["height"])
    gw, gh = (W + B - 1) // B, (H + B - 1) // B
    base = sum(((int(v["width"]) + B - 1) // B) * ((int(v["height"]) + B - 1) // B) for v in r.view_dicts[:k])
    m = run.counts[1]
    tiles = r.workspace_view(r.layout.inst_tile, torch.int32, m).cpu().numpy().astype(np.int64)
    slots = r.workspace_view(r.layout.inst_slot, torch.int32, m).cpu().numpy().astype(np.int64)
    gidx = run.meta[:, 0][slots]
    sel = (tiles >= base) & (tiles < base + gw * gh)
    tiles, gidx, slots = tiles[sel] - base, gidx[sel], slots[sel]
    assert np.all(run.meta[:, 1][slots] == k)
    # the GPU's own keys order each tile's list exactly (tile, depth bits, slot)
    gkey = run.depth_bits[slots].astype(np.int64)
    order = np.lexsort((slots, gkey, tiles))
    np.testing.assert_array_equal(order, np.arange(tiles.size))
    alive = (pr["status"] == 0) | ((pr["uncertain"] & 1) > 0)
    certain = (pr["status"] == 0) & ((pr["uncertain"] & 1) == 0)
    hi, lo = pr["rect_hi"], pr["rect_lo"]
    tx, ty = tiles % gw, tiles // gw
    assert np.all(alive[gidx])
    assert np.all((hi[gidx, 0] <= tx) & (tx < hi[gidx, 2]) & (hi[gidx, 1] <= ty) & (ty < hi[gidx, 3]))
    obits = pr["depth_f32"].view(np.uint32).astype(np.int64)
    starts = np.flatnonzero(np.r_[True, tiles[1:] != tiles[:-1]])
    ends = np.r_[starts[1:], tiles.size]
    for a, b in zip(starts, ends):
        ob = obits[gidx[a:b]]
        if b - a > 1:
            assert np.all(ob[1:] >= np.maximum.accumulate(ob)[:-1] - 2 * tol.depth_ulps), int(tiles[a])
    listed = {}
    for a, b in zip(starts, ends):
        listed[int(tiles[a])] = set(gidx[a:b].tolist())
    tile_ids = range(gw * gh) if tiles_to_check is None else tiles_to_check
    cidx = np.flatnonzero(certain)
    n_dropped = 0
    for t in tile_ids:
        x, y = t % gw, t // gw
        inside = cidx[(lo[cidx, 0] <= x) & (x < lo[cidx, 2]) & (lo[cidx, 1] <= y) & (y < lo[cidx, 3])]
        drop = np.setdiff1d(inside, np.array(sorted(listed.get(t, set())), dtype=np.int64))
        if drop.size == 0:
            continue
        n_dropped += drop.size
        xs = np.arange(x * B, min(x * B + B, W)) + 0.5
        ys = np.arange(y * B, min(y * B + B, H)) + 0.5
        px, py = np.meshgrid(xs, ys)
        px, py = px.reshape(1, -1), py.reshape(1, -1)
        pix = (np.floor(py) * W + np.floor(px)).astype(np.int64).reshape(-1)  # linear ids of the centres
        ii = np.repeat(drop, pix.size)
        pp = np.tile(pix, drop.size)
        alpha, e = oracle.alpha_bounds(pr, view, tol, ii, pp)
        bad = alpha * (1 - e) >= 1 / 255
        assert not bad.any(), "tile %d: dropped Gaussians %s have alpha >= 1/255" % (t, np.unique(ii[bad])[:5])
    return n_dropped


def test_instance_list_is_the_rect_membership_minus_skipped_pairs():
    """The instance list of a rendered scene against the tile rasterizer's
    rect membership, with no reference to the kernel's own cull test."""
    params, view, cfg = tiny_case(131, 77, 1, 1)
    run = CudaRender(params, [view], cfg)
    assert check_instance_list(run, params, view, cfg) > 100


@pytest.mark.parametrize("inst_cap", [1 << 19, 1 << 26])  # 2^26: three sub-tiles per tile-sort ticket
def test_instance_list_at_tile_8_and_several_views(inst_cap):
    sc = sy.make_scene(3000, 14, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    views = [sy.tiny_view(96, 80, t=0.4), sy.look_at((1.5, -0.5, -2.5), (0, 0, 0), (0, -1, 0), 100, 70, 0.6)]
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=inst_cap, tile=8)
    params = sc.as_dict()
    run = CudaRender(params, views, cfg)
    for k, v in enumerate(views):
        assert check_instance_list(run, params, v, cfg, k) > 100


def test_instance_list_full_size_sampled_tiles():
    """The headline view (300k Gaussians, 1352x1014): 150 tiles, every
    listed pair and every certain rect pair of those tiles."""
    sc = sy.orbit_scene()
    view = sy.orbit_view(120)
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 23)
    params = sc.as_dict()
    run = CudaRender(params, [view], cfg)
    rng = np.random.default_rng(17)
    tiles = rng.choice(85 * 64, 150, replace=False)
    assert check_instance_list(run, params, view, cfg, 0, tiles_to_check=tiles) > 1000


# ------------------------------------------------------------- edge cases

def test_empty_scene_renders_background():
    view = sy.tiny_view(50, 30)
    cfg = RenderConfig(sh_degree=1, t_order=1, bg=(0.25, 0.5, 0.75), inst_capacity=1024)
    empty = {k: v[:0] for k, v in sy.tiny_scene().as_dict().items()}
    run = CudaRender(empty, [view], cfg)
    assert run.counts[:2] == [0, 0]
    for ch, b in enumerate(cfg.bg):
        assert np.all(run.images[0][ch] == np.float32(b))
    assert np.all(run.T == 1.0) and np.all(run.last == 0)


def test_all_temporally_culled_renders_background():
    sc = sy.tiny_scene().as_dict()
    sc["mean"][:, 3] = 50.0  # far from t = 0.5 for every temporal scale
    view = sy.tiny_view(64, 48)
    cfg = RenderConfig(sh_degree=1, t_order=1, bg=(0.3, 0.3, 0.3), inst_capacity=1024)
    run = CudaRender(sc, [view], cfg)
    assert run.counts[0] == 0
    assert np.all(run.images[0] == np.float32(0.3))


def test_non_finite_parameters_are_culled_not_propagated():
    params, view, cfg = tiny_case(n=1500)
    clean = CudaRender(params, [view], cfg)
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
    poisoned = CudaRender(bad, [view], cfg)
    removed = CudaRender(subset(params, keep), [view], cfg)
    assert np.isfinite(poisoned.images[0]).all()
    np.testing.assert_array_equal(poisoned.images[0], removed.images[0])


def test_instance_capacity_overflow_is_reported_and_recoverable():
    params, view, cfg = tiny_case()
    full = CudaRender(params, [view], cfg)
    need = full.counts[1]
    small = RenderConfig(sh_degree=1, t_order=1, inst_capacity=max(1, need // 3))
    from paper_2412_20720_gb300.render import Renderer
    from helpers import to_device
    r = Renderer(params["mean"].shape[0], [view], small)
    r.forward(to_device(params))
    code, counts = r.status()
    assert code == fgs4d.ERR_CAPACITY
    assert counts[1] == need // 3 and counts[3] == need
    again = CudaRender(params, [view], RenderConfig(sh_degree=1, t_order=1, inst_capacity=counts[3]))
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
    """GPU and oracle gradients of a loss whose image gradient is random at
    every pixel where each decision is settled (zero elsewhere)."""
    run = CudaRender(params, [view], cfg)
    ost = oracle_settings(cfg)
    _, flags = check_image(run, params, view, cfg)
    pr = oracle.preprocess(params, view, ost)
    rng = np.random.default_rng(seed)
    dimg = loss_gradient_at_settled_pixels(rng, flags, (3,) + flags.shape)
    assert ((flags & 3) == 0).mean() > 0.9
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
    check_gradients(*_grad_case(params, view, cfg))


def test_backward_in_two_stages_equals_one_call():
    """fgs4d_render_bwd_composite then fgs4d_render_bwd_preprocess does what
    fgs4d_render_bwd does (up to the order of the atomic sums)."""
    import torch
    from paper_2412_20720_gb300.render import Renderer
    from helpers import ORDER_FLOOR, ORDER_RTOL, to_device
    params, view, cfg = tiny_case(131, 77, 3, 2, (0.1, 0.2, 0.3))
    p = to_device(params)
    r = Renderer(params["mean"].shape[0], [view], cfg)
    r.forward(p)
    dL = torch.from_numpy(np.random.default_rng(4).standard_normal(3 * 131 * 77).astype(np.float32)).cuda()
    one = {k: torch.zeros_like(v) for k, v in p.items()}
    r.backward(p, dL, one)
    nv = r.check()[0]
    slot_one = r.workspace_view(r.layout.slot_grad, torch.float32, 12 * nv).cpu().numpy()
    two = {k: torch.zeros_like(v) for k, v in p.items()}
    st = r.stream()
    fgs4d.render_bwd_composite(r.n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, dL.data_ptr(), st)
    fgs4d.render_bwd_preprocess(r.gaussians(p), r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes,
                                r._grads(two, None), st)
    r.check()
    slot_two = r.workspace_view(r.layout.slot_grad, torch.float32, 12 * nv).cpu().numpy()
    compare_group("slot gradients", slot_two, slot_one, ORDER_RTOL, ORDER_FLOOR)
    for k in PARAM_KEYS:
        compare_group(k, two[k].cpu().numpy(), one[k].cpu().numpy(), ORDER_RTOL, ORDER_FLOOR)


def test_render_stats_counts_the_composited_entries():
    """fgs4d_render_stats: the composited entries are the oracle's
    contributors summed over the pixels (from the admissible result each
    pixel matched); evaluations up to the last composited entry lie between
    that and all evaluations; the image is the plain forward's."""
    import torch
    from paper_2412_20720_gb300.render import Renderer
    from helpers import to_device
    params, view, cfg = tiny_case(128, 96, 1, 1)
    run = CudaRender(params, [view], cfg)
    _, flags = check_image(run, params, view, cfg)
    pr = oracle_proj(params, view, cfg)
    Tg, lastg = run.pixel_planes(0)
    W, H = view["width"], view["height"]
    _, chosen = check_pixels(pr, view, cfg, np.arange(W * H), run.images[0].reshape(3, -1).T, Tg.reshape(-1))
    r = run.renderer
    stats = torch.zeros(3, dtype=torch.int64, device="cuda")
    out = torch.empty(3 * W * H, dtype=torch.float32, device="cuda")
    fgs4d.render_stats(r.n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, out.data_ptr(),
                       stats.data_ptr(), r.stream())
    r.check()
    ev, co, evb = stats.tolist()
    assert co == int(chosen[:, 4].sum())
    assert co <= evb <= ev
    np.testing.assert_array_equal(out.cpu().numpy().reshape(3, H, W), run.images[0])


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
