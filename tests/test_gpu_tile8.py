"""The 8x8 tile edge (the other tile size the batched workload autotunes):
records, images, transmittance, the sorted instance list (bit exact),
gradients and block shapes against the FP64 oracle at tile edge 8, and the
autotune over both tile sizes."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer, autotune

from helpers import CudaRender, canonical_ranges, check_image, check_records, oracle_settings, to_device
from test_gpu_parity import KEEP_ALL, _grad_case, _synthetic_records, _write_records, check_gradients, tiny_case

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w,h,L,NT,bg", [(128, 96, 1, 1, (0.0, 0.0, 0.0)), (131, 77, 3, 2, (0.2, 0.5, 0.7))])
def test_image_matches_oracle_at_tile_8(w, h, L, NT, bg):
    params, view, cfg = tiny_case(w, h, L, NT, bg, tile=8)
    run = CudaRender(params, [view], cfg)
    check_records(run, params, view, cfg)
    check_image(run, params, view, cfg)


def test_tile_8_block_shapes_render_identically():
    """Block shape and shared batch size change the work split only."""
    params, view, cfg = tiny_case(131, 77, 2, 1, (0.1, 0.1, 0.1), tile=8)
    runs = [CudaRender(params, [view], RenderConfig(**{**cfg.__dict__, "pixels_per_thread": p, "shared_batch": b}))
            for p, b in ((1, 256), (2, 256), (2, 128))]
    for run in runs[1:]:
        np.testing.assert_array_equal(run.images[0], runs[0].images[0])
        np.testing.assert_array_equal(run.T, runs[0].T)
        np.testing.assert_array_equal(run.last, runs[0].last)


@pytest.mark.parametrize("n,W,H", [(2047, 144, 112), (30_001, 1352, 1014)])
def test_bin_sort_bit_exact_at_tile_8(n, W, H):
    import torch
    rng = np.random.default_rng(n + 8)
    gw, gh = (W + 7) // 8, (H + 7) // 8
    rec = _synthetic_records(rng, n, W, H, 8, tile=8, tau=KEEP_ALL)
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=60 * n + 16, tile=8)
    r = Renderer(n, [sy.tiny_view(W, H)], cfg)
    _write_records(r, rec, 0)
    fgs4d.bin_sort(n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, r.stream())
    counts = r.check()
    keys, vals, ranges = oracle.sort_instances(rec["rect"], rec["depth"], gw, gh)
    m = keys.shape[0]
    assert counts[1] == m
    tiles = r.workspace_view(r.layout.inst_tile, torch.int32, m).cpu().numpy()
    slots = r.workspace_view(r.layout.inst_slot, torch.int32, m).cpu().numpy()
    gr = r.workspace_view(r.layout.tile_ranges, torch.int32, 2 * gw * gh).cpu().numpy().reshape(-1, 2)
    np.testing.assert_array_equal(tiles, (keys >> np.uint64(32)).astype(np.int64))
    np.testing.assert_array_equal(slots, vals)
    np.testing.assert_array_equal(canonical_ranges(gr), ranges)


def test_gradients_match_oracle_at_tile_8():
    params, view, cfg = tiny_case(96, 80, 3, 2, (0.1, 0.2, 0.3), tile=8)
    check_gradients(*_grad_case(params, view, cfg))


def test_autotune_over_both_tile_sizes():
    import torch
    params, view, cfg = tiny_case(tile=16)
    r = Renderer(params["mean"].shape[0], [view], cfg)
    dev = to_device(params)
    res = autotune(r, dev, reps=2, tiles=(16, 8), batches=(256, 128))
    assert set(res["ms"]) == {"%d/%d/%d" % (t, p, b) for t, p in ((16, 2), (16, 4), (16, 8), (8, 1), (8, 2))
                              for b in (256, 128)}
    assert r.settings.tile == res["tile"] and r.settings.pixels_per_thread == res["pixels_per_thread"]
    assert r.settings.shared_batch == res["shared_batch"]
    # The chosen tile edge renders the oracle's image at that edge.
    run = CudaRender(params, [view], RenderConfig(**{**cfg.__dict__, "tile": res["tile"],
                                                 "pixels_per_thread": res["pixels_per_thread"],
                                                 "shared_batch": res["shared_batch"]}))
    np.testing.assert_array_equal(run.images[0], r.split(r.forward(dev))[0].cpu().numpy())
    check_image(run, params, view, run.renderer.config)
