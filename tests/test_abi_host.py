"""Host-side checks of the C ABI: the library builds and loads, exports every
entry point include/fgs4d.h declares, and rejects bad arguments before any
work is enqueued.  No GPU is needed (no call here reaches a kernel)."""
import ctypes as C
import os
import re

import pytest

from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300 import synthetic as sy

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fgs4d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fgs4d_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = fgs4d.load()
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
    assert set(fgs4d.EXPORTED) == set(names)


def _views(k=1):
    return fgs4d.make_views([sy.tiny_view(128, 96)] * k)


def test_workspace_size_and_layout_are_consistent():
    s = fgs4d.make_settings(sh_degree=1, t_order=1, inst_capacity=100_000)
    views, nv = _views(2)
    nbytes = fgs4d.workspace_size(s, 2000, views, nv)
    lay = fgs4d.workspace_layout(s, 2000, views, nv)
    assert lay.bytes == nbytes
    assert lay.vis_capacity == 4000 and lay.inst_capacity == 100_000
    assert lay.total_tiles == 2 * 8 * 6 and lay.total_pixels == 2 * 128 * 96
    offs = [lay.counters, lay.rec_geom, lay.rec_color, lay.rec_blue, lay.rec_meta, lay.depth_key, lay.sorted_slots,
            lay.inst_tile, lay.inst_slot, lay.tile_ranges, lay.pix_T, lay.pix_last, lay.slot_grad]
    assert all(o % 256 == 0 and o < nbytes for o in offs)
    assert len(set(offs)) == len(offs)


def test_block_shape_must_fit_the_tile():
    views, nv = _views()
    for tile, ok, bad in ((16, (0, 2, 4, 8), (1,)), (8, (0, 1, 2), (4, 8))):
        for p in ok:
            fgs4d.workspace_size(fgs4d.make_settings(tile=tile, pixels_per_thread=p), 10, views, nv)
        for p in bad:
            with pytest.raises(fgs4d.Fgs4dError) as e:
                fgs4d.workspace_size(fgs4d.make_settings(tile=tile, pixels_per_thread=p), 10, views, nv)
            assert e.value.code == fgs4d.ERR_UNSUPPORTED
    # 8x8 tiles: four times the tiles of 16x16 on a 128x96 view.
    assert fgs4d.workspace_layout(fgs4d.make_settings(tile=8), 10, views, nv).total_tiles == 16 * 12


@pytest.mark.parametrize("field,value,code", [
    ("sh_degree", 4, fgs4d.ERR_UNSUPPORTED),
    ("t_order", 5, fgs4d.ERR_UNSUPPORTED),
    ("tile", 32, fgs4d.ERR_UNSUPPORTED),
    ("tile", 12, fgs4d.ERR_UNSUPPORTED),
    ("period", 0.0, fgs4d.ERR_ARG),
    ("near_plane", -1.0, fgs4d.ERR_ARG),
    ("dilation", float("nan"), fgs4d.ERR_ARG),
    ("p_t_min", 1.0, fgs4d.ERR_ARG),
    ("inst_capacity", 0, fgs4d.ERR_ARG),
    ("inst_capacity", 1 << 31, fgs4d.ERR_ARG),
    ("vis_capacity", -1, fgs4d.ERR_ARG),
    ("pixels_per_thread", 3, fgs4d.ERR_UNSUPPORTED),
    ("pixels_per_thread", 16, fgs4d.ERR_UNSUPPORTED),
    ("shared_batch", 64, fgs4d.ERR_UNSUPPORTED),
    ("shared_batch", 512, fgs4d.ERR_UNSUPPORTED),
])
def test_bad_settings_are_rejected(field, value, code):
    s = fgs4d.make_settings()
    setattr(s, field, value)
    views, nv = _views()
    with pytest.raises(fgs4d.Fgs4dError) as e:
        fgs4d.workspace_size(s, 10, views, nv)
    assert e.value.code == code


def test_bad_views_and_sizes_are_rejected():
    s = fgs4d.make_settings()
    views, nv = _views()
    for n in (-1, 1 << 31):
        with pytest.raises(fgs4d.Fgs4dError):
            fgs4d.workspace_size(s, n, views, nv)
    with pytest.raises(fgs4d.Fgs4dError):
        fgs4d.workspace_size(s, 10, views, 0)
    with pytest.raises(fgs4d.Fgs4dError):
        fgs4d.workspace_size(s, 10, views, fgs4d.MAX_VIEWS + 1)
    bad = sy.tiny_view(128, 96)
    bad["width"] = 0
    v2, n2 = fgs4d.make_views([bad])
    with pytest.raises(fgs4d.Fgs4dError):
        fgs4d.workspace_size(s, 10, v2, n2)
    bad = sy.tiny_view(128, 96)
    bad["viewmat"] = bad["viewmat"].copy()
    bad["viewmat"][0, 0] = float("inf")
    v3, n3 = fgs4d.make_views([bad])
    with pytest.raises(fgs4d.Fgs4dError):
        fgs4d.workspace_size(s, 10, v3, n3)
    # A large scene needs an explicit visible capacity.
    with pytest.raises(fgs4d.Fgs4dError):
        fgs4d.workspace_size(s, 600_000_000, *_views(2))


def test_calls_reject_missing_or_small_workspace_before_launching():
    s = fgs4d.make_settings(sh_degree=1, t_order=1)
    views, nv = _views()
    g = fgs4d.make_gaussians({k: 0 for k in ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")}, 0)
    lib = fgs4d.load()
    assert lib.fgs4d_preprocess(C.byref(g), views, nv, C.byref(s), None, 0, None) == fgs4d.ERR_WORKSPACE
    assert lib.fgs4d_bin_sort(0, views, nv, C.byref(s), C.c_void_p(256), 16, None) == fgs4d.ERR_WORKSPACE
    assert lib.fgs4d_bin_sort(0, views, nv, C.byref(s), C.c_void_p(257), 1 << 40, None) == fgs4d.ERR_WORKSPACE
    # Non-empty scene with a null parameter pointer.
    g.n = 5
    assert lib.fgs4d_preprocess(C.byref(g), views, nv, C.byref(s), None, 0, None) == fgs4d.ERR_ARG
    # Misaligned parameter rows (float4 loads need 16-byte alignment).
    g2 = fgs4d.make_gaussians({k: 4096 + 4 for k in ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")}, 5)
    assert lib.fgs4d_preprocess(C.byref(g2), views, nv, C.byref(s), C.c_void_p(1 << 20), 1 << 40, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_render_fwd(0, views, nv, C.byref(s), C.c_void_p(1 << 20), 1 << 40, None, None, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_l1_loss(None, None, 10, None, None, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_get_status(None, 0, None, None) == fgs4d.ERR_WORKSPACE
    # Auxiliary render: missing output planes or a non-finite time step.
    g.n = 0
    ws, big = C.c_void_p(1 << 20), 1 << 40
    assert lib.fgs4d_render_aux(C.byref(g), views, nv, C.byref(s), ws, big, 0.1, C.c_void_p(4096), None, None,
                                None) == fgs4d.ERR_ARG
    assert lib.fgs4d_render_aux(C.byref(g), views, nv, C.byref(s), ws, big, float("nan"), C.c_void_p(4096), None,
                                C.c_void_p(4096), None) == fgs4d.ERR_ARG
    assert lib.fgs4d_render_aux(C.byref(g), views, nv, C.byref(s), None, 0, 0.1, C.c_void_p(4096), None,
                                C.c_void_p(4096), None) == fgs4d.ERR_WORKSPACE


def test_l1_loss_part_rejects_a_part_larger_than_its_mean():
    lib = fgs4d.load()
    p = C.c_void_p(4096)
    assert lib.fgs4d_l1_loss_part(p, p, 10, 5, p, p, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_l1_loss_part(p, p, 10, 0, p, p, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_l1_loss_part(None, None, 10, 40, None, None, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_l1_loss_part(None, None, 0, 40, None, None, None) == fgs4d.OK  # empty part: nothing to do


def test_bin_sort_kernel_count():
    """Histogram + 4 depth passes, pair scan, emission, then one tile-sort
    pass per 8 bits of the tile id (the last records the ranges)."""
    s = fgs4d.make_settings(sh_degree=1, t_order=1)
    views, nv = _views()  # 8 x 6 tiles: one tile pass
    assert fgs4d.bin_sort_kernels(100, views, nv, s) == 1 + 4 + 1 + 1 + 1
    big, nb = fgs4d.make_views([sy.tiny_view(1352, 1014)])  # 85 x 64 tiles: two passes
    assert fgs4d.bin_sort_kernels(100, big, nb, s) == 1 + 4 + 1 + 1 + 2
    assert fgs4d.bin_sort_kernels(0, big, nb, s) == 2  # no visible slot possible: ranges cleared, tile passes


def test_wait_selftest_rejects_bad_scratch_before_launching():
    lib = fgs4d.load()
    n = fgs4d.WAIT_SELFTEST_BYTES
    assert lib.fgs4d_wait_selftest(None, n, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_wait_selftest(C.c_void_p(4096), n - 4, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_wait_selftest(C.c_void_p(4096 + 4), n, None) == fgs4d.ERR_ARG


def test_stage_blocks_per_sm_range():
    views, nv = _views()
    for k in (0, 1, 2, 8):
        fgs4d.workspace_size(fgs4d.make_settings(stage_blocks_per_sm=k), 10, views, nv)
    for k in (-1, 9):
        with pytest.raises(fgs4d.Fgs4dError) as e:
            fgs4d.workspace_size(fgs4d.make_settings(stage_blocks_per_sm=k), 10, views, nv)
        assert e.value.code == fgs4d.ERR_UNSUPPORTED


def test_adam_set_rejects_bad_tables_before_launching():
    lib = fgs4d.load()
    step = C.c_void_p(4096)
    ok = fgs4d.AdamTensor(4096, 4096, 4096, 4096, 8, 1e-3)
    table = (fgs4d.AdamTensor * 17)(*([ok] * 17))
    assert lib.fgs4d_adam_update_set(table, 17, 0.9, 0.99, 1e-8, step, 0, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_adam_update_set(table, -1, 0.9, 0.99, 1e-8, step, 0, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_adam_update_set(table, 1, 0.9, 0.99, 1e-8, None, 0, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_adam_update_set(None, 1, 0.9, 0.99, 1e-8, step, 0, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_adam_update_set(table, 1, 1.0, 0.99, 1e-8, step, 0, None) == fgs4d.ERR_ARG
    assert lib.fgs4d_adam_update_set(table, 1, 0.9, 0.99, 0.0, step, 0, None) == fgs4d.ERR_ARG
    for bad in (fgs4d.AdamTensor(4096, 4096, 4096, 4096, -1, 1e-3),
                fgs4d.AdamTensor(4096, 4096, 4096, 4096, 8, float("nan")),
                fgs4d.AdamTensor(4096, None, 4096, 4096, 8, 1e-3),
                fgs4d.AdamTensor(4096, 4100, 4096, 4096, 8, 1e-3)):
        one = (fgs4d.AdamTensor * 1)(bad)
        assert lib.fgs4d_adam_update_set(one, 1, 0.9, 0.99, 1e-8, step, 0, None) == fgs4d.ERR_ARG
    # An empty set, or tensors with count 0 and NULL arrays, launch nothing.
    empty = (fgs4d.AdamTensor * 1)(fgs4d.AdamTensor(None, None, None, None, 0, 1e-3))
    assert lib.fgs4d_adam_update_set(empty, 0, 0.9, 0.99, 1e-8, step, 0, None) == fgs4d.OK
    assert lib.fgs4d_adam_update_set(empty, 1, 0.9, 0.99, 1e-8, step, 1, None) == fgs4d.OK


def test_status_strings():
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert fgs4d.status_string(code) not in ("", "unknown status")
    assert fgs4d.status_string(-99) == "unknown status"
