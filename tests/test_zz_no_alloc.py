"""fgs4d_sort_depth_static: the depth sort for callers that cannot give the
library a workspace (their host owns all device memory, or they may not call
cudaMalloc inside a frame loop).  It must produce exactly the permutation the
workspace-based fgs4d_bin_sort produces for the same depth keys, call after
call, although every call reuses the same library-owned device scratch.

Kept in a file of its own, collected after every other test."""
import numpy as np
import pytest

from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


def _depth_keys(rng, n):
    depth = rng.uniform(0.25, 60.0, n).astype(np.float32)
    depth[rng.integers(0, n, n // 8)] = depth[1]  # exact ties: order by index
    return depth.view(np.uint32)


def _bin_sort_order(keys_np):
    """The existing entry point: records with empty tile rects written into a
    workspace, then fgs4d_bin_sort; returns its sorted_slots region."""
    import torch

    from paper_2412_20720_gb300.render import RenderConfig, Renderer
    n = keys_np.shape[0]
    r = Renderer(n, [sy.tiny_view(64, 64)], RenderConfig(sh_degree=1, t_order=1, inst_capacity=1024))
    meta = np.zeros((n, 4), dtype=np.int32)
    meta[:, 0] = np.arange(n)
    r.workspace_view(r.layout.counters, torch.int32, 64).zero_()
    r.workspace_view(r.layout.counters, torch.int32, 1).fill_(n)
    r.workspace_view(r.layout.rec_meta, torch.int32, 4 * n).copy_(torch.from_numpy(meta.reshape(-1)).cuda())
    r.workspace_view(r.layout.depth_key, torch.int32, n).copy_(torch.from_numpy(keys_np.view(np.int32)).cuda())
    fgs4d.bin_sort(n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, r.stream())
    r.check()
    return r.workspace_view(r.layout.sorted_slots, torch.int32, n).clone()


def test_static_depth_sort_matches_bin_sort_on_consecutive_calls():
    """Sizes up to the scratch's limit (FGS4D_STATIC_SORT_MAX keys: the
    largest grid and look-back chain the array was sized for), each sorted
    twice in a row, each call's device status read back."""
    import torch
    rng = np.random.default_rng(20)
    stream = torch.cuda.current_stream().cuda_stream
    # a large sort, a smaller one over the same scratch, then the limit
    for n in (70_001, 2047, fgs4d.STATIC_SORT_MAX):
        keys = _depth_keys(rng, n)
        expect = _bin_sort_order(keys)
        keys_dev = torch.from_numpy(keys.view(np.int32)).cuda()
        for _ in range(2):
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            fgs4d.sort_depth_static(keys_dev.data_ptr(), n, out.data_ptr(), stream)
            assert fgs4d.sort_depth_static_status(stream) == fgs4d.OK
            assert torch.equal(out, expect)
        # The permutation is the stable order of the keys.
        np.testing.assert_array_equal(out.cpu().numpy(), np.argsort(keys, kind="stable"))


def test_static_depth_sort_takes_keys_at_any_4_byte_boundary():
    """Keys that start 4, 8 and 12 bytes past a 16-byte boundary (a slice of a
    larger array) sort like aligned ones."""
    import torch
    rng = np.random.default_rng(22)
    stream = torch.cuda.current_stream().cuda_stream
    n = 100_003
    keys = _depth_keys(rng, n + 3)
    base = torch.from_numpy(keys.view(np.int32)).cuda()
    assert base.data_ptr() % 16 == 0
    for off in (1, 2, 3):
        sub = keys[off:off + n]
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        fgs4d.sort_depth_static(base.data_ptr() + 4 * off, n, out.data_ptr(), stream)
        assert fgs4d.sort_depth_static_status(stream) == fgs4d.OK
        np.testing.assert_array_equal(out.cpu().numpy(), np.argsort(sub, kind="stable"))


def test_static_depth_sort_allocates_no_device_memory():
    """After a first call (which looks up the scratch's address), further
    calls leave the device memory in use unchanged."""
    import torch
    rng = np.random.default_rng(21)
    stream = torch.cuda.current_stream().cuda_stream
    n = 300_001
    keys_dev = torch.from_numpy(_depth_keys(rng, n).view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    fgs4d.sort_depth_static(keys_dev.data_ptr(), n, out.data_ptr(), stream)
    assert fgs4d.sort_depth_static_status(stream) == fgs4d.OK
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        fgs4d.sort_depth_static(keys_dev.data_ptr(), n, out.data_ptr(), stream)
        assert fgs4d.sort_depth_static_status(stream) == fgs4d.OK
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(), torch.cuda.mem_get_info()[0])
    assert after[:2] == before[:2]
    assert after[2] >= before[2]  # free device memory did not shrink


def test_static_depth_sort_rejects_sizes_beyond_its_scratch():
    with pytest.raises(fgs4d.Fgs4dError) as e:
        fgs4d.sort_depth_static(256, fgs4d.STATIC_SORT_MAX + 1, 256, None)
    assert e.value.code == fgs4d.ERR_ARG
    with pytest.raises(fgs4d.Fgs4dError):
        fgs4d.sort_depth_static(256, -1, 256, None)
    fgs4d.sort_depth_static(None, 0, None, None)  # empty input: nothing to do
