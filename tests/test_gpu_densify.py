"""Parity of the densification pieces with the FP64 oracle: the spacetime
statistics accumulated by the backward pass (|dL/dmu_2d|, |dL/dmu_t|, view
count per Gaussian, summed over the views of a call) and the split sampling
of children from the parents' full 4D Gaussians."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer, split_gaussians

from helpers import (compare_group, loss_gradient_at_settled_pixels, oracle_flags, oracle_proj, oracle_settings,
                     to_device)

pytestmark = pytest.mark.gpu


def test_densify_stats_match_oracle_over_views():
    import torch
    sc = sy.make_scene(1500, 9, (-1, -1, -1), (1, 1, 1), sh_degree=2, t_order=1)
    views = [sy.tiny_view(96, 72, t=0.45), sy.tiny_view(80, 64, t=0.55)]
    cfg = RenderConfig(sh_degree=2, t_order=1, inst_capacity=1 << 18)
    params = sc.as_dict()
    n = params["mean"].shape[0]
    st = oracle_settings(cfg)
    rng = np.random.default_rng(10)
    dimgs, expect, maybe = [], np.zeros((n, 4)), np.zeros(n)
    for v in views:
        prr = oracle_proj(params, v, cfg)
        maybe += (prr["uncertain"] & 1) > 0
        pr = oracle.preprocess(params, v, st)
        d = loss_gradient_at_settled_pixels(rng, oracle_flags(prr, v, cfg), (3, int(v["height"]), int(v["width"])))
        dimgs.append(d)
        expect += oracle.densify_stats(params, pr, v, st, d)
    r = Renderer(n, views, cfg)
    p = to_device(params)
    r.forward(p)
    grads = {k: torch.zeros_like(v) for k, v in p.items()}
    stats = torch.zeros((n, 4), dtype=torch.float32, device=r.device)
    flat = torch.from_numpy(np.concatenate([d.reshape(-1) for d in dimgs]).astype(np.float32)).cuda()
    r.backward(p, flat, grads, densify_stats=stats)
    r.check()
    got = stats.cpu().numpy().astype(np.float64)
    # view counts: equal where every view's decision is certain; where some
    # are uncertain, within that many views of the FP64 count
    cert = maybe == 0
    np.testing.assert_array_equal(got[cert, 2], expect[cert, 2])
    assert np.all(np.abs(got[~cert, 2] - expect[~cert, 2]) <= maybe[~cert])
    assert expect[:, 2].max() == 2 and (expect[:, 2] == 1).any()
    compare_group("|dL/dmu_2d|", got[:, 0], expect[:, 0], 1e-3, 1e-4)
    compare_group("|dL/dmu_t|", got[:, 1], expect[:, 1], 1e-3, 1e-4)
    assert np.all(got[:, 3] == 0)


# SH rows of 144, 54 and 3 floats: copied as float4 when the row length is a
# multiple of 4, as floats otherwise.  One parent index is out of range: its
# children are written as zeros.
@pytest.mark.parametrize("L,NT", [(3, 2), (2, 1), (0, 0)])
def test_split_children_match_oracle(L, NT):
    import torch
    sc = sy.make_scene(500, 11, (-1, -1, -1), (1, 1, 1), sh_degree=L, t_order=NT)
    params = sc.as_dict()
    rng = np.random.default_rng(12)
    idx = rng.choice(500, 77, replace=False).astype(np.int32)
    eps = rng.standard_normal((77, 3, 4)).astype(np.float32)
    bad = 5
    idx_gpu = idx.copy()
    idx_gpu[bad] = 500  # out of range
    cfg = RenderConfig(sh_degree=L, t_order=NT)
    out = split_gaussians(to_device(params), torch.from_numpy(idx_gpu).cuda(), torch.from_numpy(eps).cuda(), 1.6,
                          cfg)
    torch.cuda.synchronize()
    ref = oracle.split_sample(params, idx, eps, 1.6)
    for k in PARAM_KEYS:
        ref[k] = np.array(ref[k], copy=True)
        ref[k][3 * bad:3 * bad + 3] = 0.0
    for k in PARAM_KEYS:
        got = out[k].cpu().numpy().astype(np.float64)
        assert got.shape == ref[k].shape, k
        scale = max(np.abs(ref[k]).max(), 1.0)
        assert np.abs(got - ref[k]).max() <= 2e-6 * scale, k
