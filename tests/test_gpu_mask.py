"""Parity of the Compact-4DGS significance mask (Sec. 4.3) with the FP64
oracle: removal of Gaussians with sigmoid(m) <= eps, unchanged render of
the rest, the straight-through gradient dL/dm, and the mask loss."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer, mask_loss

from helpers import (RELAX, check_pixels, compare_group, loss_gradient_at_settled_pixels, oracle_flags,
                     oracle_settings, to_device)

pytestmark = pytest.mark.gpu

EPS = 0.4


def masked_case(seed=13, n=2000, L=2, NT=1):
    sc = sy.make_scene(n, seed, (-1, -1, -1), (1, 1, 1), sh_degree=L, t_order=NT)
    params = sc.as_dict()
    params["mask_logit"] = np.random.default_rng(seed).normal(0.0, 1.5, n).astype(np.float32)
    view = sy.tiny_view(112, 88, t=0.5)
    cfg = RenderConfig(sh_degree=L, t_order=NT, inst_capacity=1 << 18, mask_threshold=EPS)
    return params, view, cfg


def oracle_params(params):
    return dict(params, mask_threshold=float(np.float32(EPS)))


def run_gpu(params, view, cfg, dimg=None):
    import torch
    n = params["mean"].shape[0]
    r = Renderer(n, [view], cfg)
    p = to_device(params)
    p["mask_logit"] = torch.from_numpy(params["mask_logit"]).cuda()
    img = r.forward(p)
    counts = r.check()
    out = {"img": r.split(img)[0].cpu().numpy(), "visible": counts[0],
           "T": r.workspace_view(r.layout.pix_T, torch.float32, r.total_pixels).cpu().numpy()}
    if dimg is not None:
        grads = {k: torch.zeros_like(v) for k, v in p.items()}
        r.backward(p, torch.from_numpy(dimg.reshape(-1).astype(np.float32)).cuda(), grads)
        r.check()
        out["grads"] = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    return out


def test_masked_render_matches_oracle():
    params, view, cfg = masked_case()
    st = oracle_settings(cfg)
    pr = oracle.preprocess(oracle_params(params), view, st, relax=RELAX)
    g = run_gpu(params, view, cfg)
    unc = (pr["uncertain"] & 1) > 0
    certain = int(((pr["status"] == 0) & ~unc).sum())
    assert certain <= g["visible"] <= certain + int(unc.sum())
    assert (pr["status"] == 7).sum() > 100
    check_pixels(pr, view, cfg, np.arange(view["width"] * view["height"]), g["img"].reshape(3, -1).T, g["T"])


def test_mask_gradient_matches_oracle():
    params, view, cfg = masked_case(seed=14)
    st = oracle_settings(cfg)
    op = oracle_params(params)
    flags = oracle_flags(oracle.preprocess(op, view, st, relax=RELAX), view, cfg)
    pr = oracle.preprocess(op, view, st)
    dimg = loss_gradient_at_settled_pixels(np.random.default_rng(15), flags, (3,) + flags.shape)
    g_orc = oracle.render_backward(op, pr, view, st, dimg)
    g = run_gpu(params, view, cfg, dimg)["grads"]
    assert np.abs(g_orc["mask_logit"]).max() > 0
    assert np.all(g["mask_logit"][pr["status"] != 0] == 0)
    for k in PARAM_KEYS + ("mask_logit",):
        compare_group(k, g[k], g_orc[k], 1e-3, 1e-4)


def test_mask_loss_kernel():
    import torch
    m = np.random.default_rng(16).normal(0, 2, 100_003).astype(np.float32)
    loss, grad = mask_loss(torch.from_numpy(m).cuda())
    torch.cuda.synchronize()
    M = 1.0 / (1.0 + np.exp(-m.astype(np.float64)))
    assert abs(float(loss.item()) - M.mean()) <= 1e-5
    np.testing.assert_allclose(grad.cpu().numpy(), M * (1 - M) / m.size, rtol=1e-4, atol=1e-12)
