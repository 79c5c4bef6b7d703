"""Parity of the auxiliary render channels (depth, opacity 1 - T, optical flow
of the sliced mean over a time step) with the FP64 oracle, through the C ABI
entry fgs4d_render_aux."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import RenderConfig, Renderer

from helpers import (IMAGE_ATOL, RELAX, check_pixels, loss_gradient_at_settled_pixels, oracle_flags, oracle_proj,
                     oracle_settings, to_device)

pytestmark = pytest.mark.gpu


def case(width, height, L, NT, seed, n=2000, ts=(0.5,), static=False):
    sc = sy.make_scene(n, seed, (-1, -1, -1), (1, 1, 1), sh_degree=L, t_order=NT)
    params = sc.as_dict()
    if static:  # q_r = (a, b, c, -d) for q_l = (a, b, c, d): Sigma_xt = 0
        params["q_r"] = np.ascontiguousarray(params["q_l"] * np.array([1, 1, 1, -1], np.float32))
    views = [sy.tiny_view(width, height, t=t) for t in ts]
    cfg = RenderConfig(sh_degree=L, t_order=NT, inst_capacity=1 << 19)
    return params, views, cfg


def gpu_aux(params, views, cfg, flow_dt):
    import torch
    r = Renderer(params["mean"].shape[0], views, cfg)
    p = to_device(params)
    rgb, aux = r.forward_aux(p, flow_dt)
    r.check()
    plain = r.forward(p).clone()
    torch.cuda.synchronize()
    return ([x.cpu().numpy() for x in r.split(rgb)], [x.cpu().numpy() for x in r.split(aux, 4)],
            [x.cpu().numpy() for x in r.split(plain)])


def oracle_aux(params, view, cfg, flow_dt):
    st = oracle_settings(cfg)
    pr = oracle.preprocess(params, view, st)
    aux = oracle.aux_records(params, pr, view, st, float(np.float32(flow_dt)))
    return oracle.render_aux(pr, aux, view, st), aux


@pytest.mark.parametrize("w,h,L,NT,ts", [(128, 96, 1, 1, (0.5,)), (131, 77, 3, 2, (0.45,)),
                                         (64, 48, 2, 1, (0.3, 0.5, 0.7))])
def test_aux_channels_match_oracle(w, h, L, NT, ts):
    """Every pixel's image, opacity (1 - T), depth and flow against the
    admissible results of the oracle, whose extra channels are the
    per-Gaussian (z, flow_u, flow_v) composited with the colour weights."""
    params, views, cfg = case(w, h, L, NT, seed=3, ts=ts)
    dt = 0.05
    rgb, aux, plain = gpu_aux(params, views, cfg, dt)
    st = oracle_settings(cfg)
    for k, view in enumerate(views):
        np.testing.assert_array_equal(rgb[k], plain[k])  # the image is fgs4d_render_fwd's, bit for bit
        pr = oracle_proj(params, view, cfg)
        rec = oracle.aux_records(params, pr, view, st, float(np.float32(dt)), relax=RELAX)
        flags, chosen = check_pixels(pr, view, cfg, np.arange(w * h), rgb[k].reshape(3, -1).T,
                                     1.0 - aux[k][1].reshape(-1).astype(np.float64), extra=rec)
        zmax = np.abs(rec[:, 0]).max()
        assert np.abs(aux[k][0].reshape(-1) - chosen[:, 5]).max() <= IMAGE_ATOL * zmax  # depth
        fmax = max(np.abs(rec[:, 1:]).max(), 1.0)
        assert np.abs(chosen[:, 6:8]).max() > 0.05  # the scene moves
        assert np.abs(aux[k][2:].reshape(2, -1).T - chosen[:, 6:8]).max() <= IMAGE_ATOL * fmax  # flow, pixels


def test_flow_vanishes_for_gaussians_without_space_time_coupling():
    params, views, cfg = case(96, 64, 1, 1, seed=4, static=True)
    rgb, aux, plain = gpu_aux(params, views, cfg, 0.05)
    (img, T, out, mg), rec = oracle_aux(params, views[0], cfg, 0.05)
    assert np.all(out[2:] == 0.0)
    # In FP32 the rotation leaves the t axis fixed up to rounding.
    assert np.abs(aux[0][2:]).max() <= 1e-4
    assert aux[0][0].max() > 1.0 and aux[0][1].max() > 0.2


@pytest.mark.parametrize("L,NT", [(1, 1), (3, 2)])
def test_depth_and_opacity_gradients_match_oracle(L, NT):
    """Loss on the image, the depth and the opacity channels: per-slot and
    per-parameter gradients against the oracle's adjoint (pinned by central
    differences on the CPU)."""
    import torch
    from helpers import compare_group, records_from_gpu, CudaRender
    from paper_2412_20720_gb300.render import PARAM_KEYS
    params, views, cfg = case(96, 80, L, NT, seed=6)
    view = views[0]
    st = oracle_settings(cfg)
    flags = oracle_flags(oracle_proj(params, view, cfg), view, cfg)
    pr = oracle.preprocess(params, view, st)
    aux = oracle.aux_records(params, pr, view, st, 0.05)
    img, T, out, mg = oracle.render_aux(pr, aux, view, st)
    rng = np.random.default_rng(8)
    dimg = loss_gradient_at_settled_pixels(rng, flags, img.shape)
    daux = np.zeros_like(out)
    daux[:2] = loss_gradient_at_settled_pixels(rng, flags, (2,) + flags.shape)
    g_orc = oracle.render_aux_backward(params, pr, view, st, dimg, daux)

    run = CudaRender(params, views, cfg)  # records for the slot order
    r = run.renderer
    r.forward_aux(run.params, 0.05)
    grads = {k: torch.zeros_like(v) for k, v in run.params.items()}
    r.backward_aux(run.params, torch.from_numpy(dimg.reshape(-1).astype(np.float32)).cuda(),
                   torch.from_numpy(daux.reshape(-1).astype(np.float32)).cuda(), grads)
    r.check()
    nv = run.counts[0]
    slot = r.workspace_view(r.layout.slot_grad, torch.float32, 12 * nv).cpu().numpy().reshape(nv, 12)
    vis = records_from_gpu(run)["index"]
    rtol, floor = 1e-3, 1e-4
    compare_group("g_uv", slot[:, 0:2], g_orc["g_uv"][vis], rtol, floor)
    compare_group("g_conic", slot[:, 2:5], g_orc["g_conic"][vis], rtol, floor)
    compare_group("g_a", slot[:, 5], g_orc["g_a"][vis], rtol, floor)
    compare_group("g_z", slot[:, 9], g_orc["g_z"][vis], rtol, floor)
    for k in PARAM_KEYS:
        compare_group(k, grads[k].cpu().numpy().astype(np.float64), g_orc[k], rtol, floor)
