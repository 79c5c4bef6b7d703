"""The CUDA-graph form of the batched path, captured with torch.cuda.graph and
replayed, against the same calls launched one by one and against the FP64
oracle:

- the training step: forward of 4 timestamps x 1 camera in one call, L1 loss
  against targets rendered by the oracle from a second seeded scene,
  backward to every parameter;
- a group of 8 (camera, t) views of mixed resolution on a sphere around the
  scene, forward + backward in one call.

Each graph is replayed twice.  Images equal the plain calls' bit for bit;
gradients equal them up to the order of the atomic sums; every pixel matches
the oracle's admissible results and the gradients match the oracle's
adjoint."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer, l1_loss

from helpers import (ORDER_FLOOR, ORDER_RTOL, check_pixels, compare_group, loss_gradient_at_settled_pixels,
                     oracle_flags, oracle_proj, oracle_settings, to_device)

pytestmark = pytest.mark.gpu


def _capture(step):
    """step() captured as one CUDA graph after two warm-up runs on a side
    stream (what a training loop replays)."""
    import torch
    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    cur.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = step()
    return graph, out


def _pixel_T(r):
    import torch
    return r.workspace_view(r.layout.pix_T, torch.float32, r.total_pixels).cpu().numpy()


def _check_images_against_oracle(r, params, views, cfg, flat, T):
    off = 0
    for k, (v, img) in enumerate(zip(views, r.split(flat))):
        H, W = int(v["height"]), int(v["width"])
        check_pixels(oracle_proj(params, v, cfg), v, cfg, np.arange(W * H), img.cpu().numpy().reshape(3, -1).T,
                     T[off:off + W * H])
        off += W * H


def test_training_step_graph_replays_equal_the_plain_step():
    import torch
    sc = sy.make_scene(6000, 40, (-1, -1, -1), (1, 1, 1), sh_degree=3, t_order=2)
    tgt = sy.make_scene(6000, sy.TARGET_SEED, (-1, -1, -1), (1, 1, 1), sh_degree=3, t_order=2)
    ts = np.random.default_rng(sy.POSE_SEED).random(4)
    views = [sy.tiny_view(120, 90, t=float(t)) for t in ts]
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 20)
    st = oracle_settings(cfg)
    params = sc.as_dict()
    tp = tgt.as_dict()
    target = np.concatenate([oracle.render(oracle.preprocess(tp, v, st), v, st)[0].reshape(-1) for v in views])
    target_d = torch.from_numpy(target.astype(np.float32)).cuda()
    p = to_device(params)
    r = Renderer(sc.n, views, cfg)
    grads = {k: torch.zeros_like(v) for k, v in p.items()}

    def step():
        for g in grads.values():
            g.zero_()
        img = r.forward(p)
        loss, dimg = l1_loss(img, target_d)
        r.backward(p, dimg, grads)
        return img, loss

    img0, loss0 = step()
    r.check()
    plain = (img0.clone(), float(loss0.item()), {k: g.cpu().numpy().astype(np.float64) for k, g in grads.items()})
    T0 = _pixel_T(r)
    graph, (img_g, loss_g) = _capture(step)
    for _ in range(2):
        for g in grads.values():
            g.fill_(float("nan"))  # the replay must clear and refill them
        img_g.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        r.check()
        assert torch.equal(img_g, plain[0])
        np.testing.assert_array_equal(_pixel_T(r), T0)
        assert abs(float(loss_g.item()) - plain[1]) <= 1e-6 * plain[1]
        for k in PARAM_KEYS:
            compare_group(k, grads[k].cpu().numpy().astype(np.float64), plain[2][k], ORDER_RTOL, ORDER_FLOOR)
    # the replayed images against the oracle, the loss against its definition
    _check_images_against_oracle(r, params, views, cfg, img_g, T0)
    ref = np.abs(img_g.cpu().numpy().astype(np.float64) - target).mean()
    assert abs(float(loss_g.item()) - ref) <= 1e-5 * ref
    del graph


def test_mixed_resolution_view_group_graph_matches_plain_calls_and_oracle():
    import torch
    sc = sy.make_scene(5000, 41, (-1, -1, -1), (1, 1, 1), sh_degree=3, t_order=2)
    rng = np.random.default_rng(42)
    sizes = [(64, 64), (100, 100), (96, 128), (128, 96)]
    views = []
    for k in range(8):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        up = (0, -1, 0) if abs(d[1]) < 0.9 else (1, 0, 0)
        w, h = sizes[k % 4]
        views.append(sy.look_at(3.5 * d, (0, 0, 0), up, w, h, float(rng.random())))
    cfg = RenderConfig(sh_degree=3, t_order=2, inst_capacity=1 << 20, bg=(0.1, 0.2, 0.0))
    params = sc.as_dict()
    st = oracle_settings(cfg)
    # upstream gradient: random where every decision is settled
    dls, g_orc = [], None
    for v in views:
        flags = oracle_flags(oracle_proj(params, v, cfg), v, cfg)
        d = loss_gradient_at_settled_pixels(rng, flags, (3,) + flags.shape)
        dls.append(d.reshape(-1))
        g = oracle.render_backward(params, oracle.preprocess(params, v, st), v, st, d)
        g_orc = g if g_orc is None else {k: g_orc[k] + g[k] for k in g}
    dL = torch.from_numpy(np.concatenate(dls).astype(np.float32)).cuda()
    p = to_device(params)
    r = Renderer(sc.n, views, cfg)
    grads = {k: torch.zeros_like(v) for k, v in p.items()}

    def step():
        for g in grads.values():
            g.zero_()
        img = r.forward(p)
        r.backward(p, dL, grads)
        return img

    img0 = step()
    r.check()
    plain_img = img0.clone()
    plain_g = {k: g.cpu().numpy().astype(np.float64) for k, g in grads.items()}
    T0 = _pixel_T(r)
    graph, img_g = _capture(step)
    for _ in range(2):
        img_g.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        r.check()
        assert torch.equal(img_g, plain_img)
        np.testing.assert_array_equal(_pixel_T(r), T0)
        for k in PARAM_KEYS:
            got = grads[k].cpu().numpy().astype(np.float64)
            compare_group(k, got, plain_g[k], ORDER_RTOL, ORDER_FLOOR)
            compare_group(k, got, g_orc[k], 1e-3, 1e-4)
    _check_images_against_oracle(r, params, views, cfg, img_g, T0)
    assert len(set(r.sizes)) == 4
    del graph
