"""Parity of the scale-gated feature rendering (Sec. 7) and its backward
(geometry fixed) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import RenderConfig, Renderer

from helpers import (check_pixels, compare_group, loss_gradient_at_settled_pixels, oracle_flags, oracle_proj,
                     oracle_settings, to_device)

pytestmark = pytest.mark.gpu


def feat_case(D, ts=(0.5,), seed=17, n=1500, tile=16):
    sc = sy.make_scene(n, seed, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    views = [sy.tiny_view(96, 72, t=t) for t in ts]
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 18, tile=tile)
    params = sc.as_dict()
    rng = np.random.default_rng(seed)
    feats = rng.standard_normal((params["mean"].shape[0], D)).astype(np.float32)
    gate = rng.uniform(0.0, 1.0, D).astype(np.float32)
    return params, views, cfg, feats, gate


@pytest.mark.parametrize("D,ts", [(32, (0.5,)), (8, (0.4, 0.6)), (16, (0.5,))])
def test_feature_map_matches_oracle(D, ts):
    import torch
    params, views, cfg, feats, gate = feat_case(D, ts)
    r = Renderer(params["mean"].shape[0], views, cfg)
    p = to_device(params)
    out = r.forward_features(p, torch.from_numpy(feats).cuda(), torch.from_numpy(gate).cuda())
    r.check()
    got = [x.cpu().numpy() for x in r.split(out, D)]
    img = [x.cpu().numpy() for x in r.split(r.forward(p))]
    T = r.workspace_view(r.layout.pix_T, torch.float32, r.total_pixels).cpu().numpy()
    r.check()
    fhat = oracle.gated_features(feats, gate)
    off = 0
    for k, v in enumerate(views):
        H, W = int(v["height"]), int(v["width"])
        pr = oracle_proj(params, v, cfg)
        # the admissible results carry the features composited with the
        # colour weights as extra channels; the matched one is checked
        flags, chosen = check_pixels(pr, v, cfg, np.arange(W * H), img[k].reshape(3, -1).T, T[off:off + H * W],
                                     extra=fhat)
        off += H * W
        assert np.abs(chosen[:, 5:]).max() > 0.3
        assert np.abs(got[k].reshape(D, -1).T - chosen[:, 5:]).max() <= 2e-4


# The adjoint takes 4-pixel strips for D <= 16 on 16-pixel tiles, 2-pixel
# strips otherwise.
@pytest.mark.parametrize("D,tile", [(32, 16), (16, 16), (8, 16), (8, 8)])
def test_feature_backward_matches_oracle(D, tile):
    import torch
    params, views, cfg, feats, gate = feat_case(D, seed=18, tile=tile)
    view = views[0]
    st = oracle_settings(cfg)
    flags = oracle_flags(oracle_proj(params, view, cfg), view, cfg)
    pr = oracle.preprocess(params, view, st)
    F, mg = oracle.render_features(pr, view, st, feats, gate)
    dF = loss_gradient_at_settled_pixels(np.random.default_rng(19), flags, F.shape)
    gf, gg = oracle.render_features_backward(pr, view, st, feats, gate, dF)
    r = Renderer(params["mean"].shape[0], views, cfg)
    f_d, g_d = torch.from_numpy(feats).cuda(), torch.from_numpy(gate).cuda()
    r.forward_features(to_device(params), f_d, g_d)
    grad_f = torch.zeros_like(f_d)
    grad_g = torch.zeros_like(g_d)
    r.backward_features(f_d, g_d, torch.from_numpy(dF.reshape(-1).astype(np.float32)).cuda(), grad_f, grad_g)
    r.check()
    compare_group("dL/df", grad_f.cpu().numpy().astype(np.float64), gf, 1e-3, 1e-4)
    compare_group("dL/dgate", grad_g.cpu().numpy().astype(np.float64), gg, 1e-3, 1e-4)
