"""Parity of the scale-gated feature rendering (Sec. 7) and its backward
(geometry fixed) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import RenderConfig, Renderer

from helpers import PIXEL_MARGIN, compare_group, keep_clear_of_boundaries, oracle_settings, subset, to_device

pytestmark = pytest.mark.gpu


def feat_case(D, ts=(0.5,), seed=17, n=1500):
    sc = sy.make_scene(n, seed, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    views = [sy.tiny_view(96, 72, t=t) for t in ts]
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 18)
    params = sc.as_dict()
    params = subset(params, keep_clear_of_boundaries(params, views, cfg))
    rng = np.random.default_rng(seed)
    feats = rng.standard_normal((params["mean"].shape[0], D)).astype(np.float32)
    gate = rng.uniform(0.0, 1.0, D).astype(np.float32)
    return params, views, cfg, feats, gate


@pytest.mark.parametrize("D,ts", [(32, (0.5,)), (8, (0.4, 0.6)), (16, (0.5,))])
def test_feature_map_matches_oracle(D, ts):
    import torch
    params, views, cfg, feats, gate = feat_case(D, ts)
    r = Renderer(params["mean"].shape[0], views, cfg)
    out = r.forward_features(to_device(params), torch.from_numpy(feats).cuda(), torch.from_numpy(gate).cuda())
    r.check()
    got = [x.cpu().numpy() for x in r.split(out, D)]
    st = oracle_settings(cfg)
    for k, v in enumerate(views):
        pr = oracle.preprocess(params, v, st)
        F, mg = oracle.render_features(pr, v, st, feats, gate)
        ok = mg >= PIXEL_MARGIN
        assert ok.mean() >= 0.95 and np.abs(F).max() > 0.3
        assert np.abs(got[k] - F)[:, ok].max() <= 2e-4


def test_feature_backward_matches_oracle():
    import torch
    D = 32
    params, views, cfg, feats, gate = feat_case(D, seed=18)
    view = views[0]
    st = oracle_settings(cfg)
    pr = oracle.preprocess(params, view, st)
    F, mg = oracle.render_features(pr, view, st, feats, gate)
    ok = mg >= PIXEL_MARGIN
    dF = np.random.default_rng(19).standard_normal(F.shape) * ok
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
