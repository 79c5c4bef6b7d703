"""Frames rendered with several in flight (FramePipeline: one workspace and
one stream per slot) equal the same views rendered one at a time, bit for
bit (single-frame renders are held to the oracle by the parity tests)."""
import numpy as np
import pytest

from helpers import to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth", [1, 3])
def test_frames_in_flight_equal_single_frames(depth):
    import torch
    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import FramePipeline, RenderConfig, Renderer

    n = 3000
    params = sy.make_scene(n, 5, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1).as_dict()
    cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 18)
    dev = to_device(params)
    views = [sy.tiny_view(144, 100, t=float(t)) for t in np.linspace(0.05, 0.95, 7)]
    pipe = FramePipeline(n, views[0], cfg, depth=depth)
    g = pipe.slots[0].gaussians(dev)
    npx = 3 * 144 * 100
    outs = [torch.full((npx,), -1.0, device="cuda") for _ in views]
    pipe.begin()
    for k, v in enumerate(views):
        vs, nv = fgs4d.make_views([v])
        pipe.submit(g, vs, nv, outs[k].data_ptr())
    pipe.end()
    pipe.check()
    for k, v in enumerate(views):
        r = Renderer(n, [v], cfg)
        ref = r.forward(dev)
        r.check()
        assert torch.equal(outs[k], ref), "frame %d differs" % k

