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



def test_view_parallel_step_matches_one_batched_call():
    """Forward, L1 loss (mean over all views, in parts) and backward of each
    view on its own stream give the batched call's images bit for bit, and
    its loss and gradients up to the order of float atomic additions."""
    import torch
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer, ViewParallel, l1_loss

    n = 2500
    params = sy.make_scene(n, 8, (-1, -1, -1), (1, 1, 1), sh_degree=2, t_order=1).as_dict()
    tparams = sy.make_scene(n, 9, (-1, -1, -1), (1, 1, 1), sh_degree=2, t_order=1).as_dict()
    cfg = RenderConfig(sh_degree=2, t_order=1, inst_capacity=1 << 19)
    views = [sy.tiny_view(120, 88, t=0.2), sy.tiny_view(96, 64, t=0.5), sy.tiny_view(130, 90, t=0.8)]
    dev, tdev = to_device(params), to_device(tparams)
    rb = Renderer(n, views, cfg)
    target = rb.forward(tdev).clone()
    rb.check()
    targets = [t.reshape(-1).clone() for t in rb.split(target)]
    g_ref = {k: torch.zeros_like(dev[k]) for k in PARAM_KEYS}
    img_ref = rb.forward(dev)
    loss_ref, dimg = l1_loss(img_ref, target)
    rb.backward(dev, dimg, g_ref)
    rb.check()

    vp = ViewParallel(n, [[v] for v in views], cfg)
    g = {k: torch.zeros_like(dev[k]) for k in PARAM_KEYS}
    loss = torch.zeros(1, device="cuda")
    imgs = vp.step(dev, lambda j, img: l1_loss(img, targets[j], mean_count=target.numel(), loss=loss)[1], g)
    vp.check()
    for j, img in enumerate(imgs):
        assert torch.equal(img, rb.split(img_ref)[j].reshape(-1))
    # float32 sums of ~33k terms in different orders (block partial sums, atomics)
    assert abs(float(loss) - float(loss_ref)) <= 2e-5 * abs(float(loss_ref))
    for k in PARAM_KEYS:
        scale = float(g_ref[k].abs().max())
        assert scale > 0
        assert float((g[k] - g_ref[k]).abs().max()) <= 1e-4 * scale, k
