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


@pytest.mark.parametrize("tile,ppt,batch", [(16, 4, 128), (16, 2, 256), (8, 1, 128)])
def test_render_image_equals_render_fwd(tile, ppt, batch):
    """fgs4d_render_image (no backward state) gives fgs4d_render_fwd's image
    and final transmittance bit for bit and leaves the last-index plane 0."""
    import torch
    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import RenderConfig, Renderer

    n = 3000
    params = sy.make_scene(n, 13, (-1, -1, -1), (1, 1, 1), sh_degree=2, t_order=1).as_dict()
    cfg = RenderConfig(sh_degree=2, t_order=1, inst_capacity=1 << 19, tile=tile, pixels_per_thread=ppt,
                       shared_batch=batch, bg=(0.1, 0.2, 0.3))
    views = [sy.tiny_view(150, 97, t=0.3), sy.tiny_view(64, 40, t=0.7)]
    r = Renderer(n, views, cfg)
    dev = to_device(params)
    ref = r.forward(dev)
    r.check()
    npx = r.total_pixels
    T_ref = r.workspace_view(r.layout.pix_T, torch.float32, npx).clone()
    assert int(r.workspace_view(r.layout.pix_last, torch.int32, npx).max()) > 0
    out = torch.empty_like(ref)
    out_T = torch.empty(npx, device="cuda")
    fgs4d.render_image(n, r.views, r.nviews, r.settings, r.ws.data_ptr(), r.ws_bytes, out.data_ptr(),
                       out_T.data_ptr(), r.stream())
    r.check()
    assert torch.equal(out, ref)
    assert torch.equal(out_T, T_ref)
    assert int(r.workspace_view(r.layout.pix_last, torch.int32, npx).abs().max()) == 0


@pytest.mark.parametrize("nviews", [1, 3])
def test_lean_stage_grids_change_nothing(nviews):
    """stage_blocks_per_sm = 1 (persistent preprocess, radix and emission
    grids of one or two blocks per SM) gives the same slots, instance lists,
    images and gradients as the full-GPU grids, bit for bit."""
    import torch
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import PARAM_KEYS, RenderConfig, Renderer

    n = 60_000  # ~235 logical preprocess blocks per view: several per block at one block per SM
    params = sy.make_scene(n, 17, (-1.5, -1.5, -1.5), (1.5, 1.5, 1.5), sh_degree=1, t_order=1).as_dict()
    dev = to_device(params)
    views = [sy.tiny_view(400, 300, t=0.2 + 0.3 * k) for k in range(nviews)]
    out = {}
    for k in (0, 1):
        cfg = RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 22, stage_blocks_per_sm=k)
        r = Renderer(n, views, cfg)
        img = r.forward(dev)
        counts = r.check()
        m = counts[1]
        g = {key: torch.zeros_like(dev[key]) for key in PARAM_KEYS}
        r.backward(dev, torch.ones_like(img), g)
        r.check()
        out[k] = (img.clone(), counts,
                  r.workspace_view(r.layout.sorted_slots, torch.int32, counts[0]).clone(),
                  r.workspace_view(r.layout.inst_slot, torch.int32, m).clone(),
                  r.workspace_view(r.layout.inst_tile, torch.int32, m).clone(), g)
    a, b = out[0], out[1]
    assert a[1] == b[1] and a[1][1] > 100_000
    for x, y in zip(a[:1] + a[2:5], b[:1] + b[2:5]):
        assert torch.equal(x, y)
    for key in PARAM_KEYS:  # atomics add in another order: equal up to rounding
        scale = float(a[5][key].abs().max())
        assert float((a[5][key] - b[5][key]).abs().max()) <= 1e-4 * scale + 1e-12, key
