"""The training loop's Adam kernel against torch.optim.Adam (plain PyTorch
FP32 reference of the same update) over several steps, with tensor sizes
that exercise the vector body and the scalar tail."""
import numpy as np
import pytest

from paper_2412_20720_gb300.render import Adam

pytestmark = pytest.mark.gpu


def test_adam_matches_torch_reference():
    import torch
    gen = torch.Generator(device="cuda").manual_seed(5)
    shapes = {"a": (1003, 4), "b": (77,), "c": (257, 48, 3)}
    p_ours = {k: torch.randn(s, device="cuda", generator=gen) for k, s in shapes.items()}
    p_ref = {k: v.clone().requires_grad_(True) for k, v in p_ours.items()}
    ours = Adam(p_ours, lr=3e-3, betas=(0.9, 0.99), eps=1e-8)
    ref = torch.optim.Adam(list(p_ref.values()), lr=3e-3, betas=(0.9, 0.99), eps=1e-8)
    for _ in range(6):
        grads = {k: torch.randn(s, device="cuda", generator=gen) for k, s in shapes.items()}
        ours.step(grads)
        for k in shapes:
            p_ref[k].grad = grads[k].clone()
        ref.step()
    torch.cuda.synchronize()
    assert int(ours.t.item()) == 6
    for k in shapes:
        np.testing.assert_allclose(p_ours[k].cpu().numpy(), p_ref[k].detach().cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_adam_set_equals_one_call_per_tensor_and_clears_gradients():
    """fgs4d_adam_update_set over ragged tensors (empty, scalar tails, float4
    bodies) gives fgs4d_adam_update's parameters and moments bit for bit; with
    zero_grad it leaves every gradient 0, without it the gradients untouched."""
    import torch
    from paper_2412_20720_gb300 import fgs4d
    gen = torch.Generator(device="cuda").manual_seed(11)
    counts = [0, 1, 3, 4, 5, 1001, 262147]
    lrs = [1e-3 * (k + 1) for k in range(len(counts))]
    st = torch.cuda.current_stream().cuda_stream

    def state():
        return [[torch.randn(c, device="cuda", generator=gen) for _ in range(4)] for c in counts]

    ref = state()
    for s in ref:
        s[3].abs_()  # second moments are non-negative
    out = {z: [[x.clone() for x in s] for s in ref] for z in (False, True)}
    step = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    for (p, g, m, v), c, lr in zip(ref, counts, lrs):
        fgs4d.adam_update(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), c, lr, 0.9, 0.99, 1e-8,
                          step.data_ptr(), st)
    for z, tensors in out.items():
        fgs4d.adam_update_set([(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), c, lr)
                               for (p, g, m, v), c, lr in zip(tensors, counts, lrs)],
                              0.9, 0.99, 1e-8, step.data_ptr(), z, st)
    torch.cuda.synchronize()
    for k in range(len(counts)):
        for z, tensors in out.items():
            for i in (0, 2, 3):  # param, exp_avg, exp_avg_sq
                assert torch.equal(tensors[k][i], ref[k][i]), (k, z, i)
        assert torch.equal(out[False][k][1], ref[k][1])
        assert not out[True][k][1].any()
