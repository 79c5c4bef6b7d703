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
