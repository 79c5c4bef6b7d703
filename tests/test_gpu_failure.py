"""Failure detection on the GPU without a fault: the library's bounded
inter-block waits, run against a predecessor that never posts, give up after
their poll limit, report FGS4D_ERR_TIMEOUT through a status word, and leave
the context usable (a render right after succeeds)."""
import time

import numpy as np
import pytest

from helpers import to_device

pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_leave_the_context_usable():
    import torch
    from paper_2412_20720_gb300 import fgs4d
    from paper_2412_20720_gb300 import synthetic as sy
    from paper_2412_20720_gb300.render import RenderConfig, Renderer

    scratch = torch.zeros(fgs4d.WAIT_SELFTEST_BYTES // 4, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    code = fgs4d.wait_selftest(scratch.data_ptr(), fgs4d.WAIT_SELFTEST_BYTES,
                               torch.cuda.current_stream().cuda_stream)
    elapsed = time.perf_counter() - t0
    assert code == fgs4d.ERR_TIMEOUT, fgs4d.status_string(code)
    assert elapsed < 60.0
    # The context is intact: a render on the same device works and is clean.
    params = sy.make_scene(500, 3, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1).as_dict()
    r = Renderer(500, [sy.tiny_view(64, 48)], RenderConfig(sh_degree=1, t_order=1, inst_capacity=1 << 16))
    img = r.forward(to_device(params))
    counts = r.check()
    assert counts[0] > 0 and np.isfinite(img.cpu().numpy()).all()
