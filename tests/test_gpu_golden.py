"""The CUDA path (through the C ABI) against the stored oracle render of the
tiny configuration (tests/golden/tiny_2000_128x96.txt): every sampled pixel
within the image tolerance of the stored result or of one of its stored
admissible alternatives, without running the oracle."""
import os
import sys

import numpy as np
import pytest

from helpers import IMAGE_ATOL, CudaRender

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

pytestmark = pytest.mark.gpu


def test_tiny_render_matches_the_stored_oracle_values():
    g = make_golden.read()
    params, view, cfg = make_golden.tiny_scene_inputs()
    assert params["mean"].shape[0] == g["kept"]
    run = CudaRender(params, [view], cfg)
    py, px = g["py"], g["px"]
    got = np.concatenate([run.images[0][:, py, px], run.T.reshape(view["height"], view["width"])[py, px][None]]).T
    plain = np.concatenate([g["rgb"], g["T"][:, None]], axis=1)
    for q in range(py.size):
        cands = np.concatenate([plain[q:q + 1], g["alternatives"][q]])
        assert np.abs(cands - got[q]).max(axis=1).min() <= IMAGE_ATOL, (py[q], px[q], got[q], cands)
