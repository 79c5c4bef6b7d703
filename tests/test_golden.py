"""Checks against tests/golden/: the values the paper fixes for the render
path (the library's and the oracle's defaults, and the oracle's decision at
the temporal-filter threshold), and the oracle's render of the tiny
configuration as stored by tests/golden/make_golden.py (a regression guard:
the stored values were written by the oracle alone)."""
import math
import os
import sys

import numpy as np

import oracle
from paper_2412_20720_gb300 import fgs4d
from paper_2412_20720_gb300 import synthetic as sy
from paper_2412_20720_gb300.render import RenderConfig

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402


def paper_values() -> dict:
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        if line.strip() and not line.startswith("#"):
            name, value, passage = line.split(None, 2)
            assert passage.startswith("Sec. "), name  # every value cites its passage
            out[name] = value
    return out


def test_defaults_are_the_papers_values():
    v = paper_values()
    p_min = float(v["temporal_filter_p_min"])
    assert RenderConfig().p_t_min == p_min
    assert oracle.Settings().p_t_min == p_min
    assert fgs4d.make_settings().p_t_min == np.float32(p_min)
    assert RenderConfig().mask_threshold == float(v["mask_threshold"])


def test_identity_quaternions_give_the_identity_rotation():
    q = np.array([float(x) for x in paper_values()["identity_quaternions"].split(",")])
    np.testing.assert_array_equal(oracle.rotation(q, q), np.eye(4))


def _single_gaussian(dt_over_sigma: float, log_st: float = math.log(0.2), t: float = 0.5):
    """One Gaussian at the origin in front of the tiny camera with identity
    rotation (Sigma_44 = s_t^2), its temporal mean dt_over_sigma s_t before t."""
    st = math.exp(np.float32(log_st))
    mu_t = np.float32(t - dt_over_sigma * st)
    p = {"mean": np.array([[0.0, 0.0, 0.0, mu_t]], dtype=np.float32),
         "log_scale": np.array([[math.log(0.1)] * 3 + [log_st]], dtype=np.float32),
         "q_l": np.array([[1.0, 0.0, 0.0, 0.0]], dtype=np.float32),
         "q_r": np.array([[1.0, 0.0, 0.0, 0.0]], dtype=np.float32),
         "opacity_logit": np.array([3.0], dtype=np.float32),
         "sh": np.zeros((1, 8, 3), dtype=np.float32)}
    return p, sy.tiny_view(t=t)


def test_oracle_filters_below_the_papers_threshold():
    """p(t) = exp(-dt^2 / (2 Sigma_44)) just above the threshold keeps the
    Gaussian, just below culls it (status 2, the temporal filter)."""
    p_min = float(paper_values()["temporal_filter_p_min"])
    st = oracle.Settings(sh_degree=1, t_order=1)
    for rel, status in ((1.0 + 1e-4, 0), (1.0 - 1e-4, 2)):
        k = math.sqrt(2.0 * math.log(1.0 / (p_min * rel)))
        params, view = _single_gaussian(k)
        pr = oracle.preprocess(params, view, st)
        assert int(pr["status"][0]) == status, (rel, int(pr["status"][0]))


def test_oracle_tiny_render_matches_the_stored_values():
    g = make_golden.read()
    params, view, cfg = make_golden.tiny_inputs()
    assert params["mean"].shape[0] == g["kept"]
    img, T, margin = make_golden.oracle_render(params, view, cfg)
    # FP64 on the same inputs: equal up to the host's libm (x86 and Arm).
    np.testing.assert_allclose(img[:, g["py"], g["px"]].T, g["rgb"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(T[g["py"], g["px"]], g["T"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(margin[g["py"], g["px"]], g["margin"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(img.reshape(3, -1).sum(axis=1), g["sum_rgb"], rtol=1e-12)
    np.testing.assert_allclose(T.sum(), g["sum_T"], rtol=1e-12)
    pix = g["py"] * view["width"] + g["px"]
    plain = np.concatenate([img.reshape(3, -1)[:, pix], T.reshape(1, -1)[:, pix]]).T
    alts = make_golden.alternatives(params, view, cfg, pix, plain)
    assert sum(a.shape[0] for a in g["alternatives"]) > 0  # some sampled pixels sit on a threshold
    for got, want in zip(alts, g["alternatives"]):
        assert got.shape == want.shape
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
