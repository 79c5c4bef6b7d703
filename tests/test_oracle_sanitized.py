"""The FP64 oracle's C code under AddressSanitizer and UndefinedBehavior-
Sanitizer: a subprocess loads the instrumented build (libasan preloaded, any
finding aborts) and runs every entry point on small cases -- preprocess,
render, per-pixel render, the adjoints, auxiliary channels, features, split
sampling, densification statistics and the instance sort."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np
import oracle
from paper_2412_20720_gb300 import synthetic as sy

for L, NT, n, (w, h) in ((3, 2, 64, (32, 32)), (1, 1, 300, (45, 29)), (0, 0, 40, (17, 9))):
    sc = sy.make_scene(n, 7, (-0.6, -0.6, -0.6), (0.6, 0.6, 0.6), sh_degree=L, t_order=NT)
    p = sc.as_dict()
    view = sy.tiny_view(w, h, t=0.5)
    st = oracle.Settings(sh_degree=L, t_order=NT, tile=16, period=1.0, near_plane=0.2, dilation=0.3, p_t_min=0.05)
    pr = oracle.preprocess(p, view, st)
    img, T, nc, mg = oracle.render(pr, view, st)
    pix = np.array([[0, 0], [w - 1, h - 1], [w // 2, h // 2]], dtype=np.int32)
    oracle.render_pixels(pr, view, st, pix)
    prr = oracle.preprocess(p, view, st, relax=1e-3)
    oracle.render_pixels_admissible(prr, view, st, np.arange(w * h),
                                    oracle.Tolerance(eps_conic=1e-3, eps_uv=1e-5, eps_uv_abs=1e-3, eps_a=1e-4,
                                                     eps_alpha=1e-5, depth_ulps=4), extra=np.ones((n, 3)))
    dimg = np.random.default_rng(0).standard_normal(img.shape)
    oracle.render_backward(p, pr, view, st, dimg)
    aux = oracle.aux_records(p, pr, view, st, 0.05)
    rgb, aux_img = oracle.render_aux(pr, aux, view, st)[:2]
    daux = np.zeros((4, h, w))
    daux[:2] = 1.0  # depth and opacity; flow is not differentiated
    oracle.render_aux_backward(p, pr, view, st, dimg, daux)
    feat = np.random.default_rng(1).standard_normal((n, 8)).astype(np.float32)
    F, _ = oracle.render_features(pr, view, st, feat)
    oracle.render_features_backward(pr, view, st, feat, None, np.ones_like(F))
    oracle.densify_stats(p, pr, view, st, dimg)
    idx = np.arange(min(n, 5), dtype=np.int32)
    eps = np.random.default_rng(2).standard_normal((idx.size, 2, 4))
    oracle.split_sample(p, idx, eps, 1.6)
    gw, gh = (w + 15) // 16, (h + 15) // 16
    vis = pr["status"] == 0
    if vis.any():
        oracle.sort_instances(pr["rect"][vis], pr["depth_f32"][vis], gw, gh)
print("sanitized oracle ok")
"""


def _runtime(name):
    out = subprocess.run(["gcc", "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return out if os.path.isabs(out) and os.path.exists(out) else None


def test_oracle_is_clean_under_address_and_undefined_behaviour_sanitizers():
    asan = _runtime("libasan.so")
    if asan is None:
        pytest.skip("gcc's libasan is not available")
    from oracle import build
    build.build_oracle_sanitized()
    env = dict(os.environ, FGS4D_ORACLE_SANITIZED="1", LD_PRELOAD=asan, OMP_NUM_THREADS="2",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0 and "sanitized oracle ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
