"""Writes tests/golden/tiny_2000_128x96.txt: the FP64 oracle's render of the
tiny configuration (2,000 seeded 4D Gaussians in [-1,1]^3 x [0,1], spatial SH
degree 1 x temporal order 1, one 128x96 pinhole view 3 units from the origin
at t = 0.5, black background, 16-pixel tiles).

The values come from ``oracle/`` alone; the seeded scene and camera come
from the input generators.  Stored per sampled pixel: colour, final
transmittance, the pixel's distance to the nearest alpha-skip or stop
threshold, and every other result an FP32 renderer may produce there (the
oracle's admissible results under the record tolerances of the parity
tests: where a decision sits within FP32 error of its threshold, either
outcome is correct).

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2412_20720_gb300 import synthetic as sy  # noqa: E402
from paper_2412_20720_gb300.render import RenderConfig  # noqa: E402

from helpers import RELAX, oracle_settings, pixel_tolerance  # noqa: E402

FIXTURE = os.path.join(HERE, "tiny_2000_128x96.txt")
N_SAMPLES = 384
SAMPLE_SEED = 2412


def tiny_scene_inputs():
    """(params, view, cfg) of the tiny configuration, every Gaussian."""
    params = sy.tiny_scene().as_dict()
    view = sy.tiny_view(128, 96, t=0.5)
    cfg = RenderConfig(sh_degree=1, t_order=1, bg=(0.0, 0.0, 0.0), inst_capacity=1 << 18, tile=16)
    return params, view, cfg


def tiny_inputs():
    """(params, view, cfg) of the fixture: the whole tiny scene."""
    return tiny_scene_inputs()


def sample_pixels(width: int, height: int) -> np.ndarray:
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(width * height, size=N_SAMPLES, replace=False))


def oracle_render(params, view, cfg):
    st = oracle_settings(cfg)
    img, T, _, margin = oracle.render(oracle.preprocess(params, view, st), view, st)
    return img, T, margin


def alternatives(params, view, cfg, pix, plain):
    """Per pixel, the admissible results other than the plain one: a list
    of [k, 4] arrays (r, g, b, T)."""
    st = oracle_settings(cfg)
    pr = oracle.preprocess(params, view, st, relax=RELAX)
    cands, flags = oracle.render_pixels_admissible(pr, view, st, pix, pixel_tolerance(pr))
    assert not (flags & 4).any()
    out = []
    for q, c in enumerate(cands):
        keep = ~np.all(c[:, :4] == plain[q], axis=1)
        assert (~keep).sum() == 1  # the plain result is admissible, once
        out.append(c[keep, :4])
    return out


def write(path: str = FIXTURE) -> None:
    params, view, cfg = tiny_inputs()
    img, T, margin = oracle_render(params, view, cfg)
    W, H = view["width"], view["height"]
    pix = sample_pixels(W, H)
    plain = np.concatenate([img.reshape(3, -1)[:, pix], T.reshape(1, -1)[:, pix]]).T
    alts = alternatives(params, view, cfg, pix, plain)
    lines = [
        "# FP64 oracle render of the tiny configuration: 2,000 seeded 4D Gaussians in [-1,1]^3 x [0,1],",
        "# SH degree 1 x temporal order 1, 128x96 pinhole view 3 units from the origin, t = 0.5, black",
        "# background, 16-pixel tiles.  Written by tests/golden/make_golden.py from the oracle alone.",
        "# kept %d" % params["mean"].shape[0],
        "# sum_rgb %.17g %.17g %.17g" % tuple(img.reshape(3, -1).sum(axis=1)),
        "# sum_T %.17g" % T.sum(),
        "# columns: py px r g b T margin k, then k admissible alternatives (r g b T each)",
    ]
    for q, p in enumerate(pix):
        y, x = divmod(int(p), W)
        alt = " ".join("%.17g" % v for v in alts[q].reshape(-1))
        lines.append(("%d %d %.17g %.17g %.17g %.17g %.17g %d " % (y, x, img[0, y, x], img[1, y, x], img[2, y, x],
                                                                  T[y, x], margin[y, x], alts[q].shape[0]) + alt)
                     .rstrip())
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def read(path: str = FIXTURE) -> dict:
    """The fixture as arrays: py, px, rgb [P,3], T, margin, and the header's
    kept count and image sums."""
    out = {}
    rows = []
    for line in open(path):
        if line.startswith("# kept"):
            out["kept"] = int(line.split()[2])
        elif line.startswith("# sum_rgb"):
            out["sum_rgb"] = np.array([float(x) for x in line.split()[2:5]])
        elif line.startswith("# sum_T"):
            out["sum_T"] = float(line.split()[2])
        elif line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    a = np.array([r[:8] for r in rows])
    out.update(py=a[:, 0].astype(np.int64), px=a[:, 1].astype(np.int64), rgb=a[:, 2:5], T=a[:, 5], margin=a[:, 6])
    out["alternatives"] = [np.array(r[8:]).reshape(int(r[7]), 4) for r in rows]
    return out


if __name__ == "__main__":
    write()
    print(FIXTURE)
