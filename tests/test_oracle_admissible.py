"""Pins of the oracle's admissible-result layer (orc_preprocess_relaxed,
orc_render_pixels_admissible) and of the sampled-pixel renderer.

An FP32 renderer takes the discrete decisions of Eq. 6 (the 1/255 skip, the
1e-4 stop, the depth order, tile membership, the culls) from values within a
known error of the FP64 ones.  The admissible layer returns every result such
a renderer may produce.  The pins: with zero tolerances it is the plain
oracle, bit for bit; with tolerances the plain result is always among its
results; and on hand-built records whose decisions sit on a threshold it
returns exactly the closed-form results of both outcomes, and nothing else.
CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2412_20720_gb300 import synthetic as sy

BG = (0.1, 0.2, 0.3)
TIGHT = oracle.Tolerance()  # zero tolerances: the plain decisions only


def _settings(tile=16, bg=(0.0, 0.0, 0.0), L=1, NT=1):
    return oracle.Settings(sh_degree=L, t_order=NT, tile=tile, bg=bg)


# ----------------------------------------------------- sampled-pixel renderer

@pytest.mark.parametrize("w,h,tile,bg", [(128, 96, 16, (0.0, 0.0, 0.0)), (131, 77, 16, BG), (37, 53, 8, BG),
                                         (20, 9, 16, (1.0, 1.0, 1.0))])
def test_render_pixels_equals_render_at_every_pixel(w, h, tile, bg):
    """orc_render_pixels gathers each pixel's list by its own scan over all
    Gaussians; it must equal the tile-list render bit for bit at every pixel
    (ragged tiles, both tile edges, a background)."""
    sc = sy.make_scene(2000, 5, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    view = sy.tiny_view(w, h, t=0.45)
    st = _settings(tile, bg)
    pr = oracle.preprocess(sc.as_dict(), view, st)
    img, T, nc, mg = oracle.render(pr, view, st)
    pix = np.arange(w * h)
    rgb, T2, nc2, mg2 = oracle.render_pixels(pr, view, st, pix)
    assert (nc > 0).mean() > 0.3
    np.testing.assert_array_equal(rgb.T, img.reshape(3, -1))
    np.testing.assert_array_equal(T2, T.reshape(-1))
    np.testing.assert_array_equal(nc2, nc.reshape(-1))
    np.testing.assert_array_equal(mg2, mg.reshape(-1))


# ------------------------------------------------ the plain render, exactly

@pytest.mark.parametrize("w,h,tile,bg", [(128, 96, 16, BG), (37, 53, 8, (0.0, 0.0, 0.0))])
def test_zero_tolerance_walk_is_the_plain_render(w, h, tile, bg):
    sc = sy.make_scene(2000, 6, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    view = sy.tiny_view(w, h, t=0.5)
    st = _settings(tile, bg)
    pr = oracle.preprocess(sc.as_dict(), view, st)
    img, T, nc, mg, sig = oracle.render(pr, view, st, signature=True)
    cands, flags = oracle.render_pixels_admissible(pr, view, st, np.arange(w * h), TIGHT)
    assert all(c.shape[0] == 1 for c in cands)
    assert not flags.any()
    got = np.stack([c[0] for c in cands])
    np.testing.assert_array_equal(got[:, :3].T, img.reshape(3, -1))
    np.testing.assert_array_equal(got[:, 3], T.reshape(-1))
    np.testing.assert_array_equal(got[:, 4], (sig & 0xFFFF).reshape(-1))


def test_relaxed_preprocess_keeps_the_fp64_decisions():
    """The relaxation only marks decisions: status, rect and every FP64 value
    of the visible Gaussians equal the plain chain's; rect_lo <= rect <=
    rect_hi; a Gaussian culled within the relaxation has its values."""
    sc = sy.make_scene(20000, 7, (-1, -1, -1), (1, 1, 1), sh_degree=2, t_order=1)
    view = sy.tiny_view(200, 150, t=0.5)
    st = _settings(L=2)
    plain = oracle.preprocess(sc.as_dict(), view, st)
    rel = oracle.preprocess(sc.as_dict(), view, st, relax=3e-3)
    np.testing.assert_array_equal(rel["status"], plain["status"])
    np.testing.assert_array_equal(rel["rect"], plain["rect"])
    vis = plain["status"] == 0
    for k in ("uv", "conic", "a_eff", "rgb", "depth_f32", "cov2d", "mu3"):
        np.testing.assert_array_equal(rel[k][vis], plain[k][vis])
    # (a visible Gaussian whose presence is uncertain has an empty rect_lo)
    cert = vis & ((rel["uncertain"] & 1) == 0)
    assert cert.sum() < vis.sum()
    assert not rel["rect_lo"][vis & ~cert].any()
    lo, hi, r = rel["rect_lo"][cert], rel["rect_hi"][cert], plain["rect"][cert]
    assert np.all(hi[:, :2] <= r[:, :2]) and np.all(r[:, :2] <= lo[:, :2])
    assert np.all(lo[:, 2:] <= r[:, 2:]) and np.all(r[:, 2:] <= hi[:, 2:])
    assert np.all(np.abs(hi - lo) <= 1)
    assert (np.any(lo != hi, axis=1)).sum() > 10  # some rects have uncertain edges at 3e-3
    unc = rel["uncertain"] & 1
    culled_unc = (rel["status"] != 0) & (unc > 0)
    assert culled_unc.sum() > 0
    assert np.all(np.isfinite(rel["conic"][culled_unc])) and np.all(rel["conic"][culled_unc, 0] > 0)
    # plain mode marks nothing and its bounds are the rect itself
    assert not plain["uncertain"].any()
    np.testing.assert_array_equal(plain["rect_lo"], plain["rect"])
    np.testing.assert_array_equal(plain["rect_hi"], plain["rect"])


@pytest.mark.parametrize("seed,tile", [(8, 16), (9, 8)])
def test_plain_result_is_always_admissible(seed, tile):
    sc = sy.make_scene(3000, seed, (-1, -1, -1), (1, 1, 1), sh_degree=1, t_order=1)
    view = sy.tiny_view(96, 80, t=0.5)
    st = _settings(tile, BG)
    pr = oracle.preprocess(sc.as_dict(), view, st, relax=1e-3)
    img, T, nc, mg = oracle.render(oracle.preprocess(sc.as_dict(), view, st), view, st)
    tol = oracle.Tolerance(eps_conic=1e-3, eps_uv=1e-5, eps_a=1e-4, eps_alpha=1e-5, depth_ulps=4)
    cands, flags = oracle.render_pixels_admissible(pr, view, st, np.arange(96 * 80), tol)
    plain = np.concatenate([img.reshape(3, -1), T.reshape(1, -1)]).T
    for q, c in enumerate(cands):
        assert np.any(np.all(c[:, :4] == plain[q], axis=1)), q
    assert (flags & 1).sum() > 50  # wide tolerances: many pixels branch
    assert not (flags & 4).any()


# ------------------------------------------------------ hand-built records

def _proj(entries, width=32, height=32, tile=16):
    """Projection records of hand-placed Gaussians: each entry gives uv,
    isotropic sigma (pixels), effective opacity a, rgb and depth; optional
    'uncertain' bits and a 'status'.  Every record covers the whole grid."""
    n = len(entries)
    gw, gh = (width + tile - 1) // tile, (height + tile - 1) // tile
    pr = {name: np.zeros((n, w) if w > 1 else (n,), dtype=dt) for name, dt, w in oracle._PROJ_FIELDS}
    for i, e in enumerate(entries):
        s2 = e.get("sigma", 2.0) ** 2
        pr["uv"][i] = e["uv"]
        pr["conic"][i] = (1.0 / s2, 0.0, 1.0 / s2)
        pr["a_eff"][i] = e["a"]
        pr["rgb"][i] = e["rgb"]
        pr["depth"][i] = e["depth"]
        pr["depth_f32"][i] = np.float32(e["depth"])
        pr["status"][i] = e.get("status", 0)
        pr["uncertain"][i] = e.get("uncertain", 0)
        full = (0, 0, gw, gh)
        pr["rect"][i] = full if pr["status"][i] == 0 else (0, 0, 0, 0)
        pr["rect_hi"][i] = full
        pr["rect_lo"][i] = full if pr["status"][i] == 0 and not (pr["uncertain"][i] & 1) else (0, 0, 0, 0)
    return pr


def _view(w=32, h=32):
    return sy.tiny_view(w, h)


def _composite(layers, bg):
    """Eq. 6 over (alpha, rgb) layers in order, with the stop rule."""
    T, C = 1.0, np.zeros(3)
    for a, c in layers:
        if a < 1 / 255:
            continue
        if T * (1 - a) < 1e-4:
            break
        C += np.asarray(c) * a * T
        T *= 1 - a
    return np.r_[C + T * np.asarray(bg), T]


def _as_set(cands):
    return sorted(tuple(np.round(c[:4], 12)) for c in cands)


def test_skip_decision_on_the_threshold_has_both_outcomes():
    """One Gaussian whose alpha at the pixel is (1 + 1e-7) / 255: within a
    relative error of 1e-6 it may be skipped or composited."""
    st = _settings(bg=BG)
    px, py = 10, 12
    a, sigma, dx = 0.5, 2.0, 3.0
    G = math.exp(-0.5 * dx * dx / sigma ** 2)
    a = (1 + 1e-7) / 255 / G
    rgb = (0.9, 0.4, 0.1)
    pr = _proj([{"uv": (px + 0.5 + dx, py + 0.5), "sigma": sigma, "a": a, "rgb": rgb, "depth": 2.0}])
    alpha = a * G
    pix = np.array([py * 32 + px])
    take = _composite([(alpha, rgb)], BG)
    skip = np.r_[BG, 1.0]
    c0, f0 = oracle.render_pixels_admissible(pr, _view(), st, pix, TIGHT)
    np.testing.assert_allclose(c0[0][:, :4], [take], atol=1e-15)
    assert f0[0] == 0
    c1, f1 = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(eps_alpha=1e-6))
    np.testing.assert_allclose(sorted(map(tuple, c1[0][:, :4])), sorted([tuple(take), tuple(skip)]), atol=1e-15)
    assert f1[0] & 1
    # far from the threshold (1e-3 relative) the same tolerance decides
    pr["a_eff"][0] = (1 + 1e-3) / 255 / G
    c2, f2 = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(eps_alpha=1e-6))
    assert c2[0].shape[0] == 1 and f2[0] == 0


def test_conic_and_centre_errors_widen_the_skip_window():
    """The alpha error bound grows with the exponent (conic error) and with
    the exponent's slope (centre error): a pixel 1e-4 relative above the
    threshold is decided without them and uncertain with them."""
    st = _settings()
    px, py, sigma, dx = 5, 5, 1.5, 4.0
    G = math.exp(-0.5 * dx * dx / sigma ** 2)
    a = (1 + 1e-4) / 255 / G
    pr = _proj([{"uv": (px + 0.5 + dx, py + 0.5), "sigma": sigma, "a": a, "rgb": (1, 1, 1), "depth": 3.0}])
    pix = np.array([py * 32 + px])
    for tol, n in ((oracle.Tolerance(eps_alpha=1e-6), 1), (oracle.Tolerance(eps_conic=1e-4), 2),
                   (oracle.Tolerance(eps_uv=1e-5), 2)):
        c, f = oracle.render_pixels_admissible(pr, _view(), st, pix, tol)
        assert c[0].shape[0] == n, tol


def test_stop_decision_on_the_threshold_has_both_outcomes():
    """Four layers at the pixel centre with (1 - alpha)^4 = 1e-4 (1 + 1e-9):
    the fourth may be composited or the walk may stop before it; the fifth
    stops in both."""
    st = _settings(bg=BG)
    px, py = 20, 7
    alpha = 1 - (1e-4 * (1 + 1e-9)) ** 0.25
    cols = [(0.1 * k + 0.1, 0.5, 0.9 - 0.1 * k) for k in range(5)]
    pr = _proj([{"uv": (px + 0.5, py + 0.5), "a": alpha, "rgb": cols[k], "depth": 1.0 + k} for k in range(5)])
    pix = np.array([py * 32 + px])
    four = _composite([(alpha, c) for c in cols], BG)
    T3 = (1 - alpha) ** 3
    three = np.r_[sum(np.asarray(cols[k]) * alpha * (1 - alpha) ** k for k in range(3)) + T3 * np.asarray(BG), T3]
    c0, _ = oracle.render_pixels_admissible(pr, _view(), st, pix, TIGHT)
    np.testing.assert_allclose(c0[0][:, :4], [four], atol=1e-14)
    c1, f1 = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(eps_alpha=1e-8))
    got = sorted(map(tuple, c1[0][:, :4]))
    np.testing.assert_allclose(got, sorted([tuple(three), tuple(four)]), atol=1e-14)
    np.testing.assert_array_equal(sorted(c1[0][:, 4]), [3, 4])
    assert f1[0] & 1


def test_depth_order_within_the_key_error_has_both_orders():
    """Three layers whose FP32 keys are 0, 1 and 3 ulp apart; keys may be off
    by one ulp each (depth_ulps = 1), so pairs within 2 ulp may swap: the
    admissible orders are (0 1 3), (1 0 3) and (0 3 1), and no other."""
    st = _settings()
    px, py = 3, 28
    d0 = np.float32(2.5)
    ds = [d0, np.nextafter(d0, np.float32(9)), d0]
    ds[2] = np.nextafter(np.nextafter(ds[1], np.float32(9)), np.float32(9))
    ds = [float(d) for d in ds]
    assert [np.float32(d).view(np.uint32) - np.float32(d0).view(np.uint32) for d in ds] == [0, 1, 3]
    al = [0.5, 0.3, 0.6]
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    pr = _proj([{"uv": (px + 0.5, py + 0.5), "a": al[k], "rgb": cols[k], "depth": ds[k]} for k in range(3)])
    pix = np.array([py * 32 + px])
    c0, _ = oracle.render_pixels_admissible(pr, _view(), st, pix, TIGHT)
    assert c0[0].shape[0] == 1
    c1, f1 = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(depth_ulps=1))
    expect = [_composite([(al[k], cols[k]) for k in order], (0, 0, 0)) for order in ((0, 1, 2), (1, 0, 2), (0, 2, 1))]
    assert _as_set(c1[0]) == _as_set(np.array(expect))
    assert f1[0] & 1


def test_uncertain_membership_has_both_outcomes():
    """A Gaussian marked uncertain (a cull or rect edge within its error) may
    be in the pixel's list or not; when its FP64 decision culls it, the plain
    result is the one without it."""
    st = _settings(bg=BG)
    px, py = 16, 16
    base = {"uv": (px + 0.5, py + 0.5), "a": 0.4, "rgb": (0.2, 0.9, 0.5), "depth": 3.0}
    other = {"uv": (px + 0.5, py + 0.5), "a": 0.7, "rgb": (0.8, 0.1, 0.1), "depth": 2.0, "uncertain": 1, "status": 2}
    pr = _proj([base, other])
    pix = np.array([py * 32 + px])
    without = _composite([(0.4, base["rgb"])], BG)
    with_ = _composite([(0.7, other["rgb"]), (0.4, base["rgb"])], BG)
    c0, _ = oracle.render_pixels_admissible(pr, _view(), st, pix, TIGHT)
    assert _as_set(c0[0]) == _as_set(np.array([without, with_]))
    pr["uncertain"][1] = 0  # certainly culled: only the plain result
    c1, _ = oracle.render_pixels_admissible(pr, _view(), st, pix, TIGHT)
    assert _as_set(c1[0]) == _as_set(np.array([without]))


def test_derivative_flags_near_the_clamp():
    st = _settings()
    pix = np.array([5 * 32 + 5])
    pr = _proj([{"uv": (5.5, 5.5), "a": 0.99 * (1 + 1e-8), "rgb": (1, 1, 1), "depth": 2.0}])
    _, f = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(eps_alpha=1e-6))
    assert f[0] & 2
    pr["a_eff"][0] = 0.9
    _, f = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(eps_alpha=1e-6))
    assert f[0] == 0
    pr["uncertain"][0] = 2  # colour clamp within its error
    _, f = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(eps_alpha=1e-6))
    assert f[0] & 2


def test_walk_budget_is_flagged():
    st = _settings()
    pix = np.array([8 * 32 + 8])
    # 14 uncertain layers: 2^14 leaves
    pr = _proj([{"uv": (8.5, 8.5), "a": 0.05, "rgb": (1, 0, 0), "depth": 1.0 + k, "uncertain": 1} for k in range(14)])
    c, f = oracle.render_pixels_admissible(pr, _view(), st, pix, oracle.Tolerance(max_leaves=1000), max_cands=4096)
    assert f[0] & 4


# --------------------------------------------- relaxed per-Gaussian decisions

def _on_axis(view, z, sigma, t_mean=0.5, t_scale=0.3, logit=0.0):
    """One isotropic Gaussian on the optical axis at camera depth z (the
    tiny view's camera sits at world (0, 0, -3) looking along +z); SH rows
    for degree 1 x temporal order 1 (the default settings here)."""
    return {"mean": np.array([[0.0, 0.0, z - 3.0, t_mean]]),
            "log_scale": np.array([[math.log(sigma)] * 3 + [math.log(t_scale)]]),
            "q_l": np.array([[1.0, 0, 0, 0]]), "q_r": np.array([[1.0, 0, 0, 0]]),
            "opacity_logit": np.array([logit]), "sh": np.zeros((1, 8, 3))}


def test_temporal_cull_on_the_threshold_is_uncertain():
    """p(t) = 0.05 (1 -/+ 1e-9): culled / kept in FP64, uncertain when relaxed,
    with the values of a kept Gaussian either way."""
    view = _view(64, 48)
    st = _settings()
    for sgn in (-1, 1):
        dt = math.sqrt(-2 * math.log(0.05 * (1 + sgn * 1e-9))) * 0.3
        g = _on_axis(view, 4.0, 0.1, t_mean=float(view["t"]) - dt)
        plain = oracle.preprocess(g, view, st)
        rel = oracle.preprocess(g, view, st, relax=1e-6)
        assert plain["status"][0] == (2 if sgn < 0 else 0)
        assert rel["status"][0] == plain["status"][0]
        assert rel["uncertain"][0] & 1
        assert rel["conic"][0, 0] > 0 and rel["rect_hi"][0, 2] > rel["rect_hi"][0, 0]
        far = oracle.preprocess(_on_axis(view, 4.0, 0.1, t_mean=float(view["t"]) - 1.2 * dt), view, st, relax=1e-6)
        assert far["status"][0] == 2 and not far["uncertain"][0]


def test_rect_edge_on_a_tile_boundary_is_uncertain():
    """Principal point shifted so that u + r falls exactly on a tile
    boundary: the rect's right edge may end one tile earlier."""
    view = dict(_view(64, 48))
    st = _settings()
    g = _on_axis(view, 4.0, 0.05)
    pr = oracle.preprocess(g, view, st)
    u, r = pr["uv"][0, 0], pr["radius"][0]
    view["cx"] = float(view["cx"]) + (32.0 - (u + r))
    pr = oracle.preprocess(g, view, st)
    assert pr["uv"][0, 0] + pr["radius"][0] == 32.0
    assert pr["rect"][0, 2] == 3  # floor(32 / 16) + 1
    rel = oracle.preprocess(g, view, st, relax=1e-9)
    assert rel["rect_hi"][0, 2] == 3 and rel["rect_lo"][0, 2] == 2
    assert rel["rect_lo"][0, 0] == rel["rect_hi"][0, 0] == pr["rect"][0, 0]
