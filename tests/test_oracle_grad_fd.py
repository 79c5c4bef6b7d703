"""Pins of the oracle's hand-derived adjoint to FP64 central differences of
the oracle's own forward (which is pinned to closed forms separately).

A parameter whose +-h perturbation changes any discrete outcome (cull status,
tile rect, colour clamp, the per-pixel contributor count or clamped-alpha
count) is excluded: the derivative is taken as locally constant there, and the
exclusion is detected, not guessed.
"""
import math

import numpy as np

import oracle
from paper_2412_20720_gb300 import synthetic as sy

PARAM_KEYS = ("mean", "log_scale", "q_l", "q_r", "opacity_logit", "sh")


def _scene(n, seed, L=3, NT=2, box=0.6):
    sc = sy.make_scene(n, seed, (-box, -box, -box), (box, box, box), spatial_log_scale=(math.log(0.03), math.log(0.12)),
                       sh_degree=L, t_order=NT)
    return {k: v.astype(np.float64) for k, v in sc.as_dict().items()}


def _elements(rng, params, visible, sh_per_gauss=6):
    """(key, index tuple) of the parameters to perturb: every non-SH element of
    the visible Gaussians and a sample of their SH coefficients."""
    out = []
    for i in np.flatnonzero(visible):
        for k in ("mean", "log_scale", "q_l", "q_r"):
            out += [(k, (i, j)) for j in range(4)]
        out.append(("opacity_logit", (i,)))
        K = params["sh"].shape[1]
        for _ in range(sh_per_gauss):
            out.append(("sh", (i, int(rng.integers(K)), int(rng.integers(3)))))
    return out


EPS = np.finfo(np.float64).eps


def _fd(params, key, idx, fn, h_rel=1e-5):
    """Central difference and its rounding-noise bound 64 eps |L| / h."""
    x0 = params[key][idx]
    h = h_rel * max(1.0, abs(x0))
    p = {k: v.copy() for k, v in params.items()}
    p[key][idx] = x0 + h
    fp, sp = fn(p)
    p[key][idx] = x0 - h
    fm, sm = fn(p)
    return (fp - fm) / (2 * h), 64 * EPS * max(abs(fp), abs(fm)) / h, sp, sm


def _check(pairs, rtol, atol_frac):
    """|adjoint - FD| <= rtol |adjoint| + FD noise + atol_frac max|adjoint|."""
    adj = np.array([a for a, _, _ in pairs])
    fd = np.array([f for _, f, _ in pairs])
    noise = np.array([z for _, _, z in pairs])
    scale = np.abs(adj).max()
    bad = np.abs(adj - fd) > rtol * np.abs(adj) + noise + atol_frac * scale
    assert not bad.any(), (adj[bad][:5], fd[bad][:5], int(bad.sum()))


def test_preprocess_adjoint_matches_fd():
    rng = np.random.default_rng(31)
    view = sy.tiny_view(64, 64, t=0.5)
    st = oracle.Settings(sh_degree=3, t_order=2)
    params = _scene(40, 31)
    base = oracle.preprocess(params, view, st)
    vis = base["status"] == 0
    assert vis.sum() >= 8
    n = vis.shape[0]
    gu = rng.standard_normal((n, 2))
    gc = rng.standard_normal((n, 3)) * 100.0
    ga = rng.standard_normal(n)
    gr = rng.standard_normal((n, 3))

    def fn(p):
        pr = oracle.preprocess(p, view, st)
        m = vis
        loss = ((gu * pr["uv"])[m].sum() + (gc * pr["conic"])[m].sum() + (ga * pr["a_eff"])[m].sum()
                + (gr * pr["rgb"])[m].sum())
        return loss, (pr["status"].tobytes(), (pr["rgb"] > 0).tobytes())

    adj = oracle.preprocess_backward(params, view, st, gu * vis[:, None], gc * vis[:, None], ga * vis,
                                     gr * vis[:, None])
    sig0 = fn(params)[1]
    pairs = {}
    for key, idx in _elements(rng, params, vis):
        d, z, sp, sm = _fd(params, key, idx, fn)
        if sp != sig0 or sm != sig0:
            continue
        pairs.setdefault(key, []).append((adj[key][idx], d, z))
    for key in PARAM_KEYS:
        assert len(pairs.get(key, [])) >= 8, key
        _check(pairs[key], 1e-6, 1e-9)


def test_composite_adjoint_matches_fd():
    """dL/d(u, v, conic, a, rgb) of the compositing step alone, by perturbing
    the projected quantities directly."""
    rng = np.random.default_rng(32)
    view = sy.tiny_view(40, 32, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=1, bg=(0.2, 0.5, 0.1))
    params = _scene(60, 32, L=1, NT=1)
    base = oracle.preprocess(params, view, st)
    vis = np.flatnonzero(base["status"] == 0)
    assert vis.size >= 10
    dimg = rng.standard_normal((3, 32, 40))
    g = oracle.render_backward(params, base, view, st, dimg)

    def fn(pr):
        img, T, nc, mg, sig = oracle.render(pr, view, st, signature=True)
        return float((dimg * img).sum()), (nc.tobytes(), sig.tobytes())

    sig0 = fn(base)[1]
    fields = (("uv", "g_uv", 2), ("conic", "g_conic", 3), ("a_eff", "g_a", 1), ("rgb", "g_rgb", 3))
    for name, gname, w in fields:
        pairs = []
        for i in vis:
            for j in range(w):
                idx = (i, j) if w > 1 else (i,)
                d, z, sp, sm = _fd(base, name, idx, fn)
                if sp != sig0 or sm != sig0:
                    continue
                pairs.append((g[gname][idx], d, z))
        assert len(pairs) >= 10, name
        _check(pairs, 1e-6, 1e-9)


def test_full_adjoint_matches_fd_64_gaussians_32x32():
    """The whole chain on a 64-Gaussian 32x32 subset at spatial degree 3 and
    temporal order 2, as the training workload's finite-difference check."""
    rng = np.random.default_rng(33)
    view = sy.tiny_view(32, 32, t=0.45)
    st = oracle.Settings(sh_degree=3, t_order=2)
    params = _scene(64, 33, box=0.5)
    base = oracle.preprocess(params, view, st)
    vis = base["status"] == 0
    assert vis.sum() >= 16
    dimg = rng.standard_normal((3, 32, 32))
    g = oracle.render_backward(params, base, view, st, dimg)

    def fn(p):
        pr = oracle.preprocess(p, view, st)
        img, T, nc, mg, sig = oracle.render(pr, view, st, signature=True)
        return float((dimg * img).sum()), (pr["status"].tobytes(), pr["rect"].tobytes(), (pr["rgb"] > 0).tobytes(),
                                           nc.tobytes(), sig.tobytes())

    sig0 = fn(params)[1]
    pairs = {}
    skipped = 0
    for key, idx in _elements(rng, params, vis, sh_per_gauss=3):
        d, z, sp, sm = _fd(params, key, idx, fn)
        if sp != sig0 or sm != sig0:
            skipped += 1
            continue
        pairs.setdefault(key, []).append((g[key][idx], d, z))
    total = sum(len(v) for v in pairs.values())
    assert skipped <= 0.1 * (total + skipped)
    for key in PARAM_KEYS:
        assert len(pairs.get(key, [])) >= 10, key
        _check(pairs[key], 1e-6, 1e-9)


def test_depth_and_opacity_adjoint_matches_fd():
    """Loss on the image, the depth channel and the opacity channel (the
    inputs of the LiDAR and sky terms, Sec. 5): whole-chain adjoint against
    central differences of render_aux."""
    rng = np.random.default_rng(34)
    view = sy.tiny_view(32, 32, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=1, bg=(0.3, 0.1, 0.6))
    params = _scene(48, 34, L=1, NT=1, box=0.5)
    base = oracle.preprocess(params, view, st)
    vis = base["status"] == 0
    assert vis.sum() >= 12
    dimg = rng.standard_normal((3, 32, 32))
    daux = np.zeros((4, 32, 32))
    daux[:2] = rng.standard_normal((2, 32, 32))
    g = oracle.render_aux_backward(params, base, view, st, dimg, daux)
    assert np.abs(g["g_z"]).max() > 0

    def fn(p):
        pr = oracle.preprocess(p, view, st)
        aux = oracle.aux_records(p, pr, view, st, 0.05)
        img, T, out, mg = oracle.render_aux(pr, aux, view, st)
        _, _, nc, _, sig = oracle.render(pr, view, st, signature=True)
        return float((dimg * img).sum() + (daux * out).sum()), (pr["status"].tobytes(), pr["rect"].tobytes(),
                                                              (pr["rgb"] > 0).tobytes(), nc.tobytes(), sig.tobytes())

    sig0 = fn(params)[1]
    pairs = {}
    skipped = 0
    for key, idx in _elements(rng, params, vis, sh_per_gauss=2):
        d, z, sp, sm = _fd(params, key, idx, fn)
        if sp != sig0 or sm != sig0:
            skipped += 1
            continue
        pairs.setdefault(key, []).append((g[key][idx], d, z))
    total = sum(len(v) for v in pairs.values())
    assert skipped <= 0.1 * (total + skipped)
    for key in PARAM_KEYS:
        assert len(pairs.get(key, [])) >= 10, key
        _check(pairs[key], 1e-6, 1e-9)
