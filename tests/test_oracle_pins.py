"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics
(closed forms, invariants, library routines, brute force), chosen so that a
dropped term, wrong sign, wrong index or transposed operand in the oracle
fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
from paper_2412_20720_gb300 import synthetic as sy


# ------------------------------------------------------------ independent math

def hamilton(p, q):
    """Quaternion product p q, components (real, i, j, k)."""
    a1, b1, c1, d1 = p
    a2, b2, c2, d2 = q
    return np.array([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2,
                     a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                     a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2,
                     a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2])


def sandwich_matrix(ql, qr):
    """Matrix of x -> q_l x q_r on quaternions with coordinates (x, y, z, t)
    = (real, i, j, k): the left/right isoclinic decomposition of a 4D
    rotation (Sec. 3.2)."""
    ql = np.asarray(ql, float) / np.linalg.norm(ql)
    qr = np.asarray(qr, float) / np.linalg.norm(qr)
    return np.stack([hamilton(hamilton(ql, e), qr) for e in np.eye(4)], axis=1)


def cov4(ql, qr, scales):
    R = sandwich_matrix(ql, qr)
    return R @ np.diag(np.asarray(scales, float) ** 2) @ R.T


def one_gaussian(mean, log_scale, ql, qr, logit, sh):
    return {"mean": np.array([mean], float), "log_scale": np.array([log_scale], float),
            "q_l": np.array([ql], float), "q_r": np.array([qr], float),
            "opacity_logit": np.array([logit], float), "sh": np.array([sh], float)}


def stack(gs):
    return {k: np.concatenate([g[k] for g in gs], axis=0) for k in gs[0]}


Y00 = 0.5 / math.sqrt(math.pi)


# --------------------------------------------------------------- rotation pins

def test_rotation_is_quaternion_sandwich():
    """R = L(q_l) R(q_r) equals the map x -> q_l x q_r (Sec. 3.2); this checks
    every entry and sign of both printed matrices against quaternion algebra."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        ql, qr = rng.standard_normal(4), rng.standard_normal(4)
        np.testing.assert_allclose(oracle.rotation(ql, qr), sandwich_matrix(ql, qr), atol=1e-14)


def test_rotation_orthonormal_det_plus_one():
    rng = np.random.default_rng(12)
    for _ in range(50):
        R = oracle.rotation(rng.standard_normal(4), rng.standard_normal(4))
        np.testing.assert_allclose(R @ R.T, np.eye(4), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13


def test_rotation_identity_and_plane_rotation():
    np.testing.assert_allclose(oracle.rotation([1, 0, 0, 0], [1, 0, 0, 0]), np.eye(4), atol=0)
    # q_l = q_r = (cos a, sin a, 0, 0): rotation by 2a in the x-y plane, fixing z and t.
    a = 0.37
    q = [math.cos(a), math.sin(a), 0.0, 0.0]
    c, s = math.cos(2 * a), math.sin(2 * a)
    expect = np.array([[c, -s, 0, 0], [s, c, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]])
    np.testing.assert_allclose(oracle.rotation(q, q), expect, atol=1e-15)


def test_rotation_fixing_time_axis():
    """q_r = (a, b, c, -d) for q_l = (a, b, c, d) leaves the t axis fixed, so
    the covariance is block diagonal (the No-4DRot case, Sec. 8.1.3)."""
    rng = np.random.default_rng(13)
    for _ in range(20):
        q = rng.standard_normal(4)
        R = oracle.rotation(q, q * np.array([1, 1, 1, -1]))
        np.testing.assert_allclose(R[:, 3], [0, 0, 0, 1], atol=1e-15)
        np.testing.assert_allclose(R[3, :], [0, 0, 0, 1], atol=1e-15)


# ------------------------------------------------- conditional / marginal pins

def _visible_params(rng, scale_lo=0.06, scale_hi=0.12):
    mean = [rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.5 + rng.uniform(-0.05, 0.05)]
    ls = list(np.log(rng.uniform(scale_lo, scale_hi, 4)))
    return one_gaussian(mean, ls, rng.standard_normal(4), rng.standard_normal(4), 0.3, np.zeros((4, 3)))


def test_slice_and_marginal_match_quadrature():
    """Conditional mean/covariance at t and the marginal p(t) (Sec. 3.2)
    against brute-force numerical marginalisation of the unnormalized 4D
    Gaussian over a 128^3 grid at fixed t: mass-weighted mean and covariance
    equal mu_xyz|t and Sigma_xyz|t, and the mass equals
    (2 pi)^(3/2) sqrt(det Sigma_xyz|t) p(t), which also checks the
    determinant identity of the factorisation proof (Sec. 3.2)."""
    rng = np.random.default_rng(14)
    view = sy.tiny_view(64, 64, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=0)
    for _ in range(4):
        g = _visible_params(rng)
        pr = oracle.preprocess(g, view, st)
        assert pr["status"][0] in (0, 3, 4, 5)  # passed the temporal filter
        S4 = cov4(g["q_l"][0], g["q_r"][0], np.exp(g["log_scale"][0]))
        P4 = np.linalg.inv(S4)
        mu = g["mean"][0]
        half = 6.0 * math.sqrt(S4[:3, :3].diagonal().max())
        ax = np.linspace(-half, half, 128)
        h = ax[1] - ax[0]
        X, Yg, Z = np.meshgrid(ax + mu[0], ax + mu[1], ax + mu[2], indexing="ij")
        D = np.stack([X - mu[0], Yg - mu[1], Z - mu[2], np.full_like(X, 0.5 - mu[3])], axis=-1)
        f = np.exp(-0.5 * np.einsum("...i,ij,...j->...", D, P4, D))
        mass = f.sum() * h ** 3
        pts = np.stack([X, Yg, Z], axis=-1)
        mean_q = (f[..., None] * pts).sum(axis=(0, 1, 2)) * h ** 3 / mass
        dq = (pts - mean_q).reshape(-1, 3)
        cov_q = (dq.T * f.reshape(-1)) @ dq * h ** 3 / mass
        np.testing.assert_allclose(pr["mu3"][0], mean_q, rtol=0, atol=1e-6 * half)
        np.testing.assert_allclose(pr["cov3"][0].reshape(3, 3), cov_q, rtol=1e-6, atol=1e-9 * half ** 2)
        expect_mass = (2 * math.pi) ** 1.5 * math.sqrt(np.linalg.det(pr["cov3"][0].reshape(3, 3))) * pr["p_t"][0]
        assert abs(mass - expect_mass) <= 1e-6 * expect_mass


def test_determinant_factorisation():
    """det Sigma = Sigma_44 det Sigma_xyz|t (Sec. 3.2, factorisation proof)."""
    rng = np.random.default_rng(15)
    view = sy.tiny_view(64, 64, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=0)
    for _ in range(20):
        g = _visible_params(rng, 0.02, 0.3)
        pr = oracle.preprocess(g, view, st)
        if pr["status"][0] == 2:
            continue
        S4 = cov4(g["q_l"][0], g["q_r"][0], np.exp(g["log_scale"][0]))
        lhs = np.linalg.det(S4)
        rhs = S4[3, 3] * np.linalg.det(pr["cov3"][0].reshape(3, 3))
        assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
        # p(t) is the unnormalized 1D Gaussian with variance Sigma_44.
        assert abs(pr["p_t"][0] - math.exp(-0.5 * (0.5 - g["mean"][0][3]) ** 2 / S4[3, 3])) < 1e-14


def test_block_diagonal_case_is_static_3d_times_1d():
    """With Sigma_xt = 0 the slice leaves the spatial Gaussian unchanged and
    p(t) is exp(-(t - mu_t)^2 / (2 s_t^2)) (Sec. 3.2, the independent
    space/time design)."""
    rng = np.random.default_rng(16)
    view = sy.tiny_view(64, 64, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=0)
    for _ in range(10):
        q = rng.standard_normal(4)
        g = _visible_params(rng)
        g["q_l"][0] = q
        g["q_r"][0] = q * np.array([1, 1, 1, -1])
        pr = oracle.preprocess(g, view, st)
        s = np.exp(g["log_scale"][0])
        R3 = sandwich_matrix(g["q_l"][0], g["q_r"][0])[:3, :3]
        np.testing.assert_allclose(pr["mu3"][0], g["mean"][0][:3], atol=1e-15)
        np.testing.assert_allclose(pr["cov3"][0].reshape(3, 3), R3 @ np.diag(s[:3] ** 2) @ R3.T, atol=1e-15)
        assert abs(pr["p_t"][0] - math.exp(-0.5 * (0.5 - g["mean"][0][3]) ** 2 / s[3] ** 2)) < 1e-14


# ---------------------------------------------------------------- EWA pins

def test_isotropic_footprint_integral():
    """One isotropic Gaussian on the optical axis (Sec. 3.1, Eqs. 3-4): its
    2D covariance is (f sigma / z)^2 I exactly, and the image sums to the
    integral of a G over the disc where a G >= 1/255, i.e.
    a 2 pi sigma_px^2 (1 - 1/(255 a)), for opacity a = 0.25, colour 1."""
    W = H = 256
    view = sy.look_at((0, 0, -3), (0, 0, 0), (0, -1, 0), W, H, 0.5)
    f = float(view["fx"])
    sigma_px = 20.0
    sigma = sigma_px * 3.0 / f
    g = one_gaussian([0, 0, 0, 0.5], [math.log(sigma)] * 3 + [math.log(0.3)], [1, 0, 0, 0], [1, 0, 0, 0],
                     math.log(0.25 / 0.75), np.full((1, 3), 0.5 / Y00))
    st = oracle.Settings(sh_degree=0, t_order=0, dilation=0.0)
    pr = oracle.preprocess(g, view, st)
    assert pr["status"][0] == 0
    np.testing.assert_allclose(pr["cov2d"][0], [sigma_px ** 2, 0.0, sigma_px ** 2], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(pr["uv"][0], [W / 2, H / 2], atol=1e-12)
    np.testing.assert_allclose(pr["rgb"][0], [1, 1, 1], atol=1e-14)
    # Isotropic: the eigenvalue gap is 0, so the floor 0.1 under the root applies.
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(sigma_px ** 2 + math.sqrt(0.1)))
    img, T, nc, mg = oracle.render(pr, view, st)
    a = 0.25
    expect = a * 2 * math.pi * sigma_px ** 2 * (1 - 1 / (255 * a))
    for ch in range(3):
        assert abs(img[ch].sum() - expect) < 1e-3 * expect


# ------------------------------------------------------------- 4DSH pins

def real_sh_scipy(L, d):
    th = math.acos(d[2])
    ph = math.atan2(d[1], d[0])
    out = []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            if m > 0:
                out.append(math.sqrt(2) * sps.sph_harm_y(l, m, th, ph).real)
            elif m < 0:
                out.append(math.sqrt(2) * sps.sph_harm_y(l, -m, th, ph).imag)
            else:
                out.append(sps.sph_harm_y(l, 0, th, ph).real)
    return np.array(out)


def test_real_sh_matches_library():
    """Real orthonormal SH from scipy's complex SH (Condon-Shortley phase)."""
    rng = np.random.default_rng(17)
    for _ in range(30):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        np.testing.assert_allclose(oracle.real_sh(3, d), real_sh_scipy(3, d), atol=1e-13)


def test_real_sh_orthonormal():
    """Gauss-Legendre x uniform-azimuth quadrature of Y_lm Y_l'm' over the sphere."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    nph = 32
    G = np.zeros((16, 16))
    for x, w in zip(xg, wg):
        for k in range(nph):
            ph = 2 * math.pi * k / nph
            s = math.sqrt(1 - x * x)
            Y = oracle.real_sh(3, [s * math.cos(ph), s * math.sin(ph), x])
            G += w * (2 * math.pi / nph) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def _colour_scene(rng, n, L, NT, static=True, big_t=False):
    gs = []
    K = (L + 1) ** 2 * (NT + 1)
    for _ in range(n):
        q = rng.standard_normal(4)
        qr = q * np.array([1, 1, 1, -1]) if static else rng.standard_normal(4)
        ls = list(np.log(rng.uniform(0.03, 0.06, 3))) + [math.log(2.0 if big_t else 0.3)]
        gs.append(one_gaussian(list(rng.uniform(-0.5, 0.5, 3)) + [0.5], ls, q, qr, 0.0, rng.normal(0, 0.2, (K, 3))))
    return stack(gs)


def test_dc_only_colour_is_constant():
    rng = np.random.default_rng(18)
    g = _colour_scene(rng, 20, 3, 2, static=False)
    g["sh"][:, 1:, :] = 0.0
    for t in (0.45, 0.5, 0.55):
        pr = oracle.preprocess(g, sy.tiny_view(64, 64, t=t), oracle.Settings(sh_degree=3, t_order=2))
        ok = pr["status"] == 0
        assert ok.sum() > 5
        np.testing.assert_allclose(pr["rgb"][ok], np.maximum(0, Y00 * g["sh"][ok, 0, :] + 0.5), atol=1e-15)


def test_zero_temporal_order_is_time_independent():
    rng = np.random.default_rng(19)
    g = _colour_scene(rng, 20, 3, 0, static=True, big_t=True)
    st = oracle.Settings(sh_degree=3, t_order=0)
    a = oracle.preprocess(g, sy.tiny_view(64, 64, t=0.2), st)
    b = oracle.preprocess(g, sy.tiny_view(64, 64, t=0.9), st)
    ok = (a["status"] == 0) & (b["status"] == 0)
    assert ok.sum() > 5
    np.testing.assert_allclose(a["rgb"][ok], b["rgb"][ok], atol=1e-15)


def test_temporal_basis_is_periodic():
    """cos(2 pi n dt / T): colour repeats with period T in t (static slice)."""
    rng = np.random.default_rng(20)
    g = _colour_scene(rng, 20, 2, 3, static=True, big_t=True)
    st = oracle.Settings(sh_degree=2, t_order=3, period=0.5)
    a = oracle.preprocess(g, sy.tiny_view(64, 64, t=0.3), st)
    b = oracle.preprocess(g, sy.tiny_view(64, 64, t=0.8), st)
    c = oracle.preprocess(g, sy.tiny_view(64, 64, t=0.55), st)
    ok = (a["status"] == 0) & (b["status"] == 0) & (c["status"] == 0)
    assert ok.sum() > 5
    np.testing.assert_allclose(a["rgb"][ok], b["rgb"][ok], atol=1e-12)
    assert np.abs(a["rgb"][ok] - c["rgb"][ok]).max() > 1e-3  # half a period differs


# ---------------------------------------------------------- compositing pins

def _centred_layers(view, pixel, depths, opacities, colours):
    """Isotropic small Gaussians whose centres project exactly onto ``pixel``'s
    centre, at the given camera depths, with p(t) = 1."""
    fx, cx, cy = float(view["fx"]), float(view["cx"]), float(view["cy"])
    gs = []
    for z, a, c in zip(depths, opacities, colours):
        zc = z  # camera at (0,0,-3) looking +z: z_cam = z_world + 3
        x = (pixel[0] + 0.5 - cx) * zc / fx
        y = (pixel[1] + 0.5 - cy) * zc / fx
        sh = (np.asarray(c, float) - 0.5) / Y00
        gs.append(one_gaussian([x, y, zc - 3.0, 0.5], [math.log(0.02)] * 3 + [math.log(0.3)], [1, 0, 0, 0],
                               [1, 0, 0, 0], math.log(a / (1 - a)), sh[None, :]))
    return stack(gs)


def test_two_gaussian_closed_form():
    """Eq. 6 for two layers at the pixel centre: C = a1 c1 + (1 - a1) a2 c2."""
    view = sy.tiny_view(64, 48)
    st = oracle.Settings(sh_degree=0, t_order=0)
    c1, c2 = [0.9, 0.2, 0.4], [0.1, 0.7, 0.3]
    g = _centred_layers(view, (20, 30), [3.5, 4.5], [0.6, 0.7], [c1, c2])
    pr = oracle.preprocess(g, view, st)
    assert (pr["status"] == 0).all()
    img, T, nc, mg = oracle.render(pr, view, st)
    expect = 0.6 * np.array(c1) + 0.4 * 0.7 * np.array(c2)
    np.testing.assert_allclose(img[:, 30, 20], expect, atol=1e-12)
    assert abs(T[30, 20] - 0.4 * 0.3) < 1e-12
    # Order follows depth, not input order.
    g2 = _centred_layers(view, (20, 30), [4.5, 3.5], [0.7, 0.6], [c2, c1])
    img2, _, _, _ = oracle.render(oracle.preprocess(g2, view, st), view, st)
    np.testing.assert_allclose(img2[:, 30, 20], expect, atol=1e-12)


def test_permutation_invariance():
    sc = sy.tiny_scene()
    view = sy.tiny_view()
    st = oracle.Settings(sh_degree=1, t_order=1)
    img, T, _, _ = oracle.render(oracle.preprocess(sc.as_dict(), view, st), view, st)
    perm = np.random.default_rng(21).permutation(sc.n)
    sp = sc.subset(perm)
    img2, T2, _, _ = oracle.render(oracle.preprocess(sp.as_dict(), view, st), view, st)
    np.testing.assert_allclose(img2, img, atol=1e-14)
    np.testing.assert_allclose(T2, T, atol=1e-14)


def test_saturation_stops_before_transmittance_cutoff():
    """Eight alpha=0.8 layers: T after k layers is 0.2^k; the 6th would take T
    below 1e-4, so exactly five are composited."""
    view = sy.tiny_view(64, 48)
    st = oracle.Settings(sh_degree=0, t_order=0)
    cols = [[0.1 * k, 0.5, 1.0 - 0.1 * k] for k in range(8)]
    g = _centred_layers(view, (10, 12), [3.2 + 0.3 * k for k in range(8)], [0.8] * 8, cols)
    pr = oracle.preprocess(g, view, st)
    img, T, nc, mg = oracle.render(pr, view, st)
    expect = sum(np.array(cols[k]) * 0.8 * 0.2 ** k for k in range(5))
    np.testing.assert_allclose(img[:, 12, 10], expect, atol=1e-12)
    assert abs(T[12, 10] - 0.2 ** 5) < 1e-15
    assert nc[12, 10] == 5


def test_block_diagonal_render_equals_static_3dgs():
    """No-4DRot reduction (Sec. 3.2 / Sec. 8.1.3): with Sigma_xt = 0 the 4D
    render equals a static 3D Gaussian render whose opacity is scaled by the
    1D temporal Gaussian.  The static renderer below is written independently
    in plain Python (every Gaussian for every pixel; opacities are kept under
    0.35 so that anything outside the tile rect is below the 1/255 skip)."""
    rng = np.random.default_rng(22)
    W, H = 24, 20
    view = sy.look_at((0.3, -0.2, -3.0), (0, 0, 0), (0, -1, 0), W, H, 0.5, hfov_deg=20.0)
    n = 6
    gs = []
    for _ in range(n):
        q = rng.standard_normal(4)
        ls = list(np.log(rng.uniform(0.02, 0.06, 3))) + [math.log(rng.uniform(0.1, 0.3))]
        op = rng.uniform(0.1, 0.3)
        sh = rng.normal(0, 0.3, (4, 3))
        gs.append(one_gaussian(list(rng.uniform(-0.15, 0.15, 3)) + [rng.uniform(0.4, 0.6)], ls, q,
                               q * np.array([1, 1, 1, -1]), math.log(op / (1 - op)), sh))
    g = stack(gs)
    st = oracle.Settings(sh_degree=1, t_order=0, dilation=0.3)
    pr = oracle.preprocess(g, view, st)
    img, T, _, _ = oracle.render(pr, view, st)

    Wm = np.asarray(view["viewmat"], float)[:, :3]
    Tv = np.asarray(view["viewmat"], float)[:, 3]
    fx, fy, cx, cy = (float(view[k]) for k in ("fx", "fy", "cx", "cy"))
    items = []
    for i in range(n):
        s = np.exp(g["log_scale"][i])
        R3 = sandwich_matrix(g["q_l"][i], g["q_r"][i])[:3, :3]
        S3 = R3 @ np.diag(s[:3] ** 2) @ R3.T
        p = Wm @ g["mean"][i][:3] + Tv
        J = np.array([[fx / p[2], 0, -fx * p[0] / p[2] ** 2], [0, fy / p[2], -fy * p[1] / p[2] ** 2]])
        S2 = J @ Wm @ S3 @ Wm.T @ J.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S2)
        uv = np.array([fx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy])
        d = g["mean"][i][:3] - np.asarray(view["campos"], float)
        d /= np.linalg.norm(d)
        Y = real_sh_scipy(1, d)
        col = np.maximum(0.0, Y @ g["sh"][i] + 0.5)
        a = 1 / (1 + math.exp(-g["opacity_logit"][i])) * math.exp(-0.5 * (0.5 - g["mean"][i][3]) ** 2 / s[3] ** 2)
        items.append((float(np.float32(p[2])), i, uv, Q, a, col))
    items.sort(key=lambda e: (e[0], e[1]))
    ref = np.zeros((3, H, W))
    for py in range(H):
        for px in range(W):
            Tt, Cc = 1.0, np.zeros(3)
            for _, _, uv, Q, a, col in items:
                dd = uv - np.array([px + 0.5, py + 0.5])
                power = -0.5 * dd @ Q @ dd
                al = min(0.99, a * math.exp(power))
                if al < 1 / 255:
                    continue
                if Tt * (1 - al) < 1e-4:
                    break
                Cc += col * al * Tt
                Tt *= 1 - al
            ref[:, py, px] = Cc
    assert img.max() > 0.05
    np.testing.assert_allclose(img, ref, atol=1e-12)


# ------------------------------------------------------------ sort pins

def test_sort_instances_against_lexsort():
    rng = np.random.default_rng(23)
    gw, gh, n = 9, 7, 500
    x0 = rng.integers(0, gw, n)
    y0 = rng.integers(0, gh, n)
    rect = np.stack([x0, y0, np.minimum(gw, x0 + rng.integers(0, 4, n)), np.minimum(gh, y0 + rng.integers(0, 4, n))],
                    axis=1).astype(np.int32)
    depth = rng.uniform(0.5, 10, n).astype(np.float32)
    depth[::7] = depth[0]  # many exact ties, broken by index
    keys, vals, ranges = oracle.sort_instances(rect, depth, gw, gh)
    tiles, idxs = [], []
    for i in range(n):
        for ty in range(rect[i, 1], rect[i, 3]):
            for tx in range(rect[i, 0], rect[i, 2]):
                tiles.append(ty * gw + tx)
                idxs.append(i)
    tiles, idxs = np.array(tiles), np.array(idxs)
    order = np.lexsort((idxs, depth[idxs], tiles))
    assert keys.shape[0] == tiles.shape[0]
    np.testing.assert_array_equal(vals, idxs[order])
    np.testing.assert_array_equal(keys >> np.uint64(32), tiles[order].astype(np.uint64))
    np.testing.assert_array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), depth[idxs[order]].view(np.uint32))
    counts = np.bincount(tiles, minlength=gw * gh)
    np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], counts)
    nz = counts > 0
    np.testing.assert_array_equal(ranges[nz, 0], np.concatenate([[0], np.cumsum(counts)[:-1]])[nz])


# ------------------------------------------------ auxiliary channel pins

def test_flow_vanishes_without_space_time_coupling():
    """Sigma_xt = 0 (q_r = (a, b, c, -d) for q_l = (a, b, c, d)): the sliced
    mean does not move, so every Gaussian's flow and the rendered flow are
    exactly zero while depth and opacity are not."""
    rng = np.random.default_rng(31)
    g = _colour_scene(rng, 30, 1, 1, static=True, big_t=True)
    view = sy.tiny_view(64, 48, t=0.52)
    st = oracle.Settings(sh_degree=1, t_order=1)
    pr = oracle.preprocess(g, view, st)
    ok = pr["status"] == 0
    assert ok.sum() > 10
    aux = oracle.aux_records(g, pr, view, st, flow_dt=0.05)
    assert np.all(aux[:, 1:] == 0.0)
    np.testing.assert_allclose(aux[ok, 0], pr["depth"][ok], rtol=0, atol=0)
    img, T, out, mg = oracle.render_aux(pr, aux, view, st)
    assert np.all(out[2:] == 0.0)
    assert out[0].max() > 1.0 and out[1].max() > 0.2


def test_flow_is_projected_displacement_of_sliced_mean():
    """Flow of each Gaussian = pi(mu_xyz|t+dt) - pi(mu_xyz|t), with both sliced
    means taken from the oracle's own conditional (pinned by quadrature) at the
    two timestamps, projected by Eq. 3 in this test."""
    rng = np.random.default_rng(32)
    g = _colour_scene(rng, 30, 1, 1, static=False, big_t=True)
    dt = 0.04
    v0 = sy.tiny_view(64, 48, t=0.5)
    v1 = sy.tiny_view(64, 48, t=0.5 + dt)
    st = oracle.Settings(sh_degree=1, t_order=1, p_t_min=0.0)
    p0 = oracle.preprocess(g, v0, st)
    p1 = oracle.preprocess(g, v1, st)
    ok = (p0["status"] == 0) & (p1["pc"][:, 2] > 0.2)
    assert ok.sum() > 10
    aux = oracle.aux_records(g, p0, v0, st, flow_dt=float(v1["t"]) - float(v0["t"]))  # the views' stored t
    fx, fy, cx, cy = (float(v0[k]) for k in ("fx", "fy", "cx", "cy"))
    u1 = fx * p1["pc"][:, 0] / p1["pc"][:, 2] + cx
    w1 = fy * p1["pc"][:, 1] / p1["pc"][:, 2] + cy
    np.testing.assert_allclose(aux[ok, 1], (u1 - p0["uv"][:, 0])[ok], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(aux[ok, 2], (w1 - p0["uv"][:, 1])[ok], rtol=1e-9, atol=1e-9)
    assert np.abs(aux[ok, 1:]).max() > 0.05  # the coupled scene does move


def test_aux_channels_two_layer_closed_form():
    """Depth and opacity blend with the colour weights of Eq. 6:
    D = a1 z1 + (1 - a1) a2 z2 and O = 1 - (1 - a1)(1 - a2) at the pixel where
    both centres project."""
    view = sy.tiny_view(64, 48)
    st = oracle.Settings(sh_degree=0, t_order=0)
    g = _centred_layers(view, (20, 30), [3.5, 4.5], [0.6, 0.7], [[0.5] * 3, [0.5] * 3])
    pr = oracle.preprocess(g, view, st)
    aux = oracle.aux_records(g, pr, view, st, flow_dt=0.1)
    img, T, out, mg = oracle.render_aux(pr, aux, view, st)
    assert abs(out[0, 30, 20] - (0.6 * 3.5 + 0.4 * 0.7 * 4.5)) < 1e-12
    assert abs(out[1, 30, 20] - (1.0 - 0.4 * 0.3)) < 1e-12
    assert out[2, 30, 20] == 0.0 and out[3, 30, 20] == 0.0


def test_opacity_channel_matches_constant_colour_image():
    """With one colour c for every Gaussian and a black background the image
    is c O, so the opacity channel agrees with the colour compositing."""
    rng = np.random.default_rng(33)
    g = _colour_scene(rng, 40, 0, 0, static=False)
    g["sh"][:] = (0.8 - 0.5) / Y00
    view = sy.tiny_view(64, 48, t=0.5)
    st = oracle.Settings(sh_degree=0, t_order=0, bg=(0.0, 0.0, 0.0))
    pr = oracle.preprocess(g, view, st)
    aux = oracle.aux_records(g, pr, view, st, flow_dt=0.05)
    img, T, out, mg = oracle.render_aux(pr, aux, view, st)
    assert out[1].max() > 0.3
    for ch in range(3):
        np.testing.assert_allclose(img[ch], 0.8 * out[1], atol=1e-12)
    img0, T0, _, _ = oracle.render(pr, view, st)
    np.testing.assert_allclose(img, img0, atol=0)
    np.testing.assert_allclose(out[1], 1.0 - T0, atol=0)


# ---------------------------------------------------- densification pins

def _split_parents(rng, n=6, K=None):
    gs = []
    for _ in range(n):
        gs.append(one_gaussian(list(rng.uniform(-1, 1, 3)) + [rng.uniform(0, 1)],
                               list(np.log(rng.uniform(0.05, 0.5, 4))), rng.standard_normal(4),
                               rng.standard_normal(4), rng.standard_normal(), rng.normal(0, 0.2, (4, 3))))
    return stack(gs)


def test_split_sample_unit_draws_are_scaled_principal_axes():
    """eps = e_k gives mu + s_k R[:, k] with R the quaternion sandwich written
    in this test (Sec. 3.2); colour, rotation and opacity are copied and the
    log-scales reduced by log(shrink)."""
    rng = np.random.default_rng(41)
    g = _split_parents(rng)
    m = g["mean"].shape[0]
    idx = np.arange(m)[::-1].copy()
    eps = np.tile(np.eye(4)[None], (m, 1, 1))
    out = oracle.split_sample(g, idx, eps, 1.6)
    for j, i in enumerate(idx):
        R = sandwich_matrix(g["q_l"][i], g["q_r"][i])
        s = np.exp(g["log_scale"][i])
        for k in range(4):
            np.testing.assert_allclose(out["mean"][4 * j + k], g["mean"][i] + s[k] * R[:, k], atol=1e-14)
            np.testing.assert_allclose(out["log_scale"][4 * j + k], g["log_scale"][i] - math.log(1.6), atol=1e-15)
            np.testing.assert_array_equal(out["sh"][4 * j + k], g["sh"][i])
            np.testing.assert_array_equal(out["q_l"][4 * j + k], g["q_l"][i])
            assert out["opacity_logit"][4 * j + k] == g["opacity_logit"][i]


def test_split_samples_follow_the_full_4d_gaussian():
    """Many draws of one parent: sample mean and covariance match mu and
    Sigma = R S S^T R^T (statistical tolerance), including the space-time
    block Sigma_xt, so children also spread in time."""
    rng = np.random.default_rng(42)
    g = _split_parents(rng, n=1)
    N = 200_000
    eps = rng.standard_normal((1, N, 4))
    out = oracle.split_sample(g, np.array([0]), eps, 1.0)
    S = cov4(g["q_l"][0], g["q_r"][0], np.exp(g["log_scale"][0]))
    x = out["mean"]
    np.testing.assert_allclose(x.mean(axis=0), g["mean"][0], atol=5 * math.sqrt(S.diagonal().max() / N))
    C = np.cov(x.T)
    tol = 6 * np.sqrt((S.diagonal()[:, None] * S.diagonal()[None, :] + S ** 2) / N)
    assert np.all(np.abs(C - S) <= tol)
    assert np.abs(S[:3, 3]).max() > 10 * tol[:3, 3].max()  # the coupling is actually exercised


def test_densify_stats_are_gradient_magnitudes_of_the_view():
    """Per visible Gaussian: |dL/d(u, v)| and |dL/dmu_t| of the view's loss
    (the adjoint is pinned by central differences), count 1; zeros for culled
    Gaussians.  |dL/dmu_t| checked here by a central difference of the loss."""
    rng = np.random.default_rng(43)
    sc = sy.make_scene(60, 43, (-0.6, -0.6, -0.6), (0.6, 0.6, 0.6), sh_degree=1, t_order=1)
    params = {k: v.astype(np.float64) for k, v in sc.as_dict().items()}
    view = sy.tiny_view(32, 32, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=1)
    pr = oracle.preprocess(params, view, st)
    dimg = rng.standard_normal((3, 32, 32))
    d = oracle.densify_stats(params, pr, view, st, dimg)
    vis = pr["status"] == 0
    assert vis.sum() > 10 and np.all(d[~vis] == 0) and np.all(d[vis, 2] == 1)

    def loss(p):
        img, _, _, _ = oracle.render(oracle.preprocess(p, view, st), view, st)
        return float((dimg * img).sum())

    checked = 0
    for i in np.flatnonzero(vis)[:8]:
        h = 1e-6
        p = {k: v.copy() for k, v in params.items()}
        p["mean"][i, 3] += h
        lp = loss(p)
        p["mean"][i, 3] -= 2 * h
        lm = loss(p)
        fd = (lp - lm) / (2 * h)
        if abs(abs(fd) - d[i, 1]) <= 1e-5 * max(1.0, abs(fd)):
            checked += 1
    assert checked >= 6


# ------------------------------------------------------ compact mask pins

def _mask_scene(seed):
    sc = sy.make_scene(80, seed, (-0.6, -0.6, -0.6), (0.6, 0.6, 0.6), sh_degree=1, t_order=1)
    p = {k: v.astype(np.float64) for k, v in sc.as_dict().items()}
    p["mask_logit"] = np.random.default_rng(seed).normal(0.0, 1.5, p["mean"].shape[0])
    p["mask_threshold"] = 0.4
    return p


def test_mask_keeps_or_removes_whole_gaussians():
    """M_hat = 1{sigmoid(m) > eps} in value (Sec. 4.3): the masked render
    equals the plain render of the Gaussians with sigmoid(m) > eps, exactly."""
    p = _mask_scene(51)
    view = sy.tiny_view(48, 40, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=1)
    keep = 1.0 / (1.0 + np.exp(-p["mask_logit"])) > 0.4
    assert 10 < keep.sum() < keep.size - 10
    pr = oracle.preprocess(p, view, st)
    assert np.all(pr["status"][~keep] == 7)
    img, T, _, _ = oracle.render(pr, view, st)
    sub = {k: v[keep] for k, v in p.items() if k not in ("mask_logit", "mask_threshold")}
    img2, T2, _, _ = oracle.render(oracle.preprocess(sub, view, st), view, st)
    np.testing.assert_array_equal(img, img2)
    np.testing.assert_array_equal(T, T2)


def test_mask_gradient_is_straight_through_scaling_derivative():
    """dL/dm = M (1 - M) dL/dlambda at lambda = 1, where lambda scales all four
    scales and the opacity of that Gaussian (S_hat = lambda S, alpha_hat =
    lambda alpha): the straight-through estimator of Sec. 4.3, checked by a
    central difference in lambda."""
    p = _mask_scene(52)
    view = sy.tiny_view(40, 32, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=1)
    pr = oracle.preprocess(p, view, st)
    rng = np.random.default_rng(53)
    dimg = rng.standard_normal((3, 32, 40))
    g = oracle.render_backward(p, pr, view, st, dimg)
    vis = np.flatnonzero(pr["status"] == 0)
    assert vis.size >= 8
    assert np.all(g["mask_logit"][pr["status"] != 0] == 0)

    def loss_sig(q):
        pq = oracle.preprocess(q, view, st)
        img, T, nc, mg, sig = oracle.render(pq, view, st, signature=True)
        return float((dimg * img).sum()), (pq["status"].tobytes(), pq["rect"].tobytes(), nc.tobytes(), sig.tobytes())

    sig0 = loss_sig(p)[1]
    checked = 0
    for i in vis:
        h = 1e-6
        vals = []
        for lam in (1 + h, 1 - h):
            q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
            q["log_scale"][i] += math.log(lam)
            a = 1.0 / (1.0 + math.exp(-q["opacity_logit"][i])) * lam
            q["opacity_logit"][i] = math.log(a / (1.0 - a))
            vals.append(loss_sig(q))
        if vals[0][1] != sig0 or vals[1][1] != sig0:
            continue
        M = 1.0 / (1.0 + math.exp(-p["mask_logit"][i]))
        fd = (vals[0][0] - vals[1][0]) / (2 * h) * M * (1 - M)
        assert abs(g["mask_logit"][i] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, g["mask_logit"][i], fd)
        checked += 1
    assert checked >= 6


# ------------------------------------------------- feature rendering pins

def _unit_colour_scene(rng, n=60):
    """DC-only colours that are unit vectors with positive entries."""
    gs, cols = [], []
    for _ in range(n):
        c = np.abs(rng.standard_normal(3)) + 0.05
        c /= np.linalg.norm(c)
        cols.append(c)
        q = rng.standard_normal(4)
        gs.append(one_gaussian(list(rng.uniform(-0.5, 0.5, 3)) + [0.5], list(np.log(rng.uniform(0.03, 0.08, 3))) +
                               [math.log(0.3)], q, rng.standard_normal(4), rng.normal(0, 1),
                               ((c - 0.5) / Y00)[None, :]))
    return stack(gs), np.array(cols)


def test_feature_render_equals_colour_render_for_unit_colours():
    """With f_i = c_i of unit norm (so f_hat = c) and a black background the
    feature map is the image: the feature path uses the colour weights of
    Eq. 6 (Sec. 7: colour replaced by the normalised feature)."""
    rng = np.random.default_rng(61)
    g, cols = _unit_colour_scene(rng)
    view = sy.tiny_view(48, 40, t=0.5)
    st = oracle.Settings(sh_degree=0, t_order=0, bg=(0.0, 0.0, 0.0))
    pr = oracle.preprocess(g, view, st)
    assert (pr["status"] == 0).sum() > 20
    np.testing.assert_allclose(pr["rgb"][pr["status"] == 0], cols[pr["status"] == 0], atol=1e-12)
    img, T, _, _ = oracle.render(pr, view, st)
    F, mg = oracle.render_features(pr, view, st, cols * 7.0)  # scale is normalised away
    np.testing.assert_allclose(F, img, atol=1e-12)
    F2, _ = oracle.render_features(pr, view, st, cols, gate=[0.5, 0.5, 0.0])  # gate zeroes channel 2
    assert np.all(F2[2] == 0.0) and F2[:2].max() > 0.3


def test_feature_backward_matches_fd():
    rng = np.random.default_rng(62)
    sc = sy.make_scene(50, 62, (-0.6, -0.6, -0.6), (0.6, 0.6, 0.6), sh_degree=1, t_order=1)
    params = {k: v.astype(np.float64) for k, v in sc.as_dict().items()}
    view = sy.tiny_view(32, 32, t=0.5)
    st = oracle.Settings(sh_degree=1, t_order=1)
    pr = oracle.preprocess(params, view, st)
    D = 5
    f = rng.standard_normal((50, D))
    gate = rng.uniform(0.2, 1.0, D)
    dF = rng.standard_normal((D, 32, 32))
    gf, gg = oracle.render_features_backward(pr, view, st, f, gate, dF)

    def loss(ff, gt):
        F, _ = oracle.render_features(pr, view, st, ff, gt)
        return float((dF * F).sum())

    h = 1e-6
    vis = np.flatnonzero(pr["status"] == 0)
    assert vis.size > 10
    for i in vis[:6]:
        for c in range(D):
            fp, fm = f.copy(), f.copy()
            fp[i, c] += h
            fm[i, c] -= h
            fd = (loss(fp, gate) - loss(fm, gate)) / (2 * h)
            assert abs(fd - gf[i, c]) <= 1e-6 * max(1.0, abs(fd)), (i, c, fd, gf[i, c])
    for c in range(D):
        gp, gm = gate.copy(), gate.copy()
        gp[c] += h
        gm[c] -= h
        fd = (loss(f, gp) - loss(f, gm)) / (2 * h)
        assert abs(fd - gg[c]) <= 1e-6 * max(1.0, abs(fd)), (c, fd, gg[c])
    assert np.all(gf[pr["status"] != 0] == 0)
