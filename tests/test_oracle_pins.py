"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails it.  Nothing here uses the
CUDA path.
"""
import math

import numpy as np
import pytest
import torch

from oracle import model as M
from paper_2605_05876_gb300 import scenes as S
from tests import _tiny

GOLDEN = {}
with open(__file__.replace("test_oracle_pins.py", "golden/paper_constants.txt")) as fh:
    for line in fh:
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            GOLDEN[k] = float(v)


def env_state(env, prm, nq=96):
    env = np.asarray(env, np.float64)
    irr, levels = M.env_prefilter(env, prm.env_levels, prm.irr_w, prm.irr_h)
    return M.EnvState(irr, levels, M.brdf_lut(prm.lut_n, nq), env.shape)


# --------------------------------------------------------------------------
# paper constants


def test_paper_constants_match_defaults():
    prm = M.Params()
    assert prm.r_cut == GOLDEN["r_cut"]
    assert prm.k_max == GOLDEN["k_max"]
    assert abs(prm.gamma - GOLDEN["gamma"]) < 1e-8
    # Eq. alpha at W = 2 pi with gamma = 2 pi (the paper prints 0.998)
    a = 1.0 - math.exp(-prm.gamma * 2 * math.pi / (2 * math.pi))
    assert round(a, 3) == GOLDEN["alpha_at_W_2pi_gamma_2pi"]


# --------------------------------------------------------------------------
# BRDF table


def test_brdf_r_to_zero_limit():
    """As r -> 0 the GGX lobe is a mirror and G -> 1, so beta1 -> 1 - Fc(mu)
    and beta2 -> Fc(mu) with Fc = (1 - mu)^5 (Schlick)."""
    mu = np.array([0.1, 0.3, 0.5, 0.7, 0.95])
    b = M.brdf_eval(mu, 1e-4 * np.ones_like(mu), nq=128)
    Fc = (1 - mu) ** 5
    np.testing.assert_allclose(b[:, 0], 1 - Fc, atol=2e-6)
    np.testing.assert_allclose(b[:, 1], Fc, atol=2e-6)


def test_brdf_energy_bound():
    lut = M.brdf_lut(32, 96)
    s = lut.sum(-1)
    assert np.all(s <= 1.0 + 1e-9) and np.all(s > 0.0)
    # rougher surfaces lose energy to shadowing-masking at grazing angles
    assert s[-1, 0] < s[0, -1]


def test_brdf_quadrature_converged():
    mu = np.array([0.02, 0.2, 0.6, 0.98, 0.5])
    r = np.array([0.05, 0.5, 0.9, 0.3, 1.0])
    a = M.brdf_eval(mu, r, nq=128)
    b = M.brdf_eval(mu, r, nq=384)
    assert np.abs(a - b).max() < 1e-7


def test_brdf_against_monte_carlo():
    """Independent estimate: integrate the Cook-Torrance specular term
    f (n.l) over l directly, uniform on the hemisphere (no half-vector
    change of variables)."""
    rng = np.random.default_rng(7)
    for mu, r in [(0.5, 0.5), (0.8, 0.35), (0.25, 0.8)]:
        n_s = 2_000_000
        z = rng.uniform(0, 1, n_s)
        phi = rng.uniform(0, 2 * math.pi, n_s)
        st = np.sqrt(1 - z * z)
        l = np.stack([st * np.cos(phi), st * np.sin(phi), z], 1)
        v = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
        h = l + v
        h /= np.linalg.norm(h, axis=1, keepdims=True)
        nh, vh, nl = h[:, 2], h @ v, l[:, 2]
        a = r * r
        D = a * a / (math.pi * (nh * nh * (a * a - 1) + 1) ** 2)
        k = a / 2
        G = (mu / (mu * (1 - k) + k)) * (nl / (nl * (1 - k) + k))
        Fc = (1 - vh) ** 5
        f = D * G / (4 * mu * nl)                  # specular BRDF without F
        est = 2 * math.pi * f * nl                 # / pdf (1 / 2pi)
        e1, e2 = est * (1 - Fc), est * Fc
        ref = M.brdf_eval([mu], [r], nq=192)[0]
        for val, e in ((ref[0], e1), (ref[1], e2)):
            se = e.std() / math.sqrt(n_s)
            assert abs(val - e.mean()) < 4 * se + 1e-4, (mu, r, val, e.mean(), se)


# --------------------------------------------------------------------------
# environment prefilter


def test_env_constant_is_fixed_point():
    env = np.full((32, 64, 3), 0.7)
    irr, levels = M.env_prefilter(env, 6, 32, 16)
    assert np.abs(irr - 0.7).max() < 1e-12
    for lv in levels:
        assert np.abs(lv - 0.7).max() < 1e-12


def test_env_adjoint_dot_product():
    rng = np.random.default_rng(3)
    We, He = 32, 16
    x = rng.normal(size=(He, We, 3))
    irr, levels = M.env_prefilter(x, 4, 16, 8)
    y_irr = rng.normal(size=irr.shape)
    y_lv = [rng.normal(size=lv.shape) for lv in levels]
    lhs = (irr * y_irr).sum() + sum((a * b).sum() for a, b in zip(levels, y_lv))
    rhs = (x * M.env_adjoint(y_irr, y_lv, We, He)).sum()
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def _dir(a, b, W, H):
    phi = 2 * math.pi * ((a + 0.5) / W - 0.5)
    th = math.pi * (b + 0.5) / H
    return np.array([math.sin(th) * math.sin(phi), math.cos(th), -math.sin(th) * math.cos(phi)])


def test_irradiance_of_cosine_lobe():
    """Env L(w) = max(0, w.a): the cosine-weighted mean over the hemisphere
    around a is (1/pi) Int cos^2 = 2/3; around -a it is exactly 0."""
    We, He = 256, 128
    Wi, Hi = 32, 16
    ta, tb = 5, 4
    a = _dir(ta, tb, Wi, Hi)
    env = np.zeros((He, We, 3))
    for b in range(He):
        for c in range(We):
            env[b, c, :] = max(0.0, float(_dir(c, b, We, He) @ a))
    irr, _ = M.env_prefilter(env, 2, Wi, Hi)
    assert abs(irr[tb, ta, 0] - 2.0 / 3.0) < 2e-3
    # antipode of texel (ta, tb) is texel (ta + Wi/2, Hi - 1 - tb)
    assert abs(irr[Hi - 1 - tb, (ta + Wi // 2) % Wi, 1]) < 1e-12


def test_specular_level_sharp_limit():
    """With many levels, level 1 has r = 1/(L-1) -> alpha = r^2 tiny and the
    GGX-weighted average collapses onto the texel itself, i.e. the level
    equals its box-averaged source."""
    rng = np.random.default_rng(5)
    env = rng.uniform(0.1, 2.0, size=(32, 64, 3))
    _, levels = M.env_prefilter(env, 1001, 8, 4)
    src = env.reshape(16, 2, 32, 2, 3).mean(axis=(1, 3))
    assert np.abs(levels[1] - src).max() < 1e-9 * np.abs(src).max()
    assert np.array_equal(levels[0], env)


def test_specular_level_explicit_half_vector():
    """One output texel of a rough level recomputed with the half vector
    formed explicitly, D(n.h) with n = v = r = w_t."""
    rng = np.random.default_rng(6)
    env = rng.uniform(0.1, 2.0, size=(16, 32, 3))
    L = 4
    _, levels = M.env_prefilter(env, L, 8, 4)
    i = 2
    W, H = 8, 4
    src = env.reshape(4, 4, 8, 4, 3).mean(axis=(1, 3))
    alpha = (i / (L - 1)) ** 2
    for (ta, tb) in [(1, 1), (6, 2)]:
        wt = _dir(ta, tb, W, H)
        num = np.zeros(3)
        den = 0.0
        for b in range(H):
            dW = 2 * math.pi / W * (math.cos(math.pi * b / H) - math.cos(math.pi * (b + 1) / H))
            for a in range(W):
                wj = _dir(a, b, W, H)
                if wt @ wj <= 0:
                    continue
                h = (wt + wj) / np.linalg.norm(wt + wj)
                nh = wt @ h
                D = alpha ** 2 / (math.pi * (nh * nh * (alpha ** 2 - 1) + 1) ** 2)
                wgt = D * (wt @ wj) * dW
                num += wgt * src[b, a]
                den += wgt
        np.testing.assert_allclose(levels[i][tb, ta], num / den, rtol=1e-12)


# --------------------------------------------------------------------------
# single surfels, footprints, partition of unity


def _render(surf, cam, env, prm, **kw):
    return M.render_view(surf, cam, env, prm, **kw)


def test_single_surfel_normalises_to_itself():
    """A single-surfel layer reconstructs the surfel's own value wherever
    its weight is nonzero (Sec. 3.5.3: C_hat = w c / w = c)."""
    prm = M.Params()
    surf = _tiny.surfels([[0.02, -0.01, 0.0]], normals=[[0.2, 0.1, 1.0]], scale=0.12,
                         albedo=[[0.9, 0.3, 0.6]], rough=0.4, metal=0.3)
    cam = _tiny.front_camera(res=48)
    env = env_state(_tiny.lognormal_env(np.random.default_rng(1)), prm)
    out = _render(surf, cam, env, prm)
    a = out["rgba"][:, 3]
    cov = a > 0
    assert cov.sum() > 50
    assert out["n_layers"].max() == 1
    # shaded colour: the same for every covered pixel
    col = out["rgba"][cov, :3] / a[cov, None]
    assert np.abs(col - col[0]).max() < 1e-12
    alb = out["aov"][cov, 0:3] / a[cov, None]
    np.testing.assert_allclose(alb, np.broadcast_to([0.9, 0.3, 0.6], alb.shape), rtol=1e-6)
    nrm = out["aov"][cov, 5:8] / a[cov, None]
    assert np.abs(np.linalg.norm(nrm, axis=1) - 1).max() < 1e-12


@pytest.mark.parametrize("sigma_f", [0.0, 0.5, 2.0])
def test_footprint_integral(sigma_f):
    """A fronto-parallel surfel of scale s at depth z maps its unit-variance
    kernel to a screen Gaussian of std f s / z; summed over pixels the
    weights give 2 pi (f s / z)^2, independent of sigma_f because n_f
    preserves the kernel integral (Eq. mip_eval)."""
    prm = M.Params(sigma_f=sigma_f, r_cut=6.0)
    cam = _tiny.front_camera(dist=3.0, res=64)
    f = cam.fx
    s = 2.5 * 3.0 / f     # 2.5 px std
    surf = _tiny.surfels([[0.0, 0.0, 0.0]], scale=s)
    env = env_state(_tiny.const_env(), prm)
    out = _render(surf, cam, env, prm)
    w = -np.log1p(-out["rgba"][:, 3])            # alpha = 1 - exp(-W) (gamma = 2 pi)
    s_px = float(np.float32(s)) * f / 3.0
    expect = 2 * math.pi * s_px ** 2
    assert abs(w.sum() / expect - 1) < 1e-6


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_partition_of_unity(h):
    """A regular grid of unit-variance kernels with spacing h (in kernel
    units) sums to 2 pi / h^2 away from its border (Poisson summation), so
    a densely sampled plane has layer opacity 1 - exp(-2 pi / h^2)
    (0.998 at h = 1, Sec. 3.5.1)."""
    prm = M.Params(r_cut=6.0)
    cam = _tiny.front_camera(dist=3.0, res=33)
    s = 1.5 * 3.0 / cam.fx
    surf = _tiny.grid_plane(int(40 / h), h * s, scale=s)
    env = env_state(_tiny.const_env(), prm)
    out = _render(surf, cam, env, prm, pix=[16 * 33 + 16])
    assert out["n_layers"][0] == 1
    expect = 1 - math.exp(-2 * math.pi / h ** 2)
    assert abs(out["rgba"][0, 3] - expect) < 1e-7
    if h == 1.0:
        assert round(out["rgba"][0, 3], 3) == GOLDEN["alpha_at_W_2pi_gamma_2pi"]


def _tilt(surf, angle):
    """Rotate every surfel's frame about the x axis (tilts the normal)."""
    c, s = math.cos(angle / 2), math.sin(angle / 2)
    q = surf.quat.astype(np.float64)
    rx = np.array([c, s, 0.0, 0.0])
    w1, x1, y1, z1 = rx
    w2, x2, y2, z2 = q.T
    prod = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    return S.Surfels(surf.pos, prod.astype(np.float32), surf.log_scale, surf.albedo, surf.roughness,
                     surf.metallic)


def test_two_separated_planes_make_two_layers():
    """Two well separated planes form two layers composited front to back:
    A = a1 + (1 - a1) a2 and the albedo channel is
    a1 rho1 + (1 - a1) a2 rho2 (Eq. compositing)."""
    prm = M.Params()
    cam = _tiny.front_camera(dist=3.0, res=33)
    s = 1.2 * 3.0 / cam.fx
    p1 = _tiny.grid_plane(30, 1.3 * s, z=0.1, scale=s, albedo=(0.9, 0.2, 0.1))
    p2 = _tiny.grid_plane(30, 1.3 * s, z=-0.2, scale=s, albedo=(0.1, 0.4, 0.8), center=(0.3 * s, 0.2 * s))
    env = env_state(_tiny.const_env(), prm)
    pix = [16 * 33 + 16, 14 * 33 + 17]
    o1 = _render(p1, cam, env, prm, pix=pix)
    o2 = _render(p2, cam, env, prm, pix=pix)
    o = _render(S.Surfels.concat([p2, p1]), cam, env, prm, pix=pix)
    a1, a2 = o1["rgba"][:, 3], o2["rgba"][:, 3]
    assert np.all(o["n_layers"] == 2)
    np.testing.assert_allclose(o["rgba"][:, 3], a1 + (1 - a1) * a2, rtol=1e-12)
    expect = a1[:, None] * np.array([0.9, 0.2, 0.1]) + ((1 - a1) * a2)[:, None] * np.array([0.1, 0.4, 0.8])
    np.testing.assert_allclose(o["aov"][:, 0:3], expect, rtol=1e-6)


def test_thin_shell_merges():
    """Tilted planes closer than their depth extents merge into one layer
    (the thin-shell failure mode of Sec. 6)."""
    prm = M.Params()
    cam = _tiny.front_camera(dist=3.0, res=33)
    s = 1.2 * 3.0 / cam.fx
    p1 = _tilt(_tiny.grid_plane(30, 1.3 * s, z=0.0, scale=s), 0.6)
    p2 = _tilt(_tiny.grid_plane(30, 1.3 * s, z=0.5 * s, scale=s, center=(0.4 * s, 0.1 * s)), 0.6)
    env = env_state(_tiny.const_env(), prm)
    o = _render(S.Surfels.concat([p1, p2]), cam, env, prm, pix=[16 * 33 + 16])
    assert o["n_layers"][0] == 1


# --------------------------------------------------------------------------
# grouping and brute force


def _frag_sets(surf, cam, prm, env):
    Sd = M.to_torch_surfels(surf)
    cd = M.cam_dict(cam)
    rec = M.records(Sd, cd, torch.from_numpy(env.irr), [torch.from_numpy(l) for l in env.levels],
                    torch.from_numpy(env.lut), prm)
    rect = M.support_rect(rec, prm)
    fr = M.fragments(rec, rect, cd["width"], cd["height"], prm)
    return rec, rect, fr


def test_grouping_is_connected_components():
    """Layers of Algorithm 1 over z_start-sorted fragments are the connected
    components of the union of the covering depth intervals (Sec. 3.2.1)."""
    rng = np.random.default_rng(11)
    prm = M.Params(k_max=64)
    surf = _tiny.random_scene(rng, n=120, spread=0.4, scale=(0.02, 0.06))
    env = env_state(_tiny.const_env(), prm)
    rec, _, fr = _frag_sets(surf, _tiny.front_camera(res=48), prm, env)
    zs, ze = rec["zs"].numpy(), rec["ze"].numpy()
    n_multi = 0
    for p in np.unique(fr.pix):
        sel = fr.pix == p
        sids, layers = fr.sid[sel], fr.layer[sel]
        # union-find on interval overlap
        parent = list(range(len(sids)))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a
        for i in range(len(sids)):
            for j in range(i + 1, len(sids)):
                a, b = sids[i], sids[j]
                if zs[a] <= ze[b] and zs[b] <= ze[a]:
                    parent[find(i)] = find(j)
        roots = [find(i) for i in range(len(sids))]
        order = sorted(set(roots), key=lambda r: min(zs[sids[i]] for i in range(len(sids)) if roots[i] == r))
        comp = np.array([order.index(r) for r in roots])
        assert np.array_equal(comp, layers), p
        n_multi += layers.max() > 0
    assert n_multi > 50


def test_permutation_invariance():
    rng = np.random.default_rng(12)
    prm = M.Params()
    surf = _tiny.random_scene(rng, n=60)
    perm = rng.permutation(60)
    env = env_state(_tiny.lognormal_env(rng), prm)
    cam = _tiny.front_camera(res=24)
    a = _render(surf, cam, env, prm)
    b = _render(surf.subset(perm), cam, env, prm)
    np.testing.assert_allclose(a["rgba"], b["rgba"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(a["aov"], b["aov"], rtol=1e-12, atol=1e-14)


def _quat_rot(q):
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def brute_force(surf, cam, prm, ch, cons=False):
    """Independent tiny renderer: per pixel and surfel, intersect the pixel
    ray with the surfel plane by a 3x3 solve, build J by differentiating
    that intersection numerically at the surfel centre (or, for the
    per-pixel MIP filter, at the pixel), then group by connected components
    of depth intervals and composite."""
    sig = 0.0 if prm.mip_mode == "none" else prm.sigma_f
    R = np.asarray(cam.R, np.float32).astype(np.float64)
    t = np.asarray(cam.t, np.float32).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    W, H = cam.width, cam.height
    N = surf.n
    geo = []
    for i in range(N):
        Rs = _quat_rot(surf.quat[i].astype(np.float64))
        sc = np.exp(surf.log_scale[i].astype(np.float64))
        tu, tv = R @ (sc[0] * Rs[:, 0]), R @ (sc[1] * Rs[:, 1])
        c = R @ surf.pos[i].astype(np.float64) + t

        def hit(x, y, tu=tu, tv=tv, c=c):
            d = np.array([(x - cx) / fx, (y - cy) / fy, 1.0])
            A = np.stack([tu, tv, -d], 1)
            u, v, lam = np.linalg.solve(A, -c)
            return u, v, lam
        px, py = fx * c[0] / c[2] + cx, fy * c[1] / c[2] + cy
        e = 1e-4
        J = np.array([[(hit(px + e, py)[k] - hit(px - e, py)[k]) / (2 * e) for k in (0, 1)],
                      [(hit(px, py + e)[k] - hit(px, py - e)[k]) / (2 * e) for k in (0, 1)]]).T
        Sig = np.eye(2) + sig * J @ J.T
        eps = prm.r_cut * math.hypot(tu[2], tv[2])
        # support rectangle: sampled disc boundary U affine EWA ellipse, +1 px
        th = np.linspace(0, 2 * math.pi, 20001)
        P = c[None] + prm.r_cut * (np.cos(th)[:, None] * tu + np.sin(th)[:, None] * tv)
        bx, by = fx * P[:, 0] / P[:, 2] + cx, fy * P[:, 1] / P[:, 2] + cy
        Mj = np.linalg.inv(J)
        MMt = Mj @ Mj.T
        ex = prm.r_cut * np.sqrt(np.diag(MMt) + sig)
        rect = (min(bx.min(), px - ex[0]) - 1, max(bx.max(), px + ex[0]) + 1,
                min(by.min(), py - ex[1]) - 1, max(by.max(), py + ex[1]) + 1)
        geo.append(dict(hit=hit, Sinv=np.linalg.inv(Sig), nf=1 / math.sqrt(np.linalg.det(Sig)),
                        zs=c[2] - eps, ze=c[2] + eps, valid=(c[2] - eps) > prm.z_near, rect=rect))
    rgba = np.zeros((W * H, 4))
    aov = np.zeros((W * H, 9))
    unsure = np.zeros(W * H, bool)
    cons_out = np.zeros(W * H)
    for y in range(H):
        for x in range(W):
            X, Y = x + 0.5, y + 0.5
            frs = []
            for i, g in enumerate(geo):
                if not g["valid"]:
                    continue
                r = g["rect"]
                if not (r[0] <= X <= r[1] and r[2] <= Y <= r[3]):
                    continue
                u, v, lam = g["hit"](X, Y)
                if lam <= 0:
                    continue
                uv = np.array([u, v])
                Sinv, nf = g["Sinv"], g["nf"]
                if prm.mip_mode == "pixel":   # J at this pixel, numerically
                    e = 1e-4
                    Jp = np.array([[(g["hit"](X + e, Y)[k] - g["hit"](X - e, Y)[k]) / (2 * e) for k in (0, 1)],
                                   [(g["hit"](X, Y + e)[k] - g["hit"](X, Y - e)[k]) / (2 * e) for k in (0, 1)]]).T
                    Sg = np.eye(2) + sig * Jp @ Jp.T
                    Sinv, nf = np.linalg.inv(Sg), 1 / math.sqrt(np.linalg.det(Sg))
                rho2 = uv @ Sinv @ uv
                if abs(rho2 - prm.r_cut ** 2) < 1e-6 or min(X - r[0], r[1] - X, Y - r[2], r[3] - Y) < 1e-3:
                    unsure[y * W + x] = True
                if rho2 < prm.r_cut ** 2:
                    frs.append((g["zs"], g["ze"], i, nf * math.exp(-0.5 * rho2)))
            frs.sort(key=lambda f: (f[0], f[2]))
            # connected components of the union of intervals, front to back
            layers = []
            for f in frs:
                if layers and f[0] <= layers[-1]["zmax"]:
                    layers[-1]["zmax"] = max(layers[-1]["zmax"], f[1])
                    layers[-1]["f"].append(f)
                else:
                    layers.append(dict(zmax=f[1], f=[f]))
            Tb = 1.0
            out = np.zeros(12)
            lw, lz, lv = [], [], []
            for L in layers[:prm.k_max]:
                Wk = sum(f[3] for f in L["f"])
                C = sum(f[3] * ch[f[2]] for f in L["f"])
                Ch = C / Wk
                Ch[8:11] = C[8:11] / np.linalg.norm(C[8:11])
                al = 1 - math.exp(-prm.gamma * Wk / (2 * math.pi))
                out += Tb * al * Ch
                # centre depth of each fragment: the middle of its depth interval
                zc = [0.5 * (f[0] + f[1]) for f in L["f"]]
                zm = sum(f[3] * z for f, z in zip(L["f"], zc)) / Wk
                lw.append(Tb * al)
                lz.append(zm)
                lv.append(sum(f[3] * (z - zm) ** 2 for f, z in zip(L["f"], zc)) / Wk)
                Tb *= 1 - al
            cons_out[y * W + x] = (sum(lw[i] * lw[j] * abs(lz[i] - lz[j]) for i in range(len(lw))
                                       for j in range(i + 1, len(lw)))
                                   + sum(a * a * v for a, v in zip(lw, lv)))
            rgba[y * W + x, :3] = out[:3] + Tb * np.asarray(prm.bg)
            rgba[y * W + x, 3] = 1 - Tb
            aov[y * W + x] = out[3:]
    if cons:
        return rgba, aov, unsure, cons_out
    return rgba, aov, unsure


@pytest.mark.parametrize("seed,mip,aniso", [(21, "centre", False), (22, "centre", False), (23, "pixel", False),
                                             (24, "pixel", False), (25, "none", False), (26, "centre", True),
                                             (27, "pixel", True)])
def test_oracle_matches_brute_force(seed, mip, aniso):
    """The oracle against the independent brute-force renderer, for the
    centre-precomputed MIP filter (the method), the per-pixel Jacobian of
    the Sec. 4.4.2 ablation (J by finite differences of the 3x3 solve at
    every pixel) and no filter; `aniso`: a camera with f_y = 1.3 f_x and a
    wider than high image, so that a swap of the focal lengths or of the
    principal point's coordinates fails."""
    rng = np.random.default_rng(seed)
    prm = M.Params(sigma_f=0.5 if seed in (21, 23) else 1.5, mip_mode=mip)
    surf = _tiny.random_scene(rng, n=40, spread=0.35, scale=(0.08, 0.2))
    cam = _tiny.front_camera(res=28)
    if aniso:
        cam = _tiny.front_camera(res=24, width=34)
        cam = S.Camera(cam.R, cam.t, cam.fx, 1.3 * cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.scene)
    env = env_state(_tiny.lognormal_env(rng), prm)
    out = _render(surf, cam, env, prm)
    Sd = M.to_torch_surfels(surf)
    rec = M.records(Sd, M.cam_dict(cam), torch.from_numpy(env.irr),
                    [torch.from_numpy(l) for l in env.levels], torch.from_numpy(env.lut), prm)
    rgba, aov, unsure = brute_force(surf, cam, prm, rec["ch"].detach().numpy())
    ok = ~unsure
    assert ok.sum() > 0.95 * ok.size and (rgba[:, 3] > 0).sum() > 100
    np.testing.assert_allclose(out["rgba"][ok], rgba[ok], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(out["aov"][ok], aov[ok], rtol=1e-6, atol=1e-9)


# --------------------------------------------------------------------------
# gradients: autograd of the oracle vs central finite differences


def _decisions(surf, cam, env, prm):
    rec, rect, fr = _frag_sets(surf, cam, prm, env)
    return fr.pix.tobytes() + fr.sid.tobytes() + fr.layer.tobytes()


def _f64(surf):
    return S.Surfels(*(np.asarray(getattr(surf, k), np.float64).copy() for k in
                       ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(31)
    prm = M.Params()
    surf = _f64(_tiny.random_scene(rng, n=24, spread=0.3, scale=(0.06, 0.16)))
    cam = _tiny.front_camera(res=20)
    env_base = _tiny.lognormal_env(rng).astype(np.float64)
    env = env_state(env_base, prm)
    P = cam.width * cam.height
    G = rng.normal(size=(P, 13))
    out = M.render_view(surf, cam, env, prm, G=G)
    grads = out["grad"]
    base_dec = _decisions(surf, cam, env, prm)

    def loss(s, e):
        o = M.render_view(s, cam, e, prm)
        return float((np.concatenate([o["rgba"], o["aov"]], 1) * G).sum())

    checked = 0
    for name, h in [("pos", 1e-6), ("quat", 1e-6), ("log_scale", 1e-6), ("albedo", 1e-6),
                    ("roughness", 1e-6), ("metallic", 1e-6)]:
        arr = getattr(surf, name)
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            plus, minus = _f64(surf), _f64(surf)
            getattr(plus, name).reshape(-1)[idx] += h
            getattr(minus, name).reshape(-1)[idx] -= h
            if _decisions(plus, cam, env, prm) != base_dec or _decisions(minus, cam, env, prm) != base_dec:
                continue
            fd = (loss(plus, env) - loss(minus, env)) / (2 * h)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 2e-5 * max(1.0, abs(an)), (name, idx, fd, an)
            checked += 1
    assert checked >= 25
    # environment texels: decisions do not depend on them
    for idx in rng.choice(env_base.size, size=6, replace=False):
        ep, em = env_base.copy(), env_base.copy()
        ep.reshape(-1)[idx] += 1e-5
        em.reshape(-1)[idx] -= 1e-5
        fd = (loss(surf, env_state(ep, prm)) - loss(surf, env_state(em, prm))) / 2e-5
        an = grads["env"].reshape(-1)[idx]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (idx, fd, an)


def test_pixel_mip_equals_centre_mip_for_fronto_parallel_surfels():
    """A fronto-parallel surfel maps affinely to the screen (its intersection
    Jacobian is the same at every pixel), so the per-pixel MIP filter equals
    the centre-precomputed one everywhere (Sec. 3.3.2); tilted surfels make
    them differ."""
    rng = np.random.default_rng(41)
    pos = np.concatenate([rng.uniform(-0.4, 0.4, (30, 2)), rng.uniform(-0.2, 0.2, (30, 1))], 1)
    surf = _tiny.surfels(pos, scale=rng.uniform(0.02, 0.08, 30), albedo=rng.uniform(0, 1, (30, 3)))
    cam = _tiny.front_camera(res=24)
    env = env_state(_tiny.lognormal_env(rng), M.Params())
    outs = {m: _render(surf, cam, env, M.Params(sigma_f=1.5, mip_mode=m)) for m in ("centre", "pixel")}
    np.testing.assert_allclose(outs["pixel"]["rgba"], outs["centre"]["rgba"], rtol=1e-10, atol=1e-12)
    assert (outs["centre"]["rgba"][:, 3] > 0).sum() > 100
    tilted = _tilt(surf, 1.2)
    o2 = {m: _render(tilted, cam, env, M.Params(sigma_f=1.5, mip_mode=m)) for m in ("centre", "pixel")}
    assert np.abs(o2["pixel"]["rgba"] - o2["centre"]["rgba"]).max() > 1e-4


def test_no_mip_is_the_unfiltered_unit_kernel():
    """Without the MIP filter a lone fronto-parallel surfel's weight is
    exp(-rho^2 / 2) with rho the distance in its tangent frame (n_f = 1), so
    its coverage at a pixel is 1 - exp(-w) with w known in closed form."""
    s_ = 0.05
    surf = _tiny.surfels([[0.0, 0.0, 0.0]], scale=s_)
    cam = _tiny.front_camera(res=20)
    env = env_state(_tiny.const_env(1.0), M.Params())
    out = _render(surf, cam, env, M.Params(mip_mode="none"))
    f = float(np.float32(cam.fx))
    cx = float(np.float32(cam.cx))
    s32 = math.exp(float(np.float32(math.log(s_))))      # the scale as stored (float32 log-scale)
    x = (np.arange(20) + 0.5 - cx) / f * 3.0 / s32        # tangent-frame coordinates at depth 3
    U, V = np.meshgrid(x, x, indexing="xy")
    w = np.exp(-0.5 * (U ** 2 + V ** 2)).ravel()
    cov = out["rgba"][:, 3]
    inside = (U ** 2 + V ** 2).ravel() < 9.0 * (1 - 1e-6)
    np.testing.assert_allclose(cov[inside], 1 - np.exp(-w[inside]), rtol=1e-9, atol=1e-12)


# --------------------------------------------------------------------------
# compositing identities with gamma != 2 pi


def _stack_at_pixel(res=33):
    """Fronto-parallel surfels stacked on the optical axis at four depths
    (four layers at the centre pixel) plus a second surfel in the nearest
    layer, one pixel to the side.  Returns the surfels, the camera, and for
    each surfel its layer and closed-form weight at the centre pixel:
    n_f exp(-rho^2 / 2) with a = z / (f s) the tangent-frame units per pixel,
    n_f = 1 / (1 + sigma_f a^2) and rho^2 = a^2 d^2 / (1 + sigma_f a^2)
    for a centre offset of d pixels (Sec. 3.3.2, Eq. mip_cov, mip_eval)."""
    cam = _tiny.front_camera(dist=3.0, res=res)
    f = float(np.float32(cam.fx))
    zw = np.array([0.3, 0.1, -0.1, -0.3])            # world z; camera depth 3 - z
    a_want = np.array([0.7, 1.1, 0.5, 0.9])
    scale = (3.0 - zw) / (f * a_want)
    dx = (3.0 - zw[0]) / f                           # one pixel at the nearest depth
    pos = np.concatenate([np.stack([np.zeros(4), np.zeros(4), zw], 1), [[dx, 0.0, zw[0]]]])
    surf = _tiny.surfels(pos, scale=np.concatenate([scale, scale[:1]]))
    layer = np.array([0, 1, 2, 3, 0])
    return surf, cam, layer


def _closed_form_weights(surf, cam, sigma_f):
    f = float(np.float32(cam.fx))
    zc = 3.0 - surf.pos[:, 2].astype(np.float64)
    s = np.exp(surf.log_scale[:, 0].astype(np.float64))
    a = zc / (f * s)
    d = surf.pos[:, 0].astype(np.float64) * f / zc    # centre offset in pixels
    nf = 1.0 / (1.0 + sigma_f * a * a)
    return nf * np.exp(-0.5 * a * a * d * d * nf), np.exp(-0.5 * a * a * d * d * nf)


@pytest.mark.parametrize("k_max", [2, 3, 4])
def test_coverage_is_exp_of_kept_weight_sum(k_max):
    """The pixel's coverage is 1 - exp(-gamma / 2 pi * sum of W_k over the
    kept layers): the product of the per-layer 1 - alpha_k of Eq. alpha
    telescopes (Sec. 3.5.1, 3.5.2), and layers past K_max add nothing
    (Algorithm 1).  gamma is taken away from 2 pi so that a dropped or
    inverted gamma / 2 pi factor fails."""
    gamma = 3.7
    prm = M.Params(gamma=gamma, k_max=k_max)
    surf, cam, layer = _stack_at_pixel()
    env = env_state(_tiny.const_env(), prm)
    pid = 16 * 33 + 16
    out = _render(surf, cam, env, prm, pix=[pid])
    assert out["n_layers"][0] == k_max
    w, _ = _closed_form_weights(surf, cam, prm.sigma_f)
    kept = layer < k_max
    expect = 1.0 - math.exp(-gamma / (2 * math.pi) * w[kept].sum())
    assert abs(out["rgba"][0, 3] - expect) < 1e-12
    # and not the sum over every covering fragment
    if k_max < 4:
        assert abs(out["rgba"][0, 3] - (1.0 - math.exp(-gamma / (2 * math.pi) * w.sum()))) > 1e-3


@pytest.mark.parametrize("k_max", [2, 4])
def test_coverage_gradient_is_gamma_over_2pi_transmittance(k_max):
    """dA/dw_i = gamma / 2 pi * T_{K+1} for every kept fragment, whatever its
    layer (A = 1 - exp(-gamma / 2 pi * sum W)), and 0 for a fragment of a
    dropped layer.  Back-propagated through w = n_f exp(-rho^2 / 2), the
    gradient reaching each record's n_f is that times exp(-rho^2 / 2)."""
    gamma = 3.7
    prm = M.Params(gamma=gamma, k_max=k_max)
    surf, cam, layer = _stack_at_pixel()
    env = env_state(_tiny.const_env(), prm)
    pid = 16 * 33 + 16
    vs = M.prepare_view(surf, cam, env, prm, need_grad=True)
    G = np.zeros((1, 13))
    G[0, 3] = 1.0                                      # d/d(alpha channel)
    out = M.render_pixels(vs, np.array([pid], np.int32), G)
    T_end = 1.0 - out["rgba"][0, 3]
    _, gauss = _closed_form_weights(surf, cam, prm.sigma_f)
    expect = np.where(layer < k_max, gamma / (2 * math.pi) * T_end * gauss, 0.0)
    got = vs.leaf["n_f"].grad.numpy()
    np.testing.assert_allclose(got, expect, rtol=1e-10, atol=1e-15)
    assert np.all(got[layer < k_max] > 0)


def test_background_enters_through_the_residual_transmittance():
    """rgb = sum_k T_k alpha_k C_hat_k + T_{K+1} bg (Sec. 3.5.2): two
    backgrounds differ by exactly (1 - A) * (bg' - bg) at every pixel,
    covered or not, and leave the coverage and the AOVs alone (every other
    pin renders on black, where a dropped background term is invisible)."""
    rng = np.random.default_rng(5)
    surf = _tiny.random_scene(rng, n=40, spread=0.3, scale=(0.03, 0.08))
    cam = _tiny.front_camera(res=24)
    env = env_state(_tiny.lognormal_env(rng), M.Params())
    bg = np.array([0.3, 0.5, 0.7])
    o0 = _render(surf, cam, env, M.Params())
    o1 = _render(surf, cam, env, M.Params(bg=tuple(bg)))
    A = o0["rgba"][:, 3]
    assert (A == 0).sum() > 20 and ((A > 0.05) & (A < 0.95)).sum() > 20
    np.testing.assert_allclose(o1["rgba"][:, :3] - o0["rgba"][:, :3], (1 - A)[:, None] * bg, rtol=0, atol=1e-14)
    assert np.array_equal(o1["rgba"][:, 3], A) and np.array_equal(o1["aov"], o0["aov"])


def test_lone_surfel_reconstructs_its_depth_and_materials():
    """A lone fronto-parallel surfel's layer carries its own roughness,
    metallic, normal and camera-space centre depth (Sec. 3.5.3: the Shepard
    mean of one fragment is its value): the AOVs divided by the coverage
    give them back at every covered pixel."""
    z_w, rough, metal = 0.3, 0.37, 0.61
    surf = _tiny.surfels([[0.02, -0.01, z_w]], scale=0.15, rough=rough, metal=metal)
    cam = _tiny.front_camera(dist=3.0, res=32)
    env = env_state(_tiny.const_env(), M.Params())
    out = _render(surf, cam, env, M.Params())
    A = out["rgba"][:, 3]
    cov = A > 1e-3
    assert cov.sum() > 50
    f32 = lambda v: float(np.float32(v))
    got = out["aov"][cov] / A[cov, None]
    np.testing.assert_allclose(got[:, 3], f32(rough), rtol=1e-12)
    np.testing.assert_allclose(got[:, 4], f32(metal), rtol=1e-12)
    np.testing.assert_allclose(got[:, 5:8], np.broadcast_to([0.0, 0.0, 1.0], got[:, 5:8].shape), atol=1e-12)
    np.testing.assert_allclose(got[:, 8], 3.0 - f32(z_w), rtol=1e-12)


@pytest.mark.parametrize("angle", [1.2, -1.2])
def test_support_of_a_tilted_surfel_near_the_camera_is_its_projected_disc(angle):
    """Without the MIP filter (n_f = 1, Sigma = I) the support is the disc of
    radius r_cut in the surfel plane.  A large surfel tilted about 70 degrees
    close to the camera projects that disc far from its affine image at the
    centre (its near half is wider), so the support rectangle must take the
    disc's exact projected bounds (App. A), not only the EWA ellipse's: the
    covered pixels are exactly those whose ray meets the plane inside the
    disc (ray-plane intersection in FP64), and some lie beyond the affine
    bounds."""
    prm = M.Params(mip_mode="none")
    cam = _tiny.front_camera(dist=0.9, res=48)
    surf = _tilt(_tiny.surfels([[0.0, 0.05, 0.0]], scale=0.12), angle)
    env = env_state(_tiny.const_env(), prm)
    out = _render(surf, cam, env, prm)
    got = out["rgba"][:, 3] > 0
    # direct intersection: camera at (0, 0, 0.9) looking down -z, pixel rays through centres
    cd = M.cam_dict(cam)
    R, t = cd["R"].numpy(), cd["t"].numpy()
    q = surf.quat[0].astype(np.float64)
    Rs = M.quat_to_rot(torch.from_numpy(q[None])).numpy()[0]
    sc = np.exp(surf.log_scale[0].astype(np.float64))
    c = R @ surf.pos[0].astype(np.float64) + t
    tu, tv = R @ (sc[0] * Rs[:, 0]), R @ (sc[1] * Rs[:, 1])
    n = np.cross(tu, tv)
    W = H = 48
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    d = np.stack([(xs - cd["cx"]) / cd["fx"], (ys - cd["cy"]) / cd["fy"], np.ones_like(xs)], -1).reshape(-1, 3)
    lam = (n @ c) / (d @ n)
    X = lam[:, None] * d - c
    A = np.stack([tu, tv], 1)
    uv = np.linalg.lstsq(A, X.T, rcond=None)[0].T
    r2 = (uv ** 2).sum(1)
    want = (lam > 0) & (r2 < prm.r_cut ** 2)
    near_edge = np.abs(r2 - prm.r_cut ** 2) < 1e-6
    assert want.sum() > 100
    assert np.array_equal(got[~near_edge], want[~near_edge])
    # the disc reaches past the affine (EWA) bounds at the centre
    Mm = out["records"]["T"]
    T = Mm.numpy()[0]
    px, py = T[0, 2] / T[2, 2], T[1, 2] / T[2, 2]
    Mx = np.array([[T[0, 0] - px * T[2, 0], T[0, 1] - px * T[2, 1]],
                   [T[1, 0] - py * T[2, 0], T[1, 1] - py * T[2, 1]]]) / T[2, 2]
    ext = prm.r_cut * np.sqrt(np.diag(Mx @ Mx.T))
    cx_, cy_ = xs.ravel()[want], ys.ravel()[want]
    beyond = (np.abs(cx_ - px) > ext[0] + 1) | (np.abs(cy_ - py) > ext[1] + 1)
    assert beyond.sum() > 20     # (tilted one way or the other: the far side differs)
