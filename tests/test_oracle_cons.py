"""Pins of the oracle's depth-consolidation term (Sec. 3.7.1, Eq. cons_loss):
per pixel, over its composited layers,
    L_p = sum_{i<j} w_i w_j |z_i - z_j| + sum_i w_i^2 sigma_i^2,
w_i = T_i alpha_i the layer's compositing weight, z_i and sigma_i^2 the mean
and variance of its fragments' depths.  Closed forms on planes, an
independent brute-force evaluation, and finite differences of its gradient.
Nothing here uses the CUDA path."""
import math

import numpy as np

from oracle import model as M
from paper_2605_05876_gb300 import scenes as S
from tests import _tiny
from tests.test_oracle_pins import _decisions, _f64, _tilt, brute_force, env_state


def test_two_separated_planes():
    """Two fronto-parallel planes (every fragment of a plane at the plane's
    depth, so sigma_i = 0) in two layers: L = w_1 w_2 |z_1 - z_2| with
    w_1 = a_1 and w_2 = (1 - a_1) a_2, the planes' own coverages."""
    prm = M.Params(cons=True)
    cam = _tiny.front_camera(dist=3.0, res=33)
    s = 1.2 * 3.0 / cam.fx
    p1 = _tiny.grid_plane(30, 1.3 * s, z=0.1, scale=s)
    p2 = _tiny.grid_plane(30, 1.3 * s, z=-0.2, scale=s, center=(0.3 * s, 0.2 * s))
    env = env_state(_tiny.const_env(), prm)
    pix = [16 * 33 + 16, 14 * 33 + 17, 10 * 33 + 20]
    a1 = M.render_view(p1, cam, env, prm, pix=pix)["rgba"][:, 3]
    a2 = M.render_view(p2, cam, env, prm, pix=pix)["rgba"][:, 3]
    o = M.render_view(S.Surfels.concat([p2, p1]), cam, env, prm, pix=pix)
    assert np.all(o["n_layers"] == 2) and o["aov"].shape[1] == 10
    z1, z2 = 3.0 - float(np.float32(0.1)), 3.0 - float(np.float32(-0.2))
    np.testing.assert_allclose(o["aov"][:, 9], a1 * (1 - a1) * a2 * (z2 - z1), rtol=1e-10)
    # a single plane: one layer, no spread
    assert np.abs(M.render_view(p1, cam, env, prm, pix=pix)["aov"][:, 9]).max() < 1e-14


def test_thin_shell_variance():
    """Tilted planes closer than their depth extents merge into one layer;
    there L = w^2 sigma^2 with sigma^2 the Shepard-weighted variance of the
    fragments' centre depths, which is positive."""
    prm = M.Params(cons=True)
    cam = _tiny.front_camera(res=24)
    s = 0.03
    a = _tilt(_tiny.grid_plane(24, 0.8 * s, z=0.0, scale=s), 0.9)
    b = _tilt(_tiny.grid_plane(24, 0.8 * s, z=-0.01, scale=s, center=(0.4 * s, 0.3 * s)), 0.9)
    env = env_state(_tiny.const_env(), prm)
    o = M.render_view(S.Surfels.concat([a, b]), cam, env, prm)
    one = o["n_layers"] == 1
    assert one.sum() > 50
    assert np.all(o["aov"][one, 9] > 0)


def _brute_cons(surf, cam, prm):
    """The term from the brute-force renderer's own layers (its 3x3 ray-plane
    solve and connected components): per layer the weights, the centre depths
    c'_z of its fragments, their Shepard mean and variance."""
    import torch
    env = env_state(_tiny.const_env(), prm)
    Sd = M.to_torch_surfels(surf)
    rec = M.records(Sd, M.cam_dict(cam), torch.from_numpy(env.irr), [torch.from_numpy(l) for l in env.levels],
                    torch.from_numpy(env.lut), prm)
    return brute_force(surf, cam, prm, rec["ch"].detach().numpy(), cons=True)


def test_matches_brute_force():
    rng = np.random.default_rng(61)
    prm = M.Params(cons=True, sigma_f=0.7)
    front = _tiny.random_scene(rng, n=25, spread=0.3, scale=(0.05, 0.12))
    back = _tiny.random_scene(rng, n=25, spread=0.3, scale=(0.05, 0.12))
    back = S.Surfels(back.pos - np.array([0.0, 0.0, 0.9], np.float32), back.quat, back.log_scale, back.albedo,
                     back.roughness, back.metallic)
    surf = S.Surfels.concat([front, back])
    cam = _tiny.front_camera(res=28)
    env = env_state(_tiny.lognormal_env(rng), prm)
    out = M.render_view(surf, cam, env, prm)
    rgba, aov, unsure, cons = _brute_cons(surf, cam, prm)
    ok = ~unsure
    assert ok.sum() > 0.95 * ok.size
    assert (out["n_layers"][ok] >= 2).sum() > 20 and (cons[ok] > 0).sum() > 60
    np.testing.assert_allclose(out["aov"][ok, 9], cons[ok], rtol=1e-6, atol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(71)
    prm = M.Params(cons=True)
    front = _tiny.random_scene(rng, n=14, spread=0.25, scale=(0.06, 0.14))
    back = _tiny.random_scene(rng, n=14, spread=0.25, scale=(0.06, 0.14))
    back = S.Surfels(back.pos - np.array([0.0, 0.0, 0.8], np.float32), back.quat, back.log_scale, back.albedo,
                     back.roughness, back.metallic)
    surf = _f64(S.Surfels.concat([front, back]))
    cam = _tiny.front_camera(res=20)
    env = env_state(_tiny.lognormal_env(rng).astype(np.float64), prm)
    P = cam.width * cam.height
    G = np.zeros((P, 14))
    G[:, 13] = rng.normal(size=P)            # the consolidation term alone
    out = M.render_view(surf, cam, env, prm, G=G)
    base = _decisions(surf, cam, env, prm)

    def loss(s):
        o = M.render_view(s, cam, env, prm)
        return float((o["aov"][:, 9] * G[:, 13]).sum())

    checked = 0
    for name in ("pos", "quat", "log_scale"):
        flat = getattr(surf, name).reshape(-1)
        for idx in rng.choice(flat.size, size=min(10, flat.size), replace=False):
            plus, minus = _f64(surf), _f64(surf)
            getattr(plus, name).reshape(-1)[idx] += 1e-6
            getattr(minus, name).reshape(-1)[idx] -= 1e-6
            if _decisions(plus, cam, env, prm) != base or _decisions(minus, cam, env, prm) != base:
                continue
            fd = (loss(plus) - loss(minus)) / 2e-6
            an = out["grad"][name].reshape(-1)[idx]
            assert abs(fd - an) <= 2e-5 * max(1.0, abs(an)), (name, idx, fd, an)
            checked += 1
    assert checked >= 15
    assert np.abs(out["grad"]["albedo"]).max() == 0        # the term does not see the shading
