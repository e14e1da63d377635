"""Pins of the oracle's screen-space gradient statistic (Eq. ss_grad):
each fragment's g_x = dL_p/dT_{1,z} T_{4,z} (and g_y) against central finite
differences of that pixel's loss in T_{1,z} (T_{2,z}), with the fragments,
the layer assignment and the shaded channels held fixed and the MIP filter
recomputed from the perturbed T; the sum over a surfel's fragments against
finite differences of the whole image's loss."""
import numpy as np
import torch

from oracle import model as M
from tests import _tiny


def _setup(seed=7):
    rng = np.random.default_rng(seed)
    surf = _tiny.random_scene(rng, n=30, spread=0.4, scale=(0.03, 0.08))
    cam = _tiny.front_camera(res=24, width=30)
    prm = M.Params()
    env = M.prepare_env(_tiny.lognormal_env(rng, 64, 32), prm)
    S = M.to_torch_surfels(surf)
    cd = M.cam_dict(cam)
    with torch.no_grad():
        rec = M.records(S, cd, torch.from_numpy(env.irr.copy()), [torch.from_numpy(l.copy()) for l in env.levels],
                        torch.from_numpy(env.lut.copy()), prm)
    rect = M.support_rect(rec, prm)
    return rng, surf, cam, prm, env, rec, rect


def _loss(rec, fr, T, W, prm, G):
    """Loss of the queried pixels with the T-matrices replaced by T (the MIP
    filter recomputed from them), everything discrete held as in fr."""
    Sinv, n_f, _, _ = M.mip_filter(T, rec["zs"] > prm.z_near, prm)
    sid = torch.from_numpy(fr.sid.astype(np.int64))
    pf = {"T": T[sid], "Sinv": Sinv[sid], "n_f": n_f[sid], "ch": rec["ch"][sid]}
    rgba, aov = M.composite(rec, fr, W, prm, per_frag=pf)
    return float((torch.cat([rgba, aov], 1) * torch.from_numpy(G)).sum())


def _fd(rec, fr, W, prm, G, i, row, h=1e-5):
    T = rec["T"].detach().clone()
    Tp, Tm = T.clone(), T.clone()
    step = h * max(1.0, abs(float(T[i, row, 2])))
    Tp[i, row, 2] += step
    Tm[i, row, 2] -= step
    return (_loss(rec, fr, Tp, W, prm, G) - _loss(rec, fr, Tm, W, prm, G)) / (2 * step) * float(T[i, 2, 2])


def test_per_fragment_values_match_finite_differences_of_their_pixel():
    rng, surf, cam, prm, env, rec, rect = _setup()
    W, H = cam.width, cam.height
    fr_all = M.fragments(rec, rect, W, H, prm)
    # pixels where several surfels overlap (grouping and normalisation matter)
    counts = np.bincount(fr_all.pix, minlength=W * H)
    pixels = np.argsort(-counts)[:6]
    checked = 0
    for p in pixels:
        G = rng.normal(size=(1, 13))
        out = M.screen_grad_stat(surf, cam, env, prm, G, pix=[int(p)])
        fr = M.fragments(rec, rect, W, H, prm, pix=np.array([p], np.int32))
        assert np.array_equal(out["sid"], fr.sid)
        for f, i in enumerate(fr.sid):
            for row, key in ((0, "gx"), (1, "gy")):
                ref = _fd(rec, fr, W, prm, G, int(i), row)
                got = out[key][f]
                assert abs(got - ref) <= 1e-6 * max(abs(ref), 1e-3) + 1e-9, (p, i, key, got, ref)
                checked += 1
    assert checked >= 20


def test_surfel_sums_match_finite_differences_of_the_image():
    rng, surf, cam, prm, env, rec, rect = _setup(11)
    W, H = cam.width, cam.height
    G = rng.normal(size=(W * H, 13))
    out = M.screen_grad_stat(surf, cam, env, prm, G)
    fr = M.fragments(rec, rect, W, H, prm)
    sx = np.bincount(out["sid"], weights=out["gx"], minlength=surf.n)
    sy = np.bincount(out["sid"], weights=out["gy"], minlength=surf.n)
    hit = np.where(out["n_frag"] > 0)[0]
    assert hit.size >= 10
    for i in hit[:8]:
        assert abs(sx[i] - _fd(rec, fr, W, prm, G, int(i), 0)) <= 1e-6 * max(abs(sx[i]), 1e-3)
        assert abs(sy[i] - _fd(rec, fr, W, prm, G, int(i), 1)) <= 1e-6 * max(abs(sy[i]), 1e-3)
    # the statistic sums norms: never below the norm of the summed gradient,
    # zero exactly for surfels without fragments
    assert (out["sum_norm"][hit] >= np.hypot(sx[hit], sy[hit]) * (1 - 1e-12)).all()
    assert (out["sum_norm"][out["n_frag"] == 0] == 0).all()
    assert np.array_equal(out["n_frag"], np.bincount(fr.sid, minlength=surf.n))
