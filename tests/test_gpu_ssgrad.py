"""GPU densification statistic (Sec. 3.6.1, Eq. ss_grad) vs the oracle's
``screen_grad_stat``: per surfel, the sum over views and covering fragments
of |(g_x, g_y)|, g_x = dL/dT_{1,z} T_{4,z}, and the number of views in which
the surfel has a fragment, through the C ABI (ss_render_backward with
ss_render_params.screen_grad = 1)."""
import numpy as np
import pytest

from oracle import model as M
from paper_2605_05876_gb300 import scenes as S
from tests import _parity, _tiny

pytestmark = pytest.mark.gpu

# per-surfel sums of per-fragment gradient norms (FP32 per fragment, summed
# in another order): the gradient tolerances of the backward tests
BLOCK_RTOL = 1e-4
ELEM_RTOL = 1e-3
ELEM_ATOL = 1e-5


def _run(scene, seed, params=None, aov_grad=True):
    import torch
    from paper_2605_05876_gb300.api import Renderer
    r = Renderer(scene, params=params, screen_grad=True)
    r.forward()
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(r.n_pixels, 13))
    if not aov_grad:
        G[:, 4:] = 0.0
    ref_norm = np.zeros(scene.surfels.n)
    ref_views = np.zeros(scene.surfels.n)
    fragile = np.zeros(scene.surfels.n, bool)
    op = _parity.oracle_params(r.prm)
    cache = {}
    for v in range(r.n_views):
        sl = r.view_slice(v)
        cam = scene.cameras[v]
        s0, s1 = int(scene.scene_offsets[cam.scene]), int(scene.scene_offsets[cam.scene + 1])
        ref0 = _parity.oracle_view(scene, v, r.prm, env_cache=cache)
        amb = _parity.ambiguous(ref0["margin"])
        G[sl][amb] = 0.0      # no gradient from pixels within rounding of a decision (both sides)
        st = M.screen_grad_stat(scene.surfels.subset(slice(s0, s1)), cam, cache[cam.scene], op, G=G[sl])
        ref_norm[s0:s1] += st["sum_norm"]
        ref_views[s0:s1] += st["n_frag"] > 0
        # a surfel whose fragments in this view lie only on set-aside pixels may be in or out
        amb_pix = set((np.where(amb)[0]).tolist())
        on_amb = np.zeros(s1 - s0, bool)
        safe = np.zeros(s1 - s0, bool)
        for sid, pid in zip(st["sid"], st["pix"]):
            if int(pid) in amb_pix:
                on_amb[sid] = True
            else:
                safe[sid] = True
        fragile[s0:s1] |= on_amb & ~safe
    d_rgba = torch.from_numpy(G[:, :4].astype(np.float32)).cuda().contiguous()
    d_aov = torch.from_numpy(np.ascontiguousarray(G[:, 4:].T).astype(np.float32)).cuda()
    r.zero_grads()
    r.backward(d_rgba, d_aov if aov_grad else None)
    torch.cuda.synchronize()
    assert r.read_status() == 0
    return (r.screen_grad_norm.cpu().numpy().astype(np.float64), r.screen_grad_views.cpu().numpy(),
            ref_norm, ref_views, fragile)


def _compare(gpu_norm, gpu_views, ref_norm, ref_views, fragile):
    assert fragile.mean() < 1e-2
    keep = ~fragile
    assert np.array_equal(gpu_views[keep], ref_views[keep]), \
        f"view counts differ at {np.where(gpu_views[keep] != ref_views[keep])[0][:10]}"
    assert (ref_views > 0).sum() > 10
    blk = np.linalg.norm(gpu_norm - ref_norm) / np.linalg.norm(ref_norm)
    el = (np.abs(gpu_norm - ref_norm) / (ELEM_RTOL * np.abs(ref_norm) + ELEM_ATOL * np.abs(ref_norm).max()))[keep]
    print(f"screen-space statistic: block {blk:.2e}, elem/bound {el.max():.2f}, "
          f"{int((ref_views > 0).sum())} surfels seen, {int(fragile.sum())} set aside")
    assert blk <= BLOCK_RTOL and el.max() <= 1.0


@pytest.mark.parametrize("seed,sigma_f", [(1, 0.5), (2, 0.0), (3, 2.0)])
def test_screen_grad_tiny(seed, sigma_f):
    rng = np.random.default_rng(400 + seed)
    surf = _tiny.random_scene(rng, n=200, spread=0.5, scale=(0.02, 0.09))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=45)], "tiny")
    _compare(*_run(sc, seed, params=dict(sigma_f=sigma_f)))


def test_screen_grad_rgba_only():
    rng = np.random.default_rng(411)
    surf = _tiny.random_scene(rng, n=200, spread=0.5, scale=(0.02, 0.09))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=45)], "tiny")
    _compare(*_run(sc, 11, aov_grad=False))


def test_screen_grad_multi_view_multi_scene():
    a = S.sphere_4k(n=2048, res=64)
    b = S.torus_sphere_100k(n=20000, res=96)
    cams = [a.cameras[0], S.look_at((0.5, 0.3, 2.8), width=37, height=53, scene=0),
            S.look_at(b.cameras[0].R.T @ -b.cameras[0].t, width=96, height=80, scene=1)]
    rng = np.random.default_rng(6)
    sc = S.Scene(S.Surfels.concat([a.surfels, b.surfels]), np.array([0, 2048, 22048]),
                 [a.envs[0], np.exp(rng.normal(size=(32, 64, 3))).astype(np.float32)], cams, "multi")
    _compare(*_run(sc, 7))


@pytest.mark.slow
def test_screen_grad_torus_sphere_100k():
    _compare(*_run(S.torus_sphere_100k(), 9))
