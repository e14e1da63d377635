"""GPU forward path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from oracle import model as M
from paper_2605_05876_gb300 import scenes as S
from tests import _parity, _tiny

pytestmark = pytest.mark.gpu


def _renderer(scene, **kw):
    from paper_2605_05876_gb300.api import Renderer
    return Renderer(scene, **kw)


def _gpu_view(r, v):
    import torch
    torch.cuda.synchronize()
    sl = r.view_slice(v)
    rgba = r.rgba[sl].cpu().numpy().astype(np.float64)
    aov = r.aov[:, sl].t().cpu().numpy().astype(np.float64)
    return np.concatenate([rgba, aov], 1)


def _check_view(r, scene, v, pix=None, env_cache=None):
    ref = _parity.oracle_view(scene, v, r.prm, env_levels=r.ed.n_levels, pix=pix, env_cache=env_cache)
    gpu = _gpu_view(r, v)
    if pix is not None:
        gpu = gpu[np.asarray(pix)]
    amb = _parity.ambiguous(ref["margin"])
    refv = np.concatenate([ref["rgba"], ref["aov"]], 1)
    n_bad, msg = _parity.compare(gpu, refv, amb, f"view {v}")
    # (a sanity bound; samples drawn mostly from covered pixels hold more of them)
    bound = _parity.MAX_AMBIGUOUS_FRACTION * (1 if pix is None else 5)
    assert amb.mean() <= bound, f"too many ambiguous pixels: {amb.sum()}"
    assert n_bad == 0, msg
    n_amb, n_flip = _parity.check_variants(gpu, ref, amb, pix=pix, prm=r.prm)
    print(f"view {v}: {n_amb} of {amb.size} pixels with a decision within rounding (fraction {amb.mean():.2e}), "
          f"each matched an outcome at the strict tolerance; the GPU took the other outcome at {n_flip}")
    _parity.check_flip_fraction(n_flip, amb.size, f"view {v}")
    return ref, gpu


def test_brdf_lut_matches_oracle():
    import torch
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import _ptr, _stream
    lut = torch.zeros(128, 128, 2, device="cuda")
    _lib.check(_lib.lib().ss_brdf_lut(_ptr(lut), 128, _stream()))
    ref = M.brdf_lut(128, 128)
    assert np.abs(lut.cpu().numpy() - ref).max() < 2e-6


@pytest.mark.parametrize("shape", [(64, 32, 6), (256, 128, 6), (32, 16, 3)])
def test_env_prefilter_matches_oracle(shape):
    import torch
    We, He, L = shape
    rng = np.random.default_rng(We + L)
    envs = [np.exp(rng.normal(size=(He, We, 3))).astype(np.float32) for _ in range(2)]
    sc = S.Scene(_tiny.surfels([[0, 0, 0]]), np.array([0, 1, 1]), envs,
                 [S.look_at((0, 0, 3), width=16, height=16)], "env")
    r = _renderer(sc, env_levels=L)
    torch.cuda.synchronize()
    for e in range(2):
        irr, levels = M.env_prefilter(envs[e].astype(np.float64), L, 32, 16)
        gi = r.irr[e].cpu().numpy().reshape(16, 32, 3)
        assert np.abs(gi - irr).max() <= 2e-6 * np.abs(irr).max()
        gs = r.spec[e].cpu().numpy()
        off = 0
        for lv in levels:
            n = lv.size
            got = gs[off:off + n].reshape(lv.shape)
            assert np.abs(got - lv).max() <= 2e-6 * np.abs(lv).max() + 1e-7
            off += n


def test_env_prefilter_backward_matches_oracle():
    import torch
    We, He, L = 64, 32, 5
    rng = np.random.default_rng(9)
    env = np.exp(rng.normal(size=(He, We, 3))).astype(np.float32)
    sc = S.Scene(_tiny.surfels([[0, 0, 0]]), np.array([0, 1]), [env], [S.look_at((0, 0, 3), width=16, height=16)],
                 "env")
    r = _renderer(sc, env_levels=L)
    r.zero_grads()
    d_irr = torch.randn_like(r.irr)
    d_spec = torch.randn_like(r.spec)
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import _ptr, _stream
    import ctypes
    _lib.check(_lib.lib().ss_env_prefilter_backward(ctypes.byref(r.ed), 1, _ptr(d_irr), _ptr(d_spec), _ptr(r.aux),
                                                   _ptr(r.d_env), _stream()))
    torch.cuda.synchronize()
    sizes = M.level_sizes(We, He, L)
    ds = d_spec[0].cpu().numpy().astype(np.float64)
    d_lv, off = [], 0
    for (W, H) in sizes:
        d_lv.append(ds[off:off + W * H * 3].reshape(H, W, 3))
        off += W * H * 3
    ref = M.env_adjoint(d_irr[0].cpu().numpy().astype(np.float64).reshape(16, 32, 3), d_lv, We, He)
    got = r.d_env[0].cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_forward_sphere_4k():
    sc = S.sphere_4k()
    r = _renderer(sc)
    r.forward()
    assert r.read_status() == 0
    ref, gpu = _check_view(r, sc, 0)
    assert (gpu[:, 3] > 0).sum() > 4000


@pytest.mark.parametrize("seed,sigma_f,res", [(1, 0.5, 40), (2, 0.0, 33), (3, 2.0, 47), (4, 0.5, 17)])
def test_forward_tiny_random(seed, sigma_f, res):
    rng = np.random.default_rng(100 + seed)
    surf = _tiny.random_scene(rng, n=300, spread=0.5, scale=(0.01, 0.08))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=res, width=res + 7)], "tiny")
    r = _renderer(sc, params=dict(sigma_f=sigma_f, bg=(0.1, 0.2, 0.3)))
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)


def _aniso_scene(seed):
    """A camera with f_y = 1.3 f_x and a wider than high image (every other
    case has square pixels), over a random scene."""
    rng = np.random.default_rng(300 + seed)
    surf = _tiny.random_scene(rng, n=300, spread=0.5, scale=(0.01, 0.08))
    c = _tiny.front_camera(res=36, width=44)
    cam = S.Camera(c.R, c.t, c.fx, 1.3 * c.fy, c.cx, c.cy, c.width, c.height, c.scene)
    return S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)], [cam], "aniso")


def test_forward_unequal_focal_lengths():
    sc = _aniso_scene(1)
    r = _renderer(sc, params=dict(sigma_f=0.5))
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)


@pytest.mark.parametrize("k_max", [1, 2, 16])
def test_forward_layer_cap(k_max):
    rng = np.random.default_rng(7)
    planes = [_tiny.grid_plane(24, 0.03, z=0.05 * k, scale=0.025, albedo=tuple(rng.uniform(0, 1, 3)))
              for k in range(4)]
    surf = S.Surfels.concat(planes)
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 32, 16)], [_tiny.front_camera(res=40)], "cap")
    r = _renderer(sc, params=dict(k_max=k_max))
    r.forward()
    ref, gpu = _check_view(r, sc, 0)
    assert ref["n_layers"].max() == min(k_max, 4)


def test_forward_crowded_tile_sorted_in_several_chunks():
    """12800 surfels in one 16 x 16 tile (16 planes of 800, K_max layers at
    the covered pixels): the tile's list is longer than one sorting chunk,
    so it is sorted in chunks and merged; ties of z_start within a plane are
    broken by record index."""
    rng = np.random.default_rng(17)
    pos = np.concatenate([np.concatenate([rng.uniform(-1.2, -0.8, size=(800, 2)), np.full((800, 1), 0.05 * k)], 1)
                          for k in range(16)])
    surf = _tiny.surfels(pos, scale=0.03, albedo=rng.uniform(0, 1, (pos.shape[0], 3)))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 32, 16)], [_tiny.front_camera(res=32)],
                 "crowd")
    r = _renderer(sc)
    r.forward()
    assert r.stats()["instances"] >= 12800     # all in the one tile the positions project into
    ref, gpu = _check_view(r, sc, 0)
    assert ref["n_layers"].max() == 16


def test_forward_empty_and_culled():
    """All surfels behind the camera: image is the background, alpha 0."""
    surf = _tiny.surfels([[0, 0, 5.0], [0.1, 0, 4.0]], scale=0.1)
    sc = S.Scene(surf, np.array([0, 2]), [_tiny.const_env(1.0)], [_tiny.front_camera(res=20)], "empty")
    r = _renderer(sc, params=dict(bg=(0.25, 0.5, 0.75)))
    r.forward()
    gpu = _gpu_view(r, 0)
    assert np.all(gpu[:, 3] == 0) and np.allclose(gpu[:, :3], [0.25, 0.5, 0.75])
    assert np.all(gpu[:, 4:] == 0)


def test_forward_torus_sphere_100k():
    sc = S.torus_sphere_100k()
    r = _renderer(sc)
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)


def test_forward_multi_scene_uneven():
    """Two scenes, three views of different sizes (ragged tiles), one env each."""
    rng = np.random.default_rng(5)
    a = S.sphere_4k(n=2048, res=64)
    b = S.torus_sphere_100k(n=20000, res=96)
    cams = [a.cameras[0], S.look_at((0.5, 0.3, 2.8), width=37, height=53, scene=0),
            S.look_at(b.cameras[0].R.T @ -b.cameras[0].t, width=96, height=80, scene=1)]
    env_b = np.exp(rng.normal(size=(32, 64, 3))).astype(np.float32)
    sc = S.Scene(S.Surfels.concat([a.surfels, b.surfels]), np.array([0, 2048, 22048]), [a.envs[0], env_b], cams,
                 "multi")
    r = _renderer(sc)
    r.forward()
    assert r.read_status() == 0
    cache = {}
    for v in range(3):
        _check_view(r, sc, v, env_cache=cache)


@pytest.mark.slow
def test_forward_displaced_sphere_1m():
    """Full-size headline workload (1M surfels, 16 views of 800^2, rendered in
    one batch as bench.py times it): every pixel of view 0 and sampled
    pixels of view 9 against the oracle, element by element; pixels with a
    decision within rounding match one of its outcomes, and the GPU takes
    the other outcome at no more than 1e-4 of the pixels."""
    sc = S.displaced_sphere_1m()
    r = _renderer(sc)
    r.forward()
    assert r.read_status() == 0
    rng = np.random.default_rng(0)
    cache = {}
    _check_view(r, sc, 0, env_cache=cache)
    gpu = _gpu_view(r, 9)
    cov = np.where(gpu[:, 3] > 0)[0]
    pix = np.sort(np.concatenate([rng.choice(cov, 600, replace=False), rng.choice(640000, 200, replace=False)]))
    _check_view(r, sc, 9, pix=np.unique(pix), env_cache=cache)
