"""Tile shape and staging depth (the autotuner's knobs): every choice renders
and differentiates exactly as the oracle does -- they change speed, never
results."""
import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S
from tests import _tiny
from tests.test_gpu_backward import _compare, _run
from tests.test_gpu_forward import _check_view, _renderer

pytestmark = pytest.mark.gpu

TILES = [(16, 16), (16, 8), (32, 8), (8, 16), (8, 8), (8, 32), (32, 4), (8, 4)]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("depth", [1, 3])
def test_forward_tiles_and_depths(tile, depth):
    rng = np.random.default_rng(700 + tile[0] + tile[1] + depth)
    surf = _tiny.random_scene(rng, n=300, spread=0.5, scale=(0.01, 0.08))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=41, width=53)], "tiny")       # ragged in both directions
    r = _renderer(sc, params=dict(tile_w=tile[0], tile_h=tile[1], stage_depth=depth))
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)


@pytest.mark.parametrize("tile", [(8, 8), (32, 8), (16, 8)])
def test_backward_tiles(tile):
    rng = np.random.default_rng(720 + tile[0] + tile[1])
    surf = _tiny.random_scene(rng, n=200, spread=0.5, scale=(0.02, 0.09))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=45)], "tiny")
    gpu, ref = _run(sc, 3, params=dict(tile_w=tile[0], tile_h=tile[1], stage_depth=3))
    _compare(gpu, ref)


def test_multi_scene_uneven_with_other_tiles():
    a = S.sphere_4k(n=2048, res=64)
    b = S.torus_sphere_100k(n=20000, res=96)
    cams = [a.cameras[0], S.look_at((0.5, 0.3, 2.8), width=37, height=53, scene=0),
            S.look_at(b.cameras[0].R.T @ -b.cameras[0].t, width=96, height=80, scene=1)]
    rng = np.random.default_rng(5)
    env_b = np.exp(rng.normal(size=(32, 64, 3))).astype(np.float32)
    sc = S.Scene(S.Surfels.concat([a.surfels, b.surfels]), np.array([0, 2048, 22048]), [a.envs[0], env_b], cams,
                 "multi")
    r = _renderer(sc, params=dict(tile_w=32, tile_h=8, stage_depth=1))
    r.forward()
    assert r.read_status() == 0
    cache = {}
    for v in range(3):
        _check_view(r, sc, v, env_cache=cache)


def test_autotuner_picks_among_the_knobs():
    """The autotuner times every tile shape and staging depth and leaves the
    renderer on the fastest; the result still matches the oracle."""
    import torch
    sc = S.sphere_4k(n=4096, res=96)
    r = _renderer(sc)
    G = torch.randn(r.n_pixels, 13, device="cuda")
    chosen = r.autotune(G[:, :4].contiguous(), G[:, 4:].t().contiguous(), reps=1)
    assert set(chosen["tile"][1]) == {"16x16", "16x8", "32x8", "8x16", "8x8"}
    assert set(chosen["stage_depth"][1]) == {1, 2, 3}
    assert (r.prm.tile_w, r.prm.tile_h) == tuple(int(x) for x in chosen["tile"][0].split("x"))
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)
