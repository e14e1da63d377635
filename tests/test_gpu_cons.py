"""The depth-consolidation term of Eq. cons_loss (Sec. 3.7.1) on the GPU:
its per-pixel value (the tenth AOV plane) and its gradient against the
oracle, element by element, on scenes with several surface layers."""
import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S
from tests import _tiny
from tests.test_gpu_backward import _compare, _run
from tests.test_gpu_forward import _check_view, _renderer

pytestmark = pytest.mark.gpu


def _layered(rng, n=150, gap=0.7):
    """Two random clusters one behind the other (pixels with several layers)."""
    front = _tiny.random_scene(rng, n=n, spread=0.4, scale=(0.02, 0.08))
    back = _tiny.random_scene(rng, n=n, spread=0.4, scale=(0.02, 0.08))
    back = S.Surfels(back.pos - np.array([0.0, 0.0, gap], np.float32), back.quat, back.log_scale, back.albedo,
                     back.roughness, back.metallic)
    return S.Surfels.concat([front, back])


@pytest.mark.parametrize("seed", [1, 2])
def test_cons_forward_tiny(seed):
    rng = np.random.default_rng(600 + seed)
    surf = _layered(rng)
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=45)], "layered")
    r = _renderer(sc, params=dict(cons=1))
    r.forward()
    assert r.read_status() == 0
    ref, gpu = _check_view(r, sc, 0)
    assert gpu.shape[1] == 14 and (ref["n_layers"] >= 2).sum() > 50
    assert (gpu[:, 13] > 0).sum() > 50


def test_cons_forward_torus_sphere():
    """Self-occluding surfaces (torus and sphere, front and back sides)."""
    sc = S.torus_sphere_100k(n=30000, res=128)
    r = _renderer(sc, params=dict(cons=1))
    r.forward()
    assert r.read_status() == 0
    _check_view(r, sc, 0)


@pytest.mark.parametrize("seed", [3, 4])
def test_cons_backward_tiny(seed):
    rng = np.random.default_rng(610 + seed)
    surf = _layered(rng)
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=45)], "layered")
    gpu, ref = _run(sc, seed, params=dict(cons=1))
    _compare(gpu, ref)


def test_cons_backward_multi_view():
    a = S.sphere_4k(n=2048, res=64)
    b = S.torus_sphere_100k(n=20000, res=96)
    cams = [a.cameras[0], S.look_at((0.5, 0.3, 2.8), width=37, height=53, scene=0),
            S.look_at(b.cameras[0].R.T @ -b.cameras[0].t, width=96, height=80, scene=1)]
    rng = np.random.default_rng(6)
    sc = S.Scene(S.Surfels.concat([a.surfels, b.surfels]), np.array([0, 2048, 22048]),
                 [a.envs[0], np.exp(rng.normal(size=(32, 64, 3))).astype(np.float32)], cams, "multi")
    gpu, ref = _run(sc, 8, params=dict(cons=1))
    _compare(gpu, ref)
