"""Deterministic backward (ss_render_params.deterministic = 1): two runs on
the same inputs give bitwise-equal gradients for every surfel parameter, the
densification statistic and the environment; the gradients still match the
FP64 oracle and the default (atomic) mode; too few rows are reported, not
written past."""
import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S
from tests import _tiny
from tests.test_gpu_backward import _compare, _run

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")


def _scene():
    """A torus and a sphere (20k surfels, two overlapping objects, so a
    record's fragments come from many warps) seen by two views of one scene."""
    b = S.torus_sphere_100k(n=20000, res=96)
    cams = [b.cameras[0], S.look_at((0.4, 2.5, 1.6), width=120, height=88, scene=0)]
    return S.Scene(b.surfels, np.array([0, b.surfels.n]), b.envs, cams, "det")


def _grads(r, d_rgba, d_aov):
    import torch
    r.forward()
    r.zero_grads()
    r.backward(d_rgba, d_aov)
    torch.cuda.synchronize()
    assert r.read_status() == 0
    out = {k: r.grads[k].cpu().numpy().copy() for k in FIELDS}
    out["env"] = r.d_env.cpu().numpy().copy()
    out["irr"] = r.d_irr.cpu().numpy().copy()
    out["spec"] = r.d_spec.cpu().numpy().copy()
    if r.prm.screen_grad:
        out["ssg_norm"] = r.screen_grad_norm.cpu().numpy().copy()
        out["ssg_views"] = r.screen_grad_views.cpu().numpy().copy()
    return out


def _upstream(r, seed):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    G = torch.randn(r.n_pixels, 13, device="cuda", generator=g)
    return G[:, :4].contiguous(), G[:, 4:].t().contiguous()


@pytest.mark.parametrize("screen_grad", [False, True])
def test_deterministic_backward_is_bitwise_reproducible(screen_grad):
    from paper_2605_05876_gb300.api import Renderer
    sc = _scene()
    r = Renderer(sc, params=dict(deterministic=1), screen_grad=screen_grad)
    d_rgba, d_aov = _upstream(r, 5)
    a = _grads(r, d_rgba, d_aov)
    b = _grads(r, d_rgba, d_aov)
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
    assert np.abs(a["pos"]).max() > 0 and np.abs(a["env"]).max() > 0
    # the default (atomic) mode agrees up to the order of its FP32 sums
    rd = Renderer(sc, screen_grad=screen_grad)
    c = _grads(rd, d_rgba, d_aov)
    for k in a:
        nrm = np.linalg.norm(c[k])
        assert np.linalg.norm(a[k].astype(np.float64) - c[k]) <= 1e-5 * nrm + 1e-30, k


def test_deterministic_backward_rgba_only_is_reproducible():
    """Without an AOV gradient the raster writes 12 of the record's columns."""
    from paper_2605_05876_gb300.api import Renderer
    r = Renderer(_scene(), params=dict(deterministic=1))
    d_rgba, _ = _upstream(r, 6)
    a = _grads(r, d_rgba, None)
    b = _grads(r, d_rgba, None)
    for k in a:
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k


@pytest.mark.parametrize("seed", [1, 2])
def test_deterministic_backward_matches_oracle(seed):
    rng = np.random.default_rng(200 + seed)
    surf = _tiny.random_scene(rng, n=200, spread=0.5, scale=(0.02, 0.09))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 64, 32)],
                 [_tiny.front_camera(res=40, width=45)], "tiny")
    gpu, ref = _run(sc, seed, params=dict(deterministic=1, sigma_f=0.5, k_max=3))
    _compare(gpu, ref)


def test_deterministic_rows_capacity_is_reported():
    """det_rows far below the covering pairs: SS_ERR_CAPACITY, and the rows
    past the capacity are not written (the call completes)."""
    import torch
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import Renderer
    r = Renderer(_scene(), params=dict(deterministic=1, det_rows=64))
    d_rgba, d_aov = _upstream(r, 7)
    r.forward()
    r.zero_grads()
    r.backward(d_rgba, d_aov)
    torch.cuda.synchronize()
    assert r.read_status() & _lib.SS_ERR_CAPACITY
