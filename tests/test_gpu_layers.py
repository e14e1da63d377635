"""Layer state past dense_layers in the pool (ss_render_params.dense_layers,
layer_pool): the forward stores the same per-layer totals, chained per pixel
through pool slots, so images, AOVs and (in the deterministic mode)
gradients are bitwise those of the all-dense layout; too small a pool is
reported with the number of slots it needed."""
import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S
from tests import _tiny
from tests.test_gpu_forward import _check_view

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")


def _planes(n_planes=4, res=40):
    rng = np.random.default_rng(7)
    planes = [_tiny.grid_plane(24, 0.03, z=0.05 * k, scale=0.025, albedo=tuple(rng.uniform(0, 1, 3)))
              for k in range(n_planes)]
    surf = S.Surfels.concat(planes)
    return S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 32, 16)], [_tiny.front_camera(res=res)],
                   "planes")


def _render(sc, cons=False, **params):
    import torch
    from paper_2605_05876_gb300.api import Renderer
    r = Renderer(sc, params=dict(deterministic=1, cons=int(cons), **params))
    r.forward()
    torch.cuda.synchronize()
    g = torch.Generator(device="cuda").manual_seed(3)
    G = torch.randn(r.n_pixels, 13 + int(cons), device="cuda", generator=g)
    r.zero_grads()
    r.backward(G[:, :4].contiguous(), G[:, 4:].t().contiguous())
    torch.cuda.synchronize()
    out = {"rgba": r.rgba.cpu().numpy().copy(), "aov": r.aov.cpu().numpy().copy(), "env": r.d_env.cpu().numpy().copy()}
    out.update({k: r.grads[k].cpu().numpy().copy() for k in FIELDS})
    return out, r.read_status(), r.stats()


@pytest.mark.parametrize("dense", [1, 2, 3])
@pytest.mark.parametrize("cons", [False, True])
def test_layer_pool_is_bitwise_the_dense_layout(dense, cons):
    sc = _planes()
    ref, st0, s0 = _render(sc, cons)
    assert st0 == 0 and s0["pool_layers"] == 0
    got, st, s = _render(sc, cons, dense_layers=dense, layer_pool=40 * 40 * 4)
    assert st == 0
    assert s["pool_layers"] > 0   # the four planes give four layers at the covered pixels
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint32), got[k].view(np.uint32)), k


def test_layer_pool_capacity_is_reported():
    sc = _planes()
    _, _, full = _render(sc, dense_layers=1, layer_pool=40 * 40 * 4)
    need = full["pool_layers"]
    _, st, s = _render(sc, dense_layers=1, layer_pool=need // 2)
    from paper_2605_05876_gb300 import _lib
    assert st & _lib.SS_ERR_CAPACITY
    assert s["pool_layers"] == need   # the count goes on past the capacity: it sizes the pool
    _, st, s = _render(sc, dense_layers=1, layer_pool=need)
    assert st == 0


def test_crowded_tile_with_pooled_layers_matches_oracle():
    """16 planes in one tile (K_max layers at the covered pixels) with two
    dense layers: 14 of each pixel's layers live in the pool; the forward
    matches the oracle pixel by pixel."""
    from paper_2605_05876_gb300.api import Renderer
    rng = np.random.default_rng(17)
    pos = np.concatenate([np.concatenate([rng.uniform(-1.2, -0.8, size=(800, 2)), np.full((800, 1), 0.05 * k)], 1)
                          for k in range(16)])
    surf = _tiny.surfels(pos, scale=0.03, albedo=rng.uniform(0, 1, (pos.shape[0], 3)))
    sc = S.Scene(surf, np.array([0, surf.n]), [_tiny.lognormal_env(rng, 32, 16)], [_tiny.front_camera(res=32)],
                 "crowd")
    r = Renderer(sc, params=dict(dense_layers=2, layer_pool=32 * 32 * 14))
    r.forward()
    assert r.read_status() == 0 and r.stats()["pool_layers"] > 0
    ref, gpu = _check_view(r, sc, 0)
    assert ref["n_layers"].max() == 16


def test_block_lists_sized_by_their_candidates():
    """max_candidates = the count a forward reports gives bitwise the images
    and gradients of the bound-sized lists; one less is reported."""
    from paper_2605_05876_gb300 import _lib
    sc = _planes()
    ref, st0, s0 = _render(sc)
    need = s0["candidates"]
    assert st0 == 0 and need > 0
    got, st, s = _render(sc, max_candidates=need)
    assert st == 0 and s["candidates"] == need
    for k in ref:
        assert np.array_equal(ref[k].view(np.uint32), got[k].view(np.uint32)), k
    _, st, s = _render(sc, max_candidates=need - 1)
    assert st & _lib.SS_ERR_CAPACITY and s["candidates"] == need


def test_compact_workspace_renders_as_the_bounds():
    """Renderer.compact_workspace (block lists and deep layers sized by two
    counting forwards) renders the torus-and-sphere batch bitwise as the
    bound-sized workspace, in less memory."""
    import torch
    from paper_2605_05876_gb300.api import Renderer
    b = S.torus_sphere_100k(n=20000, res=96)
    a = Renderer(b)
    a.forward()
    ref = a.rgba.cpu().numpy().copy()
    c = Renderer(b)
    cands, pool, ws = c.compact_workspace(1)
    assert ws < a.ws_bytes
    c.forward()
    torch.cuda.synchronize()
    assert c.read_status() == 0
    assert np.array_equal(ref.view(np.uint32), c.rgba.cpu().numpy().view(np.uint32))


def test_instance_capacity_overflow_is_reported_and_replanned():
    """Too small an instance list (max_instances): the forward completes,
    reports SS_ERR_CAPACITY and the real count (ss_stats.instances); planned
    again with that count, the batch renders as with the default plan."""
    import torch
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import Renderer
    b = S.torus_sphere_100k(n=20000, res=96)
    ref = Renderer(b)
    ref.forward()
    torch.cuda.synchronize()
    assert ref.read_status() == 0
    r = Renderer(b)
    r.plan_capacity(max_instances=ref.counted_instances // 3)
    r.prm.collect_stats = 1
    r.forward()
    torch.cuda.synchronize()
    assert r.read_status() & _lib.SS_ERR_CAPACITY
    need = r.stats()["instances"]
    assert need == ref.counted_instances
    r.prm.collect_stats = 0
    r.plan_capacity(max_instances=need)
    r.forward()
    torch.cuda.synchronize()
    assert r.read_status() == 0
    assert torch.equal(r.rgba, ref.rgba)
