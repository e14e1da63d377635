"""A whole batched step (env prefilter with its side streams, forward,
backward, env adjoint) captured once in a CUDA graph and replayed gives the
eager step's results: the images bit for bit (the forward is deterministic),
the gradients within the FP32-atomics reordering bound."""
import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_step():
    import torch
    from paper_2605_05876_gb300.api import Renderer
    a = S.sphere_4k(n=2048, res=64)
    cams = [a.cameras[0], S.look_at((0.5, 0.3, 2.8), width=48, height=40, scene=0)]
    sc = S.Scene(a.surfels, a.scene_offsets, a.envs, cams, "graph")
    r = Renderer(sc)
    g = torch.Generator(device="cuda").manual_seed(3)
    d_rgba = torch.randn(r.rgba.shape, device="cuda", generator=g)
    d_aov = torch.randn(r.aov.shape, device="cuda", generator=g)

    def step():
        r.prefilter_env()
        r.forward()
        r.zero_grads()
        r.backward(d_rgba, d_aov)

    step()
    torch.cuda.synchronize()
    ref_img = r.rgba.clone()
    ref = {k: v.clone() for k, v in r.grads.items()}
    ref_env = r.d_env.clone()

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        step()
    r.rgba.zero_()
    for v in r.grads.values():
        v.fill_(float("nan"))
    cg.replay()
    torch.cuda.synchronize()
    assert r.read_status() == 0
    assert torch.equal(r.rgba, ref_img)
    for k, v in ref.items():
        got, want = r.grads[k].cpu().numpy(), v.cpu().numpy()
        assert np.isfinite(got).all(), k
        scale = np.abs(want).max() + 1e-30
        assert np.abs(got - want).max() <= 1e-4 * scale, k
    got, want = r.d_env.cpu().numpy(), ref_env.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-4 * (np.abs(want).max() + 1e-30)


def test_graph_recaptured_after_densify():
    """Density control changes the surfel count, so a captured step is
    captured again after it; in the deterministic mode the replay of the new
    graph gives the eager step's images and gradients bit for bit."""
    import torch
    from paper_2605_05876_gb300.api import Renderer
    a = S.sphere_4k(n=2048, res=64)
    # tangent scales 4x the sphere's default (0.12 against a neighbour spacing
    # of ~0.08), so that the split rule's size test passes
    su = a.surfels
    big = S.Surfels(su.pos, su.quat, (su.log_scale + np.float32(np.log(4.0))).astype(np.float32), su.albedo,
                    su.roughness, su.metallic)
    cams = [a.cameras[0], S.look_at((0.5, 0.3, 2.8), width=48, height=40, scene=0)]
    sc = S.Scene(big, a.scene_offsets, a.envs, cams, "graph")
    r = Renderer(sc, screen_grad=True, params=dict(deterministic=1))
    g = torch.Generator(device="cuda").manual_seed(4)
    d_rgba = torch.randn(r.rgba.shape, device="cuda", generator=g)
    d_aov = torch.randn(r.aov.shape, device="cuda", generator=g)

    def step():
        r.prefilter_env()
        r.forward()
        r.zero_grads()
        r.backward(d_rgba, d_aov)

    step()
    torch.cuda.synchronize()
    n0 = r.n_surfels
    info = r.densify(r.density_params(tau_g=1e-12))
    assert r.n_surfels > n0 and info is not None
    step()
    torch.cuda.synchronize()
    assert r.read_status() == 0
    ref_img = r.rgba.clone()
    ref = {k: v.clone() for k, v in r.grads.items()}
    ref_env = r.d_env.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        step()
    r.rgba.zero_()
    for v in r.grads.values():
        v.fill_(float("nan"))
    cg.replay()
    torch.cuda.synchronize()
    assert r.read_status() == 0
    assert torch.equal(r.rgba, ref_img)
    for k, v in ref.items():
        assert torch.equal(r.grads[k], v), k
    assert torch.equal(r.d_env, ref_env)
