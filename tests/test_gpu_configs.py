"""The uneven multi-scene batch and the inverse-rendering loop at the sizes
bench.py runs them (sampled against the oracle), and the loop's loss falling."""
import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S
from tests import _parity
from tests.test_gpu_backward import FIELDS, LOOKUP_MARGIN, _compare
from tests.test_gpu_forward import _check_view, _gpu_view, _renderer

pytestmark = pytest.mark.gpu


@pytest.mark.slow
def test_uneven_scenes_full_batch_forward_sampled():
    """8 scenes of 79k-1.5M surfels, 32 views of 256^2-1024^2, rendered in one
    batch; one view per scene checked on sampled pixels."""
    sc = S.uneven_scenes()
    r = _renderer(sc)
    r.forward()
    assert r.read_status() == 0
    rng = np.random.default_rng(1)
    cache = {}
    for k in range(sc.n_scenes):
        v = 4 * k + k % 4
        gpu = _gpu_view(r, v)
        cov = np.where(gpu[:, 3] > 0)[0]
        npx = sc.cameras[v].width * sc.cameras[v].height
        pix = np.unique(np.concatenate([rng.choice(cov, min(150, cov.size), replace=False),
                                        rng.choice(npx, 30, replace=False)])).astype(np.int32)
        _check_view(r, sc, v, pix=pix, env_cache=cache)


@pytest.mark.slow
def test_uneven_scenes_full_batch_backward_sampled():
    """The same batch with an upstream gradient on sampled pixels of one view
    of a 1.5M-surfel scene and one of a 304k-surfel scene (zero elsewhere):
    every surfel and env texel gradient of those scenes against the oracle."""
    import torch
    sc = S.uneven_scenes()
    r = _renderer(sc)
    r.forward()
    torch.cuda.synchronize()
    rng = np.random.default_rng(2)
    G = np.zeros((r.n_pixels, 13))
    cache, refs = {}, []
    for v in (17, 13):                       # scene 4 (1.5M surfels), scene 3 (304k)
        sl = r.view_slice(v)
        cov = np.where(r.rgba[sl][:, 3].cpu().numpy() > 0)[0]
        pix = np.unique(np.concatenate([rng.choice(cov, 250, replace=False),
                                        rng.choice(sl.stop - sl.start, 30, replace=False)])).astype(np.int32)
        ref0 = _parity.oracle_view(sc, v, r.prm, pix=pix, env_cache=cache)
        pix = pix[~_parity.ambiguous(ref0["margin"])]
        Gs = rng.normal(size=(pix.size, 13))
        refs.append((v, _parity.oracle_view(sc, v, r.prm, pix=pix, G=Gs, env_cache=cache)))
        G[sl.start + pix] = Gs
    d_rgba = torch.from_numpy(G[:, :4].astype(np.float32)).cuda().contiguous()
    d_aov = torch.from_numpy(np.ascontiguousarray(G[:, 4:].T).astype(np.float32)).cuda()
    r.zero_grads()
    r.backward(d_rgba, d_aov)
    torch.cuda.synchronize()
    assert r.read_status() == 0
    for v, ref in refs:
        k = sc.cameras[v].scene
        s0, s1 = int(sc.scene_offsets[k]), int(sc.scene_offsets[k + 1])
        gpu = {f: r.grads[f][s0:s1].cpu().numpy().astype(np.float64) for f in FIELDS[:-1]}
        gpu["env"] = r.d_env[k].cpu().numpy().astype(np.float64)
        refd = {f: ref["grad"][f].reshape(gpu[f].shape) for f in FIELDS[:-1]}
        refd["env"] = ref["grad"]["env"].reshape(gpu["env"].shape)
        gpu["_near"] = ref["lookup_margin"] < LOOKUP_MARGIN
        assert (np.abs(refd["pos"]).sum(1) > 0).sum() > 500
        _compare(gpu, refd)


def test_inverse_loop_loss_decreases():
    """The inverse-rendering loop at reduced size (ground truth 100k surfels
    in 16 targets of 256^2; 200k surfels initialised on a sphere of radius
    1.2 and a constant env; 4 views per iteration; L1 loss, fused Adam on every
    surfel parameter group and the env, at the loop's learning rates): over 40
    iterations the loss falls."""
    import torch
    from paper_2605_05876_gb300 import _lib as C
    from paper_2605_05876_gb300.api import Adam, Renderer, SURFEL_ACTIVATIONS, loss_l1
    B, T = 4, 16
    gt = S.loop_ground_truth(n=100_000, targets=T, res=256)
    rg = Renderer(S.Scene(gt.surfels, gt.scene_offsets, gt.envs, gt.cameras[:B], "gt"), with_backward=False)
    HW = rg.n_pixels // B
    targets = torch.empty(T, HW, 4, device="cuda")
    for b0 in range(0, T, B):
        rg.set_cameras(gt.cameras[b0:b0 + B])
        rg.forward()
        targets[b0:b0 + B] = rg.rgba.view(B, HW, 4)
    surf, env0 = S.loop_init(n=200_000, env_w=256)
    r = Renderer(S.Scene(surf, np.array([0, surf.n], np.int64), [env0], gt.cameras[:B], "loop"), capacity_slack=2.0)
    r.zero_grads()
    lr = {"pos": 1.6e-4, "quat": 1e-3, "log_scale": 5e-3, "albedo": 2.5e-3, "roughness": 2.5e-3,
          "metallic": 2.5e-3}
    groups = {}
    for k, act in SURFEL_ACTIVATIONS.items():
        a = r.params_t[k]
        if act == C.SS_ACT_SIGMOID:
            x = a.clamp(1e-4, 1 - 1e-4)
            groups[k] = (torch.log(x / (1 - x)).contiguous(), r.grads[k], a, lr[k], act)
        else:
            groups[k] = (a, r.grads[k], None, lr[k], act)
    groups["env"] = (r.env, r.d_env, None, 1e-2, C.SS_ACT_CLAMP0)
    opt = Adam(groups)
    d_rgba = torch.empty(B * HW, 4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    order = np.random.default_rng(5).permutation(np.tile(np.arange(T), 12)).reshape(-1, B)
    losses = []
    for it in range(40):
        idx = order[it % order.shape[0]]
        r.set_cameras([gt.cameras[int(i)] for i in idx])
        tb = targets[torch.from_numpy(idx).cuda()].reshape(-1, 4)
        r.prefilter_env()
        r.forward()
        loss_l1(r.rgba, tb, d_rgba, loss, scale=1.0 / d_rgba.numel())
        r.zero_grads()
        r.backward(d_rgba, None)
        opt.step()
        losses.append(float(loss.item()))
    assert r.read_status() == 0
    assert all(np.isfinite(losses))
    first, last = np.mean(losses[:5]), np.mean(losses[-5:])
    print(f"L1 loss: first iterations {first:.4f}, last {last:.4f}")
    assert last < 0.97 * first
    assert np.mean(losses[20:25]) < first     # falling along the way, not only at the end
