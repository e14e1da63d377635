"""Checkpoint and resume of the inverse-rendering loop: with the
deterministic backward, a loop restored from a checkpoint (surfel
parameters, env map, Adam's step count, raw values and moments, saved with
torch.save) continues with bit for bit the losses and parameters of the run
that was never interrupted."""
import io

import numpy as np
import pytest

from paper_2605_05876_gb300 import scenes as S

pytestmark = pytest.mark.gpu

B, T = 2, 6


def _setup(gt, targets):
    import torch
    from paper_2605_05876_gb300 import _lib as C
    from paper_2605_05876_gb300.api import Adam, Renderer, SURFEL_ACTIVATIONS
    surf, env0 = S.loop_init(n=30_000, env_w=128)
    r = Renderer(S.Scene(surf, np.array([0, surf.n], np.int64), [env0], gt.cameras[:B], "loop"), capacity_slack=2.0,
                 params=dict(deterministic=1))
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
    return r, Adam(groups)


def _iterate(r, opt, gt, targets, its):
    import torch
    from paper_2605_05876_gb300.api import loss_l1
    order = np.random.default_rng(5).permutation(np.tile(np.arange(T), 4)).reshape(-1, B)
    d_rgba = torch.empty(r.n_pixels, 4, device="cuda")
    loss = torch.zeros(1, device="cuda")
    out = []
    for it in its:
        idx = order[it % order.shape[0]]
        r.set_cameras([gt.cameras[int(i)] for i in idx])
        tb = targets[torch.from_numpy(idx).cuda()].reshape(-1, 4)
        r.prefilter_env()
        r.forward()
        loss_l1(r.rgba, tb, d_rgba, loss, scale=1.0 / d_rgba.numel())
        r.zero_grads()
        r.backward(d_rgba, None)
        opt.step()
        out.append(loss.clone())
    torch.cuda.synchronize()
    assert r.read_status() == 0
    return [float(x.item()) for x in out]


def test_resumed_loop_continues_bit_for_bit():
    import torch
    from paper_2605_05876_gb300.api import Renderer
    gt = S.loop_ground_truth(n=20_000, targets=T, res=96)
    rg = Renderer(S.Scene(gt.surfels, gt.scene_offsets, gt.envs, gt.cameras[:B], "gt"), with_backward=False)
    HW = rg.n_pixels // B
    targets = torch.empty(T, HW, 4, device="cuda")
    for b0 in range(0, T, B):
        rg.set_cameras(gt.cameras[b0:b0 + B])
        rg.forward()
        targets[b0:b0 + B] = rg.rgba.view(B, HW, 4)
    # the uninterrupted run
    r, opt = _setup(gt, targets)
    whole = _iterate(r, opt, gt, targets, range(6))
    final = {k: v.clone() for k, v in r.params_t.items()}
    # three iterations, a checkpoint through torch.save, a fresh loop resumed from it
    r1, opt1 = _setup(gt, targets)
    first = _iterate(r1, opt1, gt, targets, range(3))
    buf = io.BytesIO()
    torch.save({"renderer": r1.state_dict(), "adam": opt1.state_dict()}, buf)
    del r1, opt1
    buf.seek(0)
    ck = torch.load(buf)
    r2, opt2 = _setup(gt, targets)
    r2.load_state_dict(ck["renderer"])
    opt2.load_state_dict(ck["adam"])
    rest = _iterate(r2, opt2, gt, targets, range(3, 6))
    assert first + rest == whole
    for k, v in final.items():
        assert torch.equal(r2.params_t[k], v), k
