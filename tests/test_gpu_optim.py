"""GPU parity of the fused Adam step and the L1 loss against the FP64 oracle
(oracle/optim.py), called through the C ABI."""
import numpy as np
import pytest

from oracle import optim as O

pytestmark = pytest.mark.gpu


def test_adam_matches_oracle_over_steps():
    import torch
    from paper_2605_05876_gb300 import _lib
    from paper_2605_05876_gb300.api import Adam
    rng = np.random.default_rng(3)
    specs = {"pos": (1001, 1.6e-4, O.IDENTITY), "albedo": (3 * 777, 2.5e-3, O.SIGMOID),
             "env": (64 * 32 * 3 + 2, 1e-2, O.CLAMP0), "empty": (0, 1e-3, O.IDENTITY)}
    raw = {k: rng.normal(size=n) * (0.01 if a == O.CLAMP0 else 1.0) for k, (n, _, a) in specs.items()}
    raw["env"] = np.abs(raw["env"])
    dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda") for k, v in raw.items()}
    grads = {k: torch.zeros_like(v) for k, v in dev.items()}
    acts = {k: (torch.zeros_like(v) if specs[k][2] == O.SIGMOID else None) for k, v in dev.items()}
    # an offset view tests the unaligned path
    dev["pos_off"] = torch.tensor(rng.normal(size=400), dtype=torch.float32, device="cuda")[1:]
    grads["pos_off"] = torch.zeros_like(dev["pos_off"]); acts["pos_off"] = None
    specs["pos_off"] = (399, 1e-3, O.IDENTITY)
    groups = {k: (dev[k], grads[k], acts[k], specs[k][1], specs[k][2]) for k in dev}
    opt = Adam(groups)
    ref = {k: [dev[k].double().cpu().numpy(), 0.0, 0.0] for k in dev}
    for t in range(1, 6):
        for k in dev:
            g = rng.normal(size=dev[k].numel()).astype(np.float32) * 10.0 ** rng.uniform(-4, 1)
            grads[k].copy_(torch.from_numpy(g))
            th, m, v = ref[k]
            th, m, v, a = O.adam_step(th, g.astype(np.float64), m, v, t, specs[k][1], specs[k][2])
            ref[k] = [th, m, v]
        opt.step()
        torch.cuda.synchronize()
        for k in dev:
            got = dev[k].double().cpu().numpy()
            th = ref[k][0]
            # float32 state, up to 5 steps of size ~lr: error a few ulp of theta plus lr * 1e-5
            tol = 4e-7 * np.abs(th) + specs[k][1] * 1e-4 + 1e-12
            assert np.all(np.abs(got - th) <= tol), (k, t, np.abs(got - th).max())
            if acts[k] is not None:
                assert np.allclose(acts[k].double().cpu().numpy(), O.sigmoid(th), rtol=1e-6, atol=1e-7)
    assert (dev["env"] >= 0).all()


def test_adam_rejects_bad_groups():
    import ctypes
    from paper_2605_05876_gb300 import _lib
    lib = _lib.lib()
    g = (_lib.ss_adam_group * 1)()
    g[0].n = 10          # NULL pointers with n > 0
    p = _lib.ss_adam_params(); lib.ss_default_adam(ctypes.byref(p))
    assert lib.ss_adam_step(g, 1, ctypes.byref(p), None) == _lib.SS_ERR_INVALID_ARG
    p.step = 0
    g[0].n = 0
    assert lib.ss_adam_step(g, 1, ctypes.byref(p), None) == _lib.SS_ERR_INVALID_ARG


def test_l1_loss_matches_oracle():
    import torch
    from paper_2605_05876_gb300.api import loss_l1
    rng = np.random.default_rng(4)
    for n in (1, 1000, 3 * 1024 * 1024 + 7):
        out = rng.normal(size=n).astype(np.float32)
        tgt = rng.normal(size=n).astype(np.float32)
        tgt[: n // 10] = out[: n // 10]
        o, t = torch.from_numpy(out).cuda(), torch.from_numpy(tgt).cuda()
        d = torch.empty_like(o)
        L = torch.zeros(1, device="cuda")
        for _ in range(2):   # twice: the device-side counter must reset itself
            loss_l1(o, t, d, L, scale=1.0 / n)
        torch.cuda.synchronize()
        # the FP32 differences decide the sign: compare with the oracle on them
        ref_L, ref_d = O.loss_l1(out.astype(np.float64), tgt.astype(np.float64), 1.0 / n)
        assert abs(L.item() - ref_L) <= 1e-6 * abs(ref_L) + 1e-12
        assert np.array_equal(d.cpu().numpy(), ref_d.astype(np.float32))


def test_sil_iou_matches_oracle():
    """Silhouette soft-IoU loss (Eq. sil_loss) per view against the oracle,
    three views of different sizes, on top of an existing d_rgba (the
    gradient is added to the alpha channel only)."""
    import torch
    from oracle import optim as O
    from paper_2605_05876_gb300.api import loss_sil_iou
    rng = np.random.default_rng(11)
    sizes = [37 * 29, 64 * 64, 5]
    P = sum(sizes)
    A = rng.uniform(0, 1, P) * (rng.uniform(size=P) < 0.7)
    M = (rng.uniform(size=P) < 0.5).astype(np.float64) * rng.uniform(0.5, 1.0, P)
    rgba = np.concatenate([rng.normal(size=(P, 3)), A[:, None]], 1).astype(np.float32)
    base = rng.normal(size=(P, 4)).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    d = torch.from_numpy(base.copy()).cuda()
    loss = torch.zeros(3, device="cuda")
    loss_sil_iou(torch.from_numpy(rgba).cuda(), torch.from_numpy(M.astype(np.float32)).cuda(),
                 torch.from_numpy(offs).cuda(), d, loss, scale=0.5)
    torch.cuda.synchronize()
    dg = d.cpu().numpy()
    assert np.array_equal(dg[:, :3], base[:, :3])          # colour channels untouched
    for v in range(3):
        sl = slice(offs[v], offs[v + 1])
        ref_l, ref_g = O.loss_sil_iou(rgba[sl, 3].astype(np.float64), M[sl].astype(np.float32), 0.5)
        assert abs(loss[v].item() - ref_l) <= 1e-6 * max(1.0, abs(ref_l))
        np.testing.assert_allclose(dg[sl, 3] - base[sl, 3], ref_g, rtol=1e-5, atol=3e-7)
