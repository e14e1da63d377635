"""GPU adaptive density control (Sec. 3.6.2; appendix on splitting and
pruning surfels) against the oracle's brute-force evaluation, through the C
ABI: the same-orientation neighbour statistics of the hashed grid, the
split / prune plan and the compaction that writes the new surfels."""
import ctypes

import numpy as np
import pytest

from oracle import density as D
from paper_2605_05876_gb300 import scenes as S

pytestmark = pytest.mark.gpu

# distances: FP32 squared distances, square roots summed in FP32 in another
# order than the oracle's FP64 mean
DIST_RTOL = 2e-6
# orientation tests closer than this to cos_min may pick another set on the
# GPU (FP32 normals from FP32 quaternions against the FP64 ones)
ORIENT_MARGIN = 1e-4


def _lib():
    from paper_2605_05876_gb300 import _lib as C
    return C, C.lib()


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


def _surfels_struct(C, tensors):
    return C.ss_surfels(*(ctypes.c_void_p(tensors[k].data_ptr()) if k in tensors else ctypes.c_void_p(0)
                          for k in ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")))


def gpu_neighbours(pos, quat, offsets, **kw):
    import torch
    C, L = _lib()
    p = C.ss_density_params()
    L.ss_default_density(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    n = int(offsets[-1])
    t = {"pos": _dev(np.asarray(pos, np.float32)), "quat": _dev(np.asarray(quat, np.float32))}
    mean = torch.empty(max(n, 1), device="cuda")
    nn = torch.empty(max(n, 1), device="cuda")
    flags = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    nb = ctypes.c_size_t()
    assert L.ss_density_workspace_size(n, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    offs = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.ss_density_neighbours(ctypes.byref(_surfels_struct(C, t)), offs, len(offsets) - 1, ctypes.byref(p),
                                 ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(nn.data_ptr()),
                                 ctypes.c_void_p(flags.data_ptr()), ctypes.c_void_p(ws.data_ptr()), nb.value, st)
    assert rc == 0
    torch.cuda.synchronize()
    return mean[:n].cpu().numpy(), nn[:n].cpu().numpy(), flags[:n].cpu().numpy()


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _check_neighbours(pos, quat, offsets, k, cos_min, cell, max_rings, expect_exact=True):
    pos, quat = _f32(pos), _f32(quat)
    mean, nn, flags = gpu_neighbours(pos, quat, offsets, k=k, cos_min=cos_min, cell=cell, max_rings=max_rings)
    rmean, rcnt, rnn = D.neighbours(pos, quat, offsets, k=k, cos_min=cos_min)
    margin = D.orientation_margins(pos, quat, offsets, k, cos_min)
    sure = margin > ORIENT_MARGIN
    assert sure.mean() > 0.95
    exact_mean = (flags & 1) == 0
    exact_nn = (flags & 2) == 0
    if expect_exact:
        assert exact_mean.all() and exact_nn.all()
    # certain values equal the brute-force ones ...
    m = exact_mean & sure
    assert np.all(rcnt[m] == k)
    np.testing.assert_allclose(mean[m], rmean[m], rtol=DIST_RTOL)
    np.testing.assert_allclose(nn[exact_nn], rnn[exact_nn], rtol=DIST_RTOL)
    # ... and bounds stay below them: d_bar of the k nearest, counting the
    # missing ones at infinity when fewer than k exist
    b = ~exact_mean & sure
    full = np.where(rcnt[b] == k, rmean[b], np.inf)
    assert np.all(mean[b] <= full * (1 + DIST_RTOL))
    assert np.all(nn[~exact_nn] <= rnn[~exact_nn] * (1 + DIST_RTOL))
    return flags


def test_neighbours_two_scenes_match_oracle():
    """A sphere of surfels (scene 0) and a random cloud with random normals
    (scene 1) in one call: exact statistics everywhere, scenes apart."""
    rng = np.random.default_rng(11)
    spos, squat, _ = S.sphere_surfels(rng, 5000, radius=1.0, scale=0.02)
    cpos = rng.uniform(-1, 1, size=(2500, 3))
    cq = S.tangent_quats(rng.normal(size=(2500, 3)), rng)
    pos = np.concatenate([spos, cpos])
    quat = np.concatenate([squat, cq])
    _check_neighbours(pos, quat, [0, 5000, 7500], k=8, cos_min=0.5, cell=0.12, max_rings=8)


@pytest.mark.parametrize("k,cos_min", [(1, -2.0), (4, 0.0), (16, 0.9)])
def test_neighbours_k_and_orientation(k, cos_min):
    rng = np.random.default_rng(12 + k)
    spos, _, _ = S.sphere_surfels(rng, 3000, radius=0.7, scale=0.02)
    q = S.tangent_quats(spos + rng.normal(scale=0.4, size=spos.shape), rng)   # noisy normals
    # with the strictest test some surfels have fewer than k same-orientation
    # neighbours within the rings: bounds there, checked as such
    flags = _check_neighbours(spos, q, [0, 3000], k=k, cos_min=cos_min, cell=0.08, max_rings=12,
                              expect_exact=cos_min < 0.9)
    assert (flags != 0).mean() < 0.05


def test_neighbours_bounds_when_the_search_stops_early():
    """One ring of small cells: many queries end before their k-th neighbour
    is certain; their values are lower bounds, the rest exact.  A scene of
    three surfels has fewer than k neighbours per surfel."""
    rng = np.random.default_rng(14)
    cpos = rng.uniform(-1, 1, size=(3000, 3))
    cq = S.tangent_quats(rng.normal(size=(3000, 3)), rng)
    pos = np.concatenate([cpos, [[5.0, 5, 5], [5.1, 5, 5], [5.3, 5, 5]]])
    quat = np.concatenate([cq, np.tile([1.0, 0, 0, 0], (3, 1))])
    flags = _check_neighbours(pos, quat, [0, 3000, 3003], k=8, cos_min=0.5, cell=0.05, max_rings=1,
                              expect_exact=False)
    assert (flags & 1).mean() > 0.3
    assert np.all(flags[3000:] & 1)


def test_neighbours_at_full_size_sampled():
    """The 1M-surfel displaced sphere with the default cell rule: sampled
    queries against a brute force over all surfels; few bounds."""
    import torch
    rg, ra = S.rng_streams(3, 2)
    n = 1_000_000
    pos, quat, ls, *_ = S.displaced_sphere_surfels(rg, ra, n)
    pos, quat = _f32(pos), _f32(quat)
    cell = float(2.0 * np.exp(np.median(ls.max(1))))
    mean, nn, flags = gpu_neighbours(pos, quat, [0, n], cell=cell)
    assert (flags != 0).mean() < 1e-3
    rng = np.random.default_rng(15)
    idx = rng.choice(n, 200, replace=False)
    ref = D.neighbours_of(pos, quat, [0, n], idx, k=8, cos_min=0.5)
    ok = (flags[idx] == 0) & (ref[:, 3] > ORIENT_MARGIN) & (ref[:, 1] == 8)
    assert ok.sum() > 190
    np.testing.assert_allclose(mean[idx][ok], ref[ok, 0], rtol=DIST_RTOL)
    np.testing.assert_allclose(nn[idx][flags[idx] == 0], ref[flags[idx] == 0, 2], rtol=DIST_RTOL)
    del torch


def _plan_inputs(rng, n):
    """Log-scales, statistic and neighbour values with every comparison of the
    plan well away from its threshold (at least 1 % relative)."""
    ls = rng.normal(-4.0, 0.5, size=(n, 2)).astype(np.float32)
    s_max = np.exp(ls.astype(np.float64).max(1))
    mean = (s_max * np.where(rng.uniform(size=n) < 0.5, rng.uniform(0.3, 0.99, n), rng.uniform(1.01, 3, n)))
    nn = (3 * s_max * np.where(rng.uniform(size=n) < 0.9, rng.uniform(0.01, 0.99, n), rng.uniform(1.01, 2, n)))
    views = rng.integers(1, 9, n).astype(np.float32)
    g_norm = (rng.uniform(0, 2e-3, n) * views).astype(np.float32)
    g_norm[rng.uniform(size=n) < 0.05] = 0.0
    flags = np.where(rng.uniform(size=n) < 0.05, rng.integers(1, 4, n), 0).astype(np.int32)
    return ls, g_norm, views, mean.astype(np.float32), nn.astype(np.float32), flags


@pytest.mark.parametrize("n,ops", [(0, 7), (1, 7), (4099, 7), (50_000, 7), (50_000, 1), (50_000, 6)])
def test_plan_apply_compact_match_oracle(n, ops):
    """Actions and output offsets bit-exact; the new surfels: copied fields
    bit-exact, children within FP32 rounding of the oracle's; compacted rows
    bit-exact (copied or zero)."""
    import torch
    C, L = _lib()
    rng = np.random.default_rng(21 + n + ops)
    ls, g_norm, views, mean, nn, flags = _plan_inputs(rng, n)
    tau_g = 1e-3
    ract, roff = D.plan(ls, g_norm, views, mean, nn, flags, tau_g=tau_g, r_cut=3.0, ops=ops)
    p = C.ss_density_params()
    L.ss_default_density(ctypes.byref(p))
    p.cell, p.tau_g, p.ops = 1.0, tau_g, ops
    d = {k: _dev(v) for k, v in dict(ls=ls, g=g_norm, v=views, m=mean, nn=nn, f=flags).items()}
    act = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    nb = ctypes.c_size_t()
    assert L.ss_density_workspace_size(n, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    assert L.ss_density_plan(vp(d["ls"]), vp(d["g"]), vp(d["v"]), vp(d["m"]), vp(d["nn"]), vp(d["f"]), n,
                             ctypes.byref(p), vp(act), vp(off), vp(ws), nb.value, st) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(act[:n].cpu().numpy(), ract)
    np.testing.assert_array_equal(off.cpu().numpy(), roff)
    if n == 0:
        return
    n_new = int(roff[-1])
    fields = {"pos": rng.normal(size=(n, 3)).astype(np.float32), "quat": rng.normal(size=(n, 4)).astype(np.float32),
              "log_scale": ls, "albedo": rng.uniform(size=(n, 3)).astype(np.float32),
              "roughness": rng.uniform(size=n).astype(np.float32), "metallic": rng.uniform(size=n).astype(np.float32)}
    tin = {k: _dev(v) for k, v in fields.items()}
    tout = {k: torch.full((max(n_new, 1),) + v.shape[1:], np.nan, device="cuda") for k, v in fields.items()}
    assert L.ss_density_apply(ctypes.byref(_surfels_struct(C, tin)), n, vp(act), vp(off), ctypes.c_float(0.7),
                              ctypes.byref(_surfels_struct(C, tout)), st) == 0
    rows = rng.normal(size=(n, 5)).astype(np.float32)
    trows = _dev(rows)
    outs = []
    for zero in (0, 1):
        o = torch.full((max(n_new, 1), 5), np.nan, device="cuda")
        assert L.ss_density_compact(vp(trows), 5, n, vp(act), vp(off), zero, vp(o), st) == 0
        outs.append(o[:n_new].cpu().numpy())
    torch.cuda.synchronize()
    ref = D.apply({k: v.astype(np.float64) for k, v in fields.items()}, ract)
    got = {k: v[:n_new].cpu().numpy() for k, v in tout.items()}
    for k in ("quat", "albedo", "roughness", "metallic"):
        np.testing.assert_array_equal(got[k], ref[k].astype(np.float32))
    np.testing.assert_allclose(got["pos"], ref["pos"], rtol=0, atol=1e-6 * max(1.0, np.abs(ref["pos"]).max()))
    np.testing.assert_allclose(got["log_scale"], ref["log_scale"], rtol=0, atol=2e-6 * 8)
    kept_rows = ract == D.KEEP
    np.testing.assert_array_equal(got["pos"][roff[:-1][kept_rows]], fields["pos"][kept_rows])
    np.testing.assert_array_equal(outs[0], D.compact_rows(rows, ract))
    np.testing.assert_array_equal(outs[1], D.compact_rows(rows, ract, zero_children=True))


def test_invalid_arguments_enqueue_nothing():
    """Host-side validation: bad parameters and a short workspace are
    rejected before anything is enqueued (no device access)."""
    import torch
    C, L = _lib()
    p = C.ss_density_params()
    L.ss_default_density(ctypes.byref(p))
    t = {"pos": torch.zeros(30, device="cuda"), "quat": torch.zeros(40, device="cuda")}
    offs = (ctypes.c_int64 * 2)(0, 10)
    buf = torch.zeros(10, device="cuda")
    fl = torch.zeros(10, dtype=torch.int32, device="cuda")
    nb = ctypes.c_size_t()
    L.ss_density_workspace_size(10, ctypes.byref(nb))
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    call = lambda q, size: L.ss_density_neighbours(ctypes.byref(_surfels_struct(C, t)), offs, 1, ctypes.byref(q),
                                                   vp(buf), vp(buf), vp(fl), vp(ws), size, None)
    assert call(p, nb.value) == C.SS_ERR_INVALID_ARG          # cell 0: the caller must choose it
    p.cell = 0.1
    assert call(p, nb.value - 1) == C.SS_ERR_WORKSPACE
    for field, bad in (("k", 0), ("k", 17), ("max_rings", 0), ("max_rings", 33), ("split_scale", 1.5),
                       ("ops", 8), ("r_cut", 0.0)):
        q = C.ss_density_params()
        ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
        setattr(q, field, bad)
        assert call(q, nb.value) == C.SS_ERR_INVALID_ARG, field
    torch.cuda.synchronize()


def test_densify_end_to_end():
    """Render, differentiate with the statistic, densify with Adam state:
    the counts add up, kept surfels are unchanged, children straddle their
    parents, and the renderer and the optimiser run on the new set."""
    import torch
    from paper_2605_05876_gb300 import _lib as C
    from paper_2605_05876_gb300.api import Adam, Renderer, SURFEL_ACTIVATIONS
    scene = S.sphere_4k(res=96)
    # every other surfel wider than its neighbours' spacing (about 0.08), so
    # that some qualify for a split
    scene.surfels.log_scale[::2] = np.float32(np.log(0.12))
    r = Renderer(scene, screen_grad=True)
    r.forward()
    r.zero_grads()
    g = torch.from_numpy(np.random.default_rng(3).normal(size=(r.n_pixels, 4)).astype(np.float32)).cuda()
    r.backward(g)
    groups = {}
    for k, act in SURFEL_ACTIVATIONS.items():
        a = r.params_t[k]
        if act == C.SS_ACT_SIGMOID:
            x = a.clamp(1e-4, 1 - 1e-4)
            groups[k] = (torch.log(x / (1 - x)).contiguous(), r.grads[k], a, 1e-3, act)
        else:
            groups[k] = (a, r.grads[k], None, 1e-3, act)
    opt = Adam(groups)
    opt.step()
    before = {k: v.clone() for k, v in r.params_t.items()}
    gbar = (r.screen_grad_norm / r.screen_grad_views.clamp(min=1)).cpu().numpy()
    dp = r.density_params(tau_g=float(np.quantile(gbar[gbar > 0], 0.5)))
    mean, nn, flags = r.density_neighbours(dp)
    action, off = r.density_plan(dp, mean, nn, flags)
    act = action.cpu().numpy()
    offs = off.cpu().numpy()
    res = r.densify(dp, adam=opt)
    assert res["after"] == res["kept"] + 2 * res["split"] and res["before"] == scene.surfels.n
    assert res["split"] > 0
    np.testing.assert_array_equal(np.bincount(act, minlength=3), [res["pruned"], res["kept"], res["split"]])
    new = {k: v.cpu().numpy() for k, v in r.params_t.items()}
    old = {k: v.cpu().numpy() for k, v in before.items()}
    kept = act == C.SS_ACTION_KEEP
    for k in new:
        np.testing.assert_array_equal(new[k][offs[:-1][kept]], old[k][kept])
    sp = np.where(act == C.SS_ACTION_SPLIT)[0]
    c0, c1 = new["pos"][offs[sp]], new["pos"][offs[sp] + 1]
    np.testing.assert_allclose((c0 + c1) / 2, old["pos"][sp], atol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(c0 - c1, axis=1), np.exp(old["log_scale"][sp].max(1)), rtol=1e-5)
    assert all(opt.moments[k][0].shape[0] == res["after"] for k in SURFEL_ACTIVATIONS)
    r.forward()
    r.zero_grads()
    r.backward(torch.zeros(r.n_pixels, 4, device="cuda"))
    opt.step()
    assert r.read_status() == 0
