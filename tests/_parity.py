"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

from oracle import model as M

# image tolerance: 1e-4 relative per pixel, 1e-5 absolute where |value| < 1e-2
RTOL, ATOL, SMALL = 1e-4, 1e-5, 1e-2
# decisions closer than this to flipping are set aside (rounding of FP32 vs FP64)
M_CUT, M_GAP, M_BOX = 1e-5, 1e-5, 2e-3


MIP_MODES = {0: "centre", 1: "none", 2: "pixel"}


def oracle_params(prm) -> M.Params:
    return M.Params(r_cut=float(prm.r_cut), sigma_f=float(prm.sigma_f), gamma=float(prm.gamma),
                    k_max=int(prm.k_max), z_near=float(prm.z_near), bg=tuple(float(b) for b in prm.bg),
                    lut_n=int(prm.lut_n), mip_mode=MIP_MODES[int(prm.mip_mode)], cons=bool(prm.cons))


def oracle_view(scene, v, prm, env_levels=6, pix=None, G=None, env_cache=None):
    cam = scene.cameras[v]
    s0, s1 = int(scene.scene_offsets[cam.scene]), int(scene.scene_offsets[cam.scene + 1])
    surf = scene.surfels.subset(slice(s0, s1))
    op = oracle_params(prm)
    op.env_levels = env_levels
    key = cam.scene
    if env_cache is not None and key in env_cache:
        env = env_cache[key]
    else:
        env = M.prepare_env(scene.envs[cam.scene], op)
        if env_cache is not None:
            env_cache[key] = env
    return M.render_view(surf, cam, env, op, pix=pix, G=G)


def ambiguous(margin):
    return (margin[:, 0] < M_CUT) | (margin[:, 1] < M_GAP) | (margin[:, 2] < M_BOX)


# pixels set aside by `ambiguous` may be at most this fraction of a test's
# pixels (a bound on the rounding-scale decisions; each is still checked by
# check_variants)
MAX_AMBIGUOUS_FRACTION = 1e-2
# pixels where the GPU took another outcome of a near-tie decision than the
# FP64 oracle (both correct): at most this fraction of the checked pixels,
# or one pixel in a test of fewer than 1e4 pixels
MAX_FLIP_FRACTION = 1e-4


# columns of the composited normal in a [.., 13] row (rgba, then the AOVs:
# albedo 3, roughness, metallic, normal 3, depth; a 14th column holds the
# depth-consolidation term when it is on)
NORMAL_COLS = slice(9, 12)


def scale_of(r):
    """The magnitude each value's tolerance is relative to: the value itself,
    except the normal AOV, which is a direction (renormalised per layer,
    Sec. 4.2.3): its components are sums of unit-length terms that cancel, so
    its FP32 rounding scales with the composited normal's length, and all
    three components are measured against that length."""
    sc = np.abs(r).astype(np.float64, copy=True)
    if r.shape[-1] >= 13:
        sc[..., NORMAL_COLS] = np.linalg.norm(r[..., NORMAL_COLS], axis=-1, keepdims=True)
    return sc


def within(g, r):
    """Image tolerance: 1e-4 relative, 1e-5 absolute where the magnitude
    (scale_of) is below 1e-2."""
    sc = scale_of(r)
    return np.abs(g - r) <= np.where(sc < SMALL, ATOL, RTOL * sc)


def check_variants(gpu, ref, amb, pix=None, prm=None):
    """Pixels with a decision within rounding of flipping (FP32 vs FP64)
    have several correct results.  For each, the oracle enumerates every
    outcome of those decisions (a near-cutoff or near-rectangle-edge surfel
    in or out, a near-tie gap test taken or not) and composites each; the
    GPU's values must match one of them at the strict image tolerance.
    gpu: [P, 13] rows of the queried pixels; ref: the oracle's render_view
    result for the same pixels (pix = their ids, None for all).  Returns
    (pixels checked, pixels where the GPU matched an outcome other than the
    oracle's own)."""
    rows = np.where(amb)[0]
    if rows.size == 0:
        return 0, 0
    flipped = 0
    recs, rect, W = ref["records"], ref["rect"], ref["width"]
    op = oracle_params(prm) if prm is not None else M.Params()
    ids = np.arange(gpu.shape[0]) if pix is None else np.asarray(pix)
    for i in rows:
        pid = int(ids[i])
        variants, complete = M.decision_variants(recs, rect, W, op, pid, M_CUT, M_GAP, M_BOX)
        assert complete, f"pixel {pid}: too many near-tie decisions to enumerate"
        vals = [M.composite_variant(recs, W, op, pid, sid, lay, nl) for sid, lay, nl in variants]
        ok = [bool(within(gpu[i], v).all()) for v in vals]
        assert any(ok), (f"pixel {pid}: the GPU matches none of the {len(vals)} outcomes of its near-tie "
                         f"decisions; gpu={gpu[i][:4]} oracle={[v[:4] for v in vals[:4]]}")
        assert within(vals[0], np.concatenate([ref["rgba"][i], ref["aov"][i]])).all()   # variant 0 = the oracle's
        flipped += 0 if ok[0] else 1
    return rows.size, flipped


def check_flip_fraction(flipped, n_pixels, what=""):
    assert flipped <= max(1, MAX_FLIP_FRACTION * n_pixels), (
        f"{what}: the GPU took another outcome of a near-tie decision at {flipped} of {n_pixels} pixels")


def compare(gpu, ref, amb, what=""):
    """gpu, ref: [P, C] arrays.  Returns the number of failing entries and a
    message; ambiguous pixels are excluded (check_variants checks them)."""
    ok = ~amb
    g, r = gpu[ok], ref[ok]
    bad = ~within(g, r)
    n_bad = int(bad.sum())
    msg = ""
    if n_bad:
        idx = np.argwhere(bad)[:5]
        msg = f"{what}: {n_bad} entries out of tolerance, e.g. " + ", ".join(
            f"(p{i},c{c}) gpu={g[i, c]:.7g} ref={r[i, c]:.7g}" for i, c in idx)
    return n_bad, msg
