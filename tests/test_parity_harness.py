"""The comparison the GPU parity tests rely on (tests/_parity.py), checked on
the CPU with planted deviations: an FP32 rounding of the oracle's own render
passes; a value just outside the image tolerance is flagged, one just inside
is not; at a pixel whose decision is within rounding of flipping, a value
matching either outcome passes (the other one counted as a flip) and one
matching neither fails.  Nothing here uses the CUDA path."""
import numpy as np
import pytest

from oracle import model as M
from tests import _parity, _tiny


@pytest.fixture(scope="module")
def view():
    rng = np.random.default_rng(61)
    surf = _tiny.random_scene(rng, n=60, spread=0.4, scale=(0.03, 0.1))
    cam = _tiny.front_camera(res=24)
    prm = M.Params()
    env = M.prepare_env(_tiny.lognormal_env(rng), prm, lut_nq=64)
    out = M.render_view(surf, cam, env, prm)
    ref = np.concatenate([out["rgba"], out["aov"]], 1)
    return out, ref, cam


def test_fp32_rounding_of_the_oracle_passes(view):
    out, ref, _ = view
    gpu = ref.astype(np.float32).astype(np.float64)
    n_bad, msg = _parity.compare(gpu, ref, np.zeros(ref.shape[0], bool))
    assert n_bad == 0, msg


def test_deviation_past_the_tolerance_is_flagged(view):
    _, ref, _ = view
    none = np.zeros(ref.shape[0], bool)
    big = np.argwhere(np.abs(ref[:, :9]) > 0.05)[0]            # a relative-tolerance entry
    small = np.argwhere((np.abs(ref[:, :9]) < 5e-3) & (np.abs(ref[:, :9]) > 0))[0]   # an absolute one
    for (p, c), tol in ((big, _parity.RTOL * abs(ref[tuple(big)])), (small, _parity.ATOL)):
        for factor, expect in ((1.5, 1), (0.5, 0)):
            gpu = ref.copy()
            gpu[p, c] += factor * tol
            assert _parity.compare(gpu, ref, none)[0] == expect, (p, c, factor)
    # a normal component is measured against the composited normal's length
    p = int(np.argmax(np.linalg.norm(ref[:, _parity.NORMAL_COLS], axis=1)))
    ln = np.linalg.norm(ref[p, _parity.NORMAL_COLS])
    for factor, expect in ((1.5, 1), (0.5, 0)):
        gpu = ref.copy()
        gpu[p, 9] += factor * _parity.RTOL * ln
        assert _parity.compare(gpu, ref, none)[0] == expect
    # set aside as ambiguous, the same deviation is left to check_variants
    gpu = ref.copy()
    gpu[big[0], big[1]] += 10 * _parity.RTOL * abs(ref[tuple(big)])
    amb = none.copy()
    amb[big[0]] = True
    assert _parity.compare(gpu, ref, amb)[0] == 0


def test_ambiguous_pixel_accepts_either_outcome_and_nothing_else(view, monkeypatch):
    out, ref, cam = view
    # the covered pixel whose nearest support-cutoff test is closest to the
    # boundary; a cutoff tolerance above its margin makes that test flippable
    cov = out["rgba"][:, 3] > 0
    m = np.where(cov, out["margin"][:, 0], np.inf)
    pid = int(np.argmin(m))
    tol = 2.0 * m[pid]
    assert 0 < tol < 0.05
    monkeypatch.setattr(_parity, "M_CUT", tol)
    op = M.Params()
    variants, complete = M.decision_variants(out["records"], out["rect"], cam.width, op, pid, tol, 0.0, 0.0)
    assert complete and len(variants) == 2
    vals = [M.composite_variant(out["records"], cam.width, op, pid, *v) for v in variants]
    assert not _parity.within(vals[1], vals[0]).all()           # the two outcomes differ visibly
    amb = np.zeros(ref.shape[0], bool)
    amb[pid] = True
    gpu = ref.copy()
    assert _parity.check_variants(gpu, out, amb) == (1, 0)
    gpu[pid] = vals[1]
    assert _parity.check_variants(gpu, out, amb) == (1, 1)      # the other outcome: a flip
    gpu[pid] = 0.5 * (vals[0] + vals[1])
    with pytest.raises(AssertionError, match="matches none"):
        _parity.check_variants(gpu, out, amb)
    # the flip budget: one pixel in a small test, a fraction in a large one
    _parity.check_flip_fraction(1, 576)
    with pytest.raises(AssertionError):
        _parity.check_flip_fraction(2, 576)
    _parity.check_flip_fraction(2, 20000)
    with pytest.raises(AssertionError):
        _parity.check_flip_fraction(3, 20000)


def _grad_blocks(rng, n=500, env_shape=(1, 32, 64, 3)):
    ref = {"pos": rng.normal(size=(n, 3)), "quat": rng.normal(size=(n, 4)), "log_scale": rng.normal(size=(n, 2)),
           "albedo": rng.normal(size=(n, 3)), "roughness": rng.normal(size=n), "metallic": rng.normal(size=n),
           "env": rng.normal(size=env_shape)}
    gpu = {k: v.astype(np.float32).astype(np.float64) for k, v in ref.items()}
    gpu["_near"] = np.zeros(n, bool)
    return gpu, ref


def test_gradient_comparison_flags_block_and_element_deviations():
    """The gradient bound of the backward parity tests (per block
    |g - g_ref| / |g_ref| <= 1e-4, per element 1e-3 |g_ref| + 1e-5 max|g_ref|):
    FP32 rounding passes; one element at 1.5x its bound, or a whole block
    scaled by 1 + 2e-4, fails; 0.5x and 1 + 5e-5 pass; a surfel set aside near
    a lookup boundary is not compared, but more than 1% of them fail."""
    from tests import test_gpu_backward as B
    rng = np.random.default_rng(62)
    gpu, ref = _grad_blocks(rng)
    B._compare(gpu, ref)
    amax = np.abs(ref["albedo"]).max()
    i = 7
    bound = B.ELEM_RTOL * abs(ref["albedo"][i, 1]) + B.ELEM_ATOL * amax
    for factor, fails in ((1.5, True), (0.5, False)):
        g = dict(gpu, albedo=gpu["albedo"].copy())
        g["albedo"][i, 1] = ref["albedo"][i, 1] + factor * bound
        if fails:
            with pytest.raises(AssertionError, match="albedo"):
                B._compare(g, ref)
        else:
            B._compare(g, ref)
    for factor, fails in ((1 + 2e-4, True), (1 + 5e-5, False)):
        g = dict(gpu, metallic=ref["metallic"] * factor)
        if fails:
            with pytest.raises(AssertionError, match="metallic"):
                B._compare(g, ref)
        else:
            B._compare(g, ref)
    # a position compares against the surfel's vector norm, not the component:
    # a small component may move by half the norm-relative bound, far more
    # than a component-relative bound would allow
    r2 = dict(ref, pos=ref["pos"].copy())
    r2["pos"][3] = [1e-4, 1.0, 1.0]
    g = dict(gpu, pos=r2["pos"].copy())
    dev = 0.5 * B.ELEM_RTOL * np.linalg.norm(r2["pos"][3])
    assert dev > B.ELEM_RTOL * 1e-4 + B.ELEM_ATOL * np.abs(r2["pos"]).max()
    g["pos"][3, 0] += dev
    B._compare(g, r2)
    # near a lookup boundary: set aside, up to 1% of the surfels
    g = dict(gpu, roughness=gpu["roughness"].copy(), _near=gpu["_near"].copy())
    g["roughness"][11] += 1.0
    g["_near"][11] = True
    B._compare(g, ref)
    g["_near"][:10] = True
    with pytest.raises(AssertionError, match="near a lookup"):
        B._compare(g, ref)
    # a block the oracle says is zero must be zero
    z = dict(ref, metallic=np.zeros_like(ref["metallic"]))
    g = dict(gpu, metallic=np.zeros_like(ref["metallic"]))
    B._compare(g, z)
    g["metallic"] = g["metallic"].copy()
    g["metallic"][0] = 1e-30
    with pytest.raises(AssertionError):
        B._compare(g, z)
