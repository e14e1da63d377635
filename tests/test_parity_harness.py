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
