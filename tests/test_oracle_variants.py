"""Pins of the oracle's enumeration of near-tie decisions
(``decision_variants``), which the parity tests use where a decision of
Algorithm 1 sits within rounding of flipping between FP32 and FP64.  Nothing
here uses the CUDA path."""
import numpy as np
import torch

from oracle import model as M
from paper_2605_05876_gb300 import scenes as S
from tests import _tiny


def _setup(surf, cam, env):
    prm = M.Params()
    st = M.prepare_env(env, prm, lut_nq=64)
    out = M.render_view(surf, cam, st, prm)
    return prm, out


def test_without_tolerance_the_only_variant_is_the_oracle_decision():
    """With zero tolerances nothing is flippable: one variant per pixel, equal
    to the oracle's own render of that pixel."""
    rng = np.random.default_rng(31)
    surf = _tiny.random_scene(rng, n=120, spread=0.5, scale=(0.04, 0.12))
    cam = _tiny.front_camera(res=24)
    prm, out = _setup(surf, cam, _tiny.lognormal_env(rng))
    W = cam.width
    ref = np.concatenate([out["rgba"], out["aov"]], 1)
    covered = np.where(out["rgba"][:, 3] > 0)[0]
    assert covered.size > 150
    for pid in covered[::3]:
        v, complete = M.decision_variants(out["records"], out["rect"], W, prm, int(pid), 0.0, 0.0, 0.0)
        assert complete and len(v) == 1
        val = M.composite_variant(out["records"], W, prm, int(pid), *v[0])
        np.testing.assert_allclose(val, ref[pid], rtol=1e-12, atol=1e-14)
        assert v[0][2] == out["n_layers"][pid]


def test_near_cutoff_surfel_gives_both_coverage_outcomes():
    """The candidate whose rho2_mip lies closest to r_cut^2 over the image:
    a tolerance above its margin yields exactly two fragment sets, with and
    without that surfel; a tolerance below it yields one."""
    rng = np.random.default_rng(32)
    surf = _tiny.random_scene(rng, n=60, spread=0.4, scale=(0.03, 0.1))
    cam = _tiny.front_camera(res=24)
    prm, out = _setup(surf, cam, _tiny.lognormal_env(rng))
    W = cam.width
    rec = out["records"]
    best = (np.inf, None, None)
    rc2 = prm.r_cut ** 2
    for pid in range(W * cam.height):
        x, y = pid % W + 0.5, pid // W + 0.5
        T = rec["T"].numpy()
        k = x * T[:, 2] - T[:, 0]
        l = y * T[:, 2] - T[:, 1]
        s = np.cross(k, l)
        with np.errstate(divide="ignore", invalid="ignore"):
            u, v = s[:, 0] / s[:, 2], s[:, 1] / s[:, 2]
        Si = rec["Sinv"].numpy()
        r2 = Si[:, 0, 0] * u * u + 2 * Si[:, 0, 1] * u * v + Si[:, 1, 1] * v * v
        R = out["rect"]
        inside = (x >= R[:, 0]) & (x <= R[:, 1]) & (y >= R[:, 2]) & (y <= R[:, 3]) & out["valid"]
        m = np.where(inside, np.abs(r2 - rc2) / rc2, np.inf)
        j = int(np.nanargmin(m))
        if m[j] < best[0]:
            best = (m[j], pid, j)
    margin, pid, j = best
    assert 0 < margin < 1e-2
    v_hi, _ = M.decision_variants(rec, out["rect"], W, prm, pid, 2 * margin, 0.0, 0.0)
    v_lo, _ = M.decision_variants(rec, out["rect"], W, prm, pid, 0.5 * margin, 0.0, 0.0)
    assert len(v_lo) == 1
    assert len(v_hi) == 2
    a, b = set(v_hi[0][0].tolist()), set(v_hi[1][0].tolist())
    assert a ^ b == {j}


def test_near_tie_gap_gives_both_groupings():
    """Two fronto-parallel surfels on one line of sight, the rear one 1e-9
    (relative) deeper: Algorithm 1 starts a second layer (z_start > z_max_end)
    but a tolerance above 1e-9 also admits the merged single layer, whose
    Shepard weight is the sum of the two."""
    surf = _tiny.surfels([[0.0, 0.0, 0.0], [0.0, 0.0, -3e-9]], scale=0.05,
                         albedo=[[0.9, 0.1, 0.1], [0.1, 0.1, 0.9]])
    cam = _tiny.front_camera(res=16)
    prm, out = _setup(surf, cam, _tiny.const_env(1.0))
    W = cam.width
    pid = 8 * W + 8
    assert out["n_layers"][pid] == 2
    v, complete = M.decision_variants(out["records"], out["rect"], W, prm, pid, 0.0, 1e-6, 0.0)
    assert complete and sorted(x[2] for x in v) == [1, 2]
    assert v[0][2] == 2                              # the oracle's own outcome first
    merged = next(x for x in v if x[2] == 1)
    val = M.composite_variant(out["records"], W, prm, pid, *merged)
    # one layer of both: coverage 1 - exp(-(w_a + w_b)) (Eq. alpha with gamma = 2 pi)
    x, y = 8.5, 8.5
    rec = out["records"]
    T = rec["T"].numpy()
    w = []
    for i in range(2):
        k = x * T[i, 2] - T[i, 0]
        l = y * T[i, 2] - T[i, 1]
        s = np.cross(k, l)
        u, vv = s[0] / s[2], s[1] / s[2]
        Si = rec["Sinv"].numpy()[i]
        w.append(rec["n_f"].numpy()[i] * np.exp(-0.5 * (Si[0, 0] * u * u + 2 * Si[0, 1] * u * vv + Si[1, 1] * vv * vv)))
    assert abs(val[3] - (1 - np.exp(-(w[0] + w[1])))) < 1e-12
    split = M.composite_variant(out["records"], W, prm, pid, *v[0])
    np.testing.assert_allclose(split, np.concatenate([out["rgba"][pid], out["aov"][pid]]), rtol=1e-12, atol=1e-14)
    assert abs(split[3] - (1 - np.exp(-w[0]) * np.exp(-w[1]))) < 1e-12
