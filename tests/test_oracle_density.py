"""Pins of the oracle's adaptive density control (Sec. 3.6.2 and the
appendix on splitting and pruning surfels): the neighbour statistics against
scipy's k-d tree and lattice closed forms, the decision rules on hand-made
cases, and the split geometry against its closed form.  Nothing here uses
the CUDA path."""
import math

import numpy as np
import pytest

from oracle import density as D
from tests import _tiny


def _quats_facing(nrm, rng):
    from paper_2605_05876_gb300 import scenes as S
    return S.tangent_quats(np.asarray(nrm, np.float64), rng)


def test_unoriented_neighbours_match_kdtree():
    """With an orientation test every pair passes (cos_min = -2), the mean of
    the k nearest and the nearest distance are what a k-d tree returns."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(5)
    pos = rng.uniform(-1, 1, size=(700, 3))
    quat = _quats_facing(rng.normal(size=(700, 3)), rng)
    for k in (1, 5, 16):
        mean, cnt, nn = D.neighbours(pos, quat, [0, 700], k=k, cos_min=-2.0)
        d, _ = spatial.cKDTree(pos).query(pos, k=k + 1)      # itself first
        np.testing.assert_allclose(mean, d[:, 1:].mean(1), rtol=1e-12)
        np.testing.assert_allclose(nn, d[:, 1], rtol=1e-12)
        assert np.all(cnt == k)


def test_lattice_closed_form_and_orientation():
    """A square lattice of spacing a with normals +z: an interior site has 4
    neighbours at a and 4 at a sqrt(2), so k = 4 gives a and k = 8 gives
    a (1 + sqrt 2) / 2.  A second lattice offset by delta < a along z with
    normals -z is never a same-orientation neighbour (cos_min 0.5) but is the
    nearest surfel of any orientation."""
    a, delta = 0.1, 0.013
    top = _tiny.grid_plane(9, a, z=0.0)
    bot = _tiny.grid_plane(9, a, z=delta)
    bq = np.tile([0.0, 1.0, 0.0, 0.0], (bot.n, 1))          # 180 degrees about x: normal -z
    pos = np.concatenate([top.pos, bot.pos]).astype(np.float64)
    quat = np.concatenate([top.quat, bq]).astype(np.float64)
    inner = np.array([i for i in range(81) if 0 < i % 9 < 8 and 0 < i // 9 < 8])
    for k, want in ((4, a), (8, a * (1 + math.sqrt(2)) / 2)):
        mean, cnt, nn = D.neighbours(pos, quat, [0, 162], k=k, cos_min=0.5)
        np.testing.assert_allclose(mean[inner], want, rtol=1e-6)
        np.testing.assert_allclose(mean[81 + inner], want, rtol=1e-6)
        np.testing.assert_allclose(nn[inner], delta, rtol=1e-6)
    # without the orientation test the lower lattice's site right below counts
    mean, _, _ = D.neighbours(pos, quat, [0, 162], k=1, cos_min=-2.0)
    np.testing.assert_allclose(mean[inner], delta, rtol=1e-6)


def test_scenes_do_not_see_each_other():
    """Two scenes holding interleaved clouds: each scene's statistics equal
    those of the scene alone."""
    rng = np.random.default_rng(8)
    p1, p2 = rng.uniform(-1, 1, (200, 3)), rng.uniform(-1, 1, (150, 3))
    q1, q2 = _quats_facing(rng.normal(size=(200, 3)), rng), _quats_facing(rng.normal(size=(150, 3)), rng)
    both = D.neighbours(np.concatenate([p1, p2]), np.concatenate([q1, q2]), [0, 200, 350], k=6, cos_min=0.2)
    one = D.neighbours(p1, q1, [0, 200], k=6, cos_min=0.2)
    two = D.neighbours(p2, q2, [0, 150], k=6, cos_min=0.2)
    for a, b, c in zip(both, one, two):
        np.testing.assert_array_equal(a, np.concatenate([b, c]))


def test_fewer_neighbours_than_k():
    """Three collinear same-facing surfels at 0, 1, 3 and k = 8: each averages
    the two others; a scene of one surfel has no neighbour at all."""
    pos = np.array([[0.0, 0, 0], [1.0, 0, 0], [3.0, 0, 0], [9.0, 9, 9]])
    quat = np.tile([1.0, 0, 0, 0], (4, 1))
    mean, cnt, nn = D.neighbours(pos, quat, [0, 3, 4], k=8, cos_min=0.5)
    np.testing.assert_allclose(mean[:3], [2.0, 1.5, 2.5])
    np.testing.assert_array_equal(cnt, [2, 2, 2, 0])
    np.testing.assert_allclose(nn[:3], [1.0, 1.0, 2.0])
    assert np.isnan(mean[3]) and np.isinf(nn[3])


def test_plan_rules():
    """One surfel per rule, tau_g = 1, r_cut = 3, s_max = 0.1:
    0 zero gradient -> prune;  1 nearest neighbour beyond 0.3 -> prune;
    2 g_bar = tau_g and s_max > d_bar -> split;  3 s_max < d_bar -> keep;
    4 g_bar < tau_g -> keep;  5 as 2 but d_bar only a lower bound -> keep;
    6 nearest distance a lower bound above the support -> prune;
    7 nearest neighbour beyond s_max but within the support 0.3 -> keep.
    With pruning disabled, 1 and 6 (which also meet the split rule) split."""
    ls = np.log(np.array([[0.1, 0.05]] * 8))
    g_norm = np.array([0.0, 3.0, 3.0, 3.0, 2.9, 3.0, 3.0, 3.0])
    g_views = np.array([0.0, 3.0, 3.0, 3.0, 3.0, 3.0, 3.0, 3.0])
    mean = np.array([0.05, 0.05, 0.08, 0.12, 0.05, 0.05, 0.05, 0.12])
    nn = np.array([0.01, 0.31, 0.02, 0.02, 0.02, 0.02, 0.35, 0.2])
    flags = np.array([0, 0, 0, 0, 0, 1, 2, 0])
    act, off = D.plan(ls, g_norm, g_views, mean, nn, flags, tau_g=1.0, r_cut=3.0)
    np.testing.assert_array_equal(act, [D.PRUNE, D.PRUNE, D.SPLIT, D.KEEP, D.KEEP, D.KEEP, D.PRUNE, D.KEEP])
    np.testing.assert_array_equal(off, [0, 0, 0, 2, 3, 4, 5, 5, 6])
    act, _ = D.plan(ls, g_norm, g_views, mean, nn, flags, tau_g=1.0, ops=D.OP_PRUNE_VISIBLE)
    np.testing.assert_array_equal(act, [D.PRUNE] + [D.KEEP] * 7)
    act, _ = D.plan(ls, g_norm, g_views, mean, nn, flags, tau_g=1.0, ops=D.OP_SPLIT)
    np.testing.assert_array_equal(act, [D.KEEP, D.SPLIT, D.SPLIT, D.KEEP, D.KEEP, D.KEEP, D.SPLIT, D.KEEP])


def test_split_children_closed_form():
    """Identity rotation, scales (0.2, 0.1): children at c +- 0.1 e_x with
    scales (0.14, 0.1); with s_v the larger the split runs along e_y."""
    pos = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    quat = np.array([[1.0, 0, 0, 0], [2.0, 0, 0, 0]])             # the second unnormalised
    ls = np.log(np.array([[0.2, 0.1], [0.1, 0.4]]))
    cp, cls = D.split_children(pos, quat, ls)
    np.testing.assert_allclose(cp[0], [[1.1, 2.0, 3.0], [0.9, 2.0, 3.0]], atol=1e-15)
    np.testing.assert_allclose(cp[1], [[0.0, 0.2, 0.0], [0.0, -0.2, 0.0]], atol=1e-15)
    np.testing.assert_allclose(np.exp(cls[0]), [[0.14, 0.1]] * 2, rtol=1e-14)
    np.testing.assert_allclose(np.exp(cls[1]), [[0.1, 0.28]] * 2, rtol=1e-14)


def test_split_children_stay_on_the_parent_plane():
    """Any rotation: the children's midpoint is the parent, they are s_max
    apart, and their offset is perpendicular to the normal (coplanar)."""
    rng = np.random.default_rng(3)
    n = 50
    pos = rng.normal(size=(n, 3))
    quat = rng.normal(size=(n, 4))
    ls = rng.normal(-2, 0.5, size=(n, 2))
    cp, _ = D.split_children(pos, quat, ls)
    np.testing.assert_allclose(cp.mean(1), pos, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(cp[:, 0] - cp[:, 1], axis=1), np.exp(ls.max(1)), rtol=1e-12)
    np.testing.assert_allclose(np.einsum("ij,ij->i", cp[:, 0] - cp[:, 1], D.normals(quat)), 0, atol=1e-13)


def test_rotation_is_proper_and_matches_axis_angle():
    """R(q) is orthonormal with det 1, and a quarter turn about z maps e_x to e_y."""
    rng = np.random.default_rng(4)
    R = D.rotation(rng.normal(size=(20, 4)))
    np.testing.assert_allclose(R @ np.swapaxes(R, 1, 2), np.broadcast_to(np.eye(3), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)
    c = math.cos(math.pi / 4)
    np.testing.assert_allclose(D.rotation(np.array([[c, 0, 0, c]]))[0] @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_apply_and_compact_order():
    """Parents' order, + child first; other rows copied to both children or zeroed."""
    fields = {"pos": np.zeros((3, 3)), "quat": np.tile([1.0, 0, 0, 0], (3, 1)),
              "log_scale": np.log(np.array([[0.2, 0.1]] * 3)), "albedo": np.arange(9.0).reshape(3, 3)}
    act = np.array([D.SPLIT, D.PRUNE, D.KEEP])
    out = D.apply(fields, act)
    assert out["pos"].shape == (3, 3)
    np.testing.assert_allclose(out["pos"][:, 0], [0.1, -0.1, 0.0])
    np.testing.assert_array_equal(out["albedo"], [[0, 1, 2], [0, 1, 2], [6, 7, 8]])
    rows = np.arange(6.0).reshape(3, 2)
    np.testing.assert_array_equal(D.compact_rows(rows, act), [[0, 1], [0, 1], [4, 5]])
    np.testing.assert_array_equal(D.compact_rows(rows, act, zero_children=True), [[0, 0], [0, 0], [4, 5]])
    assert D.apply(fields, np.array([D.PRUNE] * 3))["pos"].shape == (0, 3)
