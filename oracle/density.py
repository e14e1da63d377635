"""FP64 oracle of adaptive density control -- test infrastructure only.

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference arm
of ``bench.py`` may import this module.  It shares no code with the CUDA path.

Sec. 3.6.2 and the appendix on splitting and pruning surfels define:

* the density estimate: for each surfel the mean distance d_bar to its
  nearest *same-orientation* neighbours among the surfel centres.  The paper
  names neither the neighbour count nor the orientation test; here k
  neighbours (default 8) whose unit normals n_j satisfy n_i . n_j >= cos_min
  (default 0.5), other surfels of the same scene only (``neighbours``);
* splitting: a surfel with g_bar >= tau_g (g_bar the mean of the
  screen-space statistic of Eq. ss_grad over the views it appeared in) and
  max(s_u, s_v) > d_bar is replaced by two children at
  c +- (s_max / 2) t_max, t_max the unit tangent of the larger scale; the
  scale along that axis times 0.7, the other scale, the rotation and every
  material attribute inherited (``split_children``);
* visibility pruning: a surfel whose cumulative screen-space gradient
  magnitude over all views is zero is removed;
* isolation pruning: a surfel with no neighbour (of any orientation) within
  its kernel support radius r_cut * s_max is removed (``plan``).

Everything is a brute-force evaluation of these definitions: all pairs, one
scene at a time.  The decisions are taken on float32 copies of the inputs
where the GPU path takes them in float32 too (g_bar); the comparisons with
s_max = exp(max log-scale) are taken in float64, so a caller compares with a
GPU result only away from ties (see ``decision_margins``).
"""
from __future__ import annotations

import numpy as np

PRUNE, KEEP, SPLIT = 0, 1, 2
OP_SPLIT, OP_PRUNE_VISIBLE, OP_PRUNE_ISOLATED = 1, 2, 4


def unit_quat(q):
    q = np.asarray(q, np.float64)
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def rotation(q):
    """R(q) of the unit quaternion (w, x, y, z) (rows: [N,3,3])."""
    w, x, y, z = np.moveaxis(unit_quat(q), -1, 0)
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def normals(q):
    """n = R(q) e_z (Sec. 3.1)."""
    return rotation(q)[..., :, 2]


def neighbours(pos, quat, scene_offsets, k=8, cos_min=0.5, chunk=256):
    """Per surfel: (mean_dist, n_same, nn_dist).

    mean_dist: mean Euclidean distance to the k nearest other surfels of the
    same scene with n_i . n_j >= cos_min (the mean over the ones that exist
    when fewer than k do, NaN when none does); n_same: how many such
    neighbours exist, capped at k; nn_dist: distance to the nearest other
    surfel of the same scene whatever its orientation (inf when alone)."""
    pos = np.asarray(pos, np.float64)
    nrm = normals(quat)
    n = pos.shape[0]
    mean = np.full(n, np.nan)
    cnt = np.zeros(n, np.int64)
    nn = np.full(n, np.inf)
    offs = [int(v) for v in scene_offsets]
    for s in range(len(offs) - 1):
        b, e = offs[s], offs[s + 1]
        P, Nn = pos[b:e], nrm[b:e]
        for r0 in range(0, e - b, chunk):
            r1 = min(r0 + chunk, e - b)
            d = np.sqrt(((P[r0:r1, None, :] - P[None, :, :]) ** 2).sum(-1))
            own = np.arange(r0, r1)
            d[own - r0, own] = np.inf                       # not its own neighbour
            nn[b + r0:b + r1] = d.min(1) if e - b > 1 else np.inf
            same = (Nn[r0:r1] @ Nn.T) >= cos_min
            ds = np.where(same, d, np.inf)
            m = min(k, e - b - 1)
            if m <= 0:
                continue
            part = np.sort(np.partition(ds, m - 1, axis=1)[:, :m], axis=1)
            fin = np.isfinite(part)
            c = fin.sum(1)
            with np.errstate(invalid="ignore"):
                mean[b + r0:b + r1] = np.where(c > 0, np.where(fin, part, 0).sum(1) / np.maximum(c, 1), np.nan)
            cnt[b + r0:b + r1] = c
    return mean, cnt, nn


def neighbours_of(pos, quat, scene_offsets, idx, k=8, cos_min=0.5):
    """``neighbours`` for the surfels idx only (each against every surfel of
    its scene): (mean_dist, n_same, nn_dist, orientation margin) per query,
    the margin as in ``orientation_margins``."""
    pos = np.asarray(pos, np.float64)
    nrm = normals(quat)
    offs = np.asarray([int(v) for v in scene_offsets])
    out = np.zeros((len(idx), 4))
    for a, i in enumerate(idx):
        s = int(np.searchsorted(offs, i, side="right") - 1)
        b, e = offs[s], offs[s + 1]
        P, Nn, ni = pos[b:e], nrm[b:e], nrm[i]
        d = np.sqrt(((P - pos[i]) ** 2).sum(1))
        d[i - b] = np.inf
        dot = Nn @ ni
        ds = np.sort(np.where(dot >= cos_min, d, np.inf))[:k]
        fin = ds[np.isfinite(ds)]
        mean = fin.mean() if fin.size else np.nan
        reach = fin[-1] if fin.size == k else np.inf
        near = d <= reach * (1 + 1e-5)
        margin = np.abs(dot[near] - cos_min).min() if near.any() else np.inf
        out[a] = (mean, fin.size, d.min() if e - b > 1 else np.inf, margin)
    return out


def orientation_margins(pos, quat, scene_offsets, k, cos_min, mean_slack=1e-5):
    """Per surfel, the smallest |n_i . n_j - cos_min| over the surfels j within
    (1 + slack) times its k-th same-orientation distance, or within its nearest
    distance when it has fewer than k: where this is tiny the float32 and the
    float64 orientation tests may choose different neighbour sets."""
    pos = np.asarray(pos, np.float64)
    nrm = normals(quat)
    out = np.full(pos.shape[0], np.inf)
    offs = [int(v) for v in scene_offsets]
    for s in range(len(offs) - 1):
        b, e = offs[s], offs[s + 1]
        P, Nn = pos[b:e], nrm[b:e]
        for i in range(e - b):
            d = np.sqrt(((P - P[i]) ** 2).sum(1))
            d[i] = np.inf
            dot = Nn @ Nn[i]
            ds = np.sort(np.where(dot >= cos_min, d, np.inf))
            reach = ds[min(k, e - b - 1) - 1] if e - b > 1 else 0.0
            if not np.isfinite(reach):
                reach = np.inf
            near = d <= reach * (1 + mean_slack)
            if near.any():
                out[b + i] = np.abs(dot[near] - cos_min).min()
    return out


def plan(log_scale, g_norm, g_views, mean_dist, nn_dist, flags, tau_g, r_cut=3.0, ops=7):
    """Action per surfel (PRUNE / KEEP / SPLIT) and the output position of its
    first row (exclusive prefix sum of 0 / 1 / 2 rows), total last.

    Pruning (either kind) wins over splitting.  flags: bit 0 set where the
    mean distance is only a lower bound (no split), bit 1 where the nearest
    distance is only a lower bound (still isolated when the bound exceeds the
    support)."""
    ls = np.asarray(log_scale, np.float64)
    s_max = np.exp(ls.max(1))
    gn = np.asarray(g_norm, np.float32)
    gv = np.asarray(g_views, np.float32)
    flags = np.asarray(flags, np.int64)
    act = np.full(ls.shape[0], KEEP, np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        g_bar = gn / gv                                    # float32, as the GPU divides
    split = (ops & OP_SPLIT) != 0
    split = split & (g_bar >= np.float32(tau_g)) & ((flags & 1) == 0) & (s_max > np.asarray(mean_dist, np.float64))
    act[split] = SPLIT
    if ops & OP_PRUNE_ISOLATED:
        act[np.asarray(nn_dist, np.float64) > r_cut * s_max] = PRUNE
    if ops & OP_PRUNE_VISIBLE:
        act[~(gn > 0)] = PRUNE
    rows = act.copy()                                       # PRUNE 0, KEEP 1, SPLIT 2 rows
    off = np.concatenate([[0], np.cumsum(rows)])
    return act, off


def decision_margins(log_scale, mean_dist, nn_dist, r_cut=3.0):
    """Relative distance of each float comparison of ``plan`` that involves
    exp() from its threshold: min(|s_max - d_bar| / d_bar,
    |nn - r_cut s_max| / (r_cut s_max))."""
    s_max = np.exp(np.asarray(log_scale, np.float64).max(1))
    md = np.asarray(mean_dist, np.float64)
    nn = np.asarray(nn_dist, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.abs(s_max - md) / md
        b = np.abs(nn - r_cut * s_max) / (r_cut * s_max)
    return np.fmin(np.nan_to_num(a, nan=np.inf), np.nan_to_num(b, nan=np.inf))


def split_children(pos, quat, log_scale, split_scale=0.7):
    """The two children of each row: positions c + (s_max/2) t_max and
    c - (s_max/2) t_max ([N,2,3]) and their log-scales ([N,2]): the split
    axis (u when s_u >= s_v) shrinks by split_scale, the other is kept."""
    pos = np.asarray(pos, np.float64)
    ls = np.asarray(log_scale, np.float64)
    R = rotation(quat)
    use_u = ls[:, 0] >= ls[:, 1]
    t = np.where(use_u[:, None], R[:, :, 0], R[:, :, 1])
    s_max = np.exp(ls.max(1))
    half = 0.5 * s_max[:, None] * t
    child_pos = np.stack([pos + half, pos - half], 1)
    new_ls = ls.copy()
    new_ls[use_u, 0] += np.log(split_scale)
    new_ls[~use_u, 1] += np.log(split_scale)
    return child_pos, np.stack([new_ls, new_ls], 1)


def apply(fields: dict, action, split_scale=0.7):
    """New surfel arrays: each kept surfel once, each split surfel as its two
    children (the + child first), pruned ones dropped, in the parents' order.
    fields: pos [N,3], quat [N,4], log_scale [N,2], and any further per-surfel
    rows (copied to both children)."""
    action = np.asarray(action)
    cp, cls = split_children(fields["pos"], fields["quat"], fields["log_scale"], split_scale)
    out = {k: [] for k in fields}
    for i, a in enumerate(action):
        if a == KEEP:
            for k, v in fields.items():
                out[k].append(np.asarray(v[i], np.float64))
        elif a == SPLIT:
            for c in range(2):
                for k, v in fields.items():
                    if k == "pos":
                        out[k].append(cp[i, c])
                    elif k == "log_scale":
                        out[k].append(cls[i, c])
                    else:
                        out[k].append(np.asarray(v[i], np.float64))
    return {k: (np.stack(v) if v else np.zeros((0,) + np.asarray(fields[k]).shape[1:])) for k, v in out.items()}


def compact_rows(rows, action, zero_children=False):
    """Per-surfel rows of another array (e.g. Adam moments) carried through the
    same step: kept rows once, split rows twice (or as two zero rows)."""
    rows = np.asarray(rows)
    out = []
    for i, a in enumerate(np.asarray(action)):
        if a == KEEP:
            out.append(rows[i])
        elif a == SPLIT:
            out.extend([np.zeros_like(rows[i]) if zero_children else rows[i]] * 2)
    return np.stack(out) if out else np.zeros((0,) + rows.shape[1:], rows.dtype)
