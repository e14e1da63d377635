"""The forward rasteriser's exact block culling never drops a covered pixel.

Before its per-pixel tests, a warp drops, per 8 x 4 block, the staged surfels
whose exact support cannot reach any of the block's pixel centres: the
minimum over the block of f(d) = |P d|^2 - r^2 s2(d)^2 (the per-pixel test is
f < 0) is found in closed form (interior minimiser, else a clamped 1-D
minimum per edge) and compared with a margin above the test's FP32 rounding.
This test restates both decisions in float32 arithmetic (fused multiply-adds
as one rounding of the exact product-sum, as the kernels' __fmaf_rn) and
checks, over many random screen-space records and blocks placed across their
support boundaries, that no block the cull rejects has a pixel centre the
per-pixel test covers.  CPU only; it checks the design, the GPU parity tests
check the kernels."""
import numpy as np

F = np.float32


def fma(a, b, c):
    """float32 fused multiply-add: the exact a * b + c rounded once."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F)


def records(rng, n):
    """Screen-space records as the projection builds them: P with
    P^T P = (M M^T + sigma_f I)^-1 (the kernel's triangular factor) and the
    perspective slopes (A2, B2) per pixel."""
    th, ph = rng.uniform(0, np.pi, n), rng.uniform(0, np.pi, n)
    s1, s2 = np.exp(rng.uniform(np.log(0.3), np.log(20.0), (2, n)))
    rot = lambda a: np.stack([np.stack([np.cos(a), -np.sin(a)], -1), np.stack([np.sin(a), np.cos(a)], -1)], -2)
    Mx = rot(th) @ (np.stack([s1, s2], -1)[:, :, None] * rot(ph))
    sig = rng.choice([0.0, 0.5, 2.0], n)
    G = Mx @ np.swapaxes(Mx, 1, 2) + sig[:, None, None] * np.eye(2)
    Dn = np.linalg.det(G)
    qa, qb, qc = G[:, 1, 1] / Dn, -G[:, 0, 1] / Dn, G[:, 0, 0] / Dn
    P = np.zeros((n, 4))
    up = qa >= qc
    l00 = np.sqrt(qa)
    l11 = np.sqrt(qc)
    P[up] = np.stack([l00, qb / l00, np.zeros(n), 1 / np.sqrt(Dn) / l00], -1)[up]
    P[~up] = np.stack([qb / l11, l11, 1 / np.sqrt(Dn) / l11, np.zeros(n)], -1)[~up]
    mag = np.exp(rng.uniform(np.log(1e-4), np.log(0.2), (2, n))) * rng.choice([-1.0, 1.0], (2, n))
    ext = 3.0 * np.sqrt(np.stack([G[:, 0, 0], G[:, 1, 1]], -1))
    return P.astype(F), mag[0].astype(F), mag[1].astype(F), ext


def box_may_cover(P, A2, B2, rc2, dx0, dx1, dy0, dy1):
    """The cull's decision (its conic and edge minima), elementwise."""
    a = P[:, 0] * P[:, 0] + P[:, 2] * P[:, 2] - rc2 * A2 * A2
    b = P[:, 0] * P[:, 1] + P[:, 2] * P[:, 3] - rc2 * A2 * B2
    c = P[:, 1] * P[:, 1] + P[:, 3] * P[:, 3] - rc2 * B2 * B2
    det = a * c - b * b
    pd = (a > 0) & (c > 0) & (det > 0)
    ga, gb = rc2 * A2, rc2 * B2
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        idet = F(1) / det
        xs = (c * ga - b * gb) * idet
        ys = (a * gb - b * ga) * idet
        ia, ic = F(1) / a, F(1) / c
        inside = (xs >= dx0) & (xs <= dx1) & (ys >= dy0) & (ys <= dy1)
        f = lambda x, y: x * (a * x + F(2) * b * y - F(2) * ga) + y * (c * y - F(2) * gb) - rc2
        cl = lambda v, lo, hi: np.minimum(np.maximum(v, lo), hi)
        m = f(dx0, cl((gb - b * dx0) * ic, dy0, dy1))
        m = np.minimum(m, f(dx1, cl((gb - b * dx1) * ic, dy0, dy1)))
        m = np.minimum(m, f(cl((ga - b * dy0) * ia, dx0, dx1), dy0))
        m = np.minimum(m, f(cl((ga - b * dy1) * ia, dx0, dx1), dy1))
        ex, ey = np.maximum(np.abs(dx0), np.abs(dx1)), np.maximum(np.abs(dy0), np.abs(dy1))
        sc = F(1) + np.abs(A2) * ex + np.abs(B2) * ey
        margin = F(1e-5) * rc2 * sc * sc
        return ~pd | inside | ~(m > margin)


def pixel_covers(P, A2, B2, rc2, dx, dy):
    """The per-pixel test: s2 > 0 and |P d|^2 < r^2 s2^2, in the kernels' order."""
    s0 = fma(P[:, 0], dx, P[:, 1] * dy)
    s1 = fma(P[:, 2], dx, P[:, 3] * dy)
    s2 = fma(A2, dx, fma(B2, dy, F(1)))
    q = fma(s0, s0, s1 * s1)
    return (s2 > 0) & (q < rc2 * (s2 * s2))


def test_block_cull_never_drops_a_covered_pixel():
    rng = np.random.default_rng(81)
    rc2 = F(9.0)
    n_rec, n_box = 4000, 64
    P, A2, B2, ext = records(rng, n_rec)
    idx = np.repeat(np.arange(n_rec), n_box)
    # block corners placed across each record's support boundary
    reach = ext[idx] + 10.0
    # (the surfel centre's sub-pixel position differs from record to record)
    bx = (np.floor(rng.uniform(-reach[:, 0], reach[:, 0])) + rng.uniform(0, 1, idx.size)).astype(F)
    by = (np.floor(rng.uniform(-reach[:, 1], reach[:, 1])) + rng.uniform(0, 1, idx.size)).astype(F)
    Pi, Ai, Bi = P[idx], A2[idx], B2[idx]
    may = box_may_cover(Pi, Ai, Bi, rc2, bx + F(0.5), bx + F(7.5), by + F(0.5), by + F(3.5))
    covered = np.zeros(idx.size, bool)
    for i in range(8):
        for j in range(4):
            covered |= pixel_covers(Pi, Ai, Bi, rc2, bx + F(0.5 + i), by + F(0.5 + j))
    assert not np.any(covered & ~may), int(np.sum(covered & ~may))
    # not vacuous: many blocks are dropped, and many kept blocks are covered
    assert (~may).mean() > 0.3 and covered.sum() > 0.1 * idx.size
    # and the cull is tight: few kept blocks have no covered pixel centre
    assert (may & ~covered).sum() < 0.5 * may.sum()
