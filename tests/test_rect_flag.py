"""The projection's support rectangle and its "support inside" decision.

A pixel is a candidate of a surfel only if its centre lies in the support
rectangle (the exact bounds of the projected r_cut disc, App. A, united with
the r_cut bounds of the EWA ellipse at the centre, padded by a pixel).  When
the projection finds the whole filtered support {f(d) < 0} (f the per-pixel
test, d the offset from the centre) inside the rectangle with 0.25 px to
spare, it leaves the record's rectangle flag clear and the rasterisers skip
the per-pixel rectangle check.  This test restates the projection's
rectangle, its decision and the per-pixel test in float32 (fused
multiply-adds rounded once) and checks, over random surfels in front of a
pinhole camera, that no pixel the test covers lies outside the rectangle of
a record whose flag is clear.  CPU only; it checks the design, the GPU parity
tests check the kernels."""
import numpy as np

F = np.float32


def fma(a, b, c):
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def frame(rng):
    """A random rotation (columns: tangent u, tangent v, normal)."""
    q = rng.normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def project(c, tu, tv, fx, fy, sig, rc):
    """The projection's screen-space record (float32 arithmetic): P, A2, B2,
    the rectangle's offset bounds lo, hi and the "support inside" decision."""
    rc2 = F(rc * rc)
    cz = F(c[2])
    mx, my = F(c[0] / c[2]), F(c[1] / c[2])
    tuc, tvc = tu.astype(F), tv.astype(F)
    ax, ay = fma(-mx, tuc[2], tuc[0]), fma(-my, tuc[2], tuc[1])
    bx, by = fma(-mx, tvc[2], tvc[0]), fma(-my, tvc[2], tvc[1])
    n = np.cross(tu, tv)
    n /= np.linalg.norm(n)
    Nd = F(n @ c)                                   # the camera's distance to the plane
    det0 = F(np.linalg.norm(np.cross(tu, tv)) * (n @ c) / c[2])
    A2, B2 = F(cz * F(n[0]) / (F(fx) * Nd)), F(cz * F(n[1]) / (F(fy) * Nd))
    icz = F(1) / cz
    icz2 = icz * icz
    m11 = F(fx * fx) * (ax * ax + bx * bx) * icz2
    m12 = F(fx * fy) * (ax * ay + bx * by) * icz2
    m22 = F(fy * fy) * (ay * ay + by * by) * icz2
    sdg = F(fx * fy) * det0 * icz2
    Dn = sdg * sdg + F(sig) * (m11 + m22) + F(sig * sig)
    qa, qb, qc = (m22 + F(sig)) / Dn, -m12 / Dn, (m11 + F(sig)) / Dn
    if qa >= qc:
        l00 = np.sqrt(qa)
        P = (l00, qb / l00, F(0), F(1) / np.sqrt(Dn) / l00)
    else:
        l11 = np.sqrt(qc)
        P = (qb / l11, l11, F(1) / np.sqrt(Dn) / l11, F(0))
    C00, C02 = F(fx * fx) * (ax * ax + bx * bx), F(fx) * (ax * tuc[2] + bx * tvc[2])
    C11, C12 = F(fy * fy) * (ay * ay + by * by), F(fy) * (ay * tuc[2] + by * tvc[2])
    C22 = tuc[2] * tuc[2] + tvc[2] * tvc[2] - cz * cz / rc2
    lo, hi = np.zeros(2, F), np.zeros(2, F)
    for k, (caa, ca2, maa) in enumerate(((C00, C02, m11), (C11, C12, m22))):
        dsc = np.sqrt(max(ca2 * ca2 - caa * C22, F(0)))
        r0, r1 = (ca2 + dsc) / C22, (ca2 - dsc) / C22
        ext = F(rc) * np.sqrt(maa + F(sig))
        lo[k] = min(r0, r1, -ext) - F(1)
        hi[k] = max(r0, r1, ext) + F(1)
    q00, q01, q11 = qa - rc2 * A2 * A2, qb - rc2 * A2 * B2, qc - rc2 * B2 * B2
    dq = q00 * q11 - q01 * q01
    inside = bool(q00 > 0 and dq > 0 and C22 < 0)
    if inside:
        i00, i01, i11 = q11 / dq, -q01 / dq, q00 / dq
        dcx, dcy = rc2 * (i00 * A2 + i01 * B2), rc2 * (i01 * A2 + i11 * B2)
        kap = rc2 * (F(1) + A2 * dcx + B2 * dcy)
        hx, hy = np.sqrt(max(kap * i00, F(0))), np.sqrt(max(kap * i11, F(0)))
        inside = bool(dcx - hx > lo[0] + F(0.25) and dcx + hx < hi[0] - F(0.25) and
                      dcy - hy > lo[1] + F(0.25) and dcy + hy < hi[1] - F(0.25))
    return np.array(P, F), A2, B2, lo, hi, inside, C22 < 0


def covers(P, A2, B2, rc2, dx, dy):
    s0 = fma(P[0], dx, P[1] * dy)
    s1 = fma(P[2], dx, P[3] * dy)
    s2 = fma(A2, dx, fma(B2, dy, F(1)))
    q = fma(s0, s0, s1 * s1)
    return (s2 > 0) & (q < F(9.0) * (s2 * s2))


def test_a_clear_flag_means_every_covered_pixel_is_in_the_rectangle():
    rng = np.random.default_rng(101)
    fx = 400.0
    n_inside = n_checked = n_edge = 0
    for it in range(1500):
        fy = fx * (1.3 if it % 3 == 0 else 1.0)
        z = rng.uniform(0.4, 4.0)
        c = np.array([rng.uniform(-0.4, 0.4) * z, rng.uniform(-0.4, 0.4) * z, z])
        Rf = frame(rng)
        if it % 4 == 0:                                    # nearly edge-on: the normal across the view ray
            v = c / np.linalg.norm(c)
            nrm = np.cross(v, rng.normal(size=3))
            nrm /= np.linalg.norm(nrm)
            nrm = nrm + rng.uniform(-0.05, 0.05) * v
            nrm /= np.linalg.norm(nrm)
            tu = np.cross(nrm, rng.normal(size=3))
            tu /= np.linalg.norm(tu)
            Rf = np.stack([tu, np.cross(nrm, tu), nrm], 1)
        s = np.exp(rng.uniform(np.log(0.002), np.log(0.05), 2)) * z
        tu, tv = Rf[:, 0] * s[0], Rf[:, 1] * s[1]
        sig = float(rng.choice([0.0, 0.5, 2.0]))
        P, A2, B2, lo, hi, inside, ok = project(c, tu, tv, fx, fy, sig, 3.0)
        if not ok or not inside:
            continue
        n_inside += 1
        # pixel centres around the rectangle (the centre's sub-pixel position is random)
        fx0, fy0 = rng.uniform(0, 1, 2)
        xs = (np.arange(np.floor(lo[0]) - 3, np.ceil(hi[0]) + 4) + fx0).astype(F)
        ys = (np.arange(np.floor(lo[1]) - 3, np.ceil(hi[1]) + 4) + fy0).astype(F)
        if xs.size * ys.size > 40000:
            continue
        DX, DY = np.meshgrid(xs, ys)
        cov = covers(P, A2, B2, F(9.0), DX.astype(F), DY.astype(F))
        out = (DX < lo[0]) | (DX > hi[0]) | (DY < lo[1]) | (DY > hi[1])
        assert not np.any(cov & out), (it, int((cov & out).sum()))
        n_checked += int(cov.sum())
        edge = (DX - lo[0] < 2) | (hi[0] - DX < 2) | (DY - lo[1] < 2) | (hi[1] - DY < 2)
        n_edge += int((cov & edge).sum())
    assert n_inside > 500 and n_checked > 50000
    assert n_edge > 500          # covered pixels within 2 px of the rectangle's edges were checked
