"""Pins of the oracle's forward shading (Sec. 3.4.2, Eq. ibl) against closed
forms.

Each case builds one surfel and a camera so that every lookup the split-sum
shading makes lands on a value known independently of that shading code:

* a constant environment (every prefiltered level equals it);
* a single bright texel that the reflection vector r = 2 (w_o . n) n - w_o
  hits at its centre, with roughness 0 (level 0 is the base map);
* an environment that depends on the polar angle only, so each level is
  constant along its rows and a lookup at a row centre (or inside the first
  half row at the pole) reads that row's value whatever the azimuth;

and n . w_o and the roughness sit on centres of the BRDF table's cells, so
the table lookup returns the split-sum integral at that (n . w_o, r) exactly,
evaluated independently by ``brdf_eval``.  The expected colours are the
special cases of Eq. ibl that the paper's definitions fix: F0 = 0.04 and
k_d = 0.96 for a dielectric (m = 0), F0 = albedo and k_d = 0 for a metal
(m = 1).  A transposed table lookup, swapped Fresnel terms, a reflected
vector of the wrong sign, another azimuth convention, a wrong level
coordinate, a diffuse lookup along another direction, a lookup clamped
instead of wrapped at the azimuth seam, the irradiance of a back-facing
surfel read at its unflipped normal, or near-plane culling by the centre
depth instead of z_start each fail one case.
Nothing here uses the CUDA path.
"""
import math

import numpy as np
import torch

from oracle import model as M

F64 = torch.float64
LUT_N = 128
NQ = 128


def quat_for_normal(n):
    """A unit quaternion (w, x, y, z) whose rotation takes e_z to n (input
    construction: the shortest rotation about e_z x n)."""
    n = np.asarray(n, np.float64) / np.linalg.norm(n)
    ax = np.cross([0.0, 0.0, 1.0], n)
    s = np.linalg.norm(ax)
    if s < 1e-15:
        return np.array([1.0, 0, 0, 0]) if n[2] > 0 else np.array([0.0, 1.0, 0, 0])
    ang = math.atan2(s, n[2])
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * ax / s])


def texel_dir(u, v):
    """Unit direction of equirect coordinates (u, v) under the convention
    phi = atan2(d_x, -d_z) = 2 pi (u - 1/2), theta = acos(d_y) = pi v."""
    phi, th = 2 * math.pi * (u - 0.5), math.pi * v
    return np.array([math.sin(th) * math.sin(phi), math.cos(th), -math.sin(th) * math.cos(phi)])


def polar_dir(theta, phi):
    return texel_dir(phi / (2 * math.pi) + 0.5, theta / math.pi)


def rotate_towards(d, angle, helper=(0.3, -0.5, 0.8)):
    """A unit vector at `angle` from the unit vector d."""
    e = np.asarray(helper, np.float64)
    e = e - d * (e @ d)
    e /= np.linalg.norm(e)
    return math.cos(angle) * d + math.sin(angle) * e


def view_for(refl, mu):
    """(w_o, n) with n . w_o = mu and 2 (w_o . n) n - w_o = refl."""
    w_o = rotate_towards(refl, 2 * math.acos(mu))
    n = w_o + refl
    return w_o, n / np.linalg.norm(n)


def shade(normal, w_o, albedo, rough, metal, irr, levels, lut):
    """The oracle's record of one surfel at the origin seen from 3 w_o:
    returns its 12 averaged channels (shaded RGB first)."""
    S = {"pos": torch.zeros(1, 3, dtype=F64),
         "quat": torch.tensor(quat_for_normal(normal)[None], dtype=F64),
         "log_scale": torch.full((1, 2), math.log(0.05), dtype=F64),
         "albedo": torch.tensor([albedo], dtype=F64),
         "roughness": torch.tensor([rough], dtype=F64),
         "metallic": torch.tensor([metal], dtype=F64)}
    eye = 3.0 * np.asarray(w_o, np.float64)
    cam = {"R": torch.eye(3, dtype=F64), "t": torch.tensor(-eye, dtype=F64),
           "fx": 100.0, "fy": 100.0, "cx": 32.0, "cy": 32.0, "width": 64, "height": 64}
    prm = M.Params(lut_n=LUT_N, env_levels=len(levels))
    rec = M.records(S, cam, torch.from_numpy(np.asarray(irr, np.float64)),
                    [torch.from_numpy(np.asarray(l, np.float64)) for l in levels],
                    torch.from_numpy(M.brdf_lut(LUT_N, NQ)) if lut is None else lut, prm)
    return rec["ch"][0].detach().numpy()


def cell(k):
    """Centre of cell k of the BRDF table along either axis."""
    return (k + 0.5) / LUT_N


def beta(mu, r):
    return M.brdf_eval(np.array([mu]), np.array([r]), nq=NQ)[0]


ALBEDO = np.array([0.2, 0.55, 0.9])


def test_constant_env_dielectric_and_metal():
    """Constant environment L: every prefiltered level equals L, so Eq. ibl
    is c = 0.96 rho L + L (0.04 beta1 + beta2) for m = 0 and
    c = L (rho beta1 + beta2) for m = 1, with (beta1, beta2) the split-sum
    integral at (n . w_o, r).  n . w_o and r sit on different table cells,
    so a transposed lookup reads another value."""
    L = np.array([0.7, 1.3, 2.1])
    env = np.broadcast_to(L, (32, 64, 3)).copy()
    irr, levels = M.env_prefilter(env, 6, 32, 16)
    mu, r = cell(90), cell(23)
    b1, b2 = beta(mu, r)
    b1t, b2t = beta(r, mu)
    assert abs(b1 - b1t) > 1e-2 and abs(b2 - b2t) > 1e-3      # the transposed value really differs
    w_o, n = view_for(polar_dir(1.1, 0.7), mu)
    got0 = shade(n, w_o, ALBEDO, r, 0.0, irr, levels, None)[:3]
    np.testing.assert_allclose(got0, 0.96 * ALBEDO * L + L * (0.04 * b1 + b2), rtol=1e-10, atol=0)
    got1 = shade(n, w_o, ALBEDO, r, 1.0, irr, levels, None)[:3]
    np.testing.assert_allclose(got1, L * (ALBEDO * b1 + b2), rtol=1e-10, atol=0)


def _one_texel_env(a, b, value, W=64, H=32):
    env = np.zeros((H, W, 3))
    env[b, a] = value
    return env


def test_specular_hits_the_texel_the_reflection_vector_points_at():
    """Roughness 0 reads level 0 (the base map).  With one bright texel E and
    r = 2 (w_o . n) n - w_o pointing at its centre, a metal (k_d = 0) shows
    c = E (rho beta1 + beta2); any other direction (the opposite vector,
    another azimuth convention) reads a zero texel."""
    a, b, W, H = 21, 9, 64, 32
    E = np.array([2.0, 3.0, 5.0])
    env = _one_texel_env(a, b, E, W, H)
    irr, levels = M.env_prefilter(env, 6, 32, 16)
    d = texel_dir((a + 0.5) / W, (b + 0.5) / H)
    mu = cell(77)
    w_o, n = view_for(d, mu)
    b1, b2 = beta(mu, cell(0))          # roughness 0 clamps to the table's first row
    got = shade(n, w_o, ALBEDO, 0.0, 1.0, irr, levels, None)
    np.testing.assert_allclose(got[:3], E * (ALBEDO * b1 + b2), rtol=1e-9, atol=0)
    # the bright texel is the only one the lookup may reach
    assert np.all(got[:3] > 0.5 * E * (ALBEDO * b1 + b2))


def test_back_facing_surfel_is_shaded_with_the_flipped_normal():
    """Surfels are two-sided: a surfel whose normal points away from the
    camera is shaded with -n (and reports -n), so it matches the front-facing
    case exactly."""
    a, b, W, H = 40, 20, 64, 32
    E = np.array([1.5, 0.5, 4.0])
    env = _one_texel_env(a, b, E, W, H)
    irr, levels = M.env_prefilter(env, 6, 32, 16)
    d = texel_dir((a + 0.5) / W, (b + 0.5) / H)
    mu = cell(50)
    w_o, n = view_for(d, mu)
    b1, b2 = beta(mu, cell(0))
    front = shade(n, w_o, ALBEDO, 0.0, 1.0, irr, levels, None)
    back = shade(-n, w_o, ALBEDO, 0.0, 1.0, irr, levels, None)
    np.testing.assert_allclose(back[:3], E * (ALBEDO * b1 + b2), rtol=1e-9, atol=0)
    np.testing.assert_allclose(back[:3], front[:3], rtol=1e-12, atol=0)
    np.testing.assert_allclose(back[8:11], n, atol=1e-12)     # the reported normal faces the viewer


def _polar_env(W=64, H=32):
    """Depends on the polar angle only (rows constant), so the irradiance map
    and every specular level are constant along their rows too."""
    th = (np.arange(H) + 0.5) / H * math.pi
    rows = np.stack([1.0 + 3.0 * np.cos(th) ** 2, 0.5 + np.sin(th), 2.0 - np.cos(th)], 1)
    return np.broadcast_to(rows[:, None, :], (H, W, 3)).copy()


def test_roughness_between_two_levels_blends_them_linearly():
    """The level coordinate is r (L - 1): at r = 40.5/128 (a table row
    centre), 6 levels give 1.58203125, i.e. 0.41796875 of level 1 and
    0.58203125 of level 2.  The reflection vector points 1e-3 rad from the
    pole, inside the first half row of every level, so each level returns
    its first row's value."""
    env = _polar_env()
    irr, levels = M.env_prefilter(env, 6, 32, 16)
    for lv in levels:
        assert np.ptp(lv[0], axis=0).max() < 1e-9 * np.abs(lv).max()   # rows constant
    r = cell(40)
    lc = r * 5
    i, f = int(math.floor(lc)), lc - math.floor(lc)
    assert (i, round(f, 8)) == (1, 0.58203125)
    Ls = (1 - f) * levels[1][0, 0] + f * levels[2][0, 0]
    assert np.abs(levels[1][0, 0] - levels[2][0, 0]).min() > 1e-3      # the blend is visible
    mu = cell(100)
    w_o, n = view_for(polar_dir(1e-3, 0.4), mu)
    b1, b2 = beta(mu, r)
    got = shade(n, w_o, ALBEDO, r, 1.0, irr, levels, None)[:3]
    np.testing.assert_allclose(got, Ls * (ALBEDO * b1 + b2), rtol=1e-9, atol=0)


def test_dielectric_diffuse_reads_the_irradiance_along_the_normal():
    """m = 0: c = 0.96 rho L_d(n) + L_s(r) (0.04 beta1 + beta2).  With the
    polar-only environment, n on the centre of irradiance row 5 and the
    reflection vector on the centre of base row 10 (roughness 0: level 0 is
    the base map), L_d and L_s are those rows' values."""
    env = _polar_env()
    irr, levels = M.env_prefilter(env, 6, 32, 16)
    th_n = (5 + 0.5) / 16 * math.pi
    th_r = (10 + 0.5) / 32 * math.pi
    mu = cell(95)
    # azimuth difference that puts n and r at the angle acos(mu) apart
    cdp = (mu - math.cos(th_n) * math.cos(th_r)) / (math.sin(th_n) * math.sin(th_r))
    assert abs(cdp) < 1.0
    n = polar_dir(th_n, 0.3)
    refl = polar_dir(th_r, 0.3 + math.acos(cdp))
    assert abs(n @ refl - mu) < 1e-12
    w_o = 2.0 * (n @ refl) * n - refl
    b1, b2 = beta(mu, cell(0))
    Ld, Ls = irr[5, 0], env[10, 0]
    assert abs(irr[5, 7] - Ld).max() < 1e-9 and abs(Ls - levels[0][10, 3]).max() == 0
    got = shade(n, w_o, ALBEDO, 0.0, 0.0, irr, levels, None)[:3]
    np.testing.assert_allclose(got, 0.96 * ALBEDO * Ld + Ls * (0.04 * b1 + b2), rtol=1e-9, atol=0)
    # neighbouring irradiance rows differ, so a lookup along another direction shows
    assert np.abs(irr[4, 0] - irr[5, 0]).min() > 1e-3 and np.abs(irr[6, 0] - irr[5, 0]).min() > 1e-3


def _rows_map(values, W=32):
    """A map whose row k holds values[k] everywhere (rows constant)."""
    v = np.asarray(values, np.float64)
    return np.broadcast_to(v[:, None, :], (v.shape[0], W, 3)).copy()


def _dark_levels():
    return [np.zeros((32 >> i, 64 >> i, 3)) for i in range(6)]


def test_irradiance_lookup_wraps_across_the_azimuth_seam():
    """The equirect maps wrap in azimuth: a normal at phi = pi (u = 1, the
    seam) reads half the last column and half the first, and a quarter
    texel to either side three quarters of the nearer one.  A dielectric in a
    dark specular environment shows c = 0.96 rho L_d, with L_d = (A + B) / 2
    for last column A and first column B (a clamped lookup reads A alone)."""
    Hi, Wi, k = 16, 32, 7
    irr = _rows_map(np.full((Hi, 3), 0.3), Wi)
    A, B = np.array([1.0, 2.0, 3.0]), np.array([3.0, 0.5, 0.25])
    irr[:, -1] = A
    irr[:, 0] = B
    th = (k + 0.5) / Hi * math.pi                     # a row centre: no blend between rows
    n = np.array([0.0, math.cos(th), math.sin(th)])   # phi = atan2(0, -sin th) = pi
    w_o = rotate_towards(n, 0.6)
    got = shade(n, w_o, ALBEDO, 0.4, 0.0, irr, _dark_levels(), None)[:3]
    np.testing.assert_allclose(got, 0.96 * ALBEDO * 0.5 * (A + B), rtol=1e-9, atol=0)
    # a quarter texel to either side of the seam: 3/4 of the nearer column
    for u, wA in ((1.0 - 0.25 / Wi, 0.75), (0.25 / Wi, 0.25)):
        n = texel_dir(u, (k + 0.5) / Hi)
        got = shade(n, rotate_towards(n, 0.6), ALBEDO, 0.4, 0.0, irr, _dark_levels(), None)[:3]
        np.testing.assert_allclose(got, 0.96 * ALBEDO * (wA * A + (1 - wA) * B), rtol=1e-9, atol=0)


def test_back_facing_dielectric_reads_the_irradiance_at_the_flipped_normal():
    """The diffuse term of a back-facing surfel is looked up along the
    normal turned toward the viewer (two-sided surfels): with every
    irradiance row distinct, c = 0.96 rho L_d(n_s), not L_d(-n_s)."""
    Hi = 16
    vals = np.stack([0.2 + 0.1 * np.arange(Hi), 1.0 + 0.05 * np.arange(Hi) ** 2, 3.0 - 0.15 * np.arange(Hi)], 1)
    irr = _rows_map(vals)
    k = 4
    n_s = polar_dir((k + 0.5) / Hi * math.pi, 0.9)     # row k; -n_s lies in row Hi - 1 - k
    w_o = rotate_towards(n_s, 0.5)
    got = shade(-n_s, w_o, ALBEDO, 0.3, 0.0, irr, _dark_levels(), None)
    np.testing.assert_allclose(got[:3], 0.96 * ALBEDO * vals[k], rtol=1e-9, atol=0)
    np.testing.assert_allclose(got[8:11], n_s, atol=1e-12)
    assert np.abs(vals[k] - vals[Hi - 1 - k]).min() > 0.1


def test_surfel_reaching_in_front_of_the_near_plane_is_culled():
    """z_near (0.01; not given by the paper) culls a surfel whose depth
    interval [z_c - eps, z_c + eps], eps = r_cut sqrt(t_uz^2 + t_vz^2),
    starts at or before it, although its centre lies beyond: a surfel tilted
    60 degrees with scale 0.05 has eps = 0.13, so at z_c = 0.1 it is culled
    and at z_c = 0.2 it is kept."""
    q = quat_for_normal([0.0, math.sin(math.pi / 3), math.cos(math.pi / 3)])
    cam = {"R": torch.eye(3, dtype=F64), "t": torch.zeros(3, dtype=F64),
           "fx": 100.0, "fy": 100.0, "cx": 32.0, "cy": 32.0, "width": 64, "height": 64}
    prm = M.Params(lut_n=LUT_N)
    irr, levels = M.env_prefilter(np.ones((32, 64, 3)), 6, 32, 16)
    S = {"pos": torch.tensor([[0.0, 0.0, 0.1], [0.0, 0.0, 0.2]], dtype=F64),
         "quat": torch.tensor(np.stack([q, q]), dtype=F64),
         "log_scale": torch.full((2, 2), math.log(0.05), dtype=F64),
         "albedo": torch.full((2, 3), 0.5, dtype=F64), "roughness": torch.full((2,), 0.5, dtype=F64),
         "metallic": torch.zeros(2, dtype=F64)}
    rec = M.records(S, cam, torch.from_numpy(irr), [torch.from_numpy(l) for l in levels],
                    torch.from_numpy(M.brdf_lut(LUT_N, 16)), prm)
    eps = 3.0 * 0.05 * math.sin(math.pi / 3)
    np.testing.assert_allclose(rec["zs"].numpy(), [0.1 - eps, 0.2 - eps], rtol=1e-12)
    assert rec["zs"][0] < prm.z_near < 0.1 and rec["zs"][1] > prm.z_near
    assert rec["valid"].tolist() == [False, True]
