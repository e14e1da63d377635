"""Seeded synthetic inputs shaped like the paper's object-level workloads.

This module is INPUT DATA ONLY: it draws surfel sets, cameras and HDR
environment maps.  It contains none of the renderer's arithmetic (no
projection, no kernel, no shading), so the CUDA path and the FP64 oracle can
both consume its output without sharing any of the method's code.

The paper measures on Stanford-ORB objects (~100k surfels, 512^2, Sec. 4),
on mesh-sampled scans of ~1M surfels (Sec. 4.3) and on a viewport-filling
point-sampled bunny with 50K-2M surfels at 512^2-2048^2 (Sec. 4.5).  None of
those assets exist here; the generators below stand in for them with closed
procedural surfaces of the same surfel counts, footprints and layer counts.

Conventions (shared by both sides as a specification):
  * surfel parameters are float32 SoA arrays: pos [N,3], quat [N,4] as
    (w, x, y, z) (not necessarily unit), log_scale [N,2] (s_u, s_v),
    albedo [N,3] in [0,1], roughness [N], metallic [N];
  * cameras are OpenCV pinholes (x right, y down, +z forward), world->camera
    x_c = R x_w + t, pixel (i, j) has its centre at (i + 0.5, j + 0.5),
    f = (H/2) / tan(fov/2), principal point (W/2, H/2);
  * environment maps are equirectangular float32 [He, We, 3].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# small containers


@dataclasses.dataclass
class Surfels:
    pos: np.ndarray        # [N,3] float32
    quat: np.ndarray       # [N,4] float32 (w,x,y,z)
    log_scale: np.ndarray  # [N,2] float32
    albedo: np.ndarray     # [N,3] float32
    roughness: np.ndarray  # [N]   float32
    metallic: np.ndarray   # [N]   float32

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def subset(self, idx) -> "Surfels":
        return Surfels(*(np.ascontiguousarray(getattr(self, f.name)[idx])
                         for f in dataclasses.fields(self)))

    @staticmethod
    def concat(parts) -> "Surfels":
        return Surfels(*(np.ascontiguousarray(np.concatenate([getattr(p, f.name) for p in parts]))
                         for f in dataclasses.fields(Surfels)))


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # [3,3] world->camera rotation (float64 here; cast on use)
    t: np.ndarray          # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    scene: int = 0


@dataclasses.dataclass
class Scene:
    """A batch: several surfel sets (scenes), one env map each, and views."""
    surfels: Surfels                 # all scenes concatenated
    scene_offsets: np.ndarray        # [S+1] int64 ranges into `surfels`
    envs: list                       # S float32 arrays [He, We, 3]
    cameras: list                    # V Camera objects (camera.scene indexes scenes)
    name: str = ""

    @property
    def n_scenes(self) -> int:
        return len(self.scene_offsets) - 1


# ---------------------------------------------------------------------------
# geometric helpers (input construction only)


def rng_streams(seed_id: int, n: int):
    """Independent sub-streams of PCG64 seeded by SeedSequence(1000 + id)."""
    ss = np.random.SeedSequence(1000 + int(seed_id))
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


def fibonacci_sphere(n: int) -> np.ndarray:
    """Unit vectors on the i + 0.5 Fibonacci lattice (area-uniform)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    y = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - y * y))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    phi = golden * i
    return np.stack([r * np.cos(phi), y, r * np.sin(phi)], axis=1)


def onb_from_normal(n: np.ndarray):
    """Branchless orthonormal basis of Duff et al. 2017 ("Building an
    Orthonormal Basis, Revisited", JCGT 6(1)); returns (b1, b2) with
    b1 x b2 = n for unit n."""
    x, y, z = n[:, 0], n[:, 1], n[:, 2]
    sign = np.where(z >= 0.0, 1.0, -1.0)
    a = -1.0 / (sign + z)
    b = x * y * a
    b1 = np.stack([1.0 + sign * x * x * a, sign * b, -sign * x], axis=1)
    b2 = np.stack([b, sign + y * y * a, -y], axis=1)
    # enforce a right-handed frame (b1, b2, n)
    flip = np.einsum("ij,ij->i", np.cross(b1, b2), n) < 0
    b2[flip] *= -1.0
    return b1, b2


def quat_from_frames(t1: np.ndarray, t2: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Quaternion (w,x,y,z) of the rotation whose columns are (t1, t2, n)."""
    R = np.stack([t1, t2, n], axis=2)  # [N,3,3], columns
    m00, m11, m22 = R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]
    tr = m00 + m11 + m22
    q = np.zeros((R.shape[0], 4))
    # Shepperd's method, picking the largest pivot per row
    piv = np.argmax(np.stack([tr, m00, m11, m22], axis=1), axis=1)
    for k in range(4):
        s = piv == k
        if not np.any(s):
            continue
        Rs = R[s]
        if k == 0:
            r = np.sqrt(1.0 + tr[s]) * 2
            q[s] = np.stack([0.25 * r, (Rs[:, 2, 1] - Rs[:, 1, 2]) / r,
                             (Rs[:, 0, 2] - Rs[:, 2, 0]) / r, (Rs[:, 1, 0] - Rs[:, 0, 1]) / r], 1)
        elif k == 1:
            r = np.sqrt(1.0 + m00[s] - m11[s] - m22[s]) * 2
            q[s] = np.stack([(Rs[:, 2, 1] - Rs[:, 1, 2]) / r, 0.25 * r,
                             (Rs[:, 0, 1] + Rs[:, 1, 0]) / r, (Rs[:, 0, 2] + Rs[:, 2, 0]) / r], 1)
        elif k == 2:
            r = np.sqrt(1.0 + m11[s] - m00[s] - m22[s]) * 2
            q[s] = np.stack([(Rs[:, 0, 2] - Rs[:, 2, 0]) / r, (Rs[:, 0, 1] + Rs[:, 1, 0]) / r,
                             0.25 * r, (Rs[:, 1, 2] + Rs[:, 2, 1]) / r], 1)
        else:
            r = np.sqrt(1.0 + m22[s] - m00[s] - m11[s]) * 2
            q[s] = np.stack([(Rs[:, 1, 0] - Rs[:, 0, 1]) / r, (Rs[:, 0, 2] + Rs[:, 2, 0]) / r,
                             (Rs[:, 1, 2] + Rs[:, 2, 1]) / r, 0.25 * r], 1)
    return q


def tangent_quats(normals: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """Quaternions whose local z is the normal and whose in-plane frame is
    the Duff basis rotated by a seeded angle."""
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    b1, b2 = onb_from_normal(n)
    psi = rng.uniform(0.0, 2.0 * math.pi, size=n.shape[0])
    c, s = np.cos(psi)[:, None], np.sin(psi)[:, None]
    t1 = c * b1 + s * b2
    t2 = -s * b1 + c * b2
    return quat_from_frames(t1, t2, n)


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_deg=60.0,
            width=128, height=128, scene=0) -> Camera:
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    up = np.asarray(up, np.float64)
    if abs(float(np.dot(z, up))) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    t = -R @ eye
    f = 0.5 * height / math.tan(math.radians(fov_deg) * 0.5)
    return Camera(R=R, t=t, fx=f, fy=f, cx=0.5 * width, cy=0.5 * height,
                  width=int(width), height=int(height), scene=int(scene))


def lognormal_env(rng: np.random.Generator, We: int, He: int, sigma=1.0) -> np.ndarray:
    return np.exp(rng.normal(0.0, sigma, size=(He, We, 3))).astype(np.float32)


def _pack(pos, quat, log_scale, albedo, rough, metal) -> Surfels:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Surfels(f(pos), f(quat), f(log_scale), f(albedo), f(rough), f(metal))


# ---------------------------------------------------------------------------
# surfaces


def sphere_surfels(rng, n, radius=1.0, center=(0, 0, 0), scale=0.03, fib=True):
    d = fibonacci_sphere(n) if fib else _uniform_dirs(rng, n)
    pos = np.asarray(center) + radius * d
    quat = tangent_quats(d, rng)
    ls = np.full((n, 2), math.log(scale))
    return pos, quat, ls


def _uniform_dirs(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def torus_points(rng, n, R=1.0, r=0.35):
    """Area-uniform points on a torus around the y axis (rejection on the
    area element (R + r cos th))."""
    out_t, out_p = [], []
    need = n
    while need > 0:
        th = rng.uniform(0, 2 * math.pi, size=2 * need + 16)
        ph = rng.uniform(0, 2 * math.pi, size=2 * need + 16)
        acc = rng.uniform(0, 1, size=th.size) < (R + r * np.cos(th)) / (R + r)
        out_t.append(th[acc]); out_p.append(ph[acc])
        need -= int(acc.sum())
    th = np.concatenate(out_t)[:n]
    ph = np.concatenate(out_p)[:n]
    ring = np.stack([np.cos(ph), np.zeros_like(ph), np.sin(ph)], 1)
    pos = (R + r * np.cos(th))[:, None] * ring + (r * np.sin(th))[:, None] * np.array([0, 1.0, 0])
    nrm = np.cos(th)[:, None] * ring + np.sin(th)[:, None] * np.array([0, 1.0, 0])
    return pos, nrm


def displaced_sphere_points(rng, n, amp=0.05, freq=8.0):
    """Area-uniform points on r(th, ph) = 1 + amp sin(f th) sin(f ph)
    (th polar from +y), by rejection on the analytic area element, with
    analytic normals."""
    def geom(th, ph):
        s, c = np.sin(th), np.cos(th)
        sp, cp = np.sin(ph), np.cos(ph)
        r = 1.0 + amp * np.sin(freq * th) * np.sin(freq * ph)
        r_th = amp * freq * np.cos(freq * th) * np.sin(freq * ph)
        r_ph = amp * freq * np.sin(freq * th) * np.cos(freq * ph)
        d = np.stack([s * cp, c * np.ones_like(ph), s * sp], 1)
        d_th = np.stack([c * cp, -s * np.ones_like(ph), c * sp], 1)
        d_ph = np.stack([-s * sp, np.zeros_like(ph), s * cp], 1)
        p = r[:, None] * d
        p_th = r_th[:, None] * d + r[:, None] * d_th
        p_ph = r_ph[:, None] * d + r[:, None] * d_ph
        nrm = np.cross(p_ph, p_th)
        area = np.linalg.norm(nrm, axis=1)
        nrm = nrm / area[:, None]
        flip = np.einsum("ij,ij->i", nrm, d) < 0
        nrm[flip] *= -1
        return p, nrm, area
    # area / sin(th) = r sqrt(r^2 + r_th^2 + (r_ph / sin th)^2) and
    # |sin(f th) / sin th| <= f, so this bounds the acceptance ratio by 1
    bound = (1 + amp) * math.sqrt((1 + amp) ** 2 + (amp * freq) ** 2 + (amp * freq * freq) ** 2)
    ps, ns = [], []
    need = n
    while need > 0:
        m = int(need * 4) + 64
        th = np.arccos(np.clip(rng.uniform(-1, 1, size=m), -1, 1))
        ph = rng.uniform(0, 2 * math.pi, size=m)
        p, nrm, area = geom(th, ph)
        # sampling density of (cos th uniform, ph uniform) is prop. to sin th
        w = area / (np.sin(th) * bound)
        assert np.all(w <= 1.0 + 1e-9)
        acc = rng.uniform(0, 1, size=m) < w
        ps.append(p[acc]); ns.append(nrm[acc])
        need -= int(acc.sum())
    return np.concatenate(ps)[:n], np.concatenate(ns)[:n]


def displaced_sphere_area(amp=0.05, freq=8.0, n=2048) -> float:
    th = (np.arange(n) + 0.5) * math.pi / n
    ph = (np.arange(2 * n) + 0.5) * math.pi / n
    T, P = np.meshgrid(th, ph, indexing="ij")
    s, c = np.sin(T), np.cos(T)
    r = 1.0 + amp * np.sin(freq * T) * np.sin(freq * P)
    r_th = amp * freq * np.cos(freq * T) * np.sin(freq * P)
    r_ph = amp * freq * np.sin(freq * T) * np.cos(freq * P)
    # |p_th x p_ph| = r sqrt(r^2 s^2 + r_th^2 s^2 + r_ph^2)
    dA = r * np.sqrt(r * r * s * s + r_th * r_th * s * s + r_ph * r_ph)
    return float(dA.sum() * (math.pi / n) ** 2)


def value_noise3(rng, p: np.ndarray, freq=4.0) -> np.ndarray:
    """Seeded 3D value noise: random lattice values at integer points of
    freq * p, trilinear with smoothstep weights, in [0, 1]."""
    L = 64
    lat = rng.uniform(0, 1, size=(L, L, L))
    q = p * freq + 32.0
    i = np.floor(q).astype(np.int64)
    f = q - i
    f = f * f * (3 - 2 * f)
    out = np.zeros(p.shape[0])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (np.where(dx, f[:, 0], 1 - f[:, 0]) * np.where(dy, f[:, 1], 1 - f[:, 1])
                     * np.where(dz, f[:, 2], 1 - f[:, 2]))
                out += w * lat[(i[:, 0] + dx) % L, (i[:, 1] + dy) % L, (i[:, 2] + dz) % L]
    return out


# ---------------------------------------------------------------------------
# the five workloads


def fib_cameras(n, radius, fov=60.0, width=800, height=800, scene=0, center=(0, 0, 0)):
    d = fibonacci_sphere(n)
    c = np.asarray(center, np.float64)
    return [look_at(c + radius * d[i], c, fov_deg=fov, width=width, height=height, scene=scene)
            for i in range(n)]


def sphere_4k(n=4096, res=128, seed_id=1) -> Scene:
    """4096 Fibonacci surfels on the unit sphere, isotropic tangent std 0.03,
    one 128^2 view at distance 3, 64x32 log-normal env."""
    r_geo, r_att, r_env, _ = rng_streams(seed_id, 4)
    pos, quat, ls = sphere_surfels(r_geo, n, scale=0.03)
    alb = r_att.uniform(0, 1, size=(n, 3))
    rough = r_att.uniform(0.1, 0.9, size=n)
    metal = np.zeros(n)
    s = _pack(pos, quat, ls, alb, rough, metal)
    env = lognormal_env(r_env, 64, 32)
    cam = look_at((0.0, 0.0, 3.0), width=res, height=res)
    return Scene(s, np.array([0, n], np.int64), [env], [cam], "sphere_4k")


def torus_sphere_surfels(rng_geo, rng_att, n, scale_lo=0.005, scale_hi=0.02):
    a_t = 4 * math.pi ** 2 * 1.0 * 0.35
    a_s = 4 * math.pi * 0.6 ** 2
    n_t = int(round(n * a_t / (a_t + a_s)))
    n_s = n - n_t
    pt, nt = torus_points(rng_geo, n_t)
    ds = _uniform_dirs(rng_geo, n_s)
    ps = np.array([0.8, 0.4, 0.0]) + 0.6 * ds
    pos = np.concatenate([pt, ps])
    nrm = np.concatenate([nt, ds])
    quat = tangent_quats(nrm, rng_geo)
    ls = np.log(rng_geo.uniform(scale_lo, scale_hi, size=(n, 2)))
    alb = rng_att.uniform(0, 1, size=(n, 3))
    rough = rng_att.uniform(0.05, 1.0, size=n)
    metal = (rng_att.uniform(0, 1, size=n) < 0.3).astype(np.float64)
    return pos, quat, ls, alb, rough, metal


def torus_sphere_100k(n=100_000, res=512, seed_id=2) -> Scene:
    """Torus (R=1, r=0.35) U sphere (r=0.6 at (0.8,0.4,0)), anisotropic
    scales U[0.005,0.02], one 512^2 view at distance 3, elevation 30 deg,
    azimuth 45 deg, 256x128 log-normal env."""
    r_geo, r_att, r_env, _ = rng_streams(seed_id, 4)
    s = _pack(*torus_sphere_surfels(r_geo, r_att, n))
    env = lognormal_env(r_env, 256, 128)
    el, az = math.radians(30.0), math.radians(45.0)
    eye = 3.0 * np.array([math.cos(el) * math.sin(az), math.sin(el), math.cos(el) * math.cos(az)])
    cam = look_at(eye, width=res, height=res)
    return Scene(s, np.array([0, n], np.int64), [env], [cam], "torus_sphere_100k")


def displaced_sphere_surfels(rng_geo, rng_att, n, attrs="uniform"):
    pos, nrm = displaced_sphere_points(rng_geo, n)
    quat = tangent_quats(nrm, rng_geo)
    s = math.sqrt(displaced_sphere_area() / n)
    ls = np.full((n, 2), math.log(s))
    if attrs == "uniform":
        alb = rng_att.uniform(0, 1, size=(n, 3))
        rough = rng_att.uniform(0, 1, size=n)
    else:  # spatially varying (value noise)
        alb = np.stack([value_noise3(rng_att, pos) for _ in range(3)], 1)
        rough = 0.05 + 0.9 * value_noise3(rng_att, pos)
    metal = (rng_att.uniform(0, 1, size=n) < 0.3).astype(np.float64)
    return pos, quat, ls, alb, rough, metal


def displaced_sphere_1m(n=1_000_000, views=16, res=800, env_w=512, seed_id=3) -> Scene:
    """1M surfels on the displaced sphere r = 1 + 0.05 sin(8th) sin(8ph),
    isotropic scale sqrt(area/N), 16 Fibonacci views at radius 3, 800^2,
    512x256 log-normal env."""
    r_geo, r_att, r_env, _ = rng_streams(seed_id, 4)
    s = _pack(*displaced_sphere_surfels(r_geo, r_att, n))
    env = lognormal_env(r_env, env_w, env_w // 2)
    cams = fib_cameras(views, 3.0, width=res, height=res)
    return Scene(s, np.array([0, n], np.int64), [env], cams, "displaced_sphere_1m")


def uneven_scenes(n_scenes=8, views_per_scene=4, seed_id=4, n_lo=50_000, n_hi=2_000_000,
            resolutions=(256, 512, 800, 1024)) -> Scene:
    """Uneven batch: 8 scenes with log-uniform surfel counts, alternating the
    sphere (sphere_4k) and torus U sphere (torus_sphere_100k) generators with seeded
    scale and offset, 4 views each at random resolutions, one 256x128 env per
    scene."""
    r_meta, r_geo, r_att, r_env = rng_streams(seed_id, 4)
    parts, offs, envs, cams = [], [0], [], []
    for k in range(n_scenes):
        nk = int(round(math.exp(r_meta.uniform(math.log(n_lo), math.log(n_hi)))))
        scale = r_meta.uniform(0.5, 1.5)
        off = r_meta.uniform(-0.5, 0.5, size=3)
        if k % 2 == 0:
            pos, quat, ls = sphere_surfels(r_geo, nk, scale=0.03 * math.sqrt(4096.0 / nk))
            alb = r_att.uniform(0, 1, size=(nk, 3))
            rough = r_att.uniform(0.1, 0.9, size=nk)
            metal = np.zeros(nk)
        else:
            pos, quat, ls, alb, rough, metal = torus_sphere_surfels(r_geo, r_att, nk)
        pos = pos * scale + off
        ls = ls + math.log(scale)
        parts.append(_pack(pos, quat, ls, alb, rough, metal))
        offs.append(offs[-1] + nk)
        envs.append(lognormal_env(r_env, 256, 128))
        dirs = fibonacci_sphere(views_per_scene)
        for i in range(views_per_scene):
            res = int(resolutions[r_meta.integers(0, len(resolutions))])
            eye = off + 3.0 * scale * dirs[i]
            cams.append(look_at(eye, off, width=res, height=res, scene=k))
    return Scene(Surfels.concat(parts), np.array(offs, np.int64), envs, cams, "uneven_scenes")


def loop_ground_truth(n=1_500_000, targets=64, res=1024, seed_id=5) -> Scene:
    """Ground truth of the inverse-rendering loop: displaced sphere with
    value-noise albedo/roughness, 64 targets of 1024^2, 512x256 env."""
    r_geo, r_att, r_env, _ = rng_streams(seed_id, 4)
    s = _pack(*displaced_sphere_surfels(r_geo, r_att, n, attrs="noise"))
    env = lognormal_env(r_env, 512, 256)
    cams = fib_cameras(targets, 3.0, width=res, height=res)
    return Scene(s, np.array([0, n], np.int64), [env], cams, "loop_ground_truth")


def loop_init(n=3_000_000, seed_id=55, env_w=512) -> tuple:
    """Initial state of the loop: 3M isotropic surfels on a sphere of radius
    1.2, random attributes, constant 0.5 env."""
    r_geo, r_att, _, _ = rng_streams(seed_id, 4)
    d = _uniform_dirs(r_geo, n)
    pos = 1.2 * d
    quat = tangent_quats(d, r_geo)
    s = math.sqrt(4 * math.pi * 1.44 / n)
    ls = np.full((n, 2), math.log(s))
    alb = r_att.uniform(0, 1, size=(n, 3))
    rough = r_att.uniform(0.05, 1.0, size=n)
    metal = r_att.uniform(0, 1, size=n) * 0.5
    env = np.full((env_w // 2, env_w, 3), 0.5, np.float32)
    return _pack(pos, quat, ls, alb, rough, metal), env


def checkerboard_plane(n_side=2000, spacing=0.01, cell=0.1, width=800, height=600, supersample=1,
                       seed_id=6) -> Scene:
    """A point-sampled checkerboard ground plane receding to the horizon (the
    MIP-filter ablation's workload, Sec. 4.4.2): n_side^2 surfels on a
    jittered square grid of the given spacing in the plane y = 0 (x centred,
    z from 0 to n_side * spacing), normal +y, isotropic scale = spacing,
    albedo 0.9 / 0.1 in cells of `cell`, roughness 0.5, dielectric; a
    camera 1 above the plane looking along it (60 degree vertical FOV) sees
    surfels a few pixels apart in front and ever more minified towards the
    horizon; constant env 1.  supersample multiplies the resolution and the
    focal length (the supersampled reference renders the same view at 2x)."""
    r_geo, r_att, _, _ = rng_streams(seed_id, 4)
    n = n_side * n_side
    k = np.arange(n_side, dtype=np.float64)
    X, Z = np.meshgrid((k - (n_side - 1) / 2.0) * spacing, (k + 0.5) * spacing, indexing="xy")
    jit = r_geo.uniform(-0.25, 0.25, size=(2, n)) * spacing
    x, z = X.ravel() + jit[0], Z.ravel() + jit[1]
    pos = np.stack([x, np.zeros(n), z], 1)
    nrm = np.tile([0.0, 1.0, 0.0], (n, 1))
    quat = tangent_quats(nrm, r_att)
    ls = np.full((n, 2), math.log(spacing))
    black = ((np.floor(x / cell) + np.floor(z / cell)) % 2) == 0
    alb = np.where(black[:, None], 0.1, 0.9) * np.ones((1, 3))
    s = _pack(pos, quat, ls, alb, np.full(n, 0.5), np.zeros(n))
    env = np.ones((32, 64, 3), np.float32)
    cam = look_at((0.0, 1.0, -0.5), (0.0, 0.2, 10.0), fov_deg=60.0, width=width * supersample,
                  height=height * supersample)
    return Scene(s, np.array([0, n], np.int64), [env], [cam], "checkerboard_plane")


def by_name(name: str, **kw) -> Scene:
    return {"sphere_4k": sphere_4k, "torus_sphere_100k": torus_sphere_100k, "displaced_sphere_1m": displaced_sphere_1m,
            "uneven_scenes": uneven_scenes, "loop_ground_truth": loop_ground_truth,
            "checkerboard_plane": checkerboard_plane}[name](**kw)
