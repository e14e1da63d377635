"""The seeded input generators (shared by the oracle tests and the GPU path):
deterministic, and the surfaces, frames and cameras are what their recipes
say."""
import math

import numpy as np

from paper_2605_05876_gb300 import scenes as S


def _rot(q):
    """Rotation matrices of unit quaternions (w, x, y, z), [N, 3, 3]."""
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def test_generators_are_deterministic():
    for make in (lambda: S.sphere_4k(n=512, res=32), lambda: S.torus_sphere_100k(n=3000, res=64),
                 lambda: S.uneven_scenes(n_scenes=2, views_per_scene=1, n_lo=1000, n_hi=3000)):
        a, b = make(), make()
        for f in ("pos", "quat", "log_scale", "albedo", "roughness", "metallic"):
            assert np.array_equal(getattr(a.surfels, f), getattr(b.surfels, f)), f
        assert np.array_equal(a.scene_offsets, b.scene_offsets)
        assert all(np.array_equal(x, y) for x, y in zip(a.envs, b.envs))
        assert all(np.array_equal(x.R, y.R) and np.array_equal(x.t, y.t) for x, y in zip(a.cameras, b.cameras))


def test_fibonacci_sphere_is_unit_and_balanced():
    d = S.fibonacci_sphere(4096)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    assert np.abs(d.mean(0)).max() < 1e-3          # area-uniform lattice: centroid at the origin
    # equal-area bands: as many points above y = 0.5 as below y = -0.5 (each 1/4 of the area)
    assert abs((d[:, 1] > 0.5).mean() - 0.25) < 2e-3 and abs((d[:, 1] < -0.5).mean() - 0.25) < 2e-3


def test_displaced_sphere_points_lie_on_the_surface_with_outward_normals():
    rng = np.random.default_rng(0)
    p, n = S.displaced_sphere_points(rng, 20000)
    r = np.linalg.norm(p, axis=1)
    th = np.arccos(np.clip(p[:, 1] / r, -1, 1))
    ph = np.arctan2(p[:, 2], p[:, 0])
    assert np.abs(r - (1.0 + 0.05 * np.sin(8 * th) * np.sin(8 * ph))).max() < 1e-9
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-9)
    assert (np.einsum("ij,ij->i", n, p / r[:, None]) > 0).all()
    # the normal is orthogonal to the surface: a small step in its tangent
    # plane leaves the surface only to second order, unlike a step
    # orthogonal to the plain radial direction (the undisplaced normal)
    def off_surface(nn):
        t = np.cross(nn, np.array([0.3, 0.5, 0.7]))
        t /= np.linalg.norm(t, axis=1, keepdims=True)
        q = p + 1e-5 * t
        rq = np.linalg.norm(q, axis=1)
        thq = np.arccos(np.clip(q[:, 1] / rq, -1, 1))
        phq = np.arctan2(q[:, 2], q[:, 0])
        return np.abs(rq - (1.0 + 0.05 * np.sin(8 * thq) * np.sin(8 * phq)))
    away = np.abs(p[:, 1] / r) < 0.95               # clear of the poles of (theta, phi)
    off_n, off_radial = off_surface(n)[away], off_surface(p / r[:, None])[away]
    assert np.median(off_n) < 1e-9 and np.median(off_radial) > 1e-7
    assert off_n.max() < 1e-2 * off_radial.max()


def test_tangent_frames_put_the_normal_on_local_z():
    rng = np.random.default_rng(1)
    nrm = S.fibonacci_sphere(1000)
    q = S.tangent_quats(nrm, rng)
    R = _rot(q)
    assert np.allclose(np.einsum("nij,nkj->nik", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)
    assert np.allclose(R[:, :, 2], nrm, atol=1e-12)


def test_look_at_centres_the_target():
    cam = S.look_at((0.5, 0.3, 2.8), target=(0.1, -0.2, 0.0), width=64, height=48, fov_deg=60.0)
    R, t = cam.R, cam.t
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert np.allclose(R @ np.array([0.5, 0.3, 2.8]) + t, 0.0, atol=1e-12)   # camera centre
    c = R @ np.array([0.1, -0.2, 0.0]) + t
    assert c[2] > 0
    assert abs(cam.fx * c[0] / c[2] + cam.cx - 32.0) < 1e-9 and abs(cam.fy * c[1] / c[2] + cam.cy - 24.0) < 1e-9
    # the vertical field of view spans the image height
    assert abs(2.0 * math.degrees(math.atan(0.5 * cam.height / cam.fy)) - 60.0) < 1e-9


def test_displaced_sphere_1m_recipe():
    sc = S.displaced_sphere_1m(n=20000, views=4, res=64, env_w=64)
    s = sc.surfels
    assert s.n == 20000 and len(sc.cameras) == 4 and sc.envs[0].shape == (32, 64, 3)
    scale = math.sqrt(S.displaced_sphere_area() / 20000)
    assert np.allclose(s.log_scale, math.log(scale), atol=1e-6)   # isotropic, area-matched
    assert set(np.unique(s.metallic)) <= {0.0, 1.0}
    for cam in sc.cameras:
        eye = -cam.R.T @ cam.t
        assert abs(np.linalg.norm(eye) - 3.0) < 1e-9                  # views on a sphere of radius 3
