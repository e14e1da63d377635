"""Tiny hand-built scenes for pins and parity tests (input data only)."""
import math

import numpy as np

from paper_2605_05876_gb300 import scenes as S


def surfels(pos, normals=None, scale=0.05, albedo=None, rough=0.5, metal=0.0, rng=None, quat=None):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    if quat is None:
        if normals is None:
            quat = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
        else:
            rng = rng or np.random.default_rng(0)
            quat = S.tangent_quats(np.asarray(normals, np.float64).reshape(-1, 3), rng)
    sc = np.broadcast_to(np.asarray(scale, np.float64), (n,)) if np.ndim(scale) < 2 else scale
    ls = np.log(np.stack([sc, sc], 1)) if np.ndim(scale) < 2 else np.log(scale)
    if albedo is None:
        albedo = np.full((n, 3), 0.5)
    albedo = np.broadcast_to(np.asarray(albedo, np.float64), (n, 3))
    return S._pack(pos, quat, ls, albedo, np.broadcast_to(rough, (n,)), np.broadcast_to(metal, (n,)))


def grid_plane(n_side, spacing, z=0.0, scale=None, albedo=(0.5, 0.5, 0.5), center=(0.0, 0.0)):
    """Fronto-parallel (normal +z) regular grid of surfels in the plane z."""
    k = (np.arange(n_side) - (n_side - 1) / 2.0) * spacing
    X, Y = np.meshgrid(k + center[0], k + center[1], indexing="xy")
    pos = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1)
    return surfels(pos, scale=spacing if scale is None else scale, albedo=albedo)


def front_camera(dist=3.0, res=32, fov=60.0, width=None):
    return S.look_at((0.0, 0.0, dist), (0.0, 0.0, 0.0), width=width or res, height=res, fov_deg=fov)


def const_env(value=1.0, We=32, He=16):
    return np.full((He, We, 3), value, np.float32)


def random_scene(rng, n=48, spread=0.4, scale=(0.03, 0.12)):
    pos = rng.uniform(-spread, spread, size=(n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm[:, 2] = np.abs(nrm[:, 2]) + 0.3    # mostly facing the camera on +z
    sc = rng.uniform(*scale, size=(n, 2))
    quat = S.tangent_quats(nrm, rng)
    return S._pack(pos, quat, np.log(sc), rng.uniform(0, 1, (n, 3)), rng.uniform(0.05, 1.0, n),
                   (rng.uniform(0, 1, n) < 0.3).astype(np.float64))


def lognormal_env(rng, We=32, He=16):
    return np.exp(rng.normal(0.0, 1.0, size=(He, We, 3))).astype(np.float32)
