"""The screen-space form of the per-pixel test that the CUDA kernels evaluate
equals the paper's ray-plane form, on the CPU in FP64.

The paper (Sec. 3.1, Eq. mip_weight) intersects the pixel's two planes with
the surfel plane through the T-matrix rows (k x l) and evaluates
rho^2 = (u, v) Sigma_mip^-1 (u, v)^T with Sigma_mip = I + sigma_f J J^T at the
centre (Sec. 3.3.2).  The kernels instead evaluate, for the pixel offset d
from the projected centre,

    rho^2 = d^T (M M^T + sigma_f I)^-1 d / s2(d)^2,   s2 = 1 + A2 d_x + B2 d_y,
    n_f = |det M| / sqrt(det(M M^T + sigma_f I)),

with M = d(x, y)/d(u, v) at the centre (J = M^-1) and
(A2, B2) = c'_z (n'_x / f_x, n'_y / f_y) / (n . (c - o)) from the surfel
plane's normal and the camera's distance to it: the hit point is linear in
d up to the perspective factor s2, and J^T (I + sigma_f J J^T)^-1 J =
(M M^T + sigma_f I)^-1.  This test rebuilds that form from the surfel
parameters and the pinhole model alone and compares it with the oracle's
records (T rows, Sigma^-1, n_f) and its k x l evaluation at many pixels."""
import numpy as np
import pytest
import torch

from oracle import model as M
from tests import _tiny


def _rot(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _screen_form(surf, cam, sigma_f):
    """Per surfel: projected centre p, Qs = (M M^T + sigma_f I)^-1, g = (A2, B2)
    and n_f, from the parameters and the pinhole model (float32 inputs taken
    as given, FP64 arithmetic)."""
    cd = M.cam_dict(cam)
    R, t = cd["R"].numpy(), cd["t"].numpy()
    fx, fy, cx, cy = cd["fx"], cd["fy"], cd["cx"], cd["cy"]
    pos = surf.pos.astype(np.float64)
    Rs = _rot(surf.quat.astype(np.float64))
    sc = np.exp(surf.log_scale.astype(np.float64))
    c = pos @ R.T + t                                       # camera-space centre c'
    tu = (Rs[:, :, 0] * sc[:, :1]) @ R.T                    # camera-space scaled tangents
    tv = (Rs[:, :, 1] * sc[:, 1:]) @ R.T
    n = Rs[:, :, 2] @ R.T                                   # camera-space plane normal
    m = c[:, :2] / c[:, 2:3]
    a = tu[:, :2] - m * tu[:, 2:3]
    b = tv[:, :2] - m * tv[:, 2:3]
    Mx = np.stack([np.stack([fx * a[:, 0], fx * b[:, 0]], -1), np.stack([fy * a[:, 1], fy * b[:, 1]], -1)], -2)
    Mx /= c[:, 2, None, None]
    G = Mx @ np.swapaxes(Mx, 1, 2) + sigma_f * np.eye(2)
    Qs = np.linalg.inv(G)
    Nd = (n * c).sum(-1)                                    # n . (c - o) in camera space
    g = np.stack([c[:, 2] * n[:, 0] / (fx * Nd), c[:, 2] * n[:, 1] / (fy * Nd)], -1)
    nf = np.abs(np.linalg.det(Mx)) / np.sqrt(np.linalg.det(G))
    p = np.stack([fx * m[:, 0] + cx, fy * m[:, 1] + cy], -1)
    return p, Qs, g, nf


@pytest.mark.parametrize("sigma_f", [0.0, 0.5, 2.0])
def test_screen_form_equals_the_ray_plane_form(sigma_f):
    rng = np.random.default_rng(71)
    surf = _tiny.random_scene(rng, n=60, spread=0.4, scale=(0.03, 0.12))
    cam = _tiny.front_camera(res=40, width=52)
    prm = M.Params(sigma_f=sigma_f)
    env = M.prepare_env(_tiny.const_env(), prm, lut_nq=16)
    with torch.no_grad():
        rec = M.records(M.to_torch_surfels(surf), M.cam_dict(cam), torch.from_numpy(env.irr),
                        [torch.from_numpy(lv) for lv in env.levels], torch.from_numpy(env.lut), prm)
    T, Sinv, nf_ref = rec["T"].numpy(), rec["Sinv"].numpy(), rec["n_f"].numpy()
    ok = rec["valid"].numpy()
    assert ok.sum() > 40
    p, Qs, g, nf = _screen_form(surf, cam, sigma_f)
    np.testing.assert_allclose(nf[ok], nf_ref[ok], rtol=1e-10)
    # pixel centres around each surfel's projected centre, within a few footprints
    n_checked = 0
    for i in np.where(ok)[0]:
        ext = 3.0 * np.sqrt(np.diag(np.linalg.inv(Qs[i])))
        xs = np.floor(p[i, 0] + np.linspace(-ext[0], ext[0], 7)) + 0.5
        ys = np.floor(p[i, 1] + np.linspace(-ext[1], ext[1], 7)) + 0.5
        X, Y = np.meshgrid(xs, ys)
        X, Y = X.ravel(), Y.ravel()
        # the paper's form: the two pixel planes pulled back through T meet at (u, v)
        k = X[:, None] * T[i, 2] - T[i, 0]
        l = Y[:, None] * T[i, 2] - T[i, 1]
        s = np.cross(k, l)
        u, v = s[:, 0] / s[:, 2], s[:, 1] / s[:, 2]
        S = Sinv[i]
        rho2_paper = S[0, 0] * u * u + 2 * S[0, 1] * u * v + S[1, 1] * v * v
        # the kernels' form
        d = np.stack([X - p[i, 0], Y - p[i, 1]], -1)
        s2 = 1.0 + d @ g[i]
        front = s2 > 0.05                                   # the pixel's ray meets the plane in front
        q = np.einsum("pi,ij,pj->p", d, Qs[i], d)
        rho2_screen = q / s2 ** 2
        np.testing.assert_allclose(rho2_screen[front], rho2_paper[front], rtol=1e-9, atol=1e-12)
        n_checked += int(front.sum())
    assert n_checked > 2000
