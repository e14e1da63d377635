"""FP64 oracle of the 3DSS renderer (forward values and gradients).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference arm of ``bench.py`` may import this module.  It
shares no code with the CUDA path (``paper_2605_05876_gb300``) and imports
nothing from it; both sides read the same seeded inputs.

The oracle is the method written out plainly, in double precision:

* per surfel and view (``records``): the T-matrix rows (Sec. 3.1), the depth
  interval (Sec. 3.1, Sec. 3.2.1), the centre-precomputed MIP covariance of
  Eq. mip_cov with n_f of Eq. mip_eval (Sec. 3.3.2 applies them at the
  centre), and the forward-shaded split-sum colour of Eq. ibl (Sec. 3.4);
* per pixel: the discrete decisions of Algorithm 1 (which surfels cover it,
  the order by z_start, the layer of each, the K_max cap) come from the C
  half (``ss3d_oracle.c``);
* the values -- weights (Eq. mip_weight), Shepard sums (Eq. shepard),
  coverage opacity (Eq. alpha), front-to-back compositing and residual
  transmittance (Eq. compositing) -- are PyTorch FP64 ops, so the gradient
  of any loss is PyTorch autograd with every discrete decision held fixed
  (which is the definition of the gradient used here).

Every reading where the paper is silent is restated at the function that
applies it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from functools import lru_cache

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ss3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libss3d_oracle.so")

F64 = torch.float64

# channel layout of the per-surfel payload that layers average
# 0..2 shaded RGB, 3..5 albedo, 6 roughness, 7 metallic, 8..10 normal, 11 depth
N_CH = 12
NORMAL = slice(8, 11)


@dataclasses.dataclass
class Params:
    """Renderer constants.  r_cut = 3 (App. A "Cutoff radius"),
    gamma = 2 pi (Sec. 3.5.1), K_max = 16 (App. A "Maximum layer count").
    sigma_f (the screen prefilter variance of Eq. mip_cov) is not given by
    the paper; 0.5 px^2 is the default here.  z_near and the background
    are not given either."""
    r_cut: float = 3.0
    sigma_f: float = 0.5
    gamma: float = 2.0 * math.pi
    k_max: int = 16
    z_near: float = 0.01
    bg: tuple = (0.0, 0.0, 0.0)
    env_levels: int = 6
    irr_w: int = 32
    irr_h: int = 16
    lut_n: int = 128
    # MIP filter (Sec. 3.3): "centre" -- the method, Sigma_mip and n_f at the
    # surfel centre (Sec. 3.3.2); "none" -- no band limiting (Sigma_mip = I,
    # n_f = 1, i.e. sigma_f = 0); "pixel" -- the per-pixel Jacobian of
    # AA-2DGS (Sec. 3.3.1), Sigma_mip and n_f at every hit (the Sec. 4.4.2
    # ablation)
    mip_mode: str = "centre"
    # the depth-consolidation term of Eq. cons_loss (Sec. 3.7.1) as a tenth
    # AOV column: per pixel, over its composited layers,
    # sum_{i<j} w_i w_j |z_i - z_j| + sum_i w_i^2 sigma_i^2
    cons: bool = False

    def sigma_eff(self) -> float:
        return 0.0 if self.mip_mode == "none" else self.sigma_f

    def pp_sigma(self) -> float:
        """Argument of the C half: the per-pixel filter's sigma_f, or -1."""
        return self.sigma_f if self.mip_mode == "pixel" else -1.0


# ---------------------------------------------------------------------------
# the C half


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


@lru_cache(maxsize=1)
def lib():
    L = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.oref_brdf_lut.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
    L.oref_brdf_eval.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, dp, dp, dp]
    L.oref_spec_levels_size.argtypes = [ctypes.c_int] * 3
    L.oref_spec_levels_size.restype = ctypes.c_longlong
    L.oref_env_prefilter.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, dp, dp]
    L.oref_env_adjoint.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, dp]
    L.oref_fragments.argtypes = [ctypes.c_int, dp, dp, dp, u8p, dp, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, i32p, i32p, dp,
                                 i64p, i64p, i32p, i32p, i32p]
    L.oref_fragments.restype = ctypes.c_longlong
    L.oref_pixel_candidates.argtypes = [ctypes.c_int, dp, dp, dp, u8p, dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, i32p, dp, dp, dp, dp]
    L.oref_pixel_candidates.restype = ctypes.c_int
    return L


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


# ---------------------------------------------------------------------------
# BRDF table and environment levels


@lru_cache(maxsize=4)
def _brdf_lut_np(n: int, nq: int) -> np.ndarray:
    x, w = np.polynomial.legendre.leggauss(nq)
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    out = np.zeros(n * n * 2, np.float64)
    lib().oref_brdf_lut(n, nq, _p(x, ctypes.c_double), _p(w, ctypes.c_double), _p(out, ctypes.c_double))
    return out.reshape(n, n, 2)


def brdf_lut(n: int = 128, nq: int = 128) -> np.ndarray:
    """(beta1, beta2) at cell centres, indexed [roughness][n.v][2]."""
    return _brdf_lut_np(n, nq).copy()


def brdf_eval(mu, r, nq: int = 128) -> np.ndarray:
    """(beta1, beta2) of the split-sum integral at arbitrary (n.v, r)."""
    mu = np.ascontiguousarray(np.atleast_1d(mu), np.float64)
    r = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(r), mu.shape), np.float64)
    x, w = np.polynomial.legendre.leggauss(nq)
    x = np.ascontiguousarray(x)
    w = np.ascontiguousarray(w)
    out = np.zeros((mu.shape[0], 2))
    lib().oref_brdf_eval(mu.shape[0], _p(mu, ctypes.c_double), _p(r, ctypes.c_double), nq,
                         _p(x, ctypes.c_double), _p(w, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def level_sizes(We: int, He: int, L: int):
    return [(max(We >> i, 8), max(He >> i, 4)) for i in range(L)]


def env_prefilter(env: np.ndarray, L: int = 6, Wi: int = 32, Hi: int = 16):
    """Irradiance map [Hi][Wi][3] and the L specular levels (list of
    [H_i][W_i][3]) of an equirect env [He][We][3] (see ss3d_oracle.c)."""
    env = np.ascontiguousarray(env, np.float64)
    He, We, _ = env.shape
    irr = np.zeros((Hi, Wi, 3))
    spec = np.zeros(lib().oref_spec_levels_size(We, He, L))
    lib().oref_env_prefilter(_p(env, ctypes.c_double), We, He, Wi, Hi, L,
                             _p(irr, ctypes.c_double), _p(spec, ctypes.c_double))
    levels, off = [], 0
    for (W, H) in level_sizes(We, He, L):
        levels.append(spec[off:off + W * H * 3].reshape(H, W, 3))
        off += W * H * 3
    return irr, levels


def env_adjoint(d_irr: np.ndarray, d_levels, We: int, He: int):
    """Transpose of env_prefilter: gradient w.r.t. the base env texels."""
    Hi, Wi, _ = d_irr.shape
    L = len(d_levels)
    d_irr = np.ascontiguousarray(d_irr, np.float64)
    d_spec = np.ascontiguousarray(np.concatenate([np.asarray(d, np.float64).ravel() for d in d_levels]))
    out = np.zeros((He, We, 3))
    lib().oref_env_adjoint(_p(d_irr, ctypes.c_double), _p(d_spec, ctypes.c_double), We, He, Wi, Hi, L,
                           _p(out, ctypes.c_double))
    return out


# ---------------------------------------------------------------------------
# texture lookups (bilinear, equirect convention of ss3d_oracle.c)


def dir_to_uv(d: torch.Tensor):
    """phi = atan2(d_x, -d_z), theta = acos(d_y); u = phi / 2 pi + 1/2,
    v = theta / pi."""
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    phi = torch.atan2(d[..., 0], -d[..., 2])
    th = torch.acos(torch.clamp(d[..., 1], -1.0, 1.0))
    return phi / (2.0 * math.pi) + 0.5, th / math.pi


def bilinear_wrap(tex: torch.Tensor, u: torch.Tensor, v: torch.Tensor):
    """Bilinear lookup of tex [H][W][C] at texel-centre coordinates
    (u W - 1/2, v H - 1/2), wrapping in u and clamping in v."""
    H, W, _ = tex.shape
    X = u * W - 0.5
    Y = v * H - 0.5
    x0 = torch.floor(X)
    y0 = torch.floor(Y)
    fx = (X - x0)[..., None]
    fy = (Y - y0)[..., None]
    x0 = x0.long()
    y0 = y0.long()
    xa = torch.remainder(x0, W)
    xb = torch.remainder(x0 + 1, W)
    ya = torch.clamp(y0, 0, H - 1)
    yb = torch.clamp(y0 + 1, 0, H - 1)
    return ((1 - fy) * ((1 - fx) * tex[ya, xa] + fx * tex[ya, xb])
            + fy * ((1 - fx) * tex[yb, xa] + fx * tex[yb, xb]))


def bilinear_clamp(tex: torch.Tensor, u: torch.Tensor, v: torch.Tensor):
    """Bilinear lookup of tex [H][W][C] with u along W, v along H, both in
    [0,1] at cell centres, clamped at the borders."""
    H, W, _ = tex.shape
    X = u * W - 0.5
    Y = v * H - 0.5
    x0 = torch.floor(X)
    y0 = torch.floor(Y)
    fx = (X - x0)[..., None]
    fy = (Y - y0)[..., None]
    x0 = x0.long()
    y0 = y0.long()
    xa = torch.clamp(x0, 0, W - 1)
    xb = torch.clamp(x0 + 1, 0, W - 1)
    ya = torch.clamp(y0, 0, H - 1)
    yb = torch.clamp(y0 + 1, 0, H - 1)
    return ((1 - fy) * ((1 - fx) * tex[ya, xa] + fx * tex[ya, xb])
            + fy * ((1 - fx) * tex[yb, xa] + fx * tex[yb, xb]))


def specular_lookup(levels, d: torch.Tensor, r: torch.Tensor):
    """Roughness-indexed level lookup: level coordinate r (L-1), linear
    between the two nearest levels, bilinear within each."""
    L = len(levels)
    u, v = dir_to_uv(d)
    lc = torch.clamp(r, 0.0, 1.0) * (L - 1)
    i0 = torch.clamp(torch.floor(lc).long(), 0, L - 1)
    f = (lc - i0.to(lc.dtype))[..., None]
    i1 = torch.clamp(i0 + 1, max=L - 1)
    out = torch.zeros(d.shape[:-1] + (3,), dtype=d.dtype)
    for i in range(L):
        w = (1.0 - f) * (i0 == i)[..., None] + f * (i1 == i)[..., None]
        out = out + w * bilinear_wrap(levels[i], u, v)
    return out


# ---------------------------------------------------------------------------
# per surfel and view


def quat_to_rot(q: torch.Tensor):
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def mip_filter(T: torch.Tensor, depth_ok: torch.Tensor, prm: Params):
    """Centre-precomputed MIP filter (Sec. 3.3.2) of T-matrix rows
    T [N, 3, 3] = (T1, T2, T4): J = d(u,v)/d(x,y) at the centre is the inverse
    of M = d(x,y)/d(u,v) there, with x = T1.u/T4.u; Sigma = I + sigma_f J J^T
    (Eq. mip_cov), n_f = sqrt(|I| / |Sigma|) (Eq. mip_eval).  Returns
    (Sigma^-1, n_f, M, valid) with valid = depth_ok and det M != 0."""
    T1, T2, T4 = T[:, 0], T[:, 1], T[:, 2]
    px = T1[:, 2] / T4[:, 2]
    py = T2[:, 2] / T4[:, 2]
    M = torch.stack([
        torch.stack([T1[:, 0] - px * T4[:, 0], T1[:, 1] - px * T4[:, 1]], -1),
        torch.stack([T2[:, 0] - py * T4[:, 0], T2[:, 1] - py * T4[:, 1]], -1)], -2) / T4[:, 2, None, None]
    detM = M[:, 0, 0] * M[:, 1, 1] - M[:, 0, 1] * M[:, 1, 0]
    valid = depth_ok & (detM != 0)
    Msafe = torch.where(valid[:, None, None], M, torch.eye(2, dtype=F64).expand_as(M))
    J = torch.linalg.inv(Msafe)
    Sigma = torch.eye(2, dtype=F64) + prm.sigma_eff() * (J @ J.transpose(1, 2))   # Eq. mip_cov
    Sinv = torch.linalg.inv(Sigma)
    n_f = torch.rsqrt(torch.linalg.det(Sigma))                                # sqrt(|I| / |Sigma|)
    return Sinv, n_f, M, valid


def records(S: dict, cam: dict, irr, levels, lut, prm: Params):
    """Everything the rasteriser needs for one view, as FP64 tensors that
    stay differentiable w.r.t. the surfel parameters in S and the env
    levels.

    S: pos [N,3], quat [N,4], log_scale [N,2], albedo [N,3], roughness [N],
    metallic [N].  cam: R [3,3], t [3], fx, fy, cx, cy, width, height.
    """
    R = quat_to_rot(S["quat"])
    scale = torch.exp(S["log_scale"])
    t_u = scale[:, 0:1] * R[:, :, 0]          # Sec. 3.7: quaternion + log scales
    t_v = scale[:, 1:2] * R[:, :, 1]
    n = R[:, :, 2]                            # = t_u x t_v / |.| (Sec. 3.1)
    Rc, tc = cam["R"], cam["t"]
    c_cam = S["pos"] @ Rc.T + tc              # camera-space centre c'
    tu_c = t_u @ Rc.T
    tv_c = t_v @ Rc.T
    fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    # T = P S with S = [t'_u t'_v 0 c'] (Sec. 3.1).  P is the pinhole that
    # maps camera space to homogeneous pixel coordinates; its rows x, y and w
    # give T1, T2, T4 (the depth row T3 is unused, App. A).
    row_x = torch.stack([tu_c[:, 0], tv_c[:, 0], c_cam[:, 0]], -1)
    row_y = torch.stack([tu_c[:, 1], tv_c[:, 1], c_cam[:, 1]], -1)
    row_z = torch.stack([tu_c[:, 2], tv_c[:, 2], c_cam[:, 2]], -1)
    T1 = fx * row_x + cx * row_z
    T2 = fy * row_y + cy * row_z
    T4 = row_z
    # depth interval (Sec. 3.1): eps_z = r_cut sqrt(t'_uz^2 + t'_vz^2)
    z = c_cam[:, 2]
    eps = prm.r_cut * torch.sqrt(tu_c[:, 2] ** 2 + tv_c[:, 2] ** 2)
    zs, ze = z - eps, z + eps
    T = torch.stack([T1, T2, T4], 1)                                     # [N, 3, 3]
    Sinv, n_f, M, valid = mip_filter(T, zs > prm.z_near, prm)

    # forward shading (Sec. 3.4, Eq. ibl), one colour per surfel and view
    o = -(Rc.T @ tc)                                   # camera centre
    w_o = o[None, :] - S["pos"]
    w_o = w_o / torch.linalg.norm(w_o, dim=-1, keepdim=True)
    facing = (n * w_o).sum(-1, keepdim=True)
    n_s = torch.where(facing < 0, -n, n)                # two-sided surfels
    mu = torch.clamp((n_s * w_o).sum(-1), 0.0, 1.0)
    refl = 2.0 * (w_o * n_s).sum(-1, keepdim=True) * n_s - w_o
    rho, m, r = S["albedo"], S["metallic"][:, None], S["roughness"]
    F0 = 0.04 * (1.0 - m) + rho * m
    k_d = (1.0 - F0) * (1.0 - m)
    u_n, v_n = dir_to_uv(n_s)
    L_d = bilinear_wrap(irr, u_n, v_n)
    L_s = specular_lookup(levels, refl, r)
    beta = bilinear_clamp(lut, mu, torch.clamp(r, 0.0, 1.0))   # [n.v along W, r along H]
    colour = k_d * rho * L_d + L_s * (F0 * beta[:, 0:1] + beta[:, 1:2])

    ch = torch.cat([colour, rho, r[:, None], m, n_s, z[:, None]], -1)   # [N, 12]
    return dict(T=T, Sinv=Sinv, n_f=n_f, zs=zs, ze=ze, valid=valid, ch=ch, M=M)


def support_rect(rec: dict, prm: Params) -> np.ndarray:
    """Support rectangle [x_lo, x_hi, y_lo, y_hi] (continuous pixel
    coordinates) of every surfel: the union of
      (a) the exact bounds of the projected disc of radius r_cut -- the
          bounding-rectangle construction of App. A: tangent lines of the
          image of the disc, from the dual conic C* = H Q* H^T with
          H = [T1; T2; T4] and Q* = diag(1, 1, -1/r_cut^2);
      (b) the r_cut bounds of the screen-space EWA resampling ellipse at the
          centre, covariance M M^T + sigma_f I (M = d(x,y)/d(u,v), so this is
          the screen image of Sigma_mip of Eq. mip_cov under the local affine
          map), i.e. p +- r_cut sqrt((M M^T)_aa + sigma_f);
    padded by one pixel.  A pixel is a candidate only if its centre lies in
    the rectangle.  For ordinary surfels the rectangle contains the whole
    filtered support; for nearly edge-on surfels, whose centre-precomputed
    filtered support is an unbounded strip, it bounds the footprint."""
    T = rec["T"].detach().numpy()
    N = T.shape[0]
    Q = np.diag([1.0, 1.0, -1.0 / prm.r_cut ** 2])
    C = np.einsum("nij,jk,nlk->nil", T, Q, T)
    c22 = C[:, 2, 2]
    M = rec["M"].detach().numpy()
    MMt = np.einsum("nij,nkj->nik", M, M)
    p = np.stack([T[:, 0, 2] / T[:, 2, 2], T[:, 1, 2] / T[:, 2, 2]], 1)
    out = np.zeros((N, 4))
    with np.errstate(invalid="ignore", divide="ignore"):
        for a in range(2):
            ca, cb = C[:, a, a], C[:, a, 2]
            disc = np.sqrt(np.maximum(cb * cb - ca * c22, 0.0))
            r0, r1 = (cb + disc) / c22, (cb - disc) / c22
            ext = prm.r_cut * np.sqrt(MMt[:, a, a] + prm.sigma_eff())
            lo = np.minimum(np.minimum(r0, r1), p[:, a] - ext) - 1.0
            hi = np.maximum(np.maximum(r0, r1), p[:, a] + ext) + 1.0
            bad = ~(c22 < 0)
            lo[bad] = -np.inf
            hi[bad] = np.inf
            out[:, 2 * a], out[:, 2 * a + 1] = lo, hi
    return out


# ---------------------------------------------------------------------------
# decisions (C) and values (torch)


@dataclasses.dataclass
class Fragments:
    pix: np.ndarray        # [F] pixel id (y * W + x) of each kept fragment
    sid: np.ndarray        # [F] surfel index
    layer: np.ndarray      # [F] layer index (< k_max)
    q_pix: np.ndarray      # [P] queried pixel ids
    n_layers: np.ndarray   # [P] kept layers per queried pixel
    margin: np.ndarray     # [P, 3] rho2 cutoff (rel), gap (rel), rectangle edge (px)
    count: np.ndarray      # [P] fragments per queried pixel


def fragments(rec: dict, rect: np.ndarray, W: int, H: int, prm: Params, pix=None) -> Fragments:
    T = np.ascontiguousarray(rec["T"].detach().numpy().reshape(-1, 9))
    Sinv = rec["Sinv"].detach().numpy()
    Sv = np.ascontiguousarray(np.stack([Sinv[:, 0, 0], Sinv[:, 0, 1], Sinv[:, 1, 1]], 1))
    zse = np.ascontiguousarray(np.stack([rec["zs"].detach().numpy(), rec["ze"].detach().numpy()], 1))
    valid = np.ascontiguousarray(rec["valid"].numpy().astype(np.uint8))
    rect = np.ascontiguousarray(rect, np.float64)
    N = T.shape[0]
    if pix is None:
        q = np.arange(W * H, dtype=np.int32)
        pix_ptr = None
    else:
        q = np.ascontiguousarray(pix, np.int32)
        pix_ptr = _p(q, ctypes.c_int32)
    P = q.shape[0]
    nl = np.zeros(P, np.int32)
    mg = np.zeros((P, 3), np.float64)
    cnt = np.zeros(P, np.int64)
    L = lib()
    args = (N, _p(T, ctypes.c_double), _p(Sv, ctypes.c_double), _p(zse, ctypes.c_double),
            _p(valid, ctypes.c_uint8), _p(rect, ctypes.c_double), W, H, prm.r_cut ** 2, prm.k_max,
            prm.pp_sigma(), P, pix_ptr, _p(nl, ctypes.c_int32), _p(mg, ctypes.c_double), _p(cnt, ctypes.c_int64))
    total = L.oref_fragments(*args, None, None, None, None)
    off = np.zeros(P, np.int64)
    off[1:] = np.cumsum(cnt)[:-1]
    fp = np.zeros(total, np.int32)
    fs = np.zeros(total, np.int32)
    fl = np.zeros(total, np.int32)
    L.oref_fragments(*args, _p(off, ctypes.c_int64), _p(fp, ctypes.c_int32), _p(fs, ctypes.c_int32),
                     _p(fl, ctypes.c_int32))
    return Fragments(fp, fs, fl, q, nl, mg, cnt)


def decision_variants(rec: dict, rect: np.ndarray, W: int, prm: Params, pid: int, tol_cut: float,
                      tol_gap: float, tol_box: float, max_variants: int = 512):
    """Every outcome of the discrete decisions of pixel `pid` that sit within
    rounding of flipping, as alternative fragment sets.

    A surfel's coverage (Algorithm 1: inside the support rectangle and
    rho2_mip < r_cut^2) is flippable when |rho2_mip - r_cut^2| / r_cut^2 <
    tol_cut, or when the pixel centre is within tol_box px of the
    rectangle's edge (inside or out).  For each choice of the flippable
    coverages, the covering surfels are visited in (z_start, index) order
    and grouped as Algorithm 1 groups them; a gap test z_start > z_max_end
    with |z_start - z_max_end| / |z_max_end| < tol_gap (and not an exact tie)
    is taken both ways; layers past the K_max-th are discarded.  Returns a
    list of (sid [F], layer [F], n_layers) -- the variant without any flip
    first -- and whether the enumeration was complete (at most max_variants)."""
    T = np.ascontiguousarray(rec["T"].detach().numpy().reshape(-1, 9))
    Sinv = rec["Sinv"].detach().numpy()
    Sv = np.ascontiguousarray(np.stack([Sinv[:, 0, 0], Sinv[:, 0, 1], Sinv[:, 1, 1]], 1))
    zse = np.ascontiguousarray(np.stack([rec["zs"].detach().numpy(), rec["ze"].detach().numpy()], 1))
    valid = np.ascontiguousarray(rec["valid"].numpy().astype(np.uint8))
    rect = np.ascontiguousarray(rect, np.float64)
    near = max(tol_box, 1e-9)
    cap = 256
    while True:
        idx = np.zeros(cap, np.int32)
        r2, zs, ze, dist = (np.zeros(cap) for _ in range(4))
        n = lib().oref_pixel_candidates(T.shape[0], _p(T, ctypes.c_double), _p(Sv, ctypes.c_double),
                                        _p(zse, ctypes.c_double), _p(valid, ctypes.c_uint8),
                                        _p(rect, ctypes.c_double), W, int(pid), near, prm.pp_sigma(), cap,
                                        _p(idx, ctypes.c_int32), _p(r2, ctypes.c_double), _p(zs, ctypes.c_double),
                                        _p(ze, ctypes.c_double), _p(dist, ctypes.c_double))
        if n <= cap:
            break
        cap = n
    idx, r2, zs, ze, dist = idx[:n], r2[:n], zs[:n], ze[:n], dist[:n]
    rc2 = prm.r_cut ** 2
    # coverage = (inside the rectangle) and (rho2 < r^2); either part may be
    # within rounding of flipping; a surfel is flippable when its two parts
    # can give both outcomes
    in_r, cut_ok = dist >= 0.0, r2 < rc2
    f_r, f_c = np.abs(dist) < tol_box, np.abs(r2 - rc2) / rc2 < tol_cut
    base = in_r & cut_ok
    can_cover = (in_r | f_r) & (cut_ok | f_c)
    can_miss = ~in_r | f_r | ~cut_ok | f_c
    fl = np.where(can_cover & can_miss)[0]
    out, complete = [], True
    n_sets = 1 << len(fl)
    if n_sets > max_variants:
        n_sets, complete = max_variants, False
    for m in range(n_sets):
        cov = base.copy()
        for b, j in enumerate(fl):
            if (m >> b) & 1:
                cov[j] = not cov[j]
        order = sorted(np.where(cov)[0], key=lambda j: (zs[j], idx[j]))
        # Algorithm 1 with near-tie gap tests taken both ways (depth-first)
        stack = [(0, -1, 0.0, [])]
        while stack:
            f, layer, zmax, acc = stack.pop()
            if f == len(order) or layer >= prm.k_max:
                kept = [(a, l) for a, l in acc if l < prm.k_max]
                nl = min(layer + 1, prm.k_max)
                out.append((np.array([idx[a] for a, _ in kept], np.int32),
                            np.array([l for _, l in kept], np.int32), nl))
                if len(out) >= max_variants:
                    return out, False
                continue
            j = order[f]
            choices = []
            if layer < 0:
                choices = [True]
            else:
                gap = zs[j] > zmax
                choices = [gap]
                m_g = abs(zs[j] - zmax) / abs(zmax) if zmax != 0 else np.inf
                if 0.0 < m_g < tol_gap:
                    choices.append(not gap)
            for new_layer in reversed(choices):
                l2, z2 = (layer + 1, 0.0) if new_layer else (layer, zmax)
                if l2 >= prm.k_max:
                    stack.append((len(order), l2, z2, acc))
                    continue
                stack.append((f + 1, l2, max(z2, ze[j]), acc + [(j, l2)]))
    return out, complete


def composite_variant(rec: dict, W: int, prm: Params, pid: int, sid: np.ndarray, layer: np.ndarray,
                      n_layers: int):
    """Composite one pixel from a given fragment set (see decision_variants):
    returns its 13 values (rgba, then the 9 AOV channels) in FP64."""
    fr = Fragments(np.full(sid.shape[0], pid, np.int32), sid.astype(np.int32), layer.astype(np.int32),
                   np.array([pid], np.int32), np.array([n_layers], np.int32), np.zeros((1, 3)),
                   np.array([sid.shape[0]], np.int64))
    with torch.no_grad():
        rgba, aov = composite(rec, fr, W, prm)
    return torch.cat([rgba, aov], 1)[0].numpy()


def composite(rec: dict, fr: Fragments, W: int, prm: Params, per_frag: dict | None = None):
    """Layer sums, Shepard normalisation, coverage opacity and compositing
    for the queried pixels.  Returns (rgba [P,4], aov [P,9]) as FP64
    tensors, differentiable w.r.t. the record tensors.  per_frag, if given,
    holds the fragments' own copies of T, Sinv, n_f and ch (rec[k][fr.sid]),
    so that autograd yields one gradient per fragment."""
    P = fr.q_pix.shape[0]
    Kq = max(1, int(fr.n_layers.max()) if P else 1)
    # row of each fragment within the query
    q_index = {int(p): i for i, p in enumerate(fr.q_pix)} if P < 4096 else None
    if q_index is not None:
        row = np.array([q_index[int(p)] for p in fr.pix], np.int64)
    else:
        lookup = np.full(int(fr.q_pix.max()) + 1, -1, np.int64)
        lookup[fr.q_pix] = np.arange(P)
        row = lookup[fr.pix]
    row_t = torch.from_numpy(row)
    sid = torch.from_numpy(fr.sid.astype(np.int64))
    layer = torch.from_numpy(fr.layer.astype(np.int64))
    x = torch.from_numpy((fr.pix % W).astype(np.float64)) + 0.5
    y = torch.from_numpy((fr.pix // W).astype(np.float64)) + 0.5
    fv = (lambda k: per_frag[k]) if per_frag is not None else (lambda k: rec[k][sid])
    T = fv("T")
    T1, T2, T4 = T[:, 0], T[:, 1], T[:, 2]
    # ray planes pulled back through T (Sec. 3.1) and their common zero
    k = x[:, None] * T4 - T1
    l = y[:, None] * T4 - T2
    s = torch.linalg.cross(k, l, dim=-1)
    u = s[:, 0] / s[:, 2]
    v = s[:, 1] / s[:, 2]
    if prm.mip_mode == "pixel":
        # the MIP filter at the hit (Sec. 3.3.1): J = d(u,v)/d(x,y) of this
        # intersection by the quotient rule (ds/dx = T4 x l, ds/dy = k x T4),
        # Sigma = I + sigma_f J J^T (Eq. mip_cov), n_f = |Sigma|^-1/2 (Eq. mip_eval)
        sx = torch.linalg.cross(T4, l, dim=-1)
        sy = torch.linalg.cross(k, T4, dim=-1)
        J = torch.stack([torch.stack([(sx[:, 0] - u * sx[:, 2]) / s[:, 2], (sy[:, 0] - u * sy[:, 2]) / s[:, 2]], -1),
                         torch.stack([(sx[:, 1] - v * sx[:, 2]) / s[:, 2], (sy[:, 1] - v * sy[:, 2]) / s[:, 2]], -1)],
                        -2)
        Sigma = torch.eye(2, dtype=F64) + prm.sigma_f * (J @ J.transpose(1, 2))
        Si = torch.linalg.inv(Sigma)
        n_f = torch.rsqrt(torch.linalg.det(Sigma))
    else:
        Si = fv("Sinv")
        n_f = fv("n_f")
    rho2 = Si[:, 0, 0] * u * u + 2.0 * Si[:, 0, 1] * u * v + Si[:, 1, 1] * v * v   # Eq. mip_weight
    w = n_f * torch.exp(-0.5 * rho2)
    key = row_t * Kq + layer
    Wk = torch.zeros(P * Kq, dtype=F64).index_add(0, key, w).reshape(P, Kq)
    Ck = torch.zeros(P * Kq, N_CH, dtype=F64).index_add(0, key, w[:, None] * fv("ch")).reshape(P, Kq, N_CH)
    present = torch.arange(Kq)[None, :] < torch.from_numpy(fr.n_layers.astype(np.int64))[:, None]
    Wsafe = torch.where(present, Wk, torch.ones_like(Wk))
    Chat = Ck / Wsafe[..., None]                                   # Eq. shepard
    nrm = Ck[..., NORMAL]
    nlen = torch.linalg.norm(nrm, dim=-1, keepdim=True)
    nlen = torch.where(present[..., None], nlen, torch.ones_like(nlen))
    Chat = torch.cat([Chat[..., :8], nrm / nlen, Chat[..., 11:]], -1)   # normals renormalised per layer
    alpha = 1.0 - torch.exp(-prm.gamma * Wk / (2.0 * math.pi))         # Eq. alpha
    alpha = torch.where(present, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - alpha
    Tbar = torch.cumprod(torch.cat([torch.ones(P, 1, dtype=F64), one_minus], 1), 1)   # [P, Kq+1]
    wgt = Tbar[:, :Kq] * alpha                                         # Eq. compositing
    out = (wgt[..., None] * torch.where(present[..., None], Chat, torch.zeros_like(Chat))).sum(1)
    T_end = Tbar[:, Kq]
    bg = torch.tensor(prm.bg, dtype=F64)
    rgb = out[:, :3] + T_end[:, None] * bg
    rgba = torch.cat([rgb, (1.0 - T_end)[:, None]], 1)                # soft silhouette (Sec. 3.5.2)
    if not prm.cons:
        return rgba, out[:, 3:]
    # Eq. cons_loss: w_i = T_i alpha_i, z_i the layer's mean depth (Shepard mean
    # of the fragments' depths, the depth channel), sigma_i^2 its variance
    # (Shepard-weighted mean of (z - z_i)^2 over the layer's fragments)
    z_f = fv("ch")[:, 11]
    zbar = torch.where(present, Ck[..., 11] / Wsafe, torch.zeros_like(Wsafe))          # [P, Kq]
    dev2 = w * (z_f - zbar[row_t, layer]) ** 2
    var = torch.zeros(P * Kq, dtype=F64).index_add(0, key, dev2).reshape(P, Kq) / Wsafe
    wl = torch.where(present, wgt, torch.zeros_like(wgt))
    pair = wl[:, :, None] * wl[:, None, :] * torch.abs(zbar[:, :, None] - zbar[:, None, :])
    upper = torch.triu(torch.ones(Kq, Kq, dtype=torch.bool), diagonal=1)
    inter = (pair * upper).sum((1, 2))
    intra = (wl ** 2 * torch.where(present, var, torch.zeros_like(var))).sum(1)
    return rgba, torch.cat([out[:, 3:], (inter + intra)[:, None]], 1)


def lookup_margins(S: dict, cam: dict, env_shape, prm: Params) -> np.ndarray:
    """Per surfel: the smallest distance (in texels) of any bilinear or level
    coordinate used by the shading (irradiance at n, the two specular levels
    at r, the BRDF table at (n.v, r), the level coordinate r (L-1)) to a
    cell boundary, and the distances of n.w_o from 0 and of |n.w_o| from 1
    (the two-sided flip of the normal and the clamp of n.w_o to [0, 1]).
    Each is a discrete choice; where this margin is within rounding,
    implementations in different precisions may take the other branch and
    differ in the derivative (and, for the flip, in the sign of the normal's
    contribution), though the shaded value itself is continuous."""
    with torch.no_grad():
        R = quat_to_rot(S["quat"])
        n = R[:, :, 2]
        o = -(cam["R"].T @ cam["t"])
        w_o = o[None, :] - S["pos"]
        w_o = w_o / torch.linalg.norm(w_o, dim=-1, keepdim=True)
        facing = (n * w_o).sum(-1, keepdim=True)
        n_s = torch.where(facing < 0, -n, n)
        mu = torch.clamp((n_s * w_o).sum(-1), 0.0, 1.0)
        refl = 2.0 * (w_o * n_s).sum(-1, keepdim=True) * n_s - w_o
        r = torch.clamp(S["roughness"], 0.0, 1.0)
        He, We = env_shape[0], env_shape[1]
        L = prm.env_levels
        sizes = level_sizes(We, He, L)
        frac = lambda X: torch.abs(X - torch.round(X))
        m = torch.full((n.shape[0],), float("inf"), dtype=F64)
        u, v = dir_to_uv(n_s)
        m = torch.minimum(m, torch.minimum(frac(u * prm.irr_w - 0.5), frac(v * prm.irr_h - 0.5)))
        u, v = dir_to_uv(refl)
        lc = r * (L - 1)
        i0 = torch.clamp(torch.floor(lc).long(), 0, L - 1)
        for lv in (i0, torch.clamp(i0 + 1, max=L - 1)):
            Ws = torch.tensor([sizes[k][0] for k in range(L)], dtype=F64)[lv]
            Hs = torch.tensor([sizes[k][1] for k in range(L)], dtype=F64)[lv]
            m = torch.minimum(m, torch.minimum(frac(u * Ws - 0.5), frac(v * Hs - 0.5)))
        m = torch.minimum(m, torch.minimum(frac(mu * prm.lut_n - 0.5), frac(r * prm.lut_n - 0.5)))
        m = torch.minimum(m, frac(lc))
        fa = torch.abs(facing[:, 0])
        m = torch.minimum(m, torch.minimum(fa, 1.0 - fa))
    return m.numpy()


# ---------------------------------------------------------------------------
# convenience: a whole view


def to_torch_surfels(surf, requires_grad=False) -> dict:
    d = {k: torch.from_numpy(np.asarray(getattr(surf, k), np.float64).copy())
         for k in ("pos", "quat", "log_scale", "albedo", "roughness", "metallic")}
    if requires_grad:
        for v in d.values():
            v.requires_grad_(True)
    return d


def cam_dict(cam) -> dict:
    """Camera values rounded to float32 first (the CUDA path receives
    float32), then held in FP64."""
    f32 = lambda a: float(np.float32(a))
    return dict(R=torch.from_numpy(np.asarray(cam.R, np.float32).astype(np.float64)),
                t=torch.from_numpy(np.asarray(cam.t, np.float32).astype(np.float64)),
                fx=f32(cam.fx), fy=f32(cam.fy), cx=f32(cam.cx), cy=f32(cam.cy),
                width=int(cam.width), height=int(cam.height))


@dataclasses.dataclass
class EnvState:
    irr: np.ndarray
    levels: list
    lut: np.ndarray
    shape: tuple


def prepare_env(env: np.ndarray, prm: Params, lut_nq: int = 128) -> EnvState:
    env32 = np.asarray(env, np.float32).astype(np.float64)
    irr, levels = env_prefilter(env32, prm.env_levels, prm.irr_w, prm.irr_h)
    return EnvState(irr, levels, brdf_lut(prm.lut_n, lut_nq), env32.shape)


@dataclasses.dataclass
class ViewState:
    """One view between the phases of render_view: the per-surfel records
    (differentiable), their support rectangles and the leaves the per-pixel
    part differentiates into."""
    S: dict
    cd: dict
    irr: torch.Tensor
    levels: list
    rec: dict
    rect: np.ndarray
    leaf: dict
    need_grad: bool
    env: EnvState
    prm: Params


def prepare_view(surf, cam, env: EnvState, prm: Params = Params(), need_grad: bool = False) -> ViewState:
    """Per-view part of render_view that does not depend on the pixels:
    the records of every surfel and their support rectangles."""
    S = to_torch_surfels(surf, requires_grad=need_grad)
    cd = cam_dict(cam)
    irr = torch.from_numpy(env.irr.copy()).requires_grad_(need_grad)
    levels = [torch.from_numpy(l.copy()).requires_grad_(need_grad) for l in env.levels]
    lut = torch.from_numpy(env.lut.copy())
    with torch.set_grad_enabled(need_grad):
        rec = records(S, cd, irr, levels, lut, prm)
    rect = support_rect(rec, prm)
    # leaves for the per-pixel part, so pixel chunks can be back-propagated one at a time
    leaf = {k: rec[k].detach().clone().requires_grad_(need_grad) for k in ("T", "Sinv", "n_f", "ch")}
    leaf.update(zs=rec["zs"].detach(), ze=rec["ze"].detach(), valid=rec["valid"])
    return ViewState(S, cd, irr, levels, rec, rect, leaf, need_grad, env, prm)


def render_pixels(vs: ViewState, q_all: np.ndarray, G=None, chunk: int = 1 << 16) -> dict:
    """Per-pixel part of render_view for the pixel ids q_all: decisions,
    values and (G given) the back-propagation of sum(G * [rgba, aov]) into
    the view's leaves."""
    W, H = vs.cd["width"], vs.cd["height"]
    rgba_parts, aov_parts, nl_parts, mg_parts = [], [], [], []
    for c0 in range(0, q_all.shape[0], chunk):
        q = q_all[c0:c0 + chunk]
        fr = fragments(vs.leaf, vs.rect, W, H, vs.prm, pix=q)
        with torch.set_grad_enabled(vs.need_grad):
            rgba, aov = composite(vs.leaf, fr, W, vs.prm)
            if vs.need_grad and G is not None:
                Gc = torch.from_numpy(np.asarray(G[c0:c0 + chunk], np.float64))
                (torch.cat([rgba, aov], 1) * Gc).sum().backward()
        rgba_parts.append(rgba.detach().numpy())
        aov_parts.append(aov.detach().numpy())
        nl_parts.append(fr.n_layers)
        mg_parts.append(fr.margin)
    return dict(rgba=np.concatenate(rgba_parts), aov=np.concatenate(aov_parts),
                n_layers=np.concatenate(nl_parts), margin=np.concatenate(mg_parts))


def chain_records(vs: ViewState):
    """The gradients accumulated in the view's leaves chained back through
    the records: returns (surfel parameter gradients, d_irr, d_levels)."""
    tens = [vs.rec[k] for k in ("T", "Sinv", "n_f", "ch")]
    grads = [vs.leaf[k].grad if vs.leaf[k].grad is not None else torch.zeros_like(vs.leaf[k]) for k in
             ("T", "Sinv", "n_f", "ch")]
    torch.autograd.backward(tens, grads)
    out = {k: (v.grad.numpy() if v.grad is not None else np.zeros(v.shape)) for k, v in vs.S.items()}
    d_irr = vs.irr.grad.numpy() if vs.irr.grad is not None else np.zeros(vs.irr.shape)
    d_lv = [lv.grad.numpy() if lv.grad is not None else np.zeros(lv.shape) for lv in vs.levels]
    return out, d_irr, d_lv


def finish_view(vs: ViewState) -> dict:
    """Per-view part of render_view after the pixels: chain_records, then the
    prefiltered-map gradients through the prefilter's transpose to the base
    env."""
    out, d_irr, d_lv = chain_records(vs)
    He, We, _ = vs.env.shape
    out["env"] = env_adjoint(d_irr, d_lv, We, He)
    return out


def render_view(surf, cam, env: EnvState, prm: Params = Params(), pix=None, G=None,
                chunk: int = 1 << 16):
    """Render one view (all pixels, or the pixel ids in `pix`).

    Returns a dict with rgba [P,4], aov [P,9], n_layers, margins and, if G
    (upstream gradient, [P,13] = rgba then aov) is given, the gradients of
    sum(G * [rgba, aov]) w.r.t. the surfel parameters and the base env.
    """
    need_grad = G is not None
    vs = prepare_view(surf, cam, env, prm, need_grad)
    W, H = vs.cd["width"], vs.cd["height"]
    q_all = np.arange(W * H, dtype=np.int32) if pix is None else np.asarray(pix, np.int32)
    out = render_pixels(vs, q_all, G, chunk)
    out.update(rect=vs.rect, valid=vs.rec["valid"].numpy(), lookup_margin=lookup_margins(vs.S, vs.cd, env.shape, prm),
               records={k: vs.leaf[k].detach() for k in ("T", "Sinv", "n_f", "ch", "zs", "ze", "valid")},
               width=W)
    if need_grad:
        out["grad"] = finish_view(vs)
    return out


def screen_grad_stat(surf, cam, env: EnvState, prm: Params = Params(), G=None, pix=None):
    """Per-fragment screen-space positional gradients of Eq. ss_grad and
    their per-surfel sum of norms, for one view.

    The screen centre is (T_{1,z} / T_{4,z}, T_{2,z} / T_{4,z}) (the z
    entries are the columns that multiply the centre c'); a fragment's
    contribution is g_x = dL_p/dT_{1,z} T_{4,z}, g_y = dL_p/dT_{2,z} T_{4,z},
    where L_p = sum(G[p] * [rgba, aov](p)) is the loss of the fragment's pixel
    and dL_p/dT covers both the ray-plane intersection and the centre-
    precomputed MIP filter (Sigma^-1 and n_f are functions of T), with every
    discrete decision and the shaded channels held fixed (the shading is
    not part of the T-matrix backward).  The statistic accumulates the
    per-fragment norms |(g_x, g_y)|, so that opposite contributions do not
    cancel (Sec. 3.6.1, densification criterion).

    G: upstream gradient [P, 13] for the queried pixels (all pixels, or
    `pix`).  Returns dict(sid, pix, gx, gy) per fragment and per surfel
    sum_norm [N] and n_frag [N] (fragments that reached it)."""
    S = to_torch_surfels(surf)
    cd = cam_dict(cam)
    irr = torch.from_numpy(env.irr.copy())
    levels = [torch.from_numpy(l.copy()) for l in env.levels]
    lut = torch.from_numpy(env.lut.copy())
    W, H = cd["width"], cd["height"]
    with torch.no_grad():
        rec = records(S, cd, irr, levels, lut, prm)
    rect = support_rect(rec, prm)
    q = np.arange(W * H, dtype=np.int32) if pix is None else np.asarray(pix, np.int32)
    fr = fragments(rec, rect, W, H, prm, pix=q)
    sid = torch.from_numpy(fr.sid.astype(np.int64))
    pf = {k: rec[k][sid].detach().clone().requires_grad_(k != "ch") for k in ("T", "Sinv", "n_f", "ch")}
    rgba, aov = composite(rec, fr, W, prm, per_frag=pf)
    Gt = torch.from_numpy(np.asarray(G, np.float64))
    (torch.cat([rgba, aov], 1) * Gt).sum().backward()
    # directional derivatives of the MIP filter along T_{1,z} and T_{2,z}
    T = rec["T"].detach()
    depth_ok = rec["zs"] > prm.z_near

    def mip(Tv):
        Sinv, n_f, _, _ = mip_filter(Tv, depth_ok, prm)
        return Sinv, n_f

    g = {}
    for row, name in ((0, "gx"), (1, "gy")):
        tang = torch.zeros_like(T)
        tang[:, row, 2] = 1.0
        _, (dS, dn) = torch.func.jvp(mip, (T,), (tang,))
        dLdT = (pf["T"].grad[:, row, 2] + (pf["Sinv"].grad * dS[sid]).sum((1, 2)) + pf["n_f"].grad * dn[sid])
        g[name] = (dLdT * T[sid, 2, 2]).numpy()
    norm = np.sqrt(g["gx"] ** 2 + g["gy"] ** 2)
    N = T.shape[0]
    return dict(sid=fr.sid.copy(), pix=fr.pix.copy(), gx=g["gx"], gy=g["gy"],
                sum_norm=np.bincount(fr.sid, weights=norm, minlength=N),
                n_frag=np.bincount(fr.sid, minlength=N))
