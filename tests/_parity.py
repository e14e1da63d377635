"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

from oracle import model as M

# image tolerance: 1e-4 relative per pixel, 1e-5 absolute where |value| < 1e-2
RTOL, ATOL, SMALL = 1e-4, 1e-5, 1e-2
# decisions closer than this to flipping are set aside (rounding of FP32 vs FP64)
M_CUT, M_GAP, M_BOX = 1e-5, 1e-5, 2e-3


def oracle_params(prm) -> M.Params:
    return M.Params(r_cut=float(prm.r_cut), sigma_f=float(prm.sigma_f), gamma=float(prm.gamma),
                    k_max=int(prm.k_max), z_near=float(prm.z_near), bg=tuple(float(b) for b in prm.bg),
                    lut_n=int(prm.lut_n))


def oracle_view(scene, v, prm, env_levels=6, pix=None, G=None, env_cache=None):
    cam = scene.cameras[v]
    s0, s1 = int(scene.scene_offsets[cam.scene]), int(scene.scene_offsets[cam.scene + 1])
    surf = scene.surfels.subset(slice(s0, s1))
    op = oracle_params(prm)
    op.env_levels = env_levels
    key = cam.scene
    if env_cache is not None and key in env_cache:
        env = env_cache[key]
    else:
        env = M.prepare_env(scene.envs[cam.scene], op)
        if env_cache is not None:
            env_cache[key] = env
    return M.render_view(surf, cam, env, op, pix=pix, G=G)


def ambiguous(margin):
    return (margin[:, 0] < M_CUT) | (margin[:, 1] < M_GAP) | (margin[:, 2] < M_BOX)


# a pixel whose decision flips between precisions may differ by one
# near-cutoff fragment (weight ~ n_f e^-4.5) or one layer boundary; such
# pixels must still be finite, with coverage in [0, 1], within this of the oracle
AMBIGUOUS_ABS = 0.25
MAX_AMBIGUOUS_FRACTION = 1e-2


def check_ambiguous(gpu, ref, amb):
    g, r = gpu[amb], ref[amb]
    assert np.all(np.isfinite(g))
    assert np.all((g[:, 3] >= 0) & (g[:, 3] <= 1 + 1e-6))
    if g.size:
        assert np.abs(g - r).max() <= AMBIGUOUS_ABS * max(1.0, np.abs(r).max())


def compare(gpu, ref, amb, what=""):
    """gpu, ref: [P, C] arrays.  Returns the number of failing entries and a
    message; ambiguous pixels are excluded."""
    ok = ~amb
    g, r = gpu[ok], ref[ok]
    err = np.abs(g - r)
    bound = np.where(np.abs(r) < SMALL, ATOL, RTOL * np.abs(r))
    bad = err > bound
    n_bad = int(bad.sum())
    msg = ""
    if n_bad:
        idx = np.argwhere(bad)[:5]
        msg = f"{what}: {n_bad} entries out of tolerance, e.g. " + ", ".join(
            f"(p{i},c{c}) gpu={g[i, c]:.7g} ref={r[i, c]:.7g}" for i, c in idx)
    return n_bad, msg
