"""Planted slips in the FP64 oracle, each of which some pin must catch.

    python tests/oracle_mutants.py [name ...]

Each slip is a one-line change of the kind a careful reader could still
make (a dropped factor, a wrong sign, a swapped operand, an off-by-one).
For every slip the oracle is loaded from a changed copy (a Python module
executed from its edited text, or the C half compiled from its edited text
under oracle/_build/) and the oracle pin tests (tests/test_oracle_*.py) run
against it in a separate process.  A slip that no pin fails is printed as a
survivor and the exit status is 1.  Nothing here touches the CUDA path; the
run takes several minutes, so it is not part of the default test suite.
"""
import glob
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (module, original text, planted text); "c" is the oracle's C half
SLIPS = {
    # weights, compositing (model.py)
    "cross_term": ("model", "rho2 = Si[:, 0, 0] * u * u + 2.0 * Si[:, 0, 1] * u * v",
                   "rho2 = Si[:, 0, 0] * u * u - 2.0 * Si[:, 0, 1] * u * v"),
    "gauss_half": ("model", "w = n_f * torch.exp(-0.5 * rho2)", "w = n_f * torch.exp(-rho2)"),
    "no_renorm": ("model", "Chat = torch.cat([Chat[..., :8], nrm / nlen, Chat[..., 11:]], -1)", "Chat = Chat"),
    "inclusive_T": ("model", "wgt = Tbar[:, :Kq] * alpha", "wgt = Tbar[:, 1:] * alpha"),
    "gamma_dropped": ("model", "alpha = 1.0 - torch.exp(-prm.gamma * Wk / (2.0 * math.pi))",
                      "alpha = 1.0 - torch.exp(-Wk)"),
    "no_background": ("model", "rgb = out[:, :3] + T_end[:, None] * bg", "rgb = out[:, :3]"),
    "pixel_corner": ("model", "x = torch.from_numpy((fr.pix % W).astype(np.float64)) + 0.5",
                     "x = torch.from_numpy((fr.pix % W).astype(np.float64)) + 0.0"),
    "no_shepard": ("model", "Chat = Ck / Wsafe[..., None]", "Chat = Ck"),
    "one_layer": ("model", "key = row_t * Kq + layer", "key = row_t * Kq"),
    "T_end_early": ("model", "T_end = Tbar[:, Kq]", "T_end = Tbar[:, Kq - 1]"),
    "uv_swapped": ("model", "u = s[:, 0] / s[:, 2]\n    v = s[:, 1] / s[:, 2]", "u = s[:, 1] / s[:, 2]\n    v = s[:, 0] / s[:, 2]"),
    # records: projection, MIP filter, depth interval, channels (model.py)
    "centre_undivided": ("model", "px = T1[:, 2] / T4[:, 2]", "px = T1[:, 2]"),
    "swap_f": ("model", 'fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]',
               'fy, fx, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]'),
    "swap_c": ("model", 'fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]',
               'fx, fy, cy, cx = cam["fx"], cam["fy"], cam["cx"], cam["cy"]'),
    "JtJ": ("model", "(J @ J.transpose(1, 2))", "(J.transpose(1, 2) @ J)"),
    "nf_det": ("model", "n_f = torch.rsqrt(torch.linalg.det(Sigma))", "n_f = 1.0 / torch.linalg.det(Sigma)"),
    "eps_one_tangent": ("model", "eps = prm.r_cut * torch.sqrt(tu_c[:, 2] ** 2 + tv_c[:, 2] ** 2)",
                        "eps = prm.r_cut * torch.abs(tu_c[:, 2])"),
    "near_by_centre": ("model", "Sinv, n_f, M, valid = mip_filter(T, zs > prm.z_near, prm)",
                       "Sinv, n_f, M, valid = mip_filter(T, z > prm.z_near, prm)"),
    "depth_world_z": ("model", "ch = torch.cat([colour, rho, r[:, None], m, n_s, z[:, None]], -1)",
                      "ch = torch.cat([colour, rho, r[:, None], m, n_s, S['pos'][:, 2:3]], -1)"),
    "swap_rough_metal": ("model", "ch = torch.cat([colour, rho, r[:, None], m, n_s, z[:, None]], -1)",
                         "ch = torch.cat([colour, rho, m, r[:, None], n_s, z[:, None]], -1)"),
    # shading and lookups (model.py)
    "kd_no_metal": ("model", "k_d = (1.0 - F0) * (1.0 - m)", "k_d = (1.0 - F0)"),
    "F0_swapped": ("model", "F0 = 0.04 * (1.0 - m) + rho * m", "F0 = 0.04 * m + rho * (1.0 - m)"),
    "refl_negated": ("model", "refl = 2.0 * (w_o * n_s).sum(-1, keepdim=True) * n_s - w_o",
                     "refl = w_o - 2.0 * (w_o * n_s).sum(-1, keepdim=True) * n_s"),
    "no_flip": ("model", "n_s = torch.where(facing < 0, -n, n)", "n_s = n"),
    "irr_unflipped": ("model", "u_n, v_n = dir_to_uv(n_s)", "u_n, v_n = dir_to_uv(n)"),
    "lut_axes": ("model", "beta = bilinear_clamp(lut, mu, torch.clamp(r, 0.0, 1.0))",
                 "beta = bilinear_clamp(lut, torch.clamp(r, 0.0, 1.0), mu)"),
    "beta_swapped": ("model", "colour = k_d * rho * L_d + L_s * (F0 * beta[:, 0:1] + beta[:, 1:2])",
                     "colour = k_d * rho * L_d + L_s * (F0 * beta[:, 1:2] + beta[:, 0:1])"),
    "level_rL": ("model", "lc = torch.clamp(r, 0.0, 1.0) * (L - 1)", "lc = torch.clamp(r, 0.0, 1.0) * L"),
    "phi_sign": ("model", "phi = torch.atan2(d[..., 0], -d[..., 2])", "phi = torch.atan2(d[..., 0], d[..., 2])"),
    "theta_sign": ("model", "th = torch.acos(torch.clamp(d[..., 1], -1.0, 1.0))",
                   "th = torch.acos(torch.clamp(-d[..., 1], -1.0, 1.0))"),
    "seam_clamped": ("model", "xa = torch.remainder(x0, W)", "xa = torch.clamp(x0, 0, W - 1)"),
    # support rectangle (model.py)
    "rect_unpadded": ("model", "lo = np.minimum(np.minimum(r0, r1), p[:, a] - ext) - 1.0",
                      "lo = np.minimum(np.minimum(r0, r1), p[:, a] - ext)"),
    "rect_no_ewa": ("model", "lo = np.minimum(np.minimum(r0, r1), p[:, a] - ext) - 1.0",
                    "lo = np.minimum(r0, r1) - 1.0"),
    "rect_no_disc": ("model", "hi = np.maximum(np.maximum(r0, r1), p[:, a] + ext) + 1.0",
                     "hi = p[:, a] + ext + 1.0"),
    "rect_dual_conic": ("model", "Q = np.diag([1.0, 1.0, -1.0 / prm.r_cut ** 2])", "Q = np.diag([1.0, 1.0, -1.0 / prm.r_cut])"),
    # per-pixel decisions and the environment prefilter (ss3d_oracle.c)
    "cut_radius": ("c", "if (!(rho2 < rcut2)) continue;", "if (!(rho2 < sqrt(rcut2))) continue;"),
    "gap_ge": ("c", "if (layer < 0 || fr[f].zs > zmax) {", "if (layer < 0 || fr[f].zs >= zmax) {"),
    "zmax_last": ("c", "if (fr[f].ze > zmax) zmax = fr[f].ze;", "zmax = fr[f].ze;"),
    "sort_by_ze": ("c", "if (x->zs < y->zs) return -1;\n    if (x->zs > y->zs) return 1;",
                   "if (x->ze < y->ze) return -1;\n    if (x->ze > y->ze) return 1;"),
    "kmax_plus_one": ("c", "if (layer >= kmax) break;", "if (layer > kmax) break;"),
    "c_pixel_corner": ("c", "double x = px + 0.5, y = py + 0.5;", "double x = px, y = py;"),
    "ggx_half_angle": ("c", "double c2 = 0.5 * (1.0 + mu);\n    return ggx_D(c2, alpha) * mu * dW;",
                       "double c2 = mu * mu;\n    return ggx_D(c2, alpha) * mu * dW;"),
    "irr_no_cosine": ("c", "if (kind == 0) return mu * dW;", "if (kind == 0) return dW;"),
    "solid_angle_flat": ("c", "return (2.0 * M_PI / W) * (cos(t0) - cos(t1));", "return (2.0 * M_PI / W) * (M_PI / H);"),
    "alpha_r": ("c", "1, r * r, ", "1, r, "),
    "level_roughness": ("c", "double r = (double)i / (L - 1);", "double r = (double)i / L;"),
    "box_norm": ("c", "out[(b * W + a) * 3 + c] = s / (bw * bh);", "out[(b * W + a) * 3 + c] = s / bw;"),
    "adjoint_norm": ("c", "acc[c] += w / norm[t] * d_out[t * 3 + c];", "acc[c] += w * d_out[t * 3 + c];"),
    # depth consolidation (Eq. cons_loss) and the densification statistic (Eq. ss_grad) (model.py)
    "cons_signed_gap": ("model", "torch.abs(zbar[:, :, None] - zbar[:, None, :])", "(zbar[:, :, None] - zbar[:, None, :])"),
    "cons_intra_weight": ("model", "intra = (wl ** 2 * torch.where(present, var, torch.zeros_like(var))).sum(1)",
                          "intra = (wl * torch.where(present, var, torch.zeros_like(var))).sum(1)"),
    "cons_unweighted_var": ("model", "dev2 = w * (z_f - zbar[row_t, layer]) ** 2", "dev2 = (z_f - zbar[row_t, layer]) ** 2"),
    "ssg_unscaled": ("model", "g[name] = (dLdT * T[sid, 2, 2]).numpy()", "g[name] = dLdT.numpy()"),
    "ssg_no_nf_term": ("model", "(pf[\"Sinv\"].grad * dS[sid]).sum((1, 2)) + pf[\"n_f\"].grad * dn[sid])",
                       "(pf[\"Sinv\"].grad * dS[sid]).sum((1, 2)))"),
    "ssg_signed_sum": ("model", "norm = np.sqrt(g[\"gx\"] ** 2 + g[\"gy\"] ** 2)", "norm = g[\"gx\"] + g[\"gy\"]"),
    # density control (density.py)
    "split_scale_test": ("density", "(s_max > np.asarray(mean_dist, np.float64))", "(s_max < np.asarray(mean_dist, np.float64))"),
    "prune_no_rcut": ("density", "act[np.asarray(nn_dist, np.float64) > r_cut * s_max] = PRUNE",
                      "act[np.asarray(nn_dist, np.float64) > s_max] = PRUNE"),
    "prune_visible": ("density", "act[~(gn > 0)] = PRUNE", "act[gn < 0] = PRUNE"),
    "split_full_offset": ("density", "half = 0.5 * s_max[:, None] * t", "half = s_max[:, None] * t"),
    "split_minor_axis": ("density", "use_u = ls[:, 0] >= ls[:, 1]", "use_u = ls[:, 0] < ls[:, 1]"),
    "split_over_prune": ("density", "    rows = act.copy()", "    act[split] = SPLIT\n    rows = act.copy()"),
    "neighbours_unoriented": ("density", "same = (Nn[r0:r1] @ Nn.T) >= cos_min", "same = np.abs(Nn[r0:r1] @ Nn.T) >= cos_min"),
    # Adam (optim.py)
    "adam_bias1": ("optim", "m_hat = m / (1.0 - beta1 ** step)", "m_hat = m"),
    "adam_bias2": ("optim", "v_hat = v / (1.0 - beta2 ** step)", "v_hat = v"),
    "adam_eps": ("optim", "theta = theta - lr * m_hat / (np.sqrt(v_hat) + eps)",
                 "theta = theta - lr * m_hat / np.sqrt(v_hat + eps)"),
    "adam_sigmoid": ("optim", "g = g * a * (1.0 - a)", "g = g * a"),
    "adam_abs": ("optim", "v = beta2 * v + (1.0 - beta2) * g * g", "v = beta2 * v + (1.0 - beta2) * np.abs(g)"),
}

# runs in a fresh interpreter: load the changed oracle, then the pins
_RUNNER = r"""
import glob, os, sys, types
root, kind, a, b = sys.argv[1:5]
sys.path.insert(0, root)
import oracle
def load(name, text):
    path = os.path.join(root, "oracle", name + ".py")
    m = types.ModuleType("oracle." + name)
    m.__file__, m.__package__ = path, "oracle"
    sys.modules["oracle." + name] = m
    exec(compile(text, path, "exec"), m.__dict__)
    setattr(oracle, name, m)
    return m
if kind == "c":
    src = open(os.path.join(root, "oracle", "ss3d_oracle.c")).read()
    assert src.count(a) >= 1, a
    build = os.path.join(root, "oracle", "_build", "mutants")
    os.makedirs(build, exist_ok=True)
    c_path = os.path.join(build, "ss3d_oracle_%d.c" % os.getpid())
    open(c_path, "w").write(src.replace(a, b))
    m = load("model", open(os.path.join(root, "oracle", "model.py")).read())
    m._SRC, m._BUILD, m._SO = c_path, build, os.path.join(build, "lib_%d.so" % os.getpid())
else:
    text = open(os.path.join(root, "oracle", kind + ".py")).read()
    assert text.count(a) >= 1, a
    load(kind, text.replace(a, b))
import pytest
tests = sorted(glob.glob(os.path.join(root, "tests", "test_oracle_*.py")))
rc = pytest.main(["-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"] + tests)
if kind == "c":
    for f in (c_path, m._SO):
        if os.path.exists(f):
            os.remove(f)
sys.exit(int(rc))
"""


def run(name: str) -> bool:
    """True if some pin fails with the slip planted (the slip is caught)."""
    kind, a, b = SLIPS[name]
    r = subprocess.run([sys.executable, "-c", _RUNNER, ROOT, kind, a, b], capture_output=True, text=True,
                       timeout=1800)
    caught = r.returncode == 1                        # pytest: tests failed
    if r.returncode not in (0, 1):
        raise RuntimeError(f"{name}: the run itself failed\n{r.stdout[-2000:]}{r.stderr[-2000:]}")
    first = next((line for line in r.stdout.splitlines() if line.startswith("FAILED")), "")
    print(f"{name:18s} {'caught' if caught else 'SURVIVED'}  {first[:110]}", flush=True)
    return caught


def main(names):
    names = names or list(SLIPS)
    survivors = [n for n in names if not run(n)]
    print(f"{len(names) - len(survivors)} of {len(names)} slips caught" +
          (f"; survivors: {', '.join(survivors)}" if survivors else ""))
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
