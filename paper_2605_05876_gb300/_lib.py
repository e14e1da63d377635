"""ctypes binding of libss3d.so (include/ss3d.h).  Argument marshalling only:
every step of the renderer runs in the library's CUDA kernels.  Loading fails
loudly when the library is missing; there is no CPU fallback."""
from __future__ import annotations

import ctypes
import os
from functools import lru_cache

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libss3d.so")

c_f = ctypes.c_float
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p
fp = ctypes.POINTER(ctypes.c_float)

SS_OK = 0
SS_ERR_INVALID_ARG = 1
SS_ERR_WORKSPACE = 2
SS_ERR_CAPACITY = 4
SS_ERR_TIMEOUT = 8
SS_ERR_NONFINITE = 16
SS_ERR_CUDA = 32
SS_MAX_VIEWS = 256
SS_MAX_SCENES = 64
SS_MAX_RECORDS = 0xfffffffe
SS_MAX_TILES = 1 << 27
SS_KMAX_LIMIT = 16
SS_N_AOV = 9
SS_NOALLOC_AUX_FLOATS = 1 << 20
SS_MIP_CENTRE, SS_MIP_NONE, SS_MIP_PIXEL = 0, 1, 2


class ss_camera(ctypes.Structure):
    _fields_ = [("R", c_f * 9), ("t", c_f * 3), ("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f),
                ("width", c_i32), ("height", c_i32), ("scene", c_i32), ("pad_", c_i32)]


class ss_surfels(ctypes.Structure):
    _fields_ = [("pos", c_vp), ("quat", c_vp), ("log_scale", c_vp), ("albedo", c_vp), ("roughness", c_vp),
                ("metallic", c_vp)]


class ss_surfel_grads(ctypes.Structure):
    _fields_ = [("pos", c_vp), ("quat", c_vp), ("log_scale", c_vp), ("albedo", c_vp), ("roughness", c_vp),
                ("metallic", c_vp), ("screen_grad_norm", c_vp), ("screen_grad_views", c_vp)]


class ss_batch_desc(ctypes.Structure):
    _fields_ = [("n_scenes", c_i32), ("n_views", c_i32), ("scene_offsets_host", ctypes.POINTER(c_i64)),
                ("cams_host", ctypes.POINTER(ss_camera)), ("cams_dev", c_vp)]


class ss_render_params(ctypes.Structure):
    _fields_ = [("r_cut", c_f), ("sigma_f", c_f), ("gamma", c_f), ("k_max", c_i32), ("z_near", c_f),
                ("bg", c_f * 3), ("write_aov", c_i32), ("lut_n", c_i32), ("max_instances", c_i64),
                ("collect_stats", c_i32), ("fwd_warps", c_i32), ("bwd_warps", c_i32), ("pbwd_block", c_i32),
                ("screen_grad", c_i32), ("mip_mode", c_i32), ("cons", c_i32), ("tile_w", c_i32), ("tile_h", c_i32),
                ("stage_depth", c_i32), ("deterministic", c_i32), ("det_rows", c_i64), ("dense_layers", c_i32),
                ("zero_grad_in_forward", c_i32), ("layer_pool", c_i64), ("max_candidates", c_i64)]


class ss_stats(ctypes.Structure):
    _fields_ = [("instances", c_i64), ("rect_tests", c_i64), ("lane_tests", c_i64), ("fragments", c_i64),
                ("layers", c_i64), ("bwd_fragments", c_i64), ("staged", c_i64), ("staged_covering", c_i64),
                ("bwd_batches", c_i64), ("pool_layers", c_i64), ("candidates", c_i64)]


SS_N_STAGES = 9
STAGES = ("project", "bin_sort", "raster_fwd", "raster_bwd", "project_bwd", "env_prefilter", "env_prefilter_bwd",
          "density", "screen_grad_jac")


class ss_stage_times(ctypes.Structure):
    _fields_ = [("ms", c_f * SS_N_STAGES), ("launches", c_i32 * SS_N_STAGES)]


class ss_env_desc(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("n_levels", c_i32), ("irr_width", c_i32),
                ("irr_height", c_i32)]


class ss_env_maps(ctypes.Structure):
    _fields_ = [("irr", c_vp), ("spec", c_vp), ("lut", c_vp)]


class ss_env_map_grads(ctypes.Structure):
    _fields_ = [("irr", c_vp), ("spec", c_vp)]


SS_ACT_IDENTITY = 0
SS_ACT_SIGMOID = 1
SS_ACT_CLAMP0 = 2
SS_MAX_ADAM_GROUPS = 16


class ss_adam_group(ctypes.Structure):
    _fields_ = [("param_dev", c_vp), ("grad_dev", c_vp), ("m_dev", c_vp), ("v_dev", c_vp), ("act_dev", c_vp),
                ("n", c_i64), ("lr", c_f), ("activation", c_i32)]


class ss_density_params(ctypes.Structure):
    _fields_ = [("k", c_i32), ("cos_min", c_f), ("cell", c_f), ("max_rings", c_i32), ("tau_g", c_f), ("r_cut", c_f),
                ("split_scale", c_f), ("ops", c_i32)]


SS_DENSITY_SPLIT, SS_DENSITY_PRUNE_VISIBLE, SS_DENSITY_PRUNE_ISOLATED = 1, 2, 4
SS_DENSITY_KMAX, SS_DENSITY_MAX_RINGS = 16, 32
SS_NB_MEAN_BOUND, SS_NB_NN_BOUND, SS_NB_NONFINITE = 1, 2, 4
SS_ACTION_PRUNE, SS_ACTION_KEEP, SS_ACTION_SPLIT = 0, 1, 2


class ss_adam_params(ctypes.Structure):
    _fields_ = [("beta1", c_f), ("beta2", c_f), ("eps", c_f), ("step", c_i32)]


EXPORTS = {
    "ss_default_params": (None, [ctypes.POINTER(ss_render_params)]),
    "ss_error_string": (ctypes.c_char_p, [c_i32]),
    "ss_brdf_lut": (c_i32, [c_vp, c_i32, c_vp]),
    "ss_env_sizes": (c_i32, [ctypes.POINTER(ss_env_desc), ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                             ctypes.POINTER(c_i64)]),
    "ss_env_prefilter": (c_i32, [ctypes.POINTER(ss_env_desc), c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "ss_env_prefilter_noalloc": (c_i32, [ctypes.POINTER(ss_env_desc), c_i32, c_vp, c_vp, c_vp, c_vp]),
    "ss_env_prefilter_backward": (c_i32, [ctypes.POINTER(ss_env_desc), c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "ss_env_prefilter_backward_ordered": (c_i32, [ctypes.POINTER(ss_env_desc), c_i32, c_vp, c_vp, c_vp, c_vp,
                                                  c_vp]),
    "ss_workspace_size": (c_i32, [ctypes.POINTER(ss_batch_desc), ctypes.POINTER(ss_render_params),
                                  ctypes.POINTER(ss_env_desc), c_i32,
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "ss_count_instances": (c_i32, [ctypes.POINTER(ss_batch_desc), ctypes.POINTER(ss_surfels),
                                   ctypes.POINTER(ss_render_params), ctypes.POINTER(ss_env_desc),
                                   ctypes.POINTER(ss_env_maps), c_vp, ctypes.c_size_t, ctypes.POINTER(c_i64),
                                   c_vp]),
    "ss_render_forward": (c_i32, [ctypes.POINTER(ss_batch_desc), ctypes.POINTER(ss_surfels),
                                  ctypes.POINTER(ss_render_params), ctypes.POINTER(ss_env_desc),
                                  ctypes.POINTER(ss_env_maps), c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "ss_render_backward": (c_i32, [ctypes.POINTER(ss_batch_desc), ctypes.POINTER(ss_surfels),
                                   ctypes.POINTER(ss_render_params), ctypes.POINTER(ss_env_desc),
                                   ctypes.POINTER(ss_env_maps), c_vp, c_vp, c_vp, c_vp,
                                   ctypes.POINTER(ss_surfel_grads), ctypes.POINTER(ss_env_map_grads), c_vp,
                                   ctypes.c_size_t, c_vp]),
    "ss_read_status": (c_i32, [c_vp, c_vp]),
    "ss_box_downsample": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp]),
    "ss_read_stats": (c_i32, [c_vp, ctypes.c_void_p, c_vp]),
    "ss_launch_count": (c_i32, [ctypes.POINTER(ctypes.c_int64)]),
    "ss_stream_capture_id": (c_i32, [c_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "ss_profile_begin": (c_i32, []),
    "ss_profile_end": (c_i32, [ctypes.c_void_p]),
    "ss_default_adam": (None, [ctypes.POINTER(ss_adam_params)]),
    "ss_adam_step": (c_i32, [ctypes.POINTER(ss_adam_group), c_i32, ctypes.POINTER(ss_adam_params), c_vp]),
    "ss_loss_l1": (c_i32, [c_vp, c_vp, c_i64, c_f, c_vp, c_vp, c_vp]),
    "ss_loss_sil_iou": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_f, c_vp, c_vp, c_vp]),
    "ss_default_density": (None, [ctypes.POINTER(ss_density_params)]),
    "ss_density_workspace_size": (c_i32, [c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "ss_density_neighbours": (c_i32, [ctypes.POINTER(ss_surfels), ctypes.POINTER(c_i64), c_i32,
                                      ctypes.POINTER(ss_density_params), c_vp, c_vp, c_vp, c_vp, ctypes.c_size_t,
                                      c_vp]),
    "ss_density_plan": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(ss_density_params),
                                c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "ss_density_apply": (c_i32, [ctypes.POINTER(ss_surfels), c_i64, c_vp, c_vp, c_f, ctypes.POINTER(ss_surfels),
                                 c_vp]),
    "ss_density_compact": (c_i32, [c_vp, c_i32, c_i64, c_vp, c_vp, c_i32, c_vp, c_vp]),
}


class SS3DError(RuntimeError):
    pass


@lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise SS3DError(f"libss3d.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def check(status: int, what: str = ""):
    if status != SS_OK:
        msg = lib().ss_error_string(status).decode()
        raise SS3DError(f"{what}: {msg} (status {status})")
