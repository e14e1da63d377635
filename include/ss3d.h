/*
 * ss3d.h -- C ABI of a GB300 (sm_103a) implementation of the differentiable
 * surfel rasteriser of "3D Surface Splatting" (3DSS, arxiv 2605.05876).
 *
 * Conventions for every entry point
 *  - All pointers named *_dev are device pointers; *_host are host pointers.
 *    The caller owns all memory.  Unless an entry point says otherwise, no
 *    entry point allocates device memory: scratch space is the caller's
 *    workspace (see ss_workspace_size).
 *  - All work is enqueued on the given cudaStream_t (passed as void*; NULL is
 *    the legacy default stream) and is asynchronous.  Entry points return
 *    after enqueueing.
 *  - Host-detectable errors (bad sizes, NULL pointers, a workspace that is
 *    too small, unsupported shapes) are returned immediately and nothing is
 *    enqueued.  Errors found on the device (instance-capacity overflow,
 *    non-finite inputs) are OR-ed into a status word inside the workspace;
 *    ss_read_status synchronises the stream and returns them.  No kernel
 *    traps.
 *  - Gradient outputs accumulate (+=); zeroing them is the caller's job.
 *  - Float data are IEEE binary32, little-endian, C-contiguous.
 *
 * Geometry conventions (shared with the oracle as a specification)
 *  - Surfel i: centre pos[i], unit quaternion quat[i] = (w, x, y, z) (it is
 *    normalised inside), log-scales (s_u, s_v); the tangent vectors are
 *    t_u = exp(s_u) R(q) e_x, t_v = exp(s_v) R(q) e_y and the normal is
 *    R(q) e_z (Sec. 3.1, Sec. 3.7).  Albedo, roughness and metallic are
 *    activated values in [0, 1].
 *  - Camera: OpenCV pinhole, x_cam = R x_world + t, pixel (i, j) has its
 *    centre at (i + 0.5, j + 0.5), x_pix = fx X/Z + cx.
 *  - Environment maps are equirectangular: direction d <-> (phi, theta) with
 *    phi = atan2(d_x, -d_z), theta = acos(d_y); texel (a, b) of a W x H map
 *    is centred at u = (a + 0.5)/W = phi/(2 pi) + 1/2, v = (b + 0.5)/H =
 *    theta/pi; bilinear lookups wrap in u and clamp in v.
 */
#ifndef SS3D_H
#define SS3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ss_status;
#define SS_OK 0
#define SS_ERR_INVALID_ARG 1  /* bad argument; nothing was enqueued */
#define SS_ERR_WORKSPACE 2    /* workspace smaller than ss_workspace_size */
#define SS_ERR_CAPACITY 4     /* device: more (tile, surfel) instances than
                                 ss_render_params.max_instances, more block
                                 candidates than max_candidates, more deep
                                 layers than layer_pool, or (the deterministic
                                 backward) more covering (block, surfel) pairs
                                 than det_rows; the affected outputs are
                                 incomplete */
#define SS_ERR_TIMEOUT 8      /* device: a bounded wait gave up */
#define SS_ERR_NONFINITE 16   /* device: a non-finite surfel parameter was seen
                                 (that surfel is skipped) */
#define SS_ERR_CUDA 32        /* a CUDA runtime call failed */

#define SS_MAX_VIEWS 256
#define SS_MAX_SCENES 64
#define SS_MAX_RECORDS 0xfffffffell   /* (view, surfel) records of a batch: sum over the views of
                                         their scene's surfels (32-bit record indices) */
#define SS_MAX_TILES (1ll << 27)       /* screen tiles of a batch, over all views */
#define SS_KMAX_LIMIT 16      /* App. A: at most 16 composited layers */
#define SS_N_AOV 9            /* albedo(3), roughness, metallic, normal(3), depth */
#define SS_MIP_CENTRE 0       /* values of ss_render_params.mip_mode (see there) */
#define SS_MIP_NONE 1
#define SS_MIP_PIXEL 2

/* One view.  80 bytes; arrays of it are read by both host and device. */
typedef struct ss_camera {
    float R[9];        /* world->camera rotation, row-major */
    float t[3];        /* world->camera translation */
    float fx, fy, cx, cy;
    int32_t width, height;
    int32_t scene;     /* index of the scene (surfel set + env map) it shows */
    int32_t pad_;
} ss_camera;

/* Surfel parameters of all scenes, concatenated (device, SoA). */
typedef struct ss_surfels {
    const float* pos;        /* [N][3] */
    const float* quat;       /* [N][4] (w, x, y, z) */
    const float* log_scale;  /* [N][2] (s_u, s_v) */
    const float* albedo;     /* [N][3] */
    const float* roughness;  /* [N] */
    const float* metallic;   /* [N] */
} ss_surfels;

/* Gradients w.r.t. ss_surfels (device, same layout, accumulated +=).
 * Any member may be NULL to skip it.
 *
 * The last two members are the densification statistic of Sec. 3.6.1
 * (Eq. ss_grad), filled only when ss_render_params.screen_grad = 1 (else
 * they must be NULL).  Every covering fragment of surfel i in view j adds
 * |(g_x, g_y)| with g_x = dL/dT_{1,z} T_{4,z}, g_y = dL/dT_{2,z} T_{4,z}: the
 * derivative of the fragment's own term of the loss with respect to the
 * z entries of the T-matrix rows (the column that multiplies the centre c',
 * so that (T_{1,z}, T_{2,z}) / T_{4,z} is the screen centre), through the
 * ray-plane intersection and the centre-precomputed MIP filter, with every
 * discrete decision and the shaded channels held fixed; norms, not signed
 * values, are summed, so contributions do not cancel.
 *   screen_grad_norm[i]  += sum over views and fragments of |(g_x, g_y)|
 *   screen_grad_views[i] += number of views in which surfel i has at least one
 *                           covering fragment (exact small integers in FP32)
 * The criterion of Eq. 3dgs_grad is their ratio, taken by the caller. */
typedef struct ss_surfel_grads {
    float* pos;
    float* quat;
    float* log_scale;
    float* albedo;
    float* roughness;
    float* metallic;
    float* screen_grad_norm;   /* [N] or NULL */
    float* screen_grad_views;  /* [N] or NULL */
} ss_surfel_grads;

/* A batch: several scenes, each with its surfels and views.
 * Views must be ordered by scene (all views of scene 0 first, ...). */
typedef struct ss_batch_desc {
    int32_t n_scenes;                 /* 1 .. SS_MAX_SCENES */
    int32_t n_views;                  /* 1 .. SS_MAX_VIEWS */
    const int64_t* scene_offsets_host;/* [n_scenes + 1] surfel ranges */
    const ss_camera* cams_host;       /* [n_views]: sizes and scene indices */
    const ss_camera* cams_dev;        /* [n_views]: poses/intrinsics read by the
                                         kernels (same sizes and scenes as
                                         cams_host; may change between calls,
                                         e.g. between CUDA-graph replays) */
} ss_batch_desc;

/* Renderer constants.  ss_default_params fills the paper's values. */
typedef struct ss_render_params {
    float r_cut;             /* kernel cutoff, 3 (App. A) */
    float sigma_f;           /* screen prefilter variance of Eq. mip_cov, px^2 */
    float gamma;             /* coverage gain of Eq. alpha, 2 pi (Sec. 3.5.1) */
    int32_t k_max;           /* max composited layers, 16 (App. A) */
    float z_near;            /* surfels with z_start <= z_near are culled */
    float bg[3];             /* background radiance behind the last layer */
    int32_t write_aov;       /* 1: also write the 9 AOV channels */
    int32_t lut_n;           /* BRDF table resolution (n x n) */
    int64_t max_instances;   /* capacity of the (tile, surfel) instance list: 1 .. 2^32 - 1 */
    int32_t collect_stats;   /* 1: count work (see ss_read_stats); off by default */
    /* launch shapes (0 = default); they change speed, never results */
    int32_t fwd_warps;       /* warps per CTA of the forward rasteriser: 1 (default), 2 or 4 */
    int32_t bwd_warps;       /* warps per CTA of the backward rasteriser: 2, 4 (default) or 8 */
    int32_t pbwd_block;      /* surfels per CTA of the projection adjoint: 32..1024, default 128 */
    int32_t screen_grad;     /* 1: the backward also accumulates the densification statistic
                                (ss_surfel_grads.screen_grad_*); the workspace then holds 64 more
                                bytes per (surfel, view) record */
    int32_t mip_mode;        /* MIP filter (Sec. 3.3): 0 = centre-precomputed Sigma_mip and n_f
                                (Sec. 3.3.2, the method; default), 1 = none (Sigma_mip = I, n_f = 1:
                                sigma_f is taken as 0), 2 = per-pixel Jacobian of the ray-splat
                                intersection (AA-2DGS, Sec. 3.3.1; the Sec. 4.4.2 ablation): Sigma_mip
                                = I + sigma_f J J^T and n_f evaluated at every hit.  Mode 2 is
                                forward-only: ss_render_backward returns SS_ERR_INVALID_ARG */
    int32_t cons;            /* 1: depth-consolidation term of Eq. cons_loss (Sec. 3.7.1): the
                                forward writes per pixel, over its composited layers,
                                sum_{i<j} w_i w_j |z_i - z_j| + sum_i w_i^2 sigma_i^2 (w_i = T_i alpha_i,
                                z_i / sigma_i^2 the mean / variance of the layer's fragment depths,
                                the depth channel) as a tenth AOV plane, so out_aov is [10][P]
                                (write_aov must be 1); the backward then requires d_aov [10][P]
                                whose tenth plane is the upstream gradient of that term.  Not with
                                mip_mode 2.  The workspace keeps 3 more floats per pixel layer */
    /* tiling and staging (0 = default); they change speed, never results */
    int32_t tile_w, tile_h;  /* screen tile of the binning and the rasterisers: tile_w in {8, 16, 32},
                                tile_h in {4, 8, 16, 32}, at most 8 blocks of 8 x 4 pixels per tile
                                (default 16 x 16, App. A) */
    int32_t stage_depth;     /* forward rasteriser: chunks of 32 candidate records in flight per warp
                                (1 = none ahead, 2 default, 3) */
    int32_t deterministic;   /* 1: ss_render_backward sums in a fixed order, so that two calls on the
                                same inputs give bitwise-equal gradients (the FP32 atomic adds of
                                the default mode leave the last bits to the scheduling): each
                                (warp block, staged surfel) writes its fragment sums to a row of
                                its own, and every (surfel, view) record sums its rows in row
                                order; the environment-texel gradients are summed as 64-bit
                                fixed-point integers (exact and order-free; the scale is a power of
                                two from a bound on the largest contribution: one unit is at most
                                2^(c - 56) (V + 1) of the largest record colour gradient, with 2^c
                                >= 8 (surfels + records) + 1 and V the most views of a scene, about
                                2^-24 for 1M surfels x 16 views; c <= 40 is required).  Slower; the
                                workspace holds 104 bytes per row (det_rows) more */
    int64_t det_rows;        /* deterministic = 1: capacity of those rows, one per (warp block,
                                staged surfel that covers a pixel of the block) pair
                                (ss_stats.staged_covering of the forward); 0 = the bound of
                                (blocks per tile) x max_instances.  More pairs than rows set
                                SS_ERR_CAPACITY (the gradients are then incomplete) */
    /* layer state kept by the forward for the backward (with_backward workspaces) */
    int32_t dense_layers;    /* layers per pixel held in planes of every pixel (0 = k_max: all of
                                them, no pool); the layers past it go to layer_pool */
    int32_t zero_grad_in_forward;   /* 1: a forward that keeps backward state also clears the
                                per-record gradient rows of the workspace (one 96-byte row per
                                (view, surfel) record, written by the projection pass, where the
                                stores cost little), and a backward called with it set adds into
                                those rows without clearing them first.  Valid only for the
                                backward that follows such a forward on the same workspace, in
                                stream order, with nothing in between that could write the rows
                                (inside CUDA graphs: both captured in the same graph); otherwise
                                call the backward with 0.  0 (default): the backward clears the
                                rows itself */
    int64_t layer_pool;      /* dense_layers < k_max: slots for the (pixel, layer) pairs past
                                dense_layers, 64 bytes each (80 with cons); ss_stats.pool_layers
                                of a forward is the number it needed.  More pairs than slots
                                set SS_ERR_CAPACITY (the backward then drops those layers' terms) */
    int64_t max_candidates;  /* capacity of the per-(tile, 8 x 4 block) candidate lists of the
                                rasterisers: the (tile, surfel) instances whose support can reach a
                                block, once per block (ss_stats.candidates of a forward; 4 bytes each,
                                16 with with_backward); 0 = the bound of (blocks per tile) x
                                max_instances.  A block whose list would pass the capacity is not
                                rendered and sets SS_ERR_CAPACITY */
} ss_render_params;

/* Work counters of the last forward/backward pair (collect_stats = 1). */
typedef struct ss_stats {
    int64_t instances;       /* (tile, surfel) instances */
    int64_t rect_tests;      /* (pixel, surfel) pairs with the pixel inside the support rectangle */
    int64_t lane_tests;      /* pixel tests executed by the forward raster */
    int64_t fragments;       /* covering fragments accumulated by the forward raster */
    int64_t layers;          /* composited layers summed over pixels */
    int64_t bwd_fragments;   /* fragments differentiated by the backward raster */
    int64_t staged;          /* (warp block, surfel) pairs the forward raster staged */
    int64_t staged_covering; /* ... of which cover at least one pixel of the block */
    int64_t bwd_batches;     /* groups of up to 32 fragments the backward raster differentiated together */
    int64_t pool_layers;     /* (pixel, layer) pairs past dense_layers that the forward stored in
                                layer_pool slots (counted whether or not collect_stats is set, and
                                beyond the capacity, so it sizes layer_pool) */
    int64_t candidates;      /* (tile, block, surfel) candidates of the rasterisers' block lists
                                (counted whether or not collect_stats is set; it sizes
                                max_candidates) */
} ss_stats;

/* Stage timing: CUDA events recorded on the launching stream around each
 * stage of every call made between ss_profile_begin and ss_profile_end
 * (host-side state, one profile at a time; not for use inside stream
 * capture).  Stages: 0 project, 1 bin+sort, 2 raster_fwd, 3 raster_bwd,
 * 4 project_bwd, 5 env_prefilter, 6 env_prefilter_backward, 7 density
 * control (ss_density_*), 8 the densification statistic's per-record
 * derivatives (ss_render_backward with screen_grad = 1). */
#define SS_N_STAGES 9
typedef struct ss_stage_times {
    float ms[SS_N_STAGES];       /* summed event durations */
    int32_t launches[SS_N_STAGES];
} ss_stage_times;

/* Environment map shape.  Every scene has one map of this shape. */
typedef struct ss_env_desc {
    int32_t width, height;   /* base map, width = 2 height, both powers of two */
    int32_t n_levels;        /* specular levels (roughness i/(n_levels-1)) */
    int32_t irr_width, irr_height; /* diffuse irradiance map size; irr_width a power of
                                      two <= width, irr_height in [1, 512] */
} ss_env_desc;

/* Prefiltered environment of every scene plus the BRDF table (device). */
typedef struct ss_env_maps {
    const float* irr;        /* [S][irr_h][irr_w][3] */
    const float* spec;       /* [S][spec_floats]: levels back to back, each [H_i][W_i][3] */
    const float* lut;        /* [lut_n][lut_n][2]: (beta1, beta2) at
                                (roughness row, n.v column) cell centres */
} ss_env_maps;

/* Gradients w.r.t. the prefiltered maps (device, accumulated +=). */
typedef struct ss_env_map_grads {
    float* irr;              /* [S][irr_h][irr_w][3] or NULL */
    float* spec;             /* [S][spec_floats] or NULL */
} ss_env_map_grads;

/* ---------------------------------------------------------------------- */

/* Fill p with the paper's constants (r_cut 3, gamma 2 pi, K_max 16) and this
 * library's defaults for what the paper leaves open (sigma_f 0.5 px^2,
 * z_near 0.01, black background, AOVs on, 128 x 128 BRDF table).
 * max_instances is set to 0; size it with ss_count_instances or a bound. */
void ss_default_params(ss_render_params* p);

/* Human-readable text for the lowest set bit of a status. */
const char* ss_error_string(ss_status s);

/* Split-sum BRDF table of Eq. ibl: (beta1, beta2) with F0 beta1 + beta2 the
 * specular factor (Sec. 3.4.2), for isotropic GGX (alpha = r^2) with the
 * Smith-Schlick G (k = alpha/2) and Schlick Fresnel:
 *   beta1 = Int D G (v.h) (1 - (1 - v.h)^5) / (n.v) dh,
 *   beta2 = Int D G (v.h) (1 - v.h)^5 / (n.v) dh   over n.l > 0,
 * evaluated at cell centres r = (row + 0.5)/n, n.v = (col + 0.5)/n.
 * lut_dev: [n][n][2] floats.  n in [4, 1024].  Deterministic. */
ss_status ss_brdf_lut(float* lut_dev, int32_t n, void* stream);

/* Sizes (in floats) of the prefiltered maps of ONE scene, and of the
 * scratch that ss_env_prefilter keeps for the backward pass. */
ss_status ss_env_sizes(const ss_env_desc* d, int64_t* irr_floats, int64_t* spec_floats,
                       int64_t* aux_floats);

/* Environment prefilter (Sec. 3.4.2: "pre-convolved diffuse environment
 * map" queried along n; specular radiance "pre-filtered ... at a MIP level
 * determined by the roughness"):
 *   irradiance  L_d(n_t) = sum_j L_j max(0, n_t.w_j) dW_j / sum_j max(0, n_t.w_j) dW_j
 *               over all base texels j;
 *   level 0     the base map;
 *   level i>=1  roughness r_i = i/(n_levels-1), size (max(W>>i,8), max(H>>i,4)),
 *               source S = base box-averaged to that size,
 *               L_i(w_t) = sum_j S_j D(h_j) max(0, w_t.w_j) dW_j / sum_j D(h_j) max(0, w_t.w_j) dW_j
 *               with GGX D at alpha = r_i^2 and (n.h_j)^2 = (1 + w_t.w_j)/2.
 * env_dev: [n_envs][H][W][3].  Writes irr, spec and aux (normalisers and
 * box-averaged sources, read by ss_env_prefilter_backward).
 * The per-level convolutions run side by side on side streams that the
 * library creates on the first call on a device and keeps; they are forked
 * from `stream` and joined back to it with events before the call returns,
 * so the work is ordered on `stream` as usual (and is capturable). */
ss_status ss_env_prefilter(const ss_env_desc* d, int32_t n_envs, const float* env_dev,
                           float* irr_dev, float* spec_dev, float* aux_dev, void* stream);

/* The same environment prefilter for callers that cannot allocate device
 * memory (plugins handed only input/output buffers by a host application,
 * code under a fixed budget or a pooled allocator that forbids cudaMalloc,
 * or code that must not let cudaMalloc synchronise the device).  The paper
 * has no counterpart: this is a convenience of this library.
 * Instead of a caller-provided aux buffer it uses a fixed scratch array of
 * SS_NOALLOC_AUX_FLOATS floats (4 MiB) in device memory, which every GPU that
 * loads the library holds until the process exits; the call itself
 * allocates nothing.  Inputs and outputs are as in ss_env_prefilter.
 * Returns SS_ERR_INVALID_ARG if n_envs * aux_floats (ss_env_sizes) exceeds
 * SS_NOALLOC_AUX_FLOATS (e.g. at most 5 maps of 512 x 256 with 6 levels).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * That address is kept for the rest of the process and is only valid while
 * the device's context lives: after cudaDeviceReset on that device, do not
 * call this entry point again in the same process.
 * All calls share the array and it keeps the last call's contents, so calls
 * that overlap on the GPU (on different streams) race.  The scratch it keeps
 * is not the aux that ss_env_prefilter_backward expects. */
#define SS_NOALLOC_AUX_FLOATS (1 << 20)
ss_status ss_env_prefilter_noalloc(const ss_env_desc* d, int32_t n_envs, const float* env_dev, float* irr_dev,
                                   float* spec_dev, void* stream);

/* Transpose of ss_env_prefilter: d_env += P^T (d_irr, d_spec).  aux_dev is
 * the scratch written by the forward call for the same env maps.  The level
 * terms are added on the side streams with atomics, so the last bits of d_env
 * can differ from call to call. */
ss_status ss_env_prefilter_backward(const ss_env_desc* d, int32_t n_envs, const float* d_irr_dev,
                                    const float* d_spec_dev, const float* aux_dev, float* d_env_dev,
                                    void* stream);

/* The same transpose with the level terms added one level after the other
 * on `stream` (level 0, the specular levels 1 .. n_levels - 1, then the
 * irradiance map), each base texel receiving one add per term: d_env is then
 * bitwise the same from call to call.  The companion of
 * ss_render_params.deterministic = 1; slower than the forked form. */
ss_status ss_env_prefilter_backward_ordered(const ss_env_desc* d, int32_t n_envs, const float* d_irr_dev,
                                            const float* d_spec_dev, const float* aux_dev, float* d_env_dev,
                                            void* stream);

/* Workspace bytes for a render of this batch.  with_backward != 0 adds the
 * per-pixel layer state that ss_render_backward reads and, for the env
 * description ed (required then: the one later passed to the render calls),
 * the accumulators of the env-map gradients (and, with p->deterministic = 1,
 * the rows and per-record lists of the fixed-order sums).  Requires
 * p->max_instances > 0.
 * Host only (reads no device memory).  Errors: SS_ERR_INVALID_ARG for bad
 * sizes (among them a batch past SS_MAX_RECORDS records or SS_MAX_TILES
 * tiles), an invalid ed or a launch shape (fwd_warps, bwd_warps, pbwd_block)
 * without a compiled kernel; the render calls reject the same values. */
ss_status ss_workspace_size(const ss_batch_desc* b, const ss_render_params* p, const ss_env_desc* ed,
                            int32_t with_backward, size_t* bytes);

/* Exact number of (tile, surfel) instances of a batch: runs the projection
 * step into `ws` and reads the count back (synchronises the stream).  Use it
 * to size max_instances.  `ws` must be at least ss_workspace_size bytes for
 * the same batch with max_instances = 1. */
ss_status ss_count_instances(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                             const ss_env_desc* ed, const ss_env_maps* env, void* ws, size_t ws_bytes,
                             int64_t* count, void* stream);

/* Forward render (Sec. 3, Fig. 2 stages 1-5 without tone mapping):
 * per surfel and view the T-matrix (Sec. 3.1), depth interval, centre-
 * precomputed MIP filter (Eq. mip_weight) and forward split-sum shading
 * (Eq. ibl); binning into screen tiles (16 x 16 by default, App. A) sorted by
 * z_start (Sec. 3.2.1);
 * per pixel Algorithm 1 with Eq. alpha coverage and Eq. compositing, at most
 * K_max layers.  Surfel i covers pixel x iff x lies in its support rectangle
 * (the projected r_cut disc of App. A united with the r_cut bounds of the
 * screen-space EWA ellipse M M^T + sigma_f I, padded 1 px) and
 * rho2_mip(x) < r_cut^2.
 * Outputs (device): out_rgba [P][4] (linear radiance composited over bg, and
 * coverage 1 - T_{K+1}), out_aov [9][P] planar (may be NULL if
 * p->write_aov == 0), where P = sum over views of width*height and view v's
 * pixels start at the running sum over earlier views, row-major.
 * The workspace keeps what ss_render_backward needs. */
ss_status ss_render_forward(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                            const ss_env_desc* ed, const ss_env_maps* env, float* out_rgba_dev,
                            float* out_aov_dev, void* ws, size_t ws_bytes, void* stream);

/* Backward of ss_render_forward (App. A "Backward Pass"): replays each
 * pixel's grouping front to back against the layer totals kept by the
 * forward call and accumulates the gradient of L = sum(d_rgba * rgba) +
 * sum(d_aov * aov) w.r.t. the surfel parameters and the prefiltered maps.
 * All discrete decisions (support, cutoff, grouping, K_max) are held fixed.
 * d_aov may be NULL.  out_rgba/out_aov are the forward outputs.  Must follow
 * a ss_render_forward with with_backward workspace and the same inputs, one
 * backward per forward: the backward turns the forward's per-pixel layer
 * state into its own coefficients in place. */
ss_status ss_render_backward(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                             const ss_env_desc* ed, const ss_env_maps* env, const float* out_rgba_dev,
                             const float* out_aov_dev, const float* d_rgba_dev, const float* d_aov_dev,
                             ss_surfel_grads* g, ss_env_map_grads* genv, void* ws, size_t ws_bytes,
                             void* stream);

/* Box filter of an RGBA image by an integer factor (the 4x supersampled
 * reference of Sec. 4.4.2: render at factor x the resolution without the MIP
 * filter, then average factor x factor blocks).  in_dev [H][W][4] row-major,
 * out_dev [H/factor][W/factor][4]; W and H multiples of factor, factor in
 * [1, 16].  Errors: SS_ERR_INVALID_ARG for NULL pointers or bad sizes. */
ss_status ss_box_downsample(const float* in_dev, int32_t width, int32_t height, int32_t factor, float* out_dev,
                            void* stream);

/* Start / stop collecting stage timings (see ss_stage_times).  end
 * synchronises the recorded events and fills *out. */
ss_status ss_profile_begin(void);
ss_status ss_profile_end(ss_stage_times* out);

/* Synchronise the stream and copy the work counters of ws into *out. */
ss_status ss_read_stats(void* ws, ss_stats* out, void* stream);

/* Number of kernels this library has launched in the calling process since it
 * was loaded (every entry point's launches, on every device and stream).  A
 * host-side counter with no counterpart in the paper: it lets a caller count
 * the GPU work of a region (read before and after).  out: host int64.
 * Errors: SS_ERR_INVALID_ARG for a null out. */
ss_status ss_launch_count(int64_t* out);

/* Which CUDA graph capture, if any, the stream is recording into: *id = the
 * capture's id (unique in the process), or 0 when the stream is not
 * capturing.  A host query with no counterpart in the paper; it lets a
 * caller pair a forward and a backward recorded in the same graph (see
 * ss_render_params.zero_grad_in_forward).  out: host uint64.  Errors:
 * SS_ERR_INVALID_ARG for a null id; SS_ERR_CUDA if the query fails. */
ss_status ss_stream_capture_id(void* stream, uint64_t* id);

/* Synchronise the stream and return (and clear) the device status word in
 * ws: SS_OK or an OR of SS_ERR_CAPACITY / SS_ERR_TIMEOUT / SS_ERR_NONFINITE. */
ss_status ss_read_status(void* ws, void* stream);

/* ------------------------------------------------------------------------
 * Optimisation (section "Training and Optimization": all surfel parameters
 * and the HDR environment are optimised jointly with Adam, Kingma & Ba 2014,
 * Algorithm 1).
 *
 * The renderer reads activated values; the optimiser owns the raw ones.  A
 * parameter group is one array of raw values with its Adam moments, the
 * gradient of the loss with respect to the ACTIVATED values (what
 * ss_render_backward / ss_env_prefilter_backward produce) and the activation
 * that maps raw to activated:
 *   SS_ACT_IDENTITY  a = theta          (positions, quaternions -- normalised
 *                                        inside the renderer -- and log-scales)
 *   SS_ACT_SIGMOID   a = 1/(1+e^-theta) (albedo, roughness, metallic)
 *   SS_ACT_CLAMP0    a = theta, and theta is projected onto theta >= 0 after
 *                    the step            (environment texels)
 * One step, per element, with g = dL/da * da/dtheta at the current theta:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
 *   theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * then act = a(theta) when act is not NULL.  The paper gives no Adam
 * constants; ss_default_adam gives Kingma & Ba's (0.9, 0.999, 1e-8). */
#define SS_ACT_IDENTITY 0
#define SS_ACT_SIGMOID 1
#define SS_ACT_CLAMP0 2
#define SS_MAX_ADAM_GROUPS 16

typedef struct ss_adam_group {
    float* param_dev;       /* [n] raw values, updated in place */
    const float* grad_dev;  /* [n] dL/d(activated value) */
    float* m_dev;           /* [n] first moment, updated in place */
    float* v_dev;           /* [n] second moment, updated in place */
    float* act_dev;         /* [n] activated values written after the step, or NULL */
    int64_t n;
    float lr;
    int32_t activation;     /* SS_ACT_* */
} ss_adam_group;

typedef struct ss_adam_params {
    float beta1, beta2, eps;
    int32_t step;           /* t >= 1: index of this step (bias correction) */
} ss_adam_params;

void ss_default_adam(ss_adam_params* p);

/* One fused Adam step over n_groups (1 .. SS_MAX_ADAM_GROUPS) groups in a
 * single launch; arrays of different groups must not overlap.  Errors:
 * SS_ERR_INVALID_ARG for a NULL param/grad/m/v of a group with n > 0, a
 * negative n, an unknown activation, step < 1 or a bad group count. */
ss_status ss_adam_step(const ss_adam_group* groups_host, int32_t n_groups, const ss_adam_params* p,
                       void* stream);

/* L1 photometric loss between rendered and target images (the l1 term of
 * Eq. photo_loss, on linear values; the SSIM term and the log/sRGB transfer
 * are not part of this entry point): over n floats of out and
 * target (device), loss = scale * sum |out - target| is written to
 * *loss_dev (one float, overwritten) and d_out = scale * sign(out - target)
 * (0 where equal) to d_out_dev (overwritten).  The sum is deterministic
 * (fixed order).  Its partial sums live in a fixed per-device array, so calls
 * on one device must not overlap in time (one stream, or serialised).
 * Errors: SS_ERR_INVALID_ARG for NULL pointers or n < 0. */
ss_status ss_loss_l1(const float* out_dev, const float* target_dev, int64_t n, float scale, float* d_out_dev,
                     float* loss_dev, void* stream);

/* Silhouette loss of Eq. sil_loss (Sec. 3.7.1): the soft intersection-over-
 * union loss between the rendered coverage A = 1 - T_{K+1} (the alpha
 * channel of ss_render_forward's RGBA output) and a mask M in [0, 1], per
 * view v with pixels [view_offsets[v], view_offsets[v+1]):
 *   I = sum A M,  U = sum (A + M - A M),  loss_dev[v] = scale (1 - I / U)
 * (0 where U = 0), and its gradient -scale (M U - I (1 - M)) / U^2 ADDED to
 * the alpha channel of d_rgba_dev [P][4] (so that it combines with other
 * terms of the loss).  rgba_dev [P][4] (16-byte aligned), mask_dev [P],
 * view_offsets_dev [n_views + 1] int64 (device), loss_dev [n_views].  The
 * sums are FP64 in a fixed order: deterministic.  Errors:
 * SS_ERR_INVALID_ARG for NULL or misaligned pointers or n_views outside
 * [1, 65535]. */
ss_status ss_loss_sil_iou(const float* rgba_dev, const float* mask_dev, const int64_t* view_offsets_dev,
                          int32_t n_views, float scale, float* d_rgba_dev, float* loss_dev, void* stream);

/* ------------------------------------------------------------------------
 * Adaptive density control (Sec. 3.6.2 and the appendix on splitting and
 * pruning surfels).
 *
 * A spatial index over the surfel centres gives each surfel the mean
 * distance d_bar to its k nearest same-orientation neighbours (other surfels
 * of the same scene whose unit normals satisfy n_i . n_j >= cos_min; the
 * paper names neither k nor the test) and the distance to its nearest
 * neighbour of any orientation.  With the screen-space statistic of
 * Eq. ss_grad (ss_surfel_grads.screen_grad_norm / screen_grad_views) these
 * decide, per surfel:
 *   prune  (SS_DENSITY_PRUNE_VISIBLE)   its summed statistic is zero: no
 *          backward pass ever reached it;
 *   prune  (SS_DENSITY_PRUNE_ISOLATED)  no neighbour within its kernel
 *          support r_cut * max(s_u, s_v);
 *   split  (SS_DENSITY_SPLIT)  g_bar = norm / views >= tau_g and
 *          max(s_u, s_v) > d_bar: two children at c +- (s_max/2) t_max
 *          (t_max the unit tangent of the larger scale, u on a tie), the
 *          scale along t_max times split_scale (0.7), everything else
 *          inherited;
 *   keep   otherwise.  A pruning rule wins over splitting.
 * The new surfel arrays hold, in the parents' order, each kept surfel once
 * and each split one as its two children (the + child first).
 *
 * Index: a hashed uniform grid of cell size `cell` (world units).  A query
 * visits rings of cells around its own, nearest first, skipping cells
 * farther than its current k-th distance, until the k nearest
 * same-orientation neighbours are certain (the k-th lies within the radius
 * the visited cells cover) or the ring of radius max_rings is done.  Results are
 * exact where certain; elsewhere flags say which value is only a lower
 * bound. */
#define SS_DENSITY_SPLIT 1
#define SS_DENSITY_PRUNE_VISIBLE 2
#define SS_DENSITY_PRUNE_ISOLATED 4
#define SS_DENSITY_KMAX 16
#define SS_DENSITY_MAX_RINGS 32
/* flags of ss_density_neighbours */
#define SS_NB_MEAN_BOUND 1   /* fewer than k same-orientation neighbours were
                                certain: mean_dist is a lower bound of d_bar
                                (each missing one counted at the covered
                                radius); the surfel is not split */
#define SS_NB_NN_BOUND 2     /* no neighbour within the covered radius:
                                nn_dist is that radius, a lower bound */
#define SS_NB_NONFINITE 4    /* non-finite centre: not indexed, results NaN */
/* actions of ss_density_plan */
#define SS_ACTION_PRUNE 0
#define SS_ACTION_KEEP 1
#define SS_ACTION_SPLIT 2

typedef struct ss_density_params {
    int32_t k;            /* neighbours averaged for d_bar, 1 .. SS_DENSITY_KMAX (default 8) */
    float cos_min;        /* same orientation: n_i . n_j >= cos_min (default 0.5) */
    float cell;           /* grid cell size, world units, > 0; queries cost
                             least near the typical k-th neighbour distance.
                             ss_default_density leaves it 0: the caller
                             chooses from its scene's scale */
    int32_t max_rings;    /* largest ring radius in cells, 1 .. SS_DENSITY_MAX_RINGS (default 4) */
    float tau_g;          /* split threshold on g_bar (default 2e-4) */
    float r_cut;          /* kernel support in units of the scale (default 3) */
    float split_scale;    /* factor on the split axis' scale, (0, 1] (default 0.7) */
    int32_t ops;          /* OR of SS_DENSITY_* (default all three) */
} ss_density_params;

void ss_default_density(ss_density_params* p);

/* Bytes of device workspace ss_density_neighbours and ss_density_plan need
 * for n surfels.  Errors: SS_ERR_INVALID_ARG for n < 0 or a null out. */
ss_status ss_density_workspace_size(int64_t n, size_t* bytes);

/* Neighbour statistics of the n = scene_offsets_host[n_scenes] surfels s
 * (scenes 0 .. n_scenes-1 own [scene_offsets_host[i], scene_offsets_host[i+1]),
 * neighbours only within a scene).  Writes mean_dist_dev [n] (d_bar),
 * nn_dist_dev [n] and flags_dev [n] (int32, SS_NB_*).  Uses pos and quat
 * only.  Deterministic: the k distances are summed in ascending order.
 * Errors: SS_ERR_INVALID_ARG for null pointers, bad offsets or parameters;
 * SS_ERR_WORKSPACE for a workspace below ss_density_workspace_size. */
ss_status ss_density_neighbours(const ss_surfels* s, const int64_t* scene_offsets_host, int32_t n_scenes,
                                const ss_density_params* p, float* mean_dist_dev, float* nn_dist_dev,
                                int32_t* flags_dev, void* ws, size_t ws_bytes, void* stream);

/* Decide every surfel's action (SS_ACTION_*) from its log-scales, the
 * screen-space statistic (norm and view count, as accumulated by
 * ss_render_backward with screen_grad = 1) and the outputs of
 * ss_density_neighbours.  action_dev [n] int32; out_offset_dev [n + 1] int64:
 * the first output row of each surfel, the new surfel count last.  g_bar is
 * norm / views in binary32.  Errors: SS_ERR_INVALID_ARG for null pointers
 * (any input may be NULL only when n = 0), bad parameters; SS_ERR_WORKSPACE. */
ss_status ss_density_plan(const float* log_scale_dev, const float* screen_grad_norm_dev,
                          const float* screen_grad_views_dev, const float* mean_dist_dev, const float* nn_dist_dev,
                          const int32_t* flags_dev, int64_t n, const ss_density_params* p, int32_t* action_dev,
                          int64_t* out_offset_dev, void* ws, size_t ws_bytes, void* stream);

/* Write the new surfels: `out` arrays hold out_offset[n] rows (read it back
 * first) and must not overlap `in`.  Children's positions and log-scales
 * follow the split rule above; the rotation, albedo, roughness and
 * metallic are copied.  Errors: SS_ERR_INVALID_ARG for null pointers or
 * split_scale outside (0, 1]. */
ss_status ss_density_apply(const ss_surfels* in, int64_t n, const int32_t* action_dev, const int64_t* out_offset_dev,
                           float split_scale, const ss_surfels* out, void* stream);

/* Carry another per-surfel array of `width` floats per row (an optimiser's
 * raw values or moments) through the same step: kept rows once, split rows
 * twice, or as two rows of zeros when zero_children is 1.  Errors:
 * SS_ERR_INVALID_ARG for null pointers or width outside [1, 64]. */
ss_status ss_density_compact(const float* in_dev, int32_t width, int64_t n, const int32_t* action_dev,
                             const int64_t* out_offset_dev, int32_t zero_children, float* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SS3D_H */
