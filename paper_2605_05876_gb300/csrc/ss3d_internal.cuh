// Internal declarations of the GB300 3DSS rasteriser (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include "ss3d.h"

#define SS_TILE 16                 // default 16 x 16 pixel tiles (App. A); the batch's tile shape is in ss_layout
#define SS_NCH 12                  // averaged channels: rgb, albedo 3, rough, metal, normal 3, depth
// Tile counters and cursors take the atomics of every tile instance; one per
// SS_CNT_STRIDE words spreads them over the L2 slices instead of a few.
#define SS_CNT_STRIDE 32
// Likewise the env-map gradient accumulators: one float4 per texel, 128 bytes apart.
#define SS_ACC_STRIDE 8
#define SS_NGRAD 24                // floats per (view, surfel) gradient record (21 used, 23 with
                                   // the densification statistic)
#define SS_GREC_RGB 9              // its first colour column (dL/d rgb, then the AOV channels)
#define SS_PI_F 3.14159265358979323846f

// ------------------------------------------------------------------------
// batch layout, built on the host and copied into the workspace

struct ss_view_layout {
    int32_t scene;
    int32_t width, height;
    int32_t tiles_x, tiles_y;
    int32_t tile_off;        // first global tile index of this view
    int64_t pixel_off;       // first pixel of this view in the outputs
    int64_t rec_off;         // first record of this view
    int64_t surfel_begin;    // first surfel of the view's scene
    int32_t n_surfels;       // surfels of the view's scene
    int32_t pad_;
};

struct ss_layout {
    int32_t n_views, n_scenes;
    int32_t total_tiles;
    int32_t k_max;
    // screen tile: (1 << tw_log2) x (1 << th_log2) pixels, made of bx x by
    // blocks of 8 x 4 pixels (one warp each), bpt = bx by <= 8 blocks per tile
    int32_t tw_log2, th_log2, bx, bpt, bx_log2, pad_;
    int64_t total_pixels;
    int64_t total_records;
    int64_t scene_begin[SS_MAX_SCENES + 1];
    int32_t scene_view_begin[SS_MAX_SCENES + 1];
    ss_view_layout v[SS_MAX_VIEWS];
};

// Per (view, surfel) record written by the projection step: 7 x float4.
//  r0: P00, P01, P10, P11   factor of the screen-space quadratic form, P^T P = (M M^T + sigma_f I)^-1
//  r1: A2, B2, 1, n_f       perspective denominator s2 = 1 + A2 dx + B2 dy, MIP n_f
//  r2: px_hi, py_hi, px_lo, py_lo   surfel centre in pixels (double-float)
//  r3: z_start, z_end, rect_x, rect_y (packed u16 lo | hi << 16; empty = 0xffff0000? see below)
//  r4: r, g, b, flags       forward-shaded colour (Eq. ibl), flags
//  r5: albedo rgb, roughness
//  r6: metallic, normal xyz (facing the camera, world space)
// With d = (dx, dy) = pixel centre - surfel centre p, the ray hit in the
// surfel plane is (u, v) = J d / s2(d) (J = d(u,v)/d(x,y) at the centre; the
// homogeneous hit is linear in d), so rho2_mip = u^T Sigma^-1_mip u equals
//   rho2_mip = d^T (M M^T + sigma_f I)^-1 d / s2^2 = |P d|^2 / s2^2,
// M = J^-1, and the hit is in front of the camera iff s2 > 0.
struct __align__(16) ss_rec {
    float4 r0, r1, r2, r3, r4, r5, r6;
};

#define SS_FLAG_VALID 1u
#define SS_FLAG_RECT_TEST 2u        // the support rectangle can clip: test it per pixel
#define SS_FLAG_FLIPPED 4u          // shading normal is -n

// Per-view quantities derived on the device from the camera (every call, so
// that cameras may change between graph replays): the camera centre
// o = -R^-1 t in double-float and det R.  R is used as given (its float32
// rounding need not be orthogonal), so R^-1 is not R^T.
struct ss_view_geo {
    float o_hi[3], o_lo[3];
    float detR;
    float pad_;
};

// device status bits live in the first word of the workspace; the work
// counters (ss_stats, int64 x 11) at byte 64 of the same 256-byte block (the
// layer-pool slots taken is the pool's allocation counter; the candidates are
// written by the prefix sum of the block lists)
#define SS_STATS_OFFSET 64
// work-queue heads of the persistent rasterisers (uint32: forward, backward)
// at byte 192 of the same block
#define SS_WORK_OFFSET 192
// deterministic backward: the largest |dL/d rgb| of the records (float bits,
// uint32) at byte 160 of the same block, the bound of the fixed-point scale
#define SS_DET_OFFSET 160
struct ss_ws_view {
    int* status;
    unsigned long long* stats;
    unsigned int* work;     // [2] next (tile, warp block) item of the forward / backward raster
    ss_layout* layout;
    ss_view_geo* vgeo;      // [n_views]
    ss_rec* rec;
    uint32_t* tile_count;   // [total_tiles][SS_CNT_STRIDE] (first word used): instances of records' first four tiles
    uint32_t* tile_start;   // [total_tiles + 1]
    uint32_t* tile_cursor;  // [total_tiles][SS_CNT_STRIDE] (first word used): instances past a record's
                            // first four tiles, counted by the projection, taken down by the scatter
    uint4* inst_rank;       // [total_records] rank of the record in the bins of its first four tiles
    uint2* rec_bmask;       // [total_records] block masks of the record's first four tiles (8 bits each)
                            // and its first tile (x | y << 12 | tiles across << 24), by the scatter
    unsigned long long* keys;      // [max_instances]
    unsigned long long* keys_alt;  // [max_instances]
    uint8_t* bmask;         // [max_instances] per sorted instance: bit b set iff the instance may cover a pixel
                            // centre of 8 x 4 block b of its tile (support rectangle overlaps the block and
                            // the exact support's minimum over the block's pixel centres is below the cutoff)
    uint32_t* cand_list;    // [cand_cap] per (tile, block) from cand_off[tile * 8 + block]: the records of the
                            // tile's list whose block bit is set, in list order
    uint32_t* cand_cnt;     // [total_tiles * 8] candidates of each (tile, block) (the tile sort's block bits)
    uint32_t* cand_off;     // [total_tiles * 8 + 1] their exclusive prefix sum (clamped to 32 bits)
    unsigned long long* scan_tmp;   // block sums of the prefix-sum kernels
    int64_t cand_cap;
    float* layer_state;     // [dense_layers][ls_rows][total_pixels]: raw C (12), W; with the depth-consolidation
                            // term also (sum w (z - z_r), sum w (z - z_r)^2, z_r), z_r the layer's first depth
    int32_t ls_rows;        // 13, or 16 with the depth-consolidation term
    int32_t dense_layers;   // layers per pixel in the dense planes (k_max: no pool)
    float* layer_pool;      // [pool_cap][pool_stride]: the layers past dense_layers, one slot each (ls_rows
                            // values, then the next layer's slot as uint32 bits; 0xffffffff: none)
    int32_t pool_stride;    // 16 floats, or 20 with the depth-consolidation term (16-byte aligned slots)
    int64_t pool_cap;       // slots (0: no pool)
    float* pix_state;       // [3][total_pixels]  (K as float bits, T_end, first pool slot as uint32 bits)
    float* grad_rec;        // [total_records][SS_NGRAD]
    uint2* cover_list;      // [cand_cap] per (tile, block) from cand_off: (record, 32-pixel coverage word) of every
                            // staged surfel that covers a pixel of the block, in list order (forward -> backward)
    uint32_t* cover_adv;    // [cand_cap]: per cover_list entry, the pixel lanes where that
                            // surfel's fragment opens a new layer (Algorithm 1's gap test as the
                            // forward decided it; the first fragment of a pixel opens layer 0 and
                            // is not marked)
    uint32_t* cover_count;  // [8 * tiles]: entries of each warp's list
    float4* env_acc;        // [scenes][env_texels][SS_ACC_STRIDE] RGBA accumulators of the env-map gradients (backward)
    float4* ssg_jac;        // [total_records][4] (screen_grad only): per record, the derivatives of
                            // (P00, P01, P10, P11) and (A2, B2, n_f) along the screen centre, scaled so
                            // that g_x = dL/dp_x + sum_k dL/dval_k jac_x[k] (Eq. ss_grad); x then y
    int64_t env_texels;     // irradiance + specular texels per scene
    int64_t max_instances;
    // deterministic backward (ss_render_params.deterministic): one row of
    // fragment sums per (warp block, covering staged surfel), then per record
    // the sum of its rows in row order
    uint32_t* det_icnt;     // [total_tiles * bpt] covering entries of each (tile, block) item
    uint32_t* det_coff;     // [items + 1] first row of each item (exclusive prefix sum)
    float* det_rows;        // [det_cap][SS_NGRAD]
    uint32_t* det_rid;      // [det_cap] record of each row (0xffffffff: unused)
    uint32_t* det_rcnt;     // [total_records] rows of each record
    uint32_t* det_roff;     // [total_records + 1] first list slot of each record
    uint32_t* det_rcur;     // [total_records] fill cursors
    uint32_t* det_rlist;    // [det_cap] rows of each record (sorted before the sum)
    unsigned long long* det_scan;   // block sums of the prefix-sum kernels
    unsigned int* det_maxbits;      // SS_DET_OFFSET word of the status block
    int64_t det_cap;        // rows (0: deterministic mode off)
};

// The rows of layer kk of pixel gpix (P pixels), for kk = 0, 1, 2, ... in
// turn: a dense plane (row stride P) below dense_layers, else the pool slot
// that the previous layer's slot (or the pixel's first-slot word) links to
// (row stride 1); `slot` carries the chain from one call to the next.  Null
// when the forward ran out of pool slots (SS_ERR_CAPACITY).
#define SS_NO_SLOT 0xffffffffu
__device__ __forceinline__ float* ss_layer_rows(const ss_ws_view& ws, int64_t P, int64_t gpix, int kk, uint32_t& slot,
                                                int64_t& stride) {
    if (kk < ws.dense_layers) {
        stride = P;
        return ws.layer_state + (int64_t)kk * ws.ls_rows * P + gpix;
    }
    stride = 1;
    if (kk == ws.dense_layers) slot = __float_as_uint(ws.pix_state[2 * P + gpix]);
    else if (slot != SS_NO_SLOT) slot = __float_as_uint(ws.layer_pool[(int64_t)slot * ws.pool_stride + ws.ls_rows]);
    return slot == SS_NO_SLOT ? nullptr : ws.layer_pool + (int64_t)slot * ws.pool_stride;
}

// ------------------------------------------------------------------------
// double-float helpers (error-free transforms; Dekker / Knuth)

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return two_sum(s.hi, e);
}
__device__ __forceinline__ dfl df_add_f(dfl a, float b) {
    dfl s = two_sum(a.hi, b);
    return two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
    dfl p = two_prod(a.hi, b);
    return two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    dfl p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    dfl p = df_mul_f(b, q1);
    dfl r = df_add(a, {-p.hi, -p.lo});
    float q2 = __fdiv_rn(r.hi, b.hi);
    return two_sum(q1, q2);
}
// a.x + b  with a, x float3 rows, b float, in double-float
__device__ __forceinline__ dfl df_dot3_add(float a0, float a1, float a2, float x0, float x1, float x2,
                                           float b) {
    dfl acc = two_prod(a0, x0);
    acc = df_add(acc, two_prod(a1, x1));
    acc = df_add(acc, two_prod(a2, x2));
    return df_add_f(acc, b);
}

// N_d = n . (c - o): signed distance of the camera centre o from the plane of
// a surfel with centre c and normal n = R(q/|q|) e_z.  For nearly edge-on
// surfels it is a small difference of O(1) terms, so it is formed in
// double-float from n = (2(xz+wy), 2(yz-wx), w^2-x^2-y^2+z^2) / |q|^2 and o.
struct ss_plane_n {
    dfl n0, n1, n2;   // 2(xz+wy), 2(yz-wx), w^2-x^2-y^2+z^2 in double-float
    float qq;         // |q|^2
};
__device__ __forceinline__ ss_plane_n ss_plane_normal(float4 q) {
    const float qw = q.x, qx = q.y, qy = q.z, qz = q.w;
    ss_plane_n p;
    dfl n0 = df_add(two_prod(qx, qz), two_prod(qw, qy));
    dfl n1 = df_add(two_prod(qy, qz), two_prod(-qw, qx));
    p.n2 = df_add(df_add(two_prod(qw, qw), two_prod(-qx, qx)), df_add(two_prod(-qy, qy), two_prod(qz, qz)));
    p.n0 = {2.f * n0.hi, 2.f * n0.lo};
    p.n1 = {2.f * n1.hi, 2.f * n1.lo};
    p.qq = qw * qw + qx * qx + qy * qy + qz * qz;
    return p;
}
__device__ __forceinline__ float ss_plane_distance_n(const ss_plane_n& p, float c0, float c1, float c2,
                                                     const float o_hi[3], const float o_lo[3]) {
    dfl d0 = df_add_f({-o_hi[0], -o_lo[0]}, c0);
    dfl d1 = df_add_f({-o_hi[1], -o_lo[1]}, c1);
    dfl d2 = df_add_f({-o_hi[2], -o_lo[2]}, c2);
    dfl nd = df_add(df_add(df_mul(p.n0, d0), df_mul(p.n1, d1)), df_mul(p.n2, d2));
    return (nd.hi + nd.lo) / p.qq;
}
__device__ __forceinline__ float ss_plane_distance(float4 q, float c0, float c1, float c2, const float o_hi[3],
                                                   const float o_lo[3]) {
    return ss_plane_distance_n(ss_plane_normal(q), c0, c1, c2, o_hi, o_lo);
}

// ------------------------------------------------------------------------
// small math

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    float n = rsqrtf(w * w + x * x + y * y + z * z);
    w *= n; x *= n; y *= n; z *= n;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ uint32_t pack16(int lo, int hi) {
    return (uint32_t)(lo & 0xffff) | ((uint32_t)(hi & 0xffff) << 16);
}

// Equirect coordinates (u, v) of a direction (not necessarily unit).
__device__ __forceinline__ void dir_to_uv(float dx, float dy, float dz, float& u, float& v) {
    float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    float y = fminf(fmaxf(dy * inv, -1.f), 1.f);
    u = atan2f(dx, -dz) * (0.5f / SS_PI_F) + 0.5f;
    v = acosf(y) * (1.f / SS_PI_F);
}

// Bilinear texel taps of a [H][W] map at continuous (u, v) in [0,1]:
// wrap in u (wrap != 0) or clamp, clamp in v.  Returns 4 texel indices and
// weights; also the derivative weights w.r.t. X = uW - 0.5 and Y = vH - 0.5.
struct ss_taps {
    int i00, i01, i10, i11;
    float fx, fy;
};
__device__ __forceinline__ ss_taps bilinear_taps(float u, float v, int W, int H, bool wrap) {
    float X = u * (float)W - 0.5f, Y = v * (float)H - 0.5f;
    float x0f = floorf(X), y0f = floorf(Y);
    int x0 = (int)x0f, y0 = (int)y0f;
    ss_taps t;
    t.fx = X - x0f;
    t.fy = Y - y0f;
    int xa, xb;
    if (wrap) {   // x0 mod W: one compare for (u in [0, 1] gives x0 in [-1, W - 1]), the division otherwise
        xa = x0 < 0 ? x0 + W : (x0 >= W ? x0 - W : x0);
        if ((unsigned)xa >= (unsigned)W) xa = ((x0 % W) + W) % W;
        xb = xa + 1 == W ? 0 : xa + 1;
    } else {
        xa = min(max(x0, 0), W - 1);
        xb = min(max(x0 + 1, 0), W - 1);
    }
    int ya = min(max(y0, 0), H - 1), yb = min(max(y0 + 1, 0), H - 1);
    t.i00 = ya * W + xa;
    t.i01 = ya * W + xb;
    t.i10 = yb * W + xa;
    t.i11 = yb * W + xb;
    return t;
}

// ------------------------------------------------------------------------
// The per-pixel test, identical in the forward and backward kernels (explicit
// roundings so that both make the same decision bit for bit).
struct ss_hit {
    float s0, s1, s2, q, t;  // t = s2^2
    bool cover;
};
// r0 = P, r1.xy = (A2, B2); s2 = A2 dx + B2 dy + 1
__device__ __forceinline__ ss_hit ss_pixel_test(float4 r0, float4 r1, float dx, float dy, float rc2) {
    ss_hit h;
    h.s0 = __fmaf_rn(r0.x, dx, __fmul_rn(r0.y, dy));
    h.s1 = __fmaf_rn(r0.z, dx, __fmul_rn(r0.w, dy));
    h.s2 = __fmaf_rn(r1.x, dx, __fmaf_rn(r1.y, dy, 1.f));
    h.q = __fmaf_rn(h.s0, h.s0, __fmul_rn(h.s1, h.s1));
    h.t = __fmul_rn(h.s2, h.s2);
    h.cover = (h.s2 > 0.f) && (h.q < __fmul_rn(rc2, h.t));
    return h;
}

// The per-pixel MIP filter (mip_mode 2, AA-2DGS, Sec. 3.3.1): r0 = J0 =
// d(u,v)/d(x,y) at the centre, |det J0| (= 1 / |det M|) in the staged n_f
// slot; the hit is (u, v) = J0 d / s2, whose Jacobian at d is
// J = (J0 - (u, v) g^T) / s2 with g = (A2, B2); then Sigma = I + sigma_f J J^T
// (Eq. mip_cov) and n_f = |Sigma|^-1/2 (Eq. mip_eval) at this pixel.  Nearly
// edge-on surfels have a huge J, so the forms used are free of cancellation:
//   |Sigma| = 1 + sigma_f |J|_F^2 + sigma_f^2 det(J)^2,  det J = det J0 / s2^3
//     (det(J0 - x g^T) = det J0 (1 - g^T J0^-1 x) and J0^-1 (u, v) = d / s2),
//   (u, v) adj(Sigma) (u, v)^T = |(u, v)|^2 + sigma_f |J^T (-v, u)|^2
//     (adj(Sigma) = (1 + sigma_f tr S) I - sigma_f S with S = J J^T, and
//      tr(S) |x|^2 - |J^T x|^2 = |J^T x_perp|^2 in two dimensions),
// so rho2 = the second over the first, both sums of non-negative terms.
struct ss_hit_pp {
    float rho2, nf;
    bool cover;
};
__device__ __forceinline__ ss_hit_pp ss_pixel_test_pp(float4 J0, float4 r1, float detJ0, float dx, float dy,
                                                      float rc2, float sig) {
    ss_hit_pp h;
    const float s2 = __fmaf_rn(r1.x, dx, __fmaf_rn(r1.y, dy, 1.f));
    const float is2 = 1.f / s2;
    const float u = __fmaf_rn(J0.x, dx, J0.y * dy) * is2, v = __fmaf_rn(J0.z, dx, J0.w * dy) * is2;
    const float j00 = __fmaf_rn(-u, r1.x, J0.x) * is2, j01 = __fmaf_rn(-u, r1.y, J0.y) * is2;
    const float j10 = __fmaf_rn(-v, r1.x, J0.z) * is2, j11 = __fmaf_rn(-v, r1.y, J0.w) * is2;
    const float dJ = detJ0 * is2 * is2 * is2;
    const float fro = __fmaf_rn(j00, j00, __fmaf_rn(j01, j01, __fmaf_rn(j10, j10, j11 * j11)));
    const float D = __fmaf_rn(sig * sig, dJ * dJ, __fmaf_rn(sig, fro, 1.f));
    const float p0 = __fmaf_rn(u, j10, -v * j00), p1 = __fmaf_rn(u, j11, -v * j01);   // J^T (-v, u)
    const float num = __fmaf_rn(u, u, __fmaf_rn(v, v, sig * __fmaf_rn(p0, p0, p1 * p1)));
    h.rho2 = num / D;
    h.nf = rsqrtf(D);
    h.cover = (s2 > 0.f) && (h.rho2 < rc2);
    return h;
}

// ------------------------------------------------------------------------
// host-side launchers implemented in the .cu files

// host-side count of kernel launches (ss_launch_count); call before each launch
void ss_note_launch();

// Stage timing of ss_profile_begin / ss_profile_end: events recorded on the
// launching stream around one stage's launches (nothing while no profile is
// open).  ss_stage_open returns a handle for ss_stage_close (-1: not profiling).
int ss_stage_open(int stage, cudaStream_t st);
void ss_stage_close(int handle, cudaStream_t st);
struct ss_stage_scope {
    int h;
    cudaStream_t st;
    ss_stage_scope(int stage, cudaStream_t s) : h(ss_stage_open(stage, s)), st(s) {}
    ~ss_stage_scope() { ss_stage_close(h, st); }
};

// Opt kernel `k` in to `bytes` of dynamic shared memory on the current device
// (a per-device attribute): once per device, tracked in `done` (bit = device).
template <typename K>
inline void ss_smem_optin(K k, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (bit) done.fetch_or(bit, std::memory_order_relaxed);
}

// CTAs of kernel `k` (block threads, dynamic shared memory bytes) that are
// resident at once on the current device: the grid of a persistent kernel.
// Cached per device in `cache` (device d at bits 16 d .. 16 d + 15; devices
// past 3 query every time).
template <typename K>
inline int ss_resident_ctas(K k, int threads, int smem, std::atomic<unsigned long long>& cache) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev < 4) {
        const unsigned c = (unsigned)(cache.load(std::memory_order_relaxed) >> (16 * dev)) & 0xffffu;
        if (c) return (int)c;
    }
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const int n = per_sm * sms;
    if (dev < 4 && n > 0 && n < 65536) cache.fetch_or((unsigned long long)n << (16 * dev), std::memory_order_relaxed);
    return n;
}

void ss_launch_brdf_lut(float* lut, int n, cudaStream_t st);
void ss_launch_env_prefilter(const ss_env_desc* d, int n_envs, const float* env, float* irr, float* spec,
                             float* aux, cudaStream_t st);
// ordered: the level terms one after the other on st (bitwise-reproducible
// d_env) instead of side by side on forked streams
void ss_launch_env_prefilter_bwd(const ss_env_desc* d, int n_envs, const float* d_irr, const float* d_spec,
                                 const float* aux, float* d_env, cudaStream_t st, bool ordered = false);
int64_t ss_env_irr_floats(const ss_env_desc* d);
int64_t ss_env_spec_floats(const ss_env_desc* d);
int64_t ss_env_aux_floats(const ss_env_desc* d);
void ss_env_level_size(const ss_env_desc* d, int i, int* W, int* H);

// the batch's screen tile (copied from ss_layout into kernel arguments)
struct ss_tile_shape {
    int tw_log2, th_log2, bx_log2, bpt;
};

struct ss_fwd_args {
    ss_surfels s;
    ss_render_params p;
    ss_tile_shape ts;
    ss_env_desc ed;
    ss_env_maps env;
    const ss_camera* cams;
    float* out_rgba;
    float* out_aov;
    int with_backward;
};
void ss_launch_project(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st);
void ss_launch_bin_sort(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st);
void ss_launch_raster_fwd(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st);
void ss_launch_box_downsample(const float* in, int W, int H, int f, float* out, cudaStream_t st);

struct ss_bwd_args {
    ss_fwd_args f;
    const float* out_rgba;
    const float* out_aov;
    const float* d_rgba;
    const float* d_aov;
    ss_surfel_grads g;
    ss_env_map_grads genv;
    // deterministic mode: the most views of a scene and log2 of a bound on
    // the contributions one env texel can receive (ss_det_env_exponent)
    int det_vmax, det_cbits;
};
// the densification statistic's per-record derivatives (nothing unless requested)
void ss_launch_screen_grad_jac(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st);
void ss_launch_raster_bwd(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st);
void ss_launch_project_bwd(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st);

// deterministic backward (det.cu): the rows' first index per (tile, block)
// item, before the backward raster; the per-record sums of the rows, after
// it; the bound of the fixed-point environment scale, before the projection
// adjoint.  nv: the raster's gradient values per fragment (columns 0..nv-1,
// plus 21 and 22 with the densification statistic)
void ss_launch_det_item_offsets(const ss_ws_view& ws, const ss_layout& L, cudaStream_t st);
void ss_launch_det_record_sums(const ss_ws_view& ws, const ss_layout& L, int nv, bool ssg, cudaStream_t st);
void ss_launch_det_env_bound(const ss_ws_view& ws, const ss_layout& L, cudaStream_t st);
int64_t ss_det_scan_blocks(int64_t n);
// exclusive prefix sum of n uint32 counts into out[0 .. n] (out[n] = total,
// clamped to 32 bits; a total above cap sets SS_ERR_CAPACITY in *status; the
// total also into *total_out when given); bsum: ss_det_scan_blocks(n) + 1 words
void ss_launch_scan_u32(const uint32_t* in, int64_t n, uint32_t* out, unsigned long long* bsum, unsigned long long cap,
                        int* status, unsigned long long* total_out, cudaStream_t st);

// Fixed-point scale of the deterministic environment-gradient sums: 2^k
// with k from the record bound (maxbits: the largest |dL/d rgb| of a
// record, float bits), the views per scene and the contributions a texel can
// receive (2^cbits), so that no sum can leave the 63-bit range.  A texel
// contribution is a bilinear tap weight times dL/dL_s = dL/dc (F0 beta1 +
// beta2) (one view) or dL/dL_d = sum over the views of dL/dc k_d rho, so with
// activated attributes in [0, 1] it is at most (views + 1) times the bound;
// 16 times that again is kept as headroom (a contribution beyond it is
// flagged, not summed).
__device__ __forceinline__ int ss_det_env_exponent(unsigned int maxbits, int vmax, int cbits) {
    const float m = __uint_as_float(maxbits);
    if (!(m > 0.f) || !(m < 1.0e30f)) return 0;   // no contribution, or a non-finite record (flagged)
    int e = 0;
    frexpf(m * (float)(32 * (vmax + 1)), &e);   // 2^e > 32 (vmax + 1) m
    return 62 - cbits - e;
}
