// Per-warp streaming of a tile's sorted instance list, shared by the forward
// and backward rasterisers.
//
// Each warp owns an 8 x 4 pixel block of a 16 x 16 tile and works on its own
// (no block-wide barrier).  The forward first walks the tile's list 32 keys at
// a time, reading each instance's block mask (computed once per instance by
// the sort kernel: support rectangle overlaps the block and the exact support
// can reach one of its pixel centres), and keeps the instances with its
// block's bit (ballot + prefix count, so the order by z_start is kept) in a
// candidate list; the backward reads the forward's list of covering
// instances.  Either list is then consumed 32 records at a time:
// the records are copied into shared-memory staging slots with cp.async, two
// chunks deep in the forward (while the warp works on chunk c, the records of
// chunk c+1 are in flight into the other buffer).
#pragma once

#include "ss3d_internal.cuh"

#define WSLOTS 32
// Warps per CTA of the rasterisers (a template parameter, chosen at launch
// from ss_render_params).  Every warp is independent (no block barrier), so
// small CTAs let an SM refill a finished warp's slot at once instead of
// waiting for the slowest warp of its tile.
#define RWPB_FWD_DEFAULT 1
#define RWPB_BWD_DEFAULT 4

struct ss_wstage {
    float4 h0[WSLOTS];  // P (screen quadratic-form factor)                  -- every test
    float4 h1[WSLOTS];  // record row 1 on arrival; then A2, B2, centre x, y relative to the tile
    float4 h2[WSLOTS];  // record row 2 on arrival; then z_start, z_end, +-n_f (negative: test the
                        // support rectangle), -
    float4 c0[WSLOTS];  // rgb, flags                                         -- covering fragments
    float4 c1[WSLOTS];  // albedo, roughness
    float4 c2[WSLOTS];  // metallic, normal
    float4 zr[WSLOTS];  // record row 3 (z_start, z_end, rectangle); the rectangle is read by the forward
    uint32_t id[WSLOTS];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// One chunk of up to 32 instances: this lane's record index and the
// instance's block mask (bit b: it may cover a pixel of block b of the tile),
// read from the tile list and its parallel mask list (both coalesced; the
// sort kernel computed the masks once per instance).
struct ss_chunk {
    uint32_t id;
    uint32_t bm;
    bool live;
};

__device__ __forceinline__ ss_chunk fetch_chunk(const unsigned long long* keys, const uint8_t* bmask, int64_t j,
                                                int64_t end) {
    ss_chunk c;
    c.live = j < end;
    c.id = 0;
    c.bm = 0;
    if (c.live) {
        c.id = (uint32_t)(__ldg(keys + j) & 0xffffffffull);
        c.bm = __ldg(bmask + j);
    }
    return c;
}

// Issue the copies of record `id` into slot `lane` of W (lanes with
// active), for lists that are already filtered.
__device__ __forceinline__ void stage_ids(ss_wstage& W, const ss_rec* recs, uint32_t id, int lane, bool active) {
    if (active) {
        const ss_rec* rc = recs + id;
        cp_async16(&W.h0[lane], &rc->r0);
        cp_async16(&W.h1[lane], &rc->r1);
        cp_async16(&W.h2[lane], &rc->r2);
        cp_async16(&W.c0[lane], &rc->r4);
        cp_async16(&W.c1[lane], &rc->r5);
        cp_async16(&W.c2[lane], &rc->r6);
        cp_async16(&W.zr[lane], &rc->r3);
        W.id[lane] = id;
    }
    cp_async_commit();
}

// Wait until at most `pending` (0..2) of this thread's copy groups are still
// in flight.
__device__ __forceinline__ void cp_async_wait_pending(int pending) {
    if (pending <= 0) asm volatile("cp.async.wait_group 0;\n" ::);
    else if (pending == 1) asm volatile("cp.async.wait_group 1;\n" ::);
    else asm volatile("cp.async.wait_group 2;\n" ::);
}

// Wait for the copies of the n staged slots of W (allowing `pending` later
// groups to stay in flight) and rewrite them in place: the centre relative to
// the tile origin (tx0, ty0) from its double-float value, and
// (z_start, z_end, +-n_f).
__device__ __forceinline__ void stage_finish(ss_wstage& W, int n, int lane, float tx0, float ty0, int pending = 0) {
    cp_async_wait_pending(pending);
    __syncwarp();
    if (lane < n) {
        const float4 r1 = W.h1[lane], r2 = W.h2[lane];
        const uint32_t fl = __float_as_uint(W.c0[lane].w);
        const float4 z = W.zr[lane];
        const float prx = __fadd_rn(__fsub_rn(r2.x, tx0), r2.z);
        const float pry = __fadd_rn(__fsub_rn(r2.y, ty0), r2.w);
        W.h1[lane] = make_float4(r1.x, r1.y, prx, pry);
        W.h2[lane] = make_float4(z.x, z.y, (fl & SS_FLAG_RECT_TEST) ? -r1.w : r1.w, 0.f);
    }
    __syncwarp();
}

// Can a surfel cover a pixel whose centre offset d from the surfel centre
// lies in the box [dx0, dx1] x [dy0, dy1]?  Coverage (ss_pixel_test) needs
// f(d) = |P d|^2 - r^2 s2(d)^2 < 0 with s2 = 1 + A2 dx + B2 dy; f is the
// quadratic d^T Q2 d - 2 r^2 g.d - r^2 with Q2 = P^T P - r^2 g g^T, g = (A2, B2).
// When Q2 is positive definite the minimum of f over the box is at the free
// minimiser d_s (if inside; f < 0 there) or on an edge (a clamped 1-D minimum
// per edge), and {f < t} is the ellipse (d - d_s)^T Q2 (d - d_s) < kappa + t,
// kappa = -f(d_s), whose bounding box has half-widths sqrt((kappa + t) (Q2^-1)_aa).
// A box is rejected only when that minimum exceeds a margin far above the
// rounding of the per-pixel test (f is checked in FP32 against r^2 s2^2,
// whose size over the box is at most r^2 (1 + |A2| max|dx| + |B2| max|dy|)^2),
// so a surfel it rejects covers no pixel of the box.  The per-surfel part is
// taken once (ss_conic), the per-box part for each box.
struct ss_conic {
    float a, b, c, ga, gb, xs, ys, ia, ic, idet, rc2, A2, B2;
    bool pd;   // Q2 positive definite (else every box may be covered)
};
__device__ __forceinline__ ss_conic ss_conic_of(float4 P, float A2, float B2, float rc2) {
    ss_conic q;
    q.rc2 = rc2;
    q.A2 = A2;
    q.B2 = B2;
    q.a = P.x * P.x + P.z * P.z - rc2 * A2 * A2;
    q.b = P.x * P.y + P.z * P.w - rc2 * A2 * B2;
    q.c = P.y * P.y + P.w * P.w - rc2 * B2 * B2;
    const float det = q.a * q.c - q.b * q.b;
    q.pd = (q.a > 0.f) && (q.c > 0.f) && (det > 0.f);
    q.ga = rc2 * A2;
    q.gb = rc2 * B2;
    q.idet = 1.f / det;
    q.xs = (q.c * q.ga - q.b * q.gb) * q.idet;
    q.ys = (q.a * q.gb - q.b * q.ga) * q.idet;
    q.ia = 1.f / q.a;
    q.ic = 1.f / q.c;
    return q;
}
// the test's margin for a box whose offsets reach |dx| <= ex, |dy| <= ey
__device__ __forceinline__ float ss_box_margin(const ss_conic& q, float ex, float ey) {
    const float sc = 1.f + fabsf(q.A2) * ex + fabsf(q.B2) * ey;
    return 1e-5f * q.rc2 * sc * sc;
}
// bounding box of {f < t}: false when it misses [dx0, dx1] x [dy0, dy1]
__device__ __forceinline__ bool ss_conic_aabb_meets(const ss_conic& q, float t, float dx0, float dx1, float dy0,
                                                    float dy1) {
    const float kap = q.ga * q.xs + q.gb * q.ys + q.rc2 + t;   // -f(d_s) + t
    const float hx = sqrtf(fmaxf(kap * q.c * q.idet, 0.f)) * 1.0001f + 1e-4f;
    const float hy = sqrtf(fmaxf(kap * q.a * q.idet, 0.f)) * 1.0001f + 1e-4f;
    return !(q.xs + hx < dx0 || q.xs - hx > dx1 || q.ys + hy < dy0 || q.ys - hy > dy1);
}
__device__ __forceinline__ bool ss_conic_box_may_cover(const ss_conic& q, float dx0, float dx1, float dy0, float dy1) {
    if (!q.pd) return true;
    if (q.xs >= dx0 && q.xs <= dx1 && q.ys >= dy0 && q.ys <= dy1) return true;
    const float a = q.a, b = q.b, c = q.c, ga = q.ga, gb = q.gb, rc2 = q.rc2;
    auto f = [&](float x, float y) { return x * (a * x + 2.f * b * y - 2.f * ga) + y * (c * y - 2.f * gb) - rc2; };
    float m = f(dx0, fminf(fmaxf((gb - b * dx0) * q.ic, dy0), dy1));
    m = fminf(m, f(dx1, fminf(fmaxf((gb - b * dx1) * q.ic, dy0), dy1)));
    m = fminf(m, f(fminf(fmaxf((ga - b * dy0) * q.ia, dx0), dx1), dy0));
    m = fminf(m, f(fminf(fmaxf((ga - b * dy1) * q.ia, dx0), dx1), dy1));
    return !(m > ss_box_margin(q, fmaxf(fabsf(dx0), fabsf(dx1)), fmaxf(fabsf(dy0), fabsf(dy1))));   // NaN keeps it
}

__device__ __forceinline__ bool in_rect(uint32_t rx, uint32_t ry, int px, int py) {
    int i0 = rx & 0xffff, i1 = rx >> 16, j0 = ry & 0xffff, j1 = ry >> 16;
    return px >= i0 && px <= i1 && py >= j0 && py <= j1;
}

__device__ __forceinline__ int find_view_tile(const ss_layout* L, int tile) {
    int lo = 0, hi = L->n_views - 1;
    while (lo < hi) {
        int m = (lo + hi + 1) >> 1;
        if (L->v[m].tile_off <= tile) lo = m;
        else hi = m - 1;
    }
    return lo;
}
