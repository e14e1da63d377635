// Adaptive density control (Sec. 3.6.2; appendix on splitting and pruning
// surfels): the same-orientation neighbour statistics of a hashed uniform
// grid over the surfel centres, the per-surfel split / prune decision, and
// the compaction that writes the new surfel arrays.
//
// Index build (counting sort by hash slot): cell = floor(p / h) per axis,
// slot = hash(scene, cell) mod T (T a power of two >= 2 n), counts ->
// exclusive scan -> scatter of (position, scene) and (normal, index) rows
// into slot order, so a cell's candidates are contiguous.  Slots shared by
// several cells (hash collisions) are filtered by recomputing each
// candidate's cell.  A query (one thread per indexed surfel, in slot order so
// that a warp's queries touch neighbouring cells) visits rings of cells of
// Chebyshev radius r = 0, 1, ..., skipping cells whose box lies farther than
// its current k-th distance, and stops once the k-th same-orientation
// distance is within the radius the visited box covers.  The k squared
// distances are kept sorted in registers and summed in ascending order, so
// the result does not depend on the (atomic) order inside a slot.
//
// Everything here is a few passes over the surfels (tens of bytes each) plus
// the neighbour loop; it runs once per densification interval, not per step.
#include <math.h>

#include "ss3d_internal.cuh"

#define DN_THREADS 256
#define SCAN_THREADS 256
#define SCAN_PER_THREAD 8
#define SCAN_ITEMS (SCAN_THREADS * SCAN_PER_THREAD)

namespace {

struct dn_ws {
    int32_t* slot;     // [n] hash slot of each surfel, -1 when not indexed
    int32_t* start;    // [T + 1] counts, then exclusive prefix (first entry of each slot); total last
    int32_t* cursor;   // [T] scatter cursors
    float4* spos;      // [n] slot order: (x, y, z, scene as int bits)
    float4* snrm;      // [n] slot order: (n_x, n_y, n_z, surfel index as int bits)
    int64_t* bsum;     // scan block sums
    int64_t T;
    int64_t nb;        // capacity of bsum
};

int64_t table_size(int64_t n) {
    int64_t T = 1024;
    while (T < 2 * n) T <<= 1;
    return T;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t ws_bytes_for(int64_t n, dn_ws* w, char* base) {
    const int64_t T = table_size(n);
    const int64_t nb = (std::max(T + 1, n + 1) + SCAN_ITEMS - 1) / SCAN_ITEMS + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    char* slot = take(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1));
    char* start = take(sizeof(int32_t) * (size_t)(T + 1));
    char* cursor = take(sizeof(int32_t) * (size_t)T);
    char* spos = take(sizeof(float4) * (size_t)std::max<int64_t>(n, 1));
    char* snrm = take(sizeof(float4) * (size_t)std::max<int64_t>(n, 1));
    char* bsum = take(sizeof(int64_t) * (size_t)nb);
    if (w) {
        w->slot = reinterpret_cast<int32_t*>(slot);
        w->start = reinterpret_cast<int32_t*>(start);
        w->cursor = reinterpret_cast<int32_t*>(cursor);
        w->spos = reinterpret_cast<float4*>(spos);
        w->snrm = reinterpret_cast<float4*>(snrm);
        w->bsum = reinterpret_cast<int64_t*>(bsum);
        w->T = T;
        w->nb = nb;
    }
    return off;
}

// ------------------------------------------------------------------------
// exclusive scan of m values (int32 or int64 in) into int64 or int32 out,
// out[m] = total; in and out may be the same array (each CTA reads its
// range before writing it)

template <typename Tin>
__device__ __forceinline__ int64_t load_or0(const Tin* in, int64_t i, int64_t m) {
    return i < m ? (int64_t)in[i] : 0;
}

template <typename Tin>
__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_kernel(const Tin* __restrict__ in, int64_t m,
                                                                 int64_t* __restrict__ bsum) {
    __shared__ int64_t red[SCAN_THREADS / 32];
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_ITEMS;
    int64_t s = 0;
    for (int k = 0; k < SCAN_PER_THREAD; ++k) s += load_or0(in, b0 + k * SCAN_THREADS + threadIdx.x, m);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        bsum[blockIdx.x] = t;
    }
}

// one CTA: exclusive scan of nb block sums in place, the total at bsum[nb]
__global__ void __launch_bounds__(SCAN_THREADS) scan_top_kernel(int64_t* bsum, int64_t nb) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t b = 0; b < nb; b += SCAN_THREADS) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        int64_t before = carry;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        if (i < nb) bsum[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(SCAN_THREADS) scan_apply_kernel(const Tin* in, int64_t m,
                                                                  const int64_t* __restrict__ bsum, Tout* out) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_ITEMS + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    int64_t v[SCAN_PER_THREAD];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        v[k] = load_or0(in, b0 + k, m);
        s += v[k];
    }
    int64_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int64_t run = bsum[blockIdx.x] + x - s;
    for (int w = 0; w < wid; ++w) run += wsum[w];
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (b0 + k < m) out[b0 + k] = (Tout)run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[m] = (Tout)bsum[gridDim.x];
}

template <typename Tin, typename Tout>
void scan_exclusive(const Tin* in, int64_t m, Tout* out, int64_t* bsum, cudaStream_t st) {
    const int64_t nb = std::max<int64_t>((m + SCAN_ITEMS - 1) / SCAN_ITEMS, 1);
    ss_note_launch();
    scan_sums_kernel<Tin><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, m, bsum);
    ss_note_launch();
    scan_top_kernel<<<1, SCAN_THREADS, 0, st>>>(bsum, nb);
    ss_note_launch();
    scan_apply_kernel<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, m, bsum, out);
}

// ------------------------------------------------------------------------
// grid

struct dn_scenes {
    int64_t begin[SS_MAX_SCENES + 1];
    int n_scenes;
};

__device__ __forceinline__ int scene_of(const dn_scenes& S, int64_t i) {
    int lo = 0, hi = S.n_scenes - 1;
    while (lo < hi) {   // the last scene whose begin <= i
        const int mid = (lo + hi + 1) >> 1;
        if (S.begin[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

#define DN_CELL_LIMIT 1073741824.f   // 2^30: cell coordinates are clamped to +-2^30

__device__ __forceinline__ int cell_coord(float u) {
    return (int)floorf(fminf(fmaxf(u, -DN_CELL_LIMIT), DN_CELL_LIMIT));
}

__device__ __forceinline__ uint32_t cell_hash(int scene, int cx, int cy, int cz) {
    uint32_t h = (uint32_t)cx * 0x8da6b343u;
    h ^= (uint32_t)cy * 0xd8163841u;
    h ^= (uint32_t)cz * 0xcb1ab31fu;
    h ^= (uint32_t)scene * 0x9e3779b1u;
    h ^= h >> 15;
    h *= 0x2c1b3c6du;
    h ^= h >> 12;
    return h;
}

__device__ __forceinline__ float3 unit_normal(const float* q4) {
    float w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    const float inv = rsqrtf(fmaxf(w * w + x * x + y * y + z * z, 1e-30f));
    w *= inv;
    x *= inv;
    y *= inv;
    z *= inv;
    return make_float3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));   // R(q) e_z
}

struct dn_args {
    dn_scenes S;
    int64_t n;
    uint32_t mask;
    float inv_h, h, cos_min;
    int k, max_rings;
    const float* pos;
    const float* quat;
    dn_ws w;
    float* mean;
    float* nn;
    int32_t* flags;
};

__global__ void __launch_bounds__(DN_THREADS) dn_cells_kernel(const __grid_constant__ dn_args A) {
    const int64_t i = (int64_t)blockIdx.x * DN_THREADS + threadIdx.x;
    if (i >= A.n) return;
    const float px = A.pos[3 * i], py = A.pos[3 * i + 1], pz = A.pos[3 * i + 2];
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) {
        A.w.slot[i] = -1;
        A.mean[i] = nanf("");
        A.nn[i] = nanf("");
        A.flags[i] = SS_NB_NONFINITE;
        return;
    }
    const int s = scene_of(A.S, i);
    const uint32_t slot =
        cell_hash(s, cell_coord(px * A.inv_h), cell_coord(py * A.inv_h), cell_coord(pz * A.inv_h)) & A.mask;
    A.w.slot[i] = (int32_t)slot;
    atomicAdd(&A.w.start[slot], 1);
}

__global__ void __launch_bounds__(DN_THREADS) dn_scatter_kernel(const __grid_constant__ dn_args A) {
    const int64_t i = (int64_t)blockIdx.x * DN_THREADS + threadIdx.x;
    if (i >= A.n) return;
    const int32_t slot = A.w.slot[i];
    if (slot < 0) return;
    const int32_t j = atomicAdd(&A.w.cursor[slot], 1);
    const int s = scene_of(A.S, i);
    A.w.spos[j] = make_float4(A.pos[3 * i], A.pos[3 * i + 1], A.pos[3 * i + 2], __int_as_float(s));
    const float3 nr = unit_normal(A.quat + 4 * i);
    A.w.snrm[j] = make_float4(nr.x, nr.y, nr.z, __int_as_float((int)i));
}

// distance from the scaled query coordinate u (in cell c) to the cell c + d
// along one axis, in cell units (0 inside)
__device__ __forceinline__ float axis_gap(float u, int c, int d) {
    return d > 0 ? fmaxf((float)(c + d) - u, 0.f) : (d < 0 ? fmaxf(u - (float)(c + d + 1), 0.f) : 0.f);
}

// radius (cell units) the box of cells c - r .. c + r covers around u, less a
// margin for the rounding of the scaled coordinates
__device__ __forceinline__ float covered(float u, int c, int r) {
    const float g = fminf(u - (float)(c - r), (float)(c + r + 1) - u);
    return g - 2.4e-7f * (fabsf(u) + (float)r + 2.f);
}

__global__ void __launch_bounds__(DN_THREADS) dn_query_kernel(const __grid_constant__ dn_args A) {
    const int64_t j = (int64_t)blockIdx.x * DN_THREADS + threadIdx.x;
    const int32_t total = A.w.start[A.mask + 1];
    if (j >= total) return;
    const float4 P = A.w.spos[j];
    const float4 N = A.w.snrm[j];
    const int scene = __float_as_int(P.w);
    const int self = __float_as_int(N.w);
    const float ux = P.x * A.inv_h, uy = P.y * A.inv_h, uz = P.z * A.inv_h;
    const int cx = cell_coord(ux), cy = cell_coord(uy), cz = cell_coord(uz);
    const int K = A.k;
    float kd[SS_DENSITY_KMAX];
#pragma unroll
    for (int t = 0; t < SS_DENSITY_KMAX; ++t) kd[t] = INFINITY;
    int cnt = 0;
    float nn2 = INFINITY;
    const float h2 = A.h * A.h;
    float G = 0.f;
    for (int r = 0; r <= A.max_rings; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                const int step = face ? 1 : 2 * r;   // inner rows: only the two end cells are on the ring
                for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
                    const float gx = axis_gap(ux, cx, dx), gy = axis_gap(uy, cy, dy), gz = axis_gap(uz, cz, dz);
                    const float d2min = (gx * gx + gy * gy + gz * gz) * h2;
                    if (cnt == K && d2min > kd[K - 1]) continue;
                    const int ex = cx + dx, ey = cy + dy, ez = cz + dz;
                    const uint32_t slot = cell_hash(scene, ex, ey, ez) & A.mask;
                    const int32_t b = A.w.start[slot], e = A.w.start[slot + 1];
                    for (int32_t t = b; t < e; ++t) {
                        if (t == j) continue;
                        const float4 Q = A.w.spos[t];
                        if (__float_as_int(Q.w) != scene) continue;
                        if (cell_coord(Q.x * A.inv_h) != ex || cell_coord(Q.y * A.inv_h) != ey ||
                            cell_coord(Q.z * A.inv_h) != ez)
                            continue;   // another cell in the same slot
                        const float ddx = Q.x - P.x, ddy = Q.y - P.y, ddz = Q.z - P.z;
                        const float d2 = __fmaf_rn(ddx, ddx, __fmaf_rn(ddy, ddy, ddz * ddz));
                        nn2 = fminf(nn2, d2);
                        if (cnt == K && !(d2 < kd[K - 1])) continue;
                        const float4 M = A.w.snrm[t];
                        if (!(__fmaf_rn(N.x, M.x, __fmaf_rn(N.y, M.y, N.z * M.z)) >= A.cos_min)) continue;
                        // insert d2 into the sorted list kd[0 .. K)
                        float v = d2;
#pragma unroll
                        for (int u = 0; u < SS_DENSITY_KMAX; ++u) {
                            if (u < K && v < kd[u]) {
                                const float o = kd[u];
                                kd[u] = v;
                                v = o;
                            }
                        }
                        cnt = min(cnt + 1, K);
                    }
                }
            }
        }
        G = fmaxf(fminf(fminf(covered(ux, cx, r), covered(uy, cy, r)), covered(uz, cz, r)), 0.f) * A.h *
            (1.f - 1e-6f);
        if (cnt == K && kd[K - 1] <= G * G) break;
    }
    const float G2 = G * G;
    int flags = 0;
    float sum = 0.f;
    int certain = 0;
#pragma unroll
    for (int u = 0; u < SS_DENSITY_KMAX; ++u) {
        if (u < K && kd[u] <= G2) {
            sum += sqrtf(kd[u]);
            ++certain;
        }
    }
    float mean;
    if (certain == K) {
        mean = sum / (float)K;
    } else {
        flags |= SS_NB_MEAN_BOUND;
        mean = (sum + (float)(K - certain) * G) / (float)K;
    }
    float nn;
    if (nn2 <= G2) {
        nn = sqrtf(nn2);
    } else {
        flags |= SS_NB_NN_BOUND;
        nn = G;
    }
    A.mean[self] = mean;
    A.nn[self] = nn;
    A.flags[self] = flags;
}

// ------------------------------------------------------------------------
// plan, apply, compact

struct plan_args {
    const float* ls;
    const float* gnorm;
    const float* gviews;
    const float* mean;
    const float* nn;
    const int32_t* flags;
    int64_t n;
    float tau_g, r_cut;
    int ops;
    int32_t* action;
};

__global__ void __launch_bounds__(DN_THREADS) plan_kernel(const __grid_constant__ plan_args A) {
    const int64_t i = (int64_t)blockIdx.x * DN_THREADS + threadIdx.x;
    if (i >= A.n) return;
    const float smax = expf(fmaxf(A.ls[2 * i], A.ls[2 * i + 1]));
    const float norm = A.gnorm[i];
    int act = SS_ACTION_KEEP;
    if (A.ops & SS_DENSITY_SPLIT) {
        const float gbar = norm / A.gviews[i];
        if (gbar >= A.tau_g && !(A.flags[i] & SS_NB_MEAN_BOUND) && smax > A.mean[i]) act = SS_ACTION_SPLIT;
    }
    if ((A.ops & SS_DENSITY_PRUNE_ISOLATED) && A.nn[i] > A.r_cut * smax) act = SS_ACTION_PRUNE;
    if ((A.ops & SS_DENSITY_PRUNE_VISIBLE) && !(norm > 0.f)) act = SS_ACTION_PRUNE;
    A.action[i] = act;   // also the number of output rows
}

struct apply_args {
    ss_surfels in, out;
    int64_t n;
    const int32_t* action;
    const int64_t* off;
    float log_split;
};

__device__ __forceinline__ void copy_rest(const ss_surfels& in, const ss_surfels& out, int64_t i, int64_t o) {
    float* q = const_cast<float*>(out.quat) + 4 * o;
    float* al = const_cast<float*>(out.albedo) + 3 * o;
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = in.quat[4 * i + c];
#pragma unroll
    for (int c = 0; c < 3; ++c) al[c] = in.albedo[3 * i + c];
    const_cast<float*>(out.roughness)[o] = in.roughness[i];
    const_cast<float*>(out.metallic)[o] = in.metallic[i];
}

__global__ void __launch_bounds__(DN_THREADS) apply_kernel(const __grid_constant__ apply_args A) {
    const int64_t i = (int64_t)blockIdx.x * DN_THREADS + threadIdx.x;
    if (i >= A.n) return;
    const int act = A.action[i];
    if (act == SS_ACTION_PRUNE) return;
    const int64_t o = A.off[i];
    float* op = const_cast<float*>(A.out.pos);
    float* ol = const_cast<float*>(A.out.log_scale);
    const float px = A.in.pos[3 * i], py = A.in.pos[3 * i + 1], pz = A.in.pos[3 * i + 2];
    const float su = A.in.log_scale[2 * i], sv = A.in.log_scale[2 * i + 1];
    if (act == SS_ACTION_KEEP) {
        op[3 * o] = px;
        op[3 * o + 1] = py;
        op[3 * o + 2] = pz;
        ol[2 * o] = su;
        ol[2 * o + 1] = sv;
        copy_rest(A.in, A.out, i, o);
        return;
    }
    // split: the unit tangent of the larger scale (u on a tie), R(q) e_x or R(q) e_y
    float w = A.in.quat[4 * i], x = A.in.quat[4 * i + 1], y = A.in.quat[4 * i + 2], z = A.in.quat[4 * i + 3];
    const float inv = rsqrtf(fmaxf(w * w + x * x + y * y + z * z, 1e-30f));
    w *= inv;
    x *= inv;
    y *= inv;
    z *= inv;
    const bool use_u = su >= sv;
    float3 t;
    if (use_u) t = make_float3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
    else t = make_float3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
    const float half = 0.5f * expf(use_u ? su : sv);
    const float nu = use_u ? su + A.log_split : su, nv = use_u ? sv : sv + A.log_split;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float sg = c == 0 ? half : -half;
        const int64_t oc = o + c;
        op[3 * oc] = __fmaf_rn(sg, t.x, px);
        op[3 * oc + 1] = __fmaf_rn(sg, t.y, py);
        op[3 * oc + 2] = __fmaf_rn(sg, t.z, pz);
        ol[2 * oc] = nu;
        ol[2 * oc + 1] = nv;
        copy_rest(A.in, A.out, i, oc);
    }
}

__global__ void __launch_bounds__(DN_THREADS) compact_kernel(const float* __restrict__ in, int width, int64_t n,
                                                             const int32_t* __restrict__ action,
                                                             const int64_t* __restrict__ off, int zero_children,
                                                             float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * DN_THREADS + threadIdx.x;
    if (e >= n * width) return;
    const int64_t i = e / width;
    const int c = (int)(e - i * width);
    const int act = action[i];
    if (act == SS_ACTION_PRUNE) return;
    const float v = in[e];
    const int64_t o = off[i];
    if (act == SS_ACTION_KEEP) {
        out[o * width + c] = v;
    } else {
        const float cv = zero_children ? 0.f : v;
        out[o * width + c] = cv;
        out[(o + 1) * width + c] = cv;
    }
}

bool params_ok(const ss_density_params* p) {
    return p && p->k >= 1 && p->k <= SS_DENSITY_KMAX && isfinite(p->cos_min) && isfinite(p->cell) &&
           p->cell > 0.f && p->max_rings >= 1 && p->max_rings <= SS_DENSITY_MAX_RINGS && isfinite(p->tau_g) &&
           isfinite(p->r_cut) && p->r_cut > 0.f && p->split_scale > 0.f && p->split_scale <= 1.f &&
           (p->ops & ~7) == 0;
}

unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>((n + DN_THREADS - 1) / DN_THREADS, 1); }

}  // namespace

extern "C" void ss_default_density(ss_density_params* p) {
    if (!p) return;
    p->k = 8;
    p->cos_min = 0.5f;
    p->cell = 0.f;
    p->max_rings = 4;
    p->tau_g = 2e-4f;
    p->r_cut = 3.f;
    p->split_scale = 0.7f;
    p->ops = SS_DENSITY_SPLIT | SS_DENSITY_PRUNE_VISIBLE | SS_DENSITY_PRUNE_ISOLATED;
}

extern "C" ss_status ss_density_workspace_size(int64_t n, size_t* bytes) {
    if (n < 0 || n > ((int64_t)1 << 30) || !bytes) return SS_ERR_INVALID_ARG;
    *bytes = ws_bytes_for(n, nullptr, nullptr);
    return SS_OK;
}

extern "C" ss_status ss_density_neighbours(const ss_surfels* s, const int64_t* scene_offsets_host, int32_t n_scenes,
                                           const ss_density_params* p, float* mean_dist_dev, float* nn_dist_dev,
                                           int32_t* flags_dev, void* ws, size_t ws_bytes, void* stream) {
    if (!s || !scene_offsets_host || n_scenes < 1 || n_scenes > SS_MAX_SCENES || !params_ok(p))
        return SS_ERR_INVALID_ARG;
    dn_args A{};
    A.S.n_scenes = n_scenes;
    if (scene_offsets_host[0] != 0) return SS_ERR_INVALID_ARG;
    for (int i = 0; i <= n_scenes; ++i) {
        if (i > 0 && scene_offsets_host[i] < scene_offsets_host[i - 1]) return SS_ERR_INVALID_ARG;
        A.S.begin[i] = scene_offsets_host[i];
    }
    for (int i = n_scenes + 1; i <= SS_MAX_SCENES; ++i) A.S.begin[i] = scene_offsets_host[n_scenes];
    const int64_t n = scene_offsets_host[n_scenes];
    if (n > ((int64_t)1 << 30)) return SS_ERR_INVALID_ARG;
    if (n == 0) return SS_OK;
    if (!s->pos || !s->quat || !mean_dist_dev || !nn_dist_dev || !flags_dev || !ws) return SS_ERR_INVALID_ARG;
    if (ws_bytes < ws_bytes_for(n, nullptr, nullptr)) return SS_ERR_WORKSPACE;
    ws_bytes_for(n, &A.w, static_cast<char*>(ws));
    A.n = n;
    A.mask = (uint32_t)(A.w.T - 1);
    A.inv_h = 1.f / p->cell;
    A.h = p->cell;
    A.cos_min = p->cos_min;
    A.k = p->k;
    A.max_rings = p->max_rings;
    A.pos = s->pos;
    A.quat = s->quat;
    A.mean = mean_dist_dev;
    A.nn = nn_dist_dev;
    A.flags = flags_dev;
    cudaStream_t st = (cudaStream_t)stream;
    ss_stage_scope scope(7, st);
    if (cudaMemsetAsync(A.w.start, 0, sizeof(int32_t) * (size_t)(A.w.T + 1), st) != cudaSuccess) return SS_ERR_CUDA;
    ss_note_launch();
    dn_cells_kernel<<<blocks_for(n), DN_THREADS, 0, st>>>(A);
    scan_exclusive<int32_t, int32_t>(A.w.start, A.w.T, A.w.start, A.w.bsum, st);
    if (cudaMemcpyAsync(A.w.cursor, A.w.start, sizeof(int32_t) * (size_t)A.w.T, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return SS_ERR_CUDA;
    ss_note_launch();
    dn_scatter_kernel<<<blocks_for(n), DN_THREADS, 0, st>>>(A);
    ss_note_launch();
    dn_query_kernel<<<blocks_for(n), DN_THREADS, 0, st>>>(A);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}

extern "C" ss_status ss_density_plan(const float* log_scale_dev, const float* screen_grad_norm_dev,
                                     const float* screen_grad_views_dev, const float* mean_dist_dev,
                                     const float* nn_dist_dev, const int32_t* flags_dev, int64_t n,
                                     const ss_density_params* p, int32_t* action_dev, int64_t* out_offset_dev,
                                     void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || n > ((int64_t)1 << 30) || !params_ok(p) || !out_offset_dev || !ws) return SS_ERR_INVALID_ARG;
    if (n > 0 && (!log_scale_dev || !screen_grad_norm_dev || !screen_grad_views_dev || !mean_dist_dev ||
                  !nn_dist_dev || !flags_dev || !action_dev))
        return SS_ERR_INVALID_ARG;
    dn_ws w;
    if (ws_bytes < ws_bytes_for(n, nullptr, nullptr)) return SS_ERR_WORKSPACE;
    ws_bytes_for(n, &w, static_cast<char*>(ws));
    cudaStream_t st = (cudaStream_t)stream;
    ss_stage_scope scope(7, st);
    plan_args A{log_scale_dev, screen_grad_norm_dev, screen_grad_views_dev, mean_dist_dev, nn_dist_dev, flags_dev,
                n, p->tau_g, p->r_cut, p->ops, action_dev};
    if (n > 0) {
        ss_note_launch();
        plan_kernel<<<blocks_for(n), DN_THREADS, 0, st>>>(A);
    }
    scan_exclusive<int32_t, int64_t>(action_dev, n, out_offset_dev, w.bsum, st);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}

extern "C" ss_status ss_density_apply(const ss_surfels* in, int64_t n, const int32_t* action_dev,
                                      const int64_t* out_offset_dev, float split_scale, const ss_surfels* out,
                                      void* stream) {
    if (!in || !out || n < 0 || !(split_scale > 0.f && split_scale <= 1.f)) return SS_ERR_INVALID_ARG;
    if (n == 0) return SS_OK;
    if (!action_dev || !out_offset_dev) return SS_ERR_INVALID_ARG;
    const float* ptrs[12] = {in->pos,  in->quat,  in->log_scale,  in->albedo,  in->roughness,  in->metallic,
                             out->pos, out->quat, out->log_scale, out->albedo, out->roughness, out->metallic};
    for (const float* q : ptrs)
        if (!q) return SS_ERR_INVALID_ARG;
    apply_args A{*in, *out, n, action_dev, out_offset_dev, (float)std::log((double)split_scale)};
    cudaStream_t st = (cudaStream_t)stream;
    ss_stage_scope scope(7, st);
    ss_note_launch();
    apply_kernel<<<blocks_for(n), DN_THREADS, 0, st>>>(A);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}

extern "C" ss_status ss_density_compact(const float* in_dev, int32_t width, int64_t n, const int32_t* action_dev,
                                        const int64_t* out_offset_dev, int32_t zero_children, float* out_dev,
                                        void* stream) {
    if (n < 0 || width < 1 || width > 64 || (zero_children != 0 && zero_children != 1)) return SS_ERR_INVALID_ARG;
    if (n == 0) return SS_OK;
    if (!in_dev || !action_dev || !out_offset_dev || !out_dev) return SS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ss_stage_scope scope(7, st);
    ss_note_launch();
    compact_kernel<<<blocks_for(n * width), DN_THREADS, 0, st>>>(in_dev, width, n, action_dev, out_offset_dev,
                                                                  zero_children, out_dev);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}
