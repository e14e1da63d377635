// Deterministic backward (ss_render_params.deterministic = 1), and the
// multi-block prefix sum it shares with the rasterisers' block lists.
//
// The default backward adds every run of fragment gradients into its
// (surfel, view) record with FP32 atomics, whose order -- and so the last
// bits of the sums -- depends on the scheduling.  In this mode the backward
// raster writes each (warp block, covering staged surfel) pair's sum to a row
// of its own, at a position fixed by the forward's lists (the pair's index in
// its block's list plus the prefix sum of the blocks' list lengths); then
// every record gathers its rows, orders them by row index and adds them in
// that order.  The environment-texel gradients of the projection adjoint are
// summed as 64-bit fixed-point integers, which are exact and independent of
// the order (render_bwd.cu), with a scale bounded here from the records.
#include <stdint.h>

#include "ss3d_internal.cuh"

#define DSCAN_T 1024                 // threads of the prefix-sum kernels
#define DSCAN_PER 4                  // elements per thread
#define DSCAN_B (DSCAN_T * DSCAN_PER)   // elements per block

int64_t ss_det_scan_blocks(int64_t n) { return (n + DSCAN_B - 1) / DSCAN_B; }

// block-wide exclusive scan of one 64-bit value per thread; returns the
// thread's exclusive prefix and writes the block total to *total
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* wsum,
                                                              unsigned long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < nw ? wsum[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;   // inclusive over warps
    }
    __syncthreads();
    const unsigned long long excl = (w > 0 ? wsum[w - 1] : 0ull) + x - v;
    *total = wsum[nw - 1];
    __syncthreads();   // wsum is reused by the caller's next scan
    return excl;
}

// sum of each block's DSCAN_B counts
__global__ void __launch_bounds__(DSCAN_T) scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                              unsigned long long* __restrict__ bsum) {
    __shared__ unsigned long long wsum[32];
    const int64_t i0 = (int64_t)blockIdx.x * DSCAN_B + (int64_t)threadIdx.x * DSCAN_PER;
    unsigned long long v = 0;
#pragma unroll
    for (int k = 0; k < DSCAN_PER; ++k) v += i0 + k < n ? in[i0 + k] : 0u;
    unsigned long long tot = 0;
    block_excl_scan(v, wsum, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// exclusive scan of the block sums in place (one CTA); bsum[nb] = the total
__global__ void __launch_bounds__(DSCAN_T) scan_bsum_kernel(unsigned long long* bsum, int64_t nb) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += DSCAN_T) {
        const int64_t i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? bsum[i] : 0ull;
        unsigned long long tot = 0;
        const unsigned long long ex = block_excl_scan(v, wsum, &tot);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

// out[i] = sum of in[0 .. i) (out[n] = the total), clamped to 32 bits; a
// total above cap sets SS_ERR_CAPACITY
__global__ void __launch_bounds__(DSCAN_T) scan_apply_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                             const unsigned long long* __restrict__ bsum, int64_t nb,
                                                             uint32_t* __restrict__ out, unsigned long long cap,
                                                             int* status, unsigned long long* total_out) {
    __shared__ unsigned long long wsum[32];
    const int64_t i0 = (int64_t)blockIdx.x * DSCAN_B + (int64_t)threadIdx.x * DSCAN_PER;
    uint32_t x[DSCAN_PER];
    unsigned long long v = 0;
#pragma unroll
    for (int k = 0; k < DSCAN_PER; ++k) {
        x[k] = i0 + k < n ? in[i0 + k] : 0u;
        v += x[k];
    }
    unsigned long long tot = 0;
    unsigned long long run = bsum[blockIdx.x] + block_excl_scan(v, wsum, &tot);
#pragma unroll
    for (int k = 0; k < DSCAN_PER; ++k) {
        if (i0 + k < n) out[i0 + k] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
        run += x[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long t = bsum[nb];
        out[n] = (uint32_t)(t < 0xffffffffull ? t : 0xffffffffull);
        if (t > cap) atomicOr(status, SS_ERR_CAPACITY);
        if (total_out) *total_out = t;
    }
}

void ss_launch_scan_u32(const uint32_t* in, int64_t n, uint32_t* out, unsigned long long* bsum, unsigned long long cap,
                        int* status, unsigned long long* total_out, cudaStream_t st) {
    const int64_t nb = ss_det_scan_blocks(n);
    if (nb > 0) {
        ss_note_launch();
        scan_reduce_kernel<<<(unsigned)nb, DSCAN_T, 0, st>>>(in, n, bsum);
    }
    ss_note_launch();
    scan_bsum_kernel<<<1, DSCAN_T, 0, st>>>(bsum, nb);
    ss_note_launch();
    scan_apply_kernel<<<(unsigned)(nb > 0 ? nb : 1), DSCAN_T, 0, st>>>(in, n, bsum, nb, out, cap, status, total_out);
}

// covering entries of each (tile, block) item, as the forward left them
__global__ void det_item_count_kernel(const uint32_t* __restrict__ cover_count, int64_t items, int bpt,
                                      uint32_t* __restrict__ icnt) {
    const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (it >= items) return;
    const int64_t tile = it / bpt, b = it - tile * bpt;
    icnt[it] = cover_count[tile * 8 + b];
}

void ss_launch_det_item_offsets(const ss_ws_view& ws, const ss_layout& L, cudaStream_t st) {
    const int64_t items = (int64_t)L.total_tiles * L.bpt;
    if (items > 0) {
        ss_note_launch();
        det_item_count_kernel<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(ws.cover_count, items, L.bpt,
                                                                                ws.det_icnt);
    }
    ss_launch_scan_u32(ws.det_icnt, items, ws.det_coff, ws.det_scan, (unsigned long long)ws.det_cap, ws.status, nullptr,
                       st);
}

// the rows in use: rows [0, min(total, cap)), total = det_coff[items]
__device__ __forceinline__ int64_t det_rows_used(const ss_ws_view& ws, int64_t items) {
    const int64_t t = ws.det_coff[items];
    return t < ws.det_cap ? t : ws.det_cap;
}

__global__ void det_count_kernel(ss_ws_view ws, int64_t items) {
    const int64_t n = det_rows_used(ws, items);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t rec = ws.det_rid[r];
        if (rec != 0xffffffffu) atomicAdd(ws.det_rcnt + rec, 1u);
    }
}

__global__ void det_fill_kernel(ss_ws_view ws, int64_t items) {
    const int64_t n = det_rows_used(ws, items);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t rec = ws.det_rid[r];
        if (rec != 0xffffffffu) ws.det_rlist[ws.det_roff[rec] + atomicAdd(ws.det_rcur + rec, 1u)] = (uint32_t)r;
    }
}

// One thread per record: its rows in ascending row order (the fill order
// is the scheduler's; the row indices are fixed), summed in that order.
__global__ void __launch_bounds__(256) det_sum_kernel(ss_ws_view ws, int64_t records, int nv, int ssg) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= records) return;
    const uint32_t b = ws.det_roff[r], e = ws.det_roff[r + 1];
    if (e <= b) return;
    uint32_t* lst = ws.det_rlist + b;
    const int n = (int)(e - b);
    // Shell sort with the 3h + 1 gaps (insertion sort for the short lists
    // that are the rule: a record meets a few blocks)
    int h = 1;
    while (h < n / 3) h = 3 * h + 1;
    for (; h >= 1; h /= 3)
        for (int i = h; i < n; ++i) {
            const uint32_t v = lst[i];
            int j = i;
            while (j >= h && lst[j - h] > v) {
                lst[j] = lst[j - h];
                j -= h;
            }
            lst[j] = v;
        }
    float acc[SS_NGRAD];
#pragma unroll
    for (int c = 0; c < SS_NGRAD; ++c) acc[c] = 0.f;
    for (int i = 0; i < n; ++i) {
        const float4* row = reinterpret_cast<const float4*>(ws.det_rows + (int64_t)lst[i] * SS_NGRAD);
#pragma unroll
        for (int q = 0; q < SS_NGRAD / 4; ++q) {
            const float4 x = row[q];
            acc[4 * q] += x.x; acc[4 * q + 1] += x.y; acc[4 * q + 2] += x.z; acc[4 * q + 3] += x.w;
        }
    }
    float* g = ws.grad_rec + r * SS_NGRAD;
#pragma unroll
    for (int c = 0; c < SS_NGRAD; ++c)
        if (c < nv || (ssg && (c == 21 || c == 22))) g[c] = acc[c];   // the columns the raster wrote
}

void ss_launch_det_record_sums(const ss_ws_view& ws, const ss_layout& L, int nv, bool ssg, cudaStream_t st) {
    const int64_t items = (int64_t)L.total_tiles * L.bpt, R = L.total_records;
    if (R <= 0) return;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms > 0 ? 8 * sms : 1024);
    ss_note_launch();
    det_count_kernel<<<grid, 256, 0, st>>>(ws, items);
    ss_launch_scan_u32(ws.det_rcnt, R, ws.det_roff, ws.det_scan, 0xffffffffull, ws.status, nullptr, st);
    ss_note_launch();
    det_fill_kernel<<<grid, 256, 0, st>>>(ws, items);
    ss_note_launch();
    det_sum_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(ws, R, nv, ssg ? 1 : 0);
}

// the largest |dL/d rgb| of a record (the bound of the fixed-point scale);
// a non-finite one sets SS_ERR_NONFINITE
__global__ void __launch_bounds__(256) det_env_bound_kernel(ss_ws_view ws, int64_t records) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float m = 0.f;
    bool bad = false;
    if (r < records) {
        const float* g = ws.grad_rec + r * SS_NGRAD + SS_GREC_RGB;   // dL/d rgb
        for (int c = 0; c < 3; ++c) {
            const float v = fabsf(g[c]);
            bad |= !(v <= 3.0e38f);
            m = fmaxf(m, bad ? 0.f : v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(ws.det_maxbits, __float_as_uint(m));
    if (bad) atomicOr(ws.status, SS_ERR_NONFINITE);
}

void ss_launch_det_env_bound(const ss_ws_view& ws, const ss_layout& L, cudaStream_t st) {
    if (L.total_records <= 0) return;
    ss_note_launch();
    det_env_bound_kernel<<<(unsigned)((L.total_records + 255) / 256), 256, 0, st>>>(ws, L.total_records);
}
