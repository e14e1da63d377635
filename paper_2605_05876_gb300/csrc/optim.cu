// Fused Adam step over all parameter groups (section "Training and
// Optimization"; Kingma & Ba 2014, Algorithm 1) and the L1 photometric loss
// (l1 term of Eq. photo_loss).
//
// Both are HBM-bound streams: Adam reads theta, g, m, v and writes theta, m,
// v and the activated copy (28-32 bytes per element).  One launch covers
// every group: the host assigns each CTA a contiguous range of one group's
// elements (float4 where the range allows), so no CTA searches for its group.
#include <math.h>
#include <string.h>

#include "ss3d_internal.cuh"

#define ADAM_THREADS 256
#define ADAM_ELEMS (ADAM_THREADS * 4 * 4)   // elements per CTA: 4 float4 per thread

struct adam_launch {
    ss_adam_group g[SS_MAX_ADAM_GROUPS];
    int64_t block_off[SS_MAX_ADAM_GROUPS + 1];   // first CTA of each group
    int n_groups;
    float beta1, beta2, eps, inv_bc1, inv_bc2;
};

__device__ __forceinline__ float adam_one(float& th, float g, float& m, float& v, const adam_launch& A, float lr,
                                          int act) {
    if (act == SS_ACT_SIGMOID) {
        const float a = 1.f / (1.f + __expf(-th));   // the activated value the gradient refers to
        g *= a * (1.f - a);
    }
    m = fmaf(A.beta1, m, (1.f - A.beta1) * g);
    v = fmaf(A.beta2, v, (1.f - A.beta2) * g * g);
    const float mh = m * A.inv_bc1, vh = v * A.inv_bc2;
    th -= lr * mh / (sqrtf(vh) + A.eps);
    if (act == SS_ACT_CLAMP0) th = fmaxf(th, 0.f);
    return act == SS_ACT_SIGMOID ? 1.f / (1.f + __expf(-th)) : th;
}

__global__ void __launch_bounds__(ADAM_THREADS) adam_kernel(const __grid_constant__ adam_launch A) {
    int gi = 0;
    while (gi + 1 < A.n_groups && (int64_t)blockIdx.x >= A.block_off[gi + 1]) ++gi;
    const ss_adam_group& G = A.g[gi];
    const int64_t b0 = ((int64_t)blockIdx.x - A.block_off[gi]) * ADAM_ELEMS;
    const int64_t b1 = min(b0 + (int64_t)ADAM_ELEMS, G.n);
    const bool vec = ((reinterpret_cast<uintptr_t>(G.param_dev) | reinterpret_cast<uintptr_t>(G.grad_dev) |
                       reinterpret_cast<uintptr_t>(G.m_dev) | reinterpret_cast<uintptr_t>(G.v_dev) |
                       reinterpret_cast<uintptr_t>(G.act_dev)) & 15) == 0;
    if (vec) {
        // whole float4 groups of the range (b0 is a multiple of 4)
        const int64_t n4 = (b1 - b0) / 4;
        for (int64_t k = threadIdx.x; k < n4; k += ADAM_THREADS) {
            const int64_t e = b0 + 4 * k;
            float4 th = *reinterpret_cast<const float4*>(G.param_dev + e);
            const float4 g = __ldg(reinterpret_cast<const float4*>(G.grad_dev + e));
            float4 m = *reinterpret_cast<const float4*>(G.m_dev + e);
            float4 v = *reinterpret_cast<const float4*>(G.v_dev + e);
            float4 a;
            a.x = adam_one(th.x, g.x, m.x, v.x, A, G.lr, G.activation);
            a.y = adam_one(th.y, g.y, m.y, v.y, A, G.lr, G.activation);
            a.z = adam_one(th.z, g.z, m.z, v.z, A, G.lr, G.activation);
            a.w = adam_one(th.w, g.w, m.w, v.w, A, G.lr, G.activation);
            *reinterpret_cast<float4*>(G.param_dev + e) = th;
            *reinterpret_cast<float4*>(G.m_dev + e) = m;
            *reinterpret_cast<float4*>(G.v_dev + e) = v;
            if (G.act_dev) *reinterpret_cast<float4*>(G.act_dev + e) = a;
        }
        for (int64_t e = b0 + 4 * n4 + threadIdx.x; e < b1; e += ADAM_THREADS) {   // tail of the group
            float th = G.param_dev[e], m = G.m_dev[e], v = G.v_dev[e];
            const float a = adam_one(th, G.grad_dev[e], m, v, A, G.lr, G.activation);
            G.param_dev[e] = th;
            G.m_dev[e] = m;
            G.v_dev[e] = v;
            if (G.act_dev) G.act_dev[e] = a;
        }
    } else {
        for (int64_t e = b0 + threadIdx.x; e < b1; e += ADAM_THREADS) {
            float th = G.param_dev[e], m = G.m_dev[e], v = G.v_dev[e];
            const float a = adam_one(th, G.grad_dev[e], m, v, A, G.lr, G.activation);
            G.param_dev[e] = th;
            G.m_dev[e] = m;
            G.v_dev[e] = v;
            if (G.act_dev) G.act_dev[e] = a;
        }
    }
}

extern "C" void ss_default_adam(ss_adam_params* p) {
    if (!p) return;
    p->beta1 = 0.9f;
    p->beta2 = 0.999f;
    p->eps = 1e-8f;
    p->step = 1;
}

extern "C" ss_status ss_adam_step(const ss_adam_group* groups, int32_t n_groups, const ss_adam_params* p,
                                  void* stream) {
    if (!groups || !p || n_groups < 1 || n_groups > SS_MAX_ADAM_GROUPS || p->step < 1) return SS_ERR_INVALID_ARG;
    if (!(p->beta1 >= 0.f && p->beta1 < 1.f && p->beta2 >= 0.f && p->beta2 < 1.f && p->eps >= 0.f))
        return SS_ERR_INVALID_ARG;
    adam_launch A;
    memset(&A, 0, sizeof(A));
    A.n_groups = n_groups;
    A.beta1 = p->beta1;
    A.beta2 = p->beta2;
    A.eps = p->eps;
    // bias corrections in double on the host
    A.inv_bc1 = (float)(1.0 / (1.0 - pow((double)p->beta1, (double)p->step)));
    A.inv_bc2 = (float)(1.0 / (1.0 - pow((double)p->beta2, (double)p->step)));
    int64_t blocks = 0;
    for (int i = 0; i < n_groups; ++i) {
        const ss_adam_group& g = groups[i];
        if (g.n < 0 || g.activation < SS_ACT_IDENTITY || g.activation > SS_ACT_CLAMP0) return SS_ERR_INVALID_ARG;
        if (g.n > 0 && (!g.param_dev || !g.grad_dev || !g.m_dev || !g.v_dev)) return SS_ERR_INVALID_ARG;
        A.g[i] = g;
        A.block_off[i] = blocks;
        blocks += (g.n + ADAM_ELEMS - 1) / ADAM_ELEMS;
    }
    A.block_off[n_groups] = blocks;
    if (blocks == 0) return SS_OK;
    if (blocks > 0x7fffffff) return SS_ERR_INVALID_ARG;
    ss_note_launch();
    adam_kernel<<<(unsigned)blocks, ADAM_THREADS, 0, (cudaStream_t)stream>>>(A);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}

// ------------------------------------------------------------------------
// L1 loss: per CTA a partial sum (FP32 runs of 64 terms, FP64 across them),
// combined by the last CTA to finish in CTA order, so the loss is
// deterministic.  The partials live in a fixed device array (no allocation);
// calls on one device therefore must not overlap.

#define L1_THREADS 256
#define L1_MAX_BLOCKS 1216   // 8 CTAs per SM on 152 SMs

static __device__ double g_l1_partial[L1_MAX_BLOCKS];
static __device__ unsigned g_l1_counter;

__global__ void __launch_bounds__(L1_THREADS) l1_kernel(const float* __restrict__ out,
                                                       const float* __restrict__ target, int64_t n, float scale,
                                                       float* d_out, float* loss) {
    __shared__ double red[L1_THREADS / 32];
    __shared__ bool last;
    double acc = 0.0;
    float facc = 0.f;
    int cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)L1_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * L1_THREADS) {
        const float d = out[i] - target[i];
        d_out[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        facc += fabsf(d);
        if (++cnt == 64) {
            acc += (double)facc;
            facc = 0.f;
            cnt = 0;
        }
    }
    acc += (double)facc;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < L1_THREADS / 32; ++w) s += red[w];
        g_l1_partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&g_l1_counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile double*)g_l1_partial)[b];
        *loss = (float)(s * scale);
        g_l1_counter = 0;   // ready for the next call
    }
}

extern "C" ss_status ss_loss_l1(const float* out_dev, const float* target_dev, int64_t n, float scale,
                                float* d_out_dev, float* loss_dev, void* stream) {
    if (!out_dev || !target_dev || !d_out_dev || !loss_dev || n < 0) return SS_ERR_INVALID_ARG;
    int64_t blocks = (n + L1_THREADS * 8 - 1) / (L1_THREADS * 8);
    if (blocks < 1) blocks = 1;
    if (blocks > L1_MAX_BLOCKS) blocks = L1_MAX_BLOCKS;
    ss_note_launch();
    l1_kernel<<<(unsigned)blocks, L1_THREADS, 0, (cudaStream_t)stream>>>(out_dev, target_dev, n, scale, d_out_dev,
                                                                         loss_dev);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}

// ------------------------------------------------------------------------
// Silhouette loss (Eq. sil_loss): the soft intersection-over-union loss
// between the rendered coverage A = 1 - T_{K+1} (the alpha channel of the
// RGBA output) and a mask M in [0, 1], per view:
//   I = sum A M,  U = sum (A + M - A M),  loss_v = scale (1 - I / U),
//   dloss_v/dA = -scale (M U - I (1 - M)) / U^2   (added to d_rgba's alpha).
// One CTA per view: the two sums in FP64 in a fixed order (each thread its
// strided pixels, then the warps and the CTA in order), so the loss is
// deterministic; no scratch memory.

#define SIL_THREADS 1024

__global__ void __launch_bounds__(SIL_THREADS) sil_iou_kernel(const float4* __restrict__ rgba,
                                                             const float* __restrict__ mask,
                                                             const int64_t* __restrict__ offsets, float scale,
                                                             float* d_rgba, float* loss) {
    __shared__ double red_i[SIL_THREADS / 32], red_u[SIL_THREADS / 32];
    __shared__ double tot[2];
    const int v = blockIdx.x;
    const int64_t b = offsets[v], e = offsets[v + 1];
    double si = 0.0, su = 0.0;
    for (int64_t p = b + threadIdx.x; p < e; p += SIL_THREADS) {
        const double A = rgba[p].w, M = mask[p];
        si += A * M;
        su += A + M - A * M;
    }
    for (int o = 16; o > 0; o >>= 1) {
        si += __shfl_xor_sync(0xffffffffu, si, o);
        su += __shfl_xor_sync(0xffffffffu, su, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_i[threadIdx.x >> 5] = si;
        red_u[threadIdx.x >> 5] = su;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double I = 0.0, U = 0.0;
        for (int w = 0; w < SIL_THREADS / 32; ++w) {
            I += red_i[w];
            U += red_u[w];
        }
        tot[0] = I;
        tot[1] = U;
        loss[v] = U > 0.0 ? (float)(scale * (1.0 - I / U)) : 0.f;
    }
    __syncthreads();
    const double I = tot[0], U = tot[1];
    if (!(U > 0.0)) return;   // empty coverage and mask: no gradient
    const double k = -(double)scale / (U * U);
    for (int64_t p = b + threadIdx.x; p < e; p += SIL_THREADS) {
        const double M = mask[p];
        d_rgba[p * 4 + 3] += (float)(k * (M * U - I * (1.0 - M)));
    }
}

extern "C" ss_status ss_loss_sil_iou(const float* rgba_dev, const float* mask_dev, const int64_t* view_offsets_dev,
                                     int32_t n_views, float scale, float* d_rgba_dev, float* loss_dev, void* stream) {
    if (!rgba_dev || !mask_dev || !view_offsets_dev || !d_rgba_dev || !loss_dev || n_views < 1 ||
        n_views > 65535)
        return SS_ERR_INVALID_ARG;
    if (((uintptr_t)rgba_dev & 15) || ((uintptr_t)view_offsets_dev & 7)) return SS_ERR_INVALID_ARG;
    ss_note_launch();
    sil_iou_kernel<<<(unsigned)n_views, SIL_THREADS, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(rgba_dev), mask_dev, view_offsets_dev, scale, d_rgba_dev, loss_dev);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}
