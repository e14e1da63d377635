// Backward render (App. A "Backward Pass Implementation of Multi-Layer
// Compositing"): the rasteriser replays each pixel's grouping front to back
// against the per-layer totals (C_k, W_k) kept by the forward pass, turns the
// upstream gradient into per-fragment gradients, sums them per surfel and
// adds one record of 21 floats per (surfel, view); a second kernel then
// chains those records back through the projection and the shading to the
// surfel parameters and the prefiltered environment texels.
//
// Every discrete decision (support, cutoff, grouping, K_max, normal flip) is
// held fixed: the forward pass writes, per (warp, staged surfel), the pixels
// it covers and the pixels where it opens a new layer, and the backward
// re-evaluates each fragment's weight with the same ss_pixel_test and weight
// expression as the forward kernel.
#include <math.h>

#include "ss3d_internal.cuh"
#include "raster_common.cuh"

// gradient record layout (floats) of one (view, surfel)
#define G_P 0      // dL/dP00, P01, P10, P11
#define G_A2 4
#define G_B2 5
#define G_PX 6     // dL/dp_x, dL/dp_y (surfel centre in pixels)
#define G_PY 7
#define G_NF 8
#define G_CH 9     // 12 channels: rgb, albedo 3, roughness, metallic, normal 3, depth
#define G_N 21
#define G_SSN 21   // densification statistic: sum of the fragments' |(g_x, g_y)| (Eq. ss_grad)
#define G_SSC 22   // ... and their number

// Backward rasteriser, per warp (8 x 4 pixels): the forward pass left a
// coverage word and a layer-opening word per (warp, staged surfel).  A chunk
// of 32 staged surfels is cut at the surfels that open a new layer at a live
// pixel; between two cuts every pixel stays in its layer, so the fragments of
// the slots in between are numbered in list order (a prefix sum of the slots'
// live coverage counts) and differentiated 32 at a time, one per lane: lane f
// finds its slot from the slot starts that fall inside its batch (a binary
// search over the prefix sums when an empty slot lies in between) and its
// pixel as the j-th set bit of that slot's word, writes its 22 values to column f of a
// 22 x 32 table; lane q then loads row q into registers and sums it over each
// run of columns of the same surfel (runs are contiguous), with one atomic add
// per value and run.  At a cut the opening pixels enter their next layer.
#define GCOL 36     // table row stride: 16-byte aligned rows, conflict-free column writes
#define GT 13       // floats per pixel lane in the layer-coefficient table: G_k (12), S_k

// ROWS table rows: G_N, or G_N + 2 with the densification statistic; GTR
// layer coefficients per pixel lane: GT, or GT + 3 with the consolidation term
template <int ROWS, int GTR>
struct ss_bwarp_t {
    float tab[ROWS * GCOL];
    float gtab[32 * GTR];
};

// Position of the j-th (0-based) set bit of m, for j < popc(m): the byte
// from the population counts of the low bytes, then the table of set-bit
// positions within a byte (nth8[byte * 8 + k], in shared memory).
__device__ __forceinline__ int ss_nth_bit(uint32_t m, int j, const uint8_t* nth8) {
    const int c1 = __popc(m & 0xffu), c2 = __popc(m & 0xffffu), c3 = __popc(m & 0xffffffu);
    int pos = 0, below = 0;
    if (j >= c1) { pos = 8; below = c1; }
    if (j >= c2) { pos = 16; below = c2; }
    if (j >= c3) { pos = 24; below = c3; }
    return pos + nth8[((m >> pos) & 0xffu) * 8 + (j - below)];
}

// Per pixel, per composited layer k (front to back), from the upstream
// gradient g and the layer totals (C_k, W_k) kept by the forward pass:
//   C_hat_k = C_k / W_k (normal: C_n / |C_n|), alpha_k = 1 - exp(-gamma W_k / 2 pi),
//   G_k,c  = dL/dC_k,c = g_c T_k alpha_k / W_k                   (Eq. shepard)
//   G_k,n  = dL/dC_n   = (d - n_hat (n_hat . d)) / |C_n|, d = g_n T_k alpha_k
//   dL/dW_k (alpha path) = gamma/2pi (T_{k+1} g.C_hat_k - g.R_k + g_A T_end)
//                          with R_k the radiance behind layer k (Eq. alpha, Eq. compositing)
//   S_k = sum_c G_k,c C_hat_k,c - dL/dW_k (alpha path)
// so that a fragment of weight w and channels ch in layer k has
// dL/dw = sum_c G_k,c ch_c - S_k and dL/dch_c = G_k,c w.  (G_k, S_k) are
// written over (C_k, W_k).
//
// With the depth-consolidation term (CONS, Eq. cons_loss) and its upstream
// gradient gC, per layer k with w_k = T_k alpha_k, z_k = C_k,11 / W_k,
// sigma_k^2 = Dz2 / W - (Dz / W)^2 (sums shifted by the layer's first depth
// z_r; see the forward kernel), S^b / M^b (S^a / M^a) the sums of w_i and
// w_i z_i over the layers in front of (behind) k:
//   e_k     = dL/dw_k  = z_k (S^b - S^a) - M^b + M^a + 2 w_k sigma_k^2
//   dL/dz_k = w_k (S^b - S^a),  dL/dsigma_k^2 = w_k^2,
// and through w_k = T_k alpha_k (dw_k/dW_k = kappa T_{k+1}, dw_j/dW_k =
// -kappa w_j for j > k, kappa = gamma / 2 pi), z_k and sigma_k^2:
//   dL/dC_k,11 += gC dL/dz_k / W_k
//   dL/dDz_k    = gC w_k^2 (-2 Dz / W^2),  dL/dDz2_k = gC w_k^2 / W
//   dL/dW_k    += gC (-dL/dz_k z_k / W + w_k^2 (2 Dz^2 / W^3 - Dz2 / W^2)
//                     + kappa (T_{k+1} e_k - sum_{j>k} e_j w_j)).
// dL/dDz and dL/dDz2 are written over the sums (z_r stays), so that a
// fragment of depth z adds dL/dw += dL/dDz (z - z_r) + dL/dDz2 (z - z_r)^2
// and dL/dz = w (dL/dC_11 + dL/dDz + 2 dL/dDz2 (z - z_r)).  Totals over the
// layers (sum w, sum w z, sum e w) come from two passes before the main one.
template <bool CONS>
__global__ void __launch_bounds__(256) layer_coeff_kernel(ss_ws_view ws, ss_bwd_args a) {
    const ss_layout* L = ws.layout;
    const int64_t P = L->total_pixels;
    const int64_t gpix = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gpix >= P) return;
    const int K = __float_as_int(ws.pix_state[gpix]);
    if (K <= 0) return;
    const float kw = a.f.p.gamma * (0.5f / SS_PI_F);
    const float Tend = ws.pix_state[P + gpix];
    float g[SS_NCH], rem[SS_NCH];   // rem_c = out_c - sum_{j<=k} T_j alpha_j C_hat_j
    const float4 d = reinterpret_cast<const float4*>(a.d_rgba)[gpix];
    const float4 o = reinterpret_cast<const float4*>(a.out_rgba)[gpix];
    g[0] = d.x; g[1] = d.y; g[2] = d.z;
    const float gA = d.w;
    rem[0] = o.x; rem[1] = o.y; rem[2] = o.z;   // includes T_end * bg
#pragma unroll
    for (int c = 0; c < SS_N_AOV; ++c) {
        g[3 + c] = a.d_aov ? a.d_aov[c * P + gpix] : 0.f;
        rem[3 + c] = a.out_aov ? a.out_aov[c * P + gpix] : 0.f;
    }
    // consolidation: upstream gradient and the totals of two pre-passes
    const float gC = CONS ? a.d_aov[SS_N_AOV * P + gpix] : 0.f;
    float Wt = 0.f, WZt = 0.f, Et = 0.f;
    auto cons_layer = [&](int kk, uint32_t& slot, float Tk, float& wk, float& zk, float& var, float& alk,
                          float& ek_e) {
        int64_t rs;
        const float* ls = ss_layer_rows(ws, P, gpix, kk, slot, rs);
        if (!ls) {   // a layer the forward could not store (pool capacity): no term
            wk = zk = var = alk = 0.f;
            ek_e = 1.f;
            return;
        }
        const float W = ls[12 * rs], iW = 1.f / W;
        zk = ls[11 * rs] * iW;
        const float mdz = ls[13 * rs] * iW;
        var = fmaf(ls[14 * rs], iW, -mdz * mdz);
        ek_e = expf(-kw * W);
        alk = -expm1f(-kw * W);
        wk = Tk * alk;
    };
    if (CONS && gC != 0.f) {
        float Tk = 1.f;
        uint32_t slot = SS_NO_SLOT;
        for (int kk = 0; kk < K; ++kk) {
            float wk, zk, var, al, e;
            cons_layer(kk, slot, Tk, wk, zk, var, al, e);
            Wt += wk;
            WZt = fmaf(wk, zk, WZt);
            Tk *= e;
        }
        Tk = 1.f;
        slot = SS_NO_SLOT;
        float Sb = 0.f, Mb = 0.f;
        for (int kk = 0; kk < K; ++kk) {
            float wk, zk, var, al, e;
            cons_layer(kk, slot, Tk, wk, zk, var, al, e);
            const float Sa = Wt - Sb - wk, Ma = WZt - Mb - wk * zk;
            const float ek = fmaf(zk, Sb - Sa, Ma - Mb) + 2.f * wk * var;
            Et = fmaf(ek, wk, Et);
            Sb += wk;
            Mb = fmaf(wk, zk, Mb);
            Tk *= e;
        }
    }
    float Tb = 1.f;
    float Sb = 0.f, Mb = 0.f, Pew = 0.f;   // consolidation: running sums over the layers in front
    uint32_t slot = SS_NO_SLOT;
    for (int kk = 0; kk < K; ++kk) {
        int64_t rs;
        float* ls = ss_layer_rows(ws, P, gpix, kk, slot, rs);
        if (!ls) break;   // the forward ran out of pool slots (SS_ERR_CAPACITY): no deeper terms
        float C[SS_NCH];
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) C[c] = ls[c * rs];
        const float W = ls[12 * rs];
        const float invW = 1.f / W;
        float hat[SS_NCH];
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) hat[c] = C[c] * invW;
        const float nl = sqrtf(C[8] * C[8] + C[9] * C[9] + C[10] * C[10]);
        const float inl = nl > 0.f ? 1.f / nl : 0.f;
        hat[8] = C[8] * inl; hat[9] = C[9] * inl; hat[10] = C[10] * inl;
        const float al = -expm1f(-kw * W);
        const float e = expf(-kw * W);
        const float tw = Tb * al;
        float gChat = 0.f, gR = 0.f;
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) {
            rem[c] = fmaf(-tw, hat[c], rem[c]);
            gChat = fmaf(g[c], hat[c], gChat);
            gR = fmaf(g[c], rem[c], gR);
        }
        const float dW_alpha = kw * (Tb * e * gChat - gR + gA * Tend);
        float G[SS_NCH];
        float sG = 0.f;
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) {
            if (c >= 8 && c <= 10) continue;
            G[c] = g[c] * tw * invW;
            sG = fmaf(G[c], hat[c], sG);
        }
        const float dn0 = g[8] * tw, dn1 = g[9] * tw, dn2 = g[10] * tw;
        const float nd = dn0 * hat[8] + dn1 * hat[9] + dn2 * hat[10];
        G[8] = (dn0 - hat[8] * nd) * inl;
        G[9] = (dn1 - hat[9] * nd) * inl;
        G[10] = (dn2 - hat[10] * nd) * inl;
        float S = sG - dW_alpha;
        if (CONS) {
            float gDz = 0.f, gDz2 = 0.f;
            if (gC != 0.f) {
                const float wk = tw, zk = hat[11];
                const float Dz = ls[13 * rs], Dz2 = ls[14 * rs];
                const float mdz = Dz * invW, var = fmaf(Dz2, invW, -mdz * mdz);
                const float Sa = Wt - Sb - wk, Ma = WZt - Mb - wk * zk;
                const float ek = fmaf(zk, Sb - Sa, Ma - Mb) + 2.f * wk * var;
                Pew = fmaf(ek, wk, Pew);
                const float dz = wk * (Sb - Sa);                  // dL/dz_k
                const float w2 = wk * wk;
                G[11] = fmaf(gC * dz, invW, G[11]);
                gDz = gC * w2 * (-2.f * mdz * invW);
                gDz2 = gC * w2 * invW;
                const float dW = gC * (-dz * zk * invW + w2 * invW * fmaf(2.f * mdz, mdz, -Dz2 * invW) +
                                       kw * (Tb * e * ek - (Et - Pew)));
                S -= dW;
                Sb += wk;
                Mb = fmaf(wk, zk, Mb);
            }
            ls[13 * rs] = gDz;
            ls[14 * rs] = gDz2;
        }
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) ls[c * rs] = G[c];
        ls[12 * rs] = S;
        Tb *= e;
    }
}

// ------------------------------------------------------------------------
// Densification statistic (Sec. 3.6.1, Eq. ss_grad): per (surfel, view)
// record, the derivatives of the record values the per-pixel weight depends
// on -- P (factor of the screen quadratic form), A2, B2 (perspective term),
// n_f -- along the camera-space centre c'_x and c'_y with the tangents held
// fixed.  T_{1,z} = f_x c'_x + c_x c'_z is the only T entry that c'_x moves
// (T_{2,z}: c'_y), so d/dT_{1,z} = (1/f_x) d/dc'_x; with T_{4,z} = c'_z and
// dp_x/dc'_x = f_x / c'_z, a fragment's
//   g_x = dL/dT_{1,z} T_{4,z} = dL/dp_x + sum_k dL/dval_k (c'_z / f_x) dval_k/dc'_x,
// likewise g_y.  The derivatives are taken in forward mode (value and two
// partials carried through the projection's arithmetic), with the
// factorisation branch the forward pass chose for P.

struct d3 {   // value and its partials along c'_x, c'_y
    float v, x, y;
};
__device__ __forceinline__ d3 dc(float v) { return {v, 0.f, 0.f}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return {a.v + b.v, a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return {a.v - b.v, a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ d3 operator-(d3 a) { return {-a.v, -a.x, -a.y}; }
__device__ __forceinline__ d3 operator*(d3 a, d3 b) {
    return {a.v * b.v, a.x * b.v + a.v * b.x, a.y * b.v + a.v * b.y};
}
__device__ __forceinline__ d3 operator*(float k, d3 a) { return {k * a.v, k * a.x, k * a.y}; }
// (the values only carry the partials, which the statistic needs to a few
// ulp: approximate reciprocals and square roots serve)
__device__ __forceinline__ d3 operator/(d3 a, d3 b) {
    const float ib = __fdividef(1.f, b.v), q = a.v * ib;
    return {q, (a.x - q * b.x) * ib, (a.y - q * b.y) * ib};
}
__device__ __forceinline__ d3 dsqrt(d3 a) {
    const float ir = rsqrtf(a.v), h = 0.5f * ir;
    return {a.v * ir, a.x * h, a.y * h};
}
__device__ __forceinline__ d3 dabs(d3 a) { return a.v < 0.f ? -a : a; }

__global__ void __launch_bounds__(256) ssg_jac_kernel(ss_ws_view ws, ss_fwd_args a, int64_t n_total) {
    const ss_layout* L = ws.layout;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_total) return;
    int scene = 0;
    while (scene + 1 < L->n_scenes && i >= L->scene_begin[scene + 1]) ++scene;
    const float c0 = a.s.pos[i * 3], c1 = a.s.pos[i * 3 + 1], c2 = a.s.pos[i * 3 + 2];
    const float4 q = *reinterpret_cast<const float4*>(a.s.quat + i * 4);
    const float2 ls = *reinterpret_cast<const float2*>(a.s.log_scale + i * 2);
    float Rq[9];
    quat_rot(q.x, q.y, q.z, q.w, Rq);
    const float su = expf(ls.x), sv = expf(ls.y);
    const float tu[3] = {su * Rq[0], su * Rq[3], su * Rq[6]};
    const float tv[3] = {sv * Rq[1], sv * Rq[4], sv * Rq[7]};
    const float nrm[3] = {Rq[2], Rq[5], Rq[8]};
    const float sig = a.p.sigma_f;
    for (int v = L->scene_view_begin[scene]; v < L->scene_view_begin[scene + 1]; ++v) {
        const ss_view_layout& vl = L->v[v];
        const int64_t r = vl.rec_off + (i - vl.surfel_begin);
        float4 out[4] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                         make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
        const uint32_t flags = __float_as_uint(ws.rec[r].r4.w);
        if (flags & SS_FLAG_VALID) {
            const ss_camera& cam = a.cams[v];
            const float* Rc = cam.R;
            float cp[3], tuc[3], tvc[3];
            for (int k = 0; k < 3; ++k) {
                cp[k] = Rc[k * 3] * c0 + Rc[k * 3 + 1] * c1 + Rc[k * 3 + 2] * c2 + cam.t[k];
                tuc[k] = Rc[k * 3] * tu[0] + Rc[k * 3 + 1] * tu[1] + Rc[k * 3 + 2] * tu[2];
                tvc[k] = Rc[k * 3] * tv[0] + Rc[k * 3 + 1] * tv[1] + Rc[k * 3 + 2] * tv[2];
            }
            const ss_view_geo& vg = ws.vgeo[v];
            const float Ndv = ss_plane_distance(q, c0, c1, c2, vg.o_hi, vg.o_lo);
            const float ncx = Rc[0] * nrm[0] + Rc[1] * nrm[1] + Rc[2] * nrm[2];   // n' = R n
            const float ncy = Rc[3] * nrm[0] + Rc[4] * nrm[1] + Rc[5] * nrm[2];
            const float fx = a.cams[v].fx, fy = a.cams[v].fy;
            const d3 cx{cp[0], 1.f, 0.f}, cy{cp[1], 0.f, 1.f}, cz = dc(cp[2]);
            const d3 Nd{Ndv, ncx, ncy};                      // N_d = n'.c'
            const d3 mx = cx / cz, my = cy / cz;
            const d3 ax = dc(tuc[0]) - mx * dc(tuc[2]), ay = dc(tuc[1]) - my * dc(tuc[2]);
            const d3 bx = dc(tvc[0]) - mx * dc(tvc[2]), by = dc(tvc[1]) - my * dc(tvc[2]);
            const d3 icz2 = dc(1.f / (cp[2] * cp[2]));
            const d3 m11 = (fx * fx) * ((ax * ax + bx * bx) * icz2);
            const d3 m12 = (fx * fy) * ((ax * ay + bx * by) * icz2);
            const d3 m22 = (fy * fy) * ((ay * ay + by * by) * icz2);
            const d3 det0 = (vg.detR * su * sv) * (Nd / cz);
            const d3 sdg = (fx * fy) * (det0 * icz2);
            const d3 Dn = sdg * sdg + sig * (m11 + m22) + dc(sig * sig);
            const d3 nf = dabs(sdg) / dsqrt(Dn);
            const d3 A2 = (1.f / fx) * (cz * dc(ncx) / Nd), B2 = (1.f / fy) * (cz * dc(ncy) / Nd);
            const d3 qa = (m22 + dc(sig)) / Dn, qb = -m12 / Dn, qc = (m11 + dc(sig)) / Dn;
            const d3 rsD = dc(1.f) / dsqrt(Dn);
            d3 P00, P01, P10, P11;
            if (ws.rec[r].r0.z == 0.f) {   // the branch the forward took (its P10 is zero)
                P00 = dsqrt(qa);
                P01 = qb / P00;
                P10 = dc(0.f);
                P11 = rsD / P00;
            } else {
                const d3 l11 = dsqrt(qc);
                P00 = qb / l11;
                P01 = l11;
                P10 = rsD / l11;
                P11 = dc(0.f);
            }
            const float kx = cp[2] / fx, ky = cp[2] / fy;
            out[0] = make_float4(kx * P00.x, kx * P01.x, kx * P10.x, kx * P11.x);
            out[1] = make_float4(kx * A2.x, kx * B2.x, kx * nf.x, 0.f);
            out[2] = make_float4(ky * P00.y, ky * P01.y, ky * P10.y, ky * P11.y);
            out[3] = make_float4(ky * A2.y, ky * B2.y, ky * nf.y, 0.f);
        }
        float4* J = ws.ssg_jac + r * 4;
        J[0] = out[0];
        J[1] = out[1];
        J[2] = out[2];
        J[3] = out[3];
    }
}

// AOV = false when no AOV gradient is given: the AOV channels' coefficients
// are zero, so only P, A2, B2, the centre, n_f and RGB (the first 12 values
// of the record) are differentiated and summed.
// The kernel is persistent, like the forward one: warps take (tile, block)
// items from a queue.
template <bool AOV, bool SSG, bool CONS, bool DET, bool POOL, int RWPB_BWD>
__device__ __forceinline__ void raster_bwd_block(const ss_ws_view& ws, const ss_bwd_args& a, const int gw,
                                                 unsigned char* bwd_smem, const uint8_t* nth8) {
    constexpr int NV = AOV ? G_N : G_CH + 3;   // gradient values per fragment
    constexpr int NVT = NV + (SSG ? 2 : 0);    // + |(g_x, g_y)| and a count of 1 (Eq. ss_grad)
    constexpr int NC = AOV ? SS_NCH : 3;       // channels with a coefficient
    constexpr int GTR = CONS ? GT + 3 : GT;    // layer coefficients per lane (+ dL/dDz, dL/dDz2, z_r)
    using bwarp = ss_bwarp_t<SSG ? G_N + 2 : G_N, GTR>;
    ss_wstage* Wst = reinterpret_cast<ss_wstage*>(bwd_smem);
    bwarp* Bws = reinterpret_cast<bwarp*>(bwd_smem + RWPB_BWD * sizeof(ss_wstage));
    const ss_layout* L = ws.layout;
    const int lw = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = gw / a.f.ts.bpt, warp = gw - tile * a.f.ts.bpt;   // bpt blocks per tile
    const int view = find_view_tile(L, tile);
    const ss_view_layout& vl = L->v[view];
    const int lt = tile - vl.tile_off;
    const int tx = lt % vl.tiles_x, ty = lt / vl.tiles_x;
    const int x0 = tx << a.f.ts.tw_log2, y0 = ty << a.f.ts.th_log2;
    ss_wstage* Wc = Wst + lw;         // staging buffer
    bwarp& B = Bws[lw];
    const int wx0 = 8 * (warp & ((1 << a.f.ts.bx_log2) - 1)), wy0 = 4 * (warp >> a.f.ts.bx_log2);
    const int lx = wx0 + (lane & 7), ly = wy0 + (lane >> 3);
    const int px = x0 + lx, py = y0 + ly;
    const bool inside = px < vl.width && py < vl.height;
    const float rc2 = a.f.p.r_cut * a.f.p.r_cut;
    const int64_t P = L->total_pixels;
    const int64_t gpix = vl.pixel_off + (int64_t)(inside ? py : 0) * vl.width + (inside ? px : 0);

    // per-pixel state: layer count from the forward pass; the per-layer
    // gradient coefficients (G_k, S_k) were written over the layer totals by
    // layer_coeff_kernel
    const int K = inside ? __float_as_int(ws.pix_state[gpix]) : 0;
    bool done = !inside || K == 0;
    unsigned n_frag = 0, n_batch = 0;

    // replay state (Algorithm 1): the layer index; the forward pass marked
    // in cover_adv the fragments that open a new layer (its gap test), so
    // the replay only counts them
    int k = 0;

    uint32_t slot = SS_NO_SLOT;   // pool slot of the current layer (layers past dense_layers)
    auto enter_layer = [&](int kk) {   // this lane's layer coefficients -> B.gtab (layers entered in order)
        if (!POOL || kk < ws.dense_layers) {
            const float* ls = ws.layer_state + (int64_t)kk * ws.ls_rows * P + gpix;
#pragma unroll
            for (int c = 0; c < GTR; ++c) B.gtab[lane * GTR + c] = ls[c * P];
        } else {
            int64_t rs;
            const float* ls = ss_layer_rows(ws, P, gpix, kk, slot, rs);
#pragma unroll
            for (int c = 0; c < GTR; ++c) B.gtab[lane * GTR + c] = ls ? ls[c] : 0.f;
        }
    };
    if (!done) enter_layer(0);

    const ss_rec* recs = ws.rec;   // keys hold batch-wide record indices
    float* grad = ws.grad_rec;
    // the forward pass's list of covering staged surfels of this warp
    const int64_t loff = ws.cand_off[(int64_t)tile * 8 + warp];   // the block's list (the forward's offsets)
    const uint2* clist = ws.cover_list + loff;
    const uint32_t* alist = ws.cover_adv + loff;
    const int64_t n_list = ws.cover_count[(int64_t)tile * 8 + warp];
    // deterministic mode: this item's rows start at det_coff[item] (one per list entry)
    const int64_t row0 = DET ? (int64_t)ws.det_coff[gw] : 0;
    int64_t chunk_base = 0;   // list index of the staged chunk's first slot

    // Differentiate the fragments of staged slots [sa, sb) at the live pixels
    // (dmask: pixels past their last layer), 32 at a time in list order (one
    // per lane), then sum the gradient rows of each run of equal surfels and
    // add the sums.  Every pixel stays in its layer within [sa, sb).
    auto run_slots = [&](int sa, int sb, uint32_t cmw, uint32_t dmask) {
        const uint32_t eff = (lane >= sa && lane < sb) ? (cmw & ~dmask) : 0u;
        const int cnt = __popc(eff);
        int incl = cnt;   // inclusive prefix sum of the slots' fragment counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - cnt;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) return;
        n_frag += lane == 0 ? (unsigned)total : 0u;
        // nonempty slots; when they are consecutive, a fragment's slot is the
        // one holding the batch's first fragment plus the slot starts between
        const uint32_t ne = __ballot_sync(0xffffffffu, cnt > 0);
        const bool contig = ((ne + (ne & (0u - ne))) & ne) == 0u;
        const int ne0 = __ffs(ne) - 1;
        __syncwarp();   // layer tables written by other lanes
        for (int b0 = 0; b0 < total; b0 += 32) {
            ++n_batch;
            const int nb = min(32, total - b0);
            const bool valid = lane < nb;
            const int F = b0 + lane;
            int s = 0;   // the slot of fragment F: the first with incl > F
            if (contig) {
                const uint32_t starts = __reduce_or_sync(
                    0xffffffffu, (cnt > 0 && excl > b0 && excl < b0 + 32) ? 1u << (excl - b0) : 0u);
                const int c0 = __popc(__ballot_sync(0xffffffffu, cnt > 0 && excl <= b0));
                s = min(31, ne0 + c0 - 1 + __popc(starts & ((2u << lane) - 1u)));
            } else {
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, incl, s + st - 1);
                    if (v <= F) s += st;
                }
            }
            const uint32_t es = __shfl_sync(0xffffffffu, eff, s);
            const int first = __shfl_sync(0xffffffffu, excl, s);
            const int pl = valid ? ss_nth_bit(es, F - first, nth8) : 0;   // its pixel lane
            if (valid) {
                const float4 h0 = Wc->h0[s], h1 = Wc->h1[s], h2 = Wc->h2[s];
                const float dx = (float)(wx0 + (pl & 7)) + 0.5f - h1.z;
                const float dy = (float)(wy0 + (pl >> 3)) + 0.5f - h1.w;
                const ss_hit h = ss_pixel_test(h0, h1, dx, dy, rc2);
                const float nf = fabsf(h2.z);
                const float rho2 = __fdividef(h.q, h.t);
                const float ex = __expf(-0.5f * rho2);
                const float w = nf * ex;   // the forward kernel's weight, same operations
                // the pixel's layer coefficients (row stride 13 or 16 floats: 4-byte loads of distinct
                // pixels fall in distinct banks for the odd stride)
                const float* gt = B.gtab + pl * GTR;
                const float4 c0v = Wc->c0[s], c1v = Wc->c1[s], c2v = Wc->c2[s];
                const float ch[SS_NCH] = {c0v.x, c0v.y, c0v.z, c1v.x, c1v.y, c1v.z,
                                          c1v.w, c2v.x, c2v.y, c2v.z, c2v.w, 0.5f * (h2.x + h2.y)};
                float gr[G_N];
                // dL/dw = sum_c G_c ch_c - S_k, in three interleaved chains
                float dl[3] = {-gt[12], 0.f, 0.f};
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float G = gt[c];
                    dl[c % 3] = fmaf(G, ch[c], dl[c % 3]);
                    gr[G_CH + c] = G * w;
                }
                float dLdw = dl[0] + (dl[1] + dl[2]);
                if (CONS) {   // the consolidation term's shifted depth sums of the layer
                    const float dz = ch[11] - gt[15];
                    dLdw = fmaf(gt[13], dz, fmaf(gt[14] * dz, dz, dLdw));
                    gr[G_CH + 11] = w * fmaf(2.f * gt[14], dz, gt[11] + gt[13]);
                }
                // w = n_f exp(-rho2 / 2), rho2 = q / s2^2 (Eq. mip_weight)
                gr[G_NF] = dLdw * ex;
                const float grho = -0.5f * w * dLdw;
                const float it2 = __fdividef(2.f * grho, h.t);
                const float gs0 = it2 * h.s0, gs1 = it2 * h.s1;
                const float gs2 = -2.f * grho * __fdividef(rho2, h.s2);
                gr[G_P + 0] = gs0 * dx; gr[G_P + 1] = gs0 * dy;
                gr[G_P + 2] = gs1 * dx; gr[G_P + 3] = gs1 * dy;
                gr[G_A2] = gs2 * dx; gr[G_B2] = gs2 * dy;
                gr[G_PX] = -(gs0 * h0.x + gs1 * h0.z + gs2 * h1.x);
                gr[G_PY] = -(gs0 * h0.y + gs1 * h0.w + gs2 * h1.y);
#pragma unroll
                for (int q = 0; q < NV; ++q) B.tab[q * GCOL + lane] = gr[q];
                if (SSG) {   // Eq. ss_grad: g = dL/dp + sum_k dL/dval_k jac[k]
                    // the record's row (64 B, read by the ~8 lanes of its run: L1 hits after the first)
                    const float4* J = ws.ssg_jac + (int64_t)Wc->id[s] * 4;
                    const float4 j0 = __ldg(J), j1 = __ldg(J + 1), j2 = __ldg(J + 2), j3 = __ldg(J + 3);
                    const float gxs = gr[G_PX] + gr[G_P + 0] * j0.x + gr[G_P + 1] * j0.y + gr[G_P + 2] * j0.z +
                                      gr[G_P + 3] * j0.w + gr[G_A2] * j1.x + gr[G_B2] * j1.y + gr[G_NF] * j1.z;
                    const float gys = gr[G_PY] + gr[G_P + 0] * j2.x + gr[G_P + 1] * j2.y + gr[G_P + 2] * j2.z +
                                      gr[G_P + 3] * j2.w + gr[G_A2] * j3.x + gr[G_B2] * j3.y + gr[G_NF] * j3.z;
                    B.tab[NV * GCOL + lane] = sqrtf(gxs * gxs + gys * gys);
                    B.tab[(NV + 1) * GCOL + lane] = 1.f;
                }
            }
            const uint32_t rid = Wc->id[s];   // this lane's record (run ends shuffle it to the row lanes)
            const int snext = __shfl_down_sync(0xffffffffu, s, 1);
            // run ends: the last valid column and every column followed by another surfel
            const uint32_t ends = __ballot_sync(0xffffffffu, valid && (lane == nb - 1 || snext != s));
            __syncwarp();
            float v[32];
            {
                const float4* t4 = reinterpret_cast<const float4*>(B.tab + (lane < NVT ? lane : 0) * GCOL);
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const float4 x = lane < NVT ? t4[m] : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[4 * m] = x.x; v[4 * m + 1] = x.y; v[4 * m + 2] = x.z; v[4 * m + 3] = x.w;
                }
            }
            // run sums, four columns at a time where no run ends inside them
            float tot = 0.f;
            int rs = 0;   // first column of the current run
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (((ends >> (4 * m)) & 15u) == 0u) {   // warp-uniform
                    tot += (v[4 * m] + v[4 * m + 1]) + (v[4 * m + 2] + v[4 * m + 3]);
                    continue;
                }
#pragma unroll
                for (int j = 4 * m; j < 4 * m + 4; ++j) {
                    tot += v[j];
                    if ((ends >> j) & 1u) {   // warp-uniform
                        const int colq = lane < NV ? lane : G_SSN + lane - NV;   // table row -> record column
                        if constexpr (DET) {
                            // the entry's row: written by its first run, added to by the run that
                            // continues it at the start of the next batch
                            const int sl = __shfl_sync(0xffffffffu, s, j);
                            const int64_t row = row0 + chunk_base + sl;
                            const bool cont = rs == 0 && __shfl_sync(0xffffffffu, excl, sl) < b0;
                            if (row < ws.det_cap) {
                                float* dst = ws.det_rows + row * SS_NGRAD + colq;
                                if (lane < NVT) *dst = cont ? *dst + tot : tot;
                                if (lane == 0 && !cont) ws.det_rid[row] = Wc->id[sl];
                            }
                        } else {
                            const uint32_t rj = __shfl_sync(0xffffffffu, rid, j);
                            if (lane < NVT && tot != 0.f) atomicAdd(grad + (int64_t)rj * SS_NGRAD + colq, tot);
                        }
                        tot = 0.f;
                        rs = j + 1;
                    }
                }
            }
            __syncwarp();
        }
    };

    // one staging buffer; the records of the next chunk are prefetched into L2
    uint2 nxt = lane < n_list ? __ldg(clist + lane) : make_uint2(0u, 0u);
    uint32_t nxa = lane < n_list ? __ldg(alist + lane) : 0u;
    for (int64_t base = 0; base < n_list; base += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        const int n = (int)min((int64_t)32, n_list - base);
        chunk_base = base;
        const uint2 cur = nxt;
        const uint32_t ca = lane < n ? nxa : 0u;   // layer-opening lanes of slot `lane`
        if (SSG && lane < n) {   // the record's densification derivatives into L2 ahead of their use
            const char* pj = reinterpret_cast<const char*>(ws.ssg_jac + (int64_t)cur.x * 4);
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pj));
        }
        stage_ids(*Wc, recs, cur.x, lane, lane < n);
        nxt = base + 32 + lane < n_list ? __ldg(clist + base + 32 + lane) : make_uint2(0u, 0u);
        nxa = base + 32 + lane < n_list ? __ldg(alist + base + 32 + lane) : 0u;
        if (base + 32 + lane < n_list) {
            const char* pr = reinterpret_cast<const char*>(recs + nxt.x);
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pr));
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pr + sizeof(ss_rec) - 1));
        }
        stage_finish(*Wc, n, lane, (float)x0, (float)y0);
        const uint32_t cm = lane < n ? cur.y : 0u;   // forward coverage of slot `lane`
        // replay of Algorithm 1: cut the chunk at each slot that opens a new
        // layer at a live pixel (the forward kernel's gap decisions); the
        // opening slot's own fragments belong to the new layers
        int sa = 0, applied = -1;
        for (;;) {
            const uint32_t dmask = __ballot_sync(0xffffffffu, done);
            if (dmask == 0xffffffffu) break;
            const uint32_t am = __ballot_sync(0xffffffffu, lane > applied && (ca & ~dmask) != 0u);
            const int sb = am ? __ffs(am) - 1 : n;
            run_slots(sa, sb, cm, dmask);
            if (sb >= n) break;
            const uint32_t av = __shfl_sync(0xffffffffu, ca, sb);
            if (!done && ((av >> lane) & 1u)) {
                ++k;
                if (k >= K) done = true;
                else enter_layer(k);
            }
            sa = sb;
            applied = sb;
            __syncwarp();
        }
        __syncwarp();   // the next chunk rewrites the staged slots
    }
    if (a.f.p.collect_stats) {
        unsigned long long x = n_frag;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(ws.stats + 5, x);
        if (lane == 0 && n_batch) atomicAdd(ws.stats + 8, (unsigned long long)n_batch);
    }
}

template <bool AOV, bool SSG, bool CONS, bool DET, bool POOL, int RWPB_BWD>
__global__ void __launch_bounds__(32 * RWPB_BWD, 24 / RWPB_BWD) raster_bwd_kernel(ss_ws_view ws, ss_bwd_args a,
                                                                                  int n_items) {
    extern __shared__ __align__(16) unsigned char bwd_smem[];
    __shared__ uint8_t nth8[256 * 8];   // set-bit positions within a byte
    for (int e = threadIdx.x; e < 256 * 8; e += blockDim.x) {
        const uint32_t v = (uint32_t)e >> 3;
        const int k = e & 7;
        int p = 0;
        for (int c = -1; p < 8; ++p)
            if (((v >> p) & 1u) && ++c == k) break;
        nth8[e] = (uint8_t)(p & 7);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(ws.work + 1, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        raster_bwd_block<AOV, SSG, CONS, DET, POOL, RWPB_BWD>(ws, a, item, bwd_smem, nth8);
        __syncwarp();
    }
}

template <bool AOV, bool SSG, bool CONS, bool DET, bool POOL, int W>
static void launch_raster_bwd(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st) {
    const int smem = W * (int)(sizeof(ss_wstage) + sizeof(ss_bwarp_t<SSG ? G_N + 2 : G_N, CONS ? GT + 3 : GT>));
    static std::atomic<unsigned long long> optin{0}, resident{0};
    ss_smem_optin(raster_bwd_kernel<AOV, SSG, CONS, DET, POOL, W>, smem, optin);
    const int n_items = (int)(L.total_tiles * L.bpt);
    const int ctas = ss_resident_ctas(raster_bwd_kernel<AOV, SSG, CONS, DET, POOL, W>, 32 * W, smem, resident);
    const int grid = max(1, min(ctas > 0 ? ctas : 1, (n_items + W - 1) / W));
    raster_bwd_kernel<AOV, SSG, CONS, DET, POOL, W><<<grid, 32 * W, smem, st>>>(ws, a, n_items);
}

template <bool AOV, bool SSG, bool CONS, bool DET, bool POOL>
static void launch_raster_bwd_w3(int w, const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a,
                                 cudaStream_t st) {
    if (w == 2) launch_raster_bwd<AOV, SSG, CONS, DET, POOL, 2>(ws, L, a, st);
    else if (w == 4) launch_raster_bwd<AOV, SSG, CONS, DET, POOL, 4>(ws, L, a, st);
    else launch_raster_bwd<AOV, SSG, CONS, DET, POOL, 8>(ws, L, a, st);
}

template <bool AOV, bool SSG, bool CONS, bool DET>
static void launch_raster_bwd_w2(int w, const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a,
                                 cudaStream_t st) {
    if (ws.dense_layers < a.f.p.k_max) launch_raster_bwd_w3<AOV, SSG, CONS, DET, true>(w, ws, L, a, st);
    else launch_raster_bwd_w3<AOV, SSG, CONS, DET, false>(w, ws, L, a, st);
}

// the deterministic mode (fixed-order row sums) and the pooled layer state
// are instances of their own, so that the default one carries none of their code
template <bool AOV, bool SSG, bool CONS>
static void launch_raster_bwd_w(int w, const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a,
                                cudaStream_t st) {
    if (ws.det_cap) launch_raster_bwd_w2<AOV, SSG, CONS, true>(w, ws, L, a, st);
    else launch_raster_bwd_w2<AOV, SSG, CONS, false>(w, ws, L, a, st);
}

void ss_launch_screen_grad_jac(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st) {
    if (L.total_tiles <= 0 || !ws.ssg_jac || !(a.g.screen_grad_norm || a.g.screen_grad_views)) return;
    const int64_t n = L.scene_begin[L.n_scenes];
    if (n <= 0) return;
    ss_note_launch();
    ssg_jac_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ws, a.f, n);
}

void ss_launch_raster_bwd(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st) {
    if (L.total_tiles <= 0) return;
    const bool ssg = ws.ssg_jac && (a.g.screen_grad_norm || a.g.screen_grad_views);
    const bool cons = a.f.p.cons != 0;   // (the host requires d_aov then)
    ss_note_launch();
    if (cons) layer_coeff_kernel<true><<<(unsigned)((L.total_pixels + 255) / 256), 256, 0, st>>>(ws, a);
    else layer_coeff_kernel<false><<<(unsigned)((L.total_pixels + 255) / 256), 256, 0, st>>>(ws, a);
    const int w = a.f.p.bwd_warps ? a.f.p.bwd_warps : RWPB_BWD_DEFAULT;
    ss_note_launch();
    if (cons) {
        if (ssg) launch_raster_bwd_w<true, true, true>(w, ws, L, a, st);
        else launch_raster_bwd_w<true, false, true>(w, ws, L, a, st);
    } else if (a.d_aov) {
        if (ssg) launch_raster_bwd_w<true, true, false>(w, ws, L, a, st);
        else launch_raster_bwd_w<true, false, false>(w, ws, L, a, st);
    } else {
        if (ssg) launch_raster_bwd_w<false, true, false>(w, ws, L, a, st);
        else launch_raster_bwd_w<false, false, false>(w, ws, L, a, st);
    }
}

// ------------------------------------------------------------------------
// projection + shading adjoint: one thread per surfel, loop over its views

__device__ __forceinline__ int64_t spec_level_off_b(const ss_env_desc& ed, int i, int& W, int& H) {
    int64_t off = 0;
    for (int k = 0; k < i; ++k) off += (int64_t)max(ed.width >> k, 8) * max(ed.height >> k, 4) * 3;
    W = max(ed.width >> i, 8);
    H = max(ed.height >> i, 4);
    return off;
}

// bilinear value of a 3-channel map
__device__ __forceinline__ float3 bilerp3b(const float* T, ss_taps t) {
    float w00 = (1.f - t.fx) * (1.f - t.fy), w01 = t.fx * (1.f - t.fy), w10 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
    float3 r;
    r.x = w00 * T[t.i00 * 3] + w01 * T[t.i01 * 3] + w10 * T[t.i10 * 3] + w11 * T[t.i11 * 3];
    r.y = w00 * T[t.i00 * 3 + 1] + w01 * T[t.i01 * 3 + 1] + w10 * T[t.i10 * 3 + 1] + w11 * T[t.i11 * 3 + 1];
    r.z = w00 * T[t.i00 * 3 + 2] + w01 * T[t.i01 * 3 + 2] + w10 * T[t.i10 * 3 + 2] + w11 * T[t.i11 * 3 + 2];
    return r;
}

// bilinear value, d/du, d/dv of a 3-channel map at precomputed taps
struct lk3 {
    float v[3], du[3], dv[3];
};
__device__ __forceinline__ lk3 lookup3(const float* T, const ss_taps& t, int W, int H) {
    lk3 r;
    for (int c = 0; c < 3; ++c) {
        float a = T[t.i00 * 3 + c], b = T[t.i01 * 3 + c], d = T[t.i10 * 3 + c], e = T[t.i11 * 3 + c];
        r.v[c] = (1.f - t.fy) * ((1.f - t.fx) * a + t.fx * b) + t.fy * ((1.f - t.fx) * d + t.fx * e);
        r.du[c] = (float)W * ((1.f - t.fy) * (b - a) + t.fy * (e - d));
        r.dv[c] = (float)H * ((1.f - t.fx) * (d - a) + t.fx * (e - b));
    }
    return r;
}
// Where the env-texel gradients go: RGBA float accumulators (one 16-byte
// atomic per tap, accumulators SS_ACC_STRIDE float4 apart), or in the
// deterministic mode the same memory as 64-bit fixed-point integers (RGB,
// 2 SS_ACC_STRIDE words apart): a contribution v is added as rint(v 2^k),
// exact and independent of the order; one beyond 2^lim_bits is flagged.
struct ss_env_sink {
    float4* acc;
    long long* accx;   // deterministic mode (acc is then null)
    int k;
    double lim;        // 2^(62 - cbits)
    int* status;
};
__device__ __forceinline__ void scatter4_fx(const ss_env_sink& S, int64_t base, const ss_taps& t, const float g[3],
                                            float scale) {
    const float w[4] = {(1.f - t.fx) * (1.f - t.fy) * scale, t.fx * (1.f - t.fy) * scale, (1.f - t.fx) * t.fy * scale,
                        t.fx * t.fy * scale};
    const int idx[4] = {t.i00, t.i01, t.i10, t.i11};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double v = ldexp((double)(w[q] * g[c]), S.k);
            if (!(fabs(v) < S.lim)) {
                atomicOr(S.status, SS_ERR_CAPACITY);
                continue;
            }
            const long long iv = llrint(v);
            if (iv)
                atomicAdd(reinterpret_cast<unsigned long long*>(S.accx + (base + idx[q]) * (2 * SS_ACC_STRIDE) + c),
                          (unsigned long long)iv);
        }
}
__device__ __forceinline__ void scatter4(float4* D, const ss_taps& t, const float g[3], float scale) {
    if (scale == 0.f || (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f)) return;
    const float w00 = (1.f - t.fx) * (1.f - t.fy) * scale, w01 = t.fx * (1.f - t.fy) * scale,
                w10 = (1.f - t.fx) * t.fy * scale, w11 = t.fx * t.fy * scale;
    atomicAdd(D + (int64_t)t.i00 * SS_ACC_STRIDE, make_float4(w00 * g[0], w00 * g[1], w00 * g[2], 0.f));
    atomicAdd(D + (int64_t)t.i01 * SS_ACC_STRIDE, make_float4(w01 * g[0], w01 * g[1], w01 * g[2], 0.f));
    atomicAdd(D + (int64_t)t.i10 * SS_ACC_STRIDE, make_float4(w10 * g[0], w10 * g[1], w10 * g[2], 0.f));
    atomicAdd(D + (int64_t)t.i11 * SS_ACC_STRIDE, make_float4(w11 * g[0], w11 * g[1], w11 * g[2], 0.f));
}
// the taps of a map whose first texel is `base` of the scene's accumulators
__device__ __forceinline__ void scatter_to(const ss_env_sink& S, int64_t base, const ss_taps& t, const float g[3],
                                           float scale) {
    if (scale == 0.f || (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f)) return;
    if (S.accx) scatter4_fx(S, base, t, g, scale);
    else if (S.acc) scatter4(S.acc + base * SS_ACC_STRIDE, t, g, scale);
}

// d(u, v)/d(direction) for the equirect map of a unit direction d
__device__ __forceinline__ void uv_grad(const float d[3], float gu, float gv, float out[3]) {
    const float rxz = fmaxf(d[0] * d[0] + d[2] * d[2], 1e-20f);
    // u = atan2(d_x, -d_z) / 2pi + 1/2
    const float irs = rsqrtf(rxz);
    const float k = gu * (0.5f / SS_PI_F) * irs * irs;
    out[0] = k * (-d[2]);
    out[2] = k * d[0];
    out[1] = 0.f;
    // v = acos(d_y / |d|) / pi; with |d| = 1: dv/dd = -(e_y - d_y d) / (pi sqrt(1 - d_y^2))
    const float kv = -gv * (1.f / SS_PI_F) * irs;
    out[0] += kv * (-d[1] * d[0]);
    out[1] += kv * (1.f - d[1] * d[1]);
    out[2] += kv * (-d[1] * d[2]);
}

// One thread per surfel: the raster gradient record of each of its views is
// chained back to the surfel parameters; the views are summed in order
// (deterministic) and added to the caller's gradients.  The irradiance lookup
// depends on the surfel's normal and on the side it shows, not on the view,
// so its adjoint is taken once per side, from the sum over the views that
// see that side.


// Irradiance adjoint of one side of a surfel (fs = +1 front, -1 back) given
// g = sum over that side's views of dL/dLd: the texel gradients (bilinear
// adjoint) and the normal column of dL/dR through uv(fs n).
__device__ __forceinline__ void irr_side_adjoint(const float* irr, int W, int H, const float nrm[3], float fs,
                                                 const float g[3], const ss_env_sink* sink, int64_t base,
                                                 float gRn[3]) {
    if (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f) return;
    const float ns[3] = {fs * nrm[0], fs * nrm[1], fs * nrm[2]};
    float un, vn;
    dir_to_uv(ns[0], ns[1], ns[2], un, vn);
    const ss_taps t = bilinear_taps(un, vn, W, H, true);
    const lk3 Ld = lookup3(irr, t, W, H);
    if (sink) scatter_to(*sink, base, t, g, 1.f);
    float gun = 0.f, gvn = 0.f;
    for (int k = 0; k < 3; ++k) {
        gun += g[k] * Ld.du[k];
        gvn += g[k] * Ld.dv[k];
    }
    float dnsv[3];
    uv_grad(ns, gun, gvn, dnsv);
    for (int k = 0; k < 3; ++k) gRn[k] += fs * dnsv[k];
}

template <bool DET>
__device__ __forceinline__ void pbwd_surfel(const ss_ws_view& ws, const ss_bwd_args& A, const int64_t i,
                                            const int scene) {
    const ss_layout* L = ws.layout;
    const ss_fwd_args& a = A.f;
    const float c[3] = {a.s.pos[i * 3], a.s.pos[i * 3 + 1], a.s.pos[i * 3 + 2]};
    const float4 q4 = *reinterpret_cast<const float4*>(a.s.quat + i * 4);
    const float2 ls = *reinterpret_cast<const float2*>(a.s.log_scale + i * 2);
    const float rho[3] = {a.s.albedo[i * 3], a.s.albedo[i * 3 + 1], a.s.albedo[i * 3 + 2]};
    const float rough = a.s.roughness[i], metal = a.s.metallic[i];
    float Rq[9];
    quat_rot(q4.x, q4.y, q4.z, q4.w, Rq);
    const float su = expf(ls.x), sv = expf(ls.y);
    const float tu[3] = {su * Rq[0], su * Rq[3], su * Rq[6]};
    const float tv[3] = {sv * Rq[1], sv * Rq[4], sv * Rq[7]};
    const float nrm[3] = {Rq[2], Rq[5], Rq[8]};
    const float sig = a.p.sigma_f;
    const int nL = a.ed.n_levels;
    const int IW = a.ed.irr_width, IH = a.ed.irr_height;
    const int64_t irr_stride = (int64_t)IW * IH * 3;
    int Wt, Ht;
    const int64_t spec_stride = spec_level_off_b(a.ed, nL, Wt, Ht);
    const float* irr = a.env.irr + scene * irr_stride;
    const float* spec = a.env.spec + scene * spec_stride;
    const bool d_irr = A.genv.irr != nullptr, d_spec = A.genv.spec != nullptr;
    // env-texel gradients: float accumulators, or fixed-point integers (deterministic mode)
    ss_env_sink sink;
    sink.acc = DET ? nullptr : ws.env_acc;
    sink.accx = DET ? reinterpret_cast<long long*>(ws.env_acc) : nullptr;
    sink.k = DET ? ss_det_env_exponent(*ws.det_maxbits, A.det_vmax, A.det_cbits) : 0;
    sink.lim = DET ? ldexp(1.0, 62 - A.det_cbits) : 0.0;
    sink.status = ws.status;
    const int lutn = a.p.lut_n;
    const float* LUT = a.env.lut;
    // roughness-only shading quantities: the two specular levels and their blend
    const float rcl = fminf(fmaxf(rough, 0.f), 1.f);
    const float lc = rcl * (float)(nL - 1);
    const int l0 = min((int)floorf(lc), nL - 1), l1 = min(l0 + 1, nL - 1);
    const float lf = lc - (float)l0;
    int W0, H0, W1, H1;
    const int64_t o0 = spec_level_off_b(a.ed, l0, W0, H0), o1 = spec_level_off_b(a.ed, l1, W1, H1);
    // irradiance at the front and the back side of the normal (the same in every view)
    float LdF[3], LdB[3];
    {
        float u, v;
        dir_to_uv(nrm[0], nrm[1], nrm[2], u, v);
        const float3 f = bilerp3b(irr, bilinear_taps(u, v, IW, IH, true));
        dir_to_uv(-nrm[0], -nrm[1], -nrm[2], u, v);
        const float3 b = bilerp3b(irr, bilinear_taps(u, v, IW, IH, true));
        LdF[0] = f.x; LdF[1] = f.y; LdF[2] = f.z;
        LdB[0] = b.x; LdB[1] = b.y; LdB[2] = b.z;
    }

    // parameter gradients, summed over the scene's views in order
    float gc[3] = {0, 0, 0}, gRq[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gsu = 0.f, gsv = 0.f;
    float grho[3] = {0, 0, 0}, grough = 0.f, gmetal = 0.f;
    float gLdF[3] = {0, 0, 0}, gLdB[3] = {0, 0, 0};   // dL/dLd summed per side
    float ssg_norm = 0.f, ssg_views = 0.f;            // densification statistic (Eq. ss_grad)
    const bool ssg = A.g.screen_grad_norm || A.g.screen_grad_views;
    bool any_view = false;
    for (int v = L->scene_view_begin[scene]; v < L->scene_view_begin[scene + 1]; ++v) {
        const ss_view_layout& vl = L->v[v];
        const int64_t r = vl.rec_off + (i - vl.surfel_begin);
        // every load of the view first (one round trip), then the decisions
        const uint32_t flags = __float_as_uint(ws.rec[r].r4.w);
        const float4 r0 = ws.rec[r].r0, r1 = ws.rec[r].r1;
        const float4* gr4 = reinterpret_cast<const float4*>(ws.grad_rec + r * SS_NGRAD);
        float G[24];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 t = gr4[k];
            G[4 * k] = t.x; G[4 * k + 1] = t.y; G[4 * k + 2] = t.z; G[4 * k + 3] = t.w;
        }
        if (!(flags & SS_FLAG_VALID)) continue;
        if (ssg) {
            ssg_norm += G[G_SSN];
            ssg_views += G[G_SSC] > 0.f ? 1.f : 0.f;   // the surfel has a fragment in this view
        }
        bool any = false;
#pragma unroll
        for (int k = 0; k < G_N; ++k) any = any || (G[k] != 0.f);
        if (!any) continue;
        any_view = true;
        const ss_camera& cam = a.cams[v];
        const float* Rc = cam.R;
        const float fx = cam.fx, fy = cam.fy;
        // ---- recompute the forward quantities (FP32 suffices for derivatives)
        float cp[3], tuc[3], tvc[3];
        for (int k = 0; k < 3; ++k) {
            cp[k] = Rc[k * 3] * c[0] + Rc[k * 3 + 1] * c[1] + Rc[k * 3 + 2] * c[2] + cam.t[k];
            tuc[k] = Rc[k * 3] * tu[0] + Rc[k * 3 + 1] * tu[1] + Rc[k * 3 + 2] * tu[2];
            tvc[k] = Rc[k * 3] * tv[0] + Rc[k * 3 + 1] * tv[1] + Rc[k * 3 + 2] * tv[2];
        }
        const float cz = cp[2];
        const float icz = 1.f / cz, icz2 = icz * icz;
        const float mx = cp[0] * icz, my = cp[1] * icz;
        const float ax = tuc[0] - mx * tuc[2], ay = tuc[1] - my * tuc[2];
        const float bx = tvc[0] - mx * tvc[2], by = tvc[1] - my * tvc[2];
        const ss_view_geo& vg = ws.vgeo[v];
        const float cmo[3] = {(c[0] - vg.o_hi[0]) - vg.o_lo[0], (c[1] - vg.o_hi[1]) - vg.o_lo[1],
                              (c[2] - vg.o_hi[2]) - vg.o_lo[2]};
        const float A2 = r1.x, B2 = r1.y;
        const float Nd = ss_plane_distance(q4, c[0], c[1], c[2], vg.o_hi, vg.o_lo);
        const float iNd = 1.f / Nd;
        const float detR = vg.detR;
        const float det0 = detR * su * sv * Nd * icz;
        const float m11 = fx * fx * (ax * ax + bx * bx) * icz2;
        const float m12 = fx * fy * (ax * ay + bx * by) * icz2;
        const float m22 = fy * fy * (ay * ay + by * by) * icz2;
        const float sdg = fx * fy * det0 * icz2;
        const float Dn = sdg * sdg + sig * (m11 + m22) + sig * sig;
        const float iDn = 1.f / Dn;
        const float rsD = rsqrtf(Dn);
        const float nf = fabsf(sdg) * rsD;
        const float qa = (m22 + sig) * iDn, qb = -m12 * iDn, qc = (m11 + sig) * iDn;

        // ---- raster parameters -> (qa, qb, qc, Dn); the factorisation the
        // forward chose is the one whose P10 it stored as zero
        float dqa = 0.f, dqb = 0.f, dqc = 0.f, dDn = 0.f;
        if (r0.z == 0.f) {
            const float P00 = sqrtf(qa), iP = 1.f / P00, P01 = qb * iP, P11 = rsD * iP;
            dqb += G[G_P + 1] * iP;
            dDn += G[G_P + 3] * (-0.5f * rsD * iDn) * iP;
            const float dP00 = G[G_P + 0] - (G[G_P + 1] * P01 + G[G_P + 3] * P11) * iP;
            dqa += 0.5f * dP00 * iP;
        } else {
            const float l = sqrtf(qc), il = 1.f / l, P00 = qb * il, P10 = rsD * il;
            dqb += G[G_P + 0] * il;
            dDn += G[G_P + 2] * (-0.5f * rsD * iDn) * il;
            const float dl = G[G_P + 1] - (G[G_P + 0] * P00 + G[G_P + 2] * P10) * il;
            dqc += 0.5f * dl * il;
        }
        float dm11 = dqc * iDn, dm12 = -dqb * iDn, dm22 = dqa * iDn;
        dDn += -(dqa * qa + dqb * qb + dqc * qc) * iDn;
        // n_f = |sdg| / sqrt(Dn)
        float dsdg = G[G_NF] * copysignf(1.f, sdg) * rsD;
        dDn += -0.5f * G[G_NF] * nf * iDn;
        // Dn = sdg^2 + sig (m11 + m22) + sig^2
        dsdg += 2.f * sdg * dDn;
        dm11 += sig * dDn;
        dm22 += sig * dDn;
        // ---- (m11, m12, m22, sdg) -> (a, b, det0, cz)
        float dcz = 0.f;
        const float ddet0 = dsdg * fx * fy * icz2;
        dcz += -2.f * dsdg * sdg * icz;
        float dax = icz2 * (dm11 * fx * fx * 2.f * ax + dm12 * fx * fy * ay);
        float dbx = icz2 * (dm11 * fx * fx * 2.f * bx + dm12 * fx * fy * by);
        float day = icz2 * (dm22 * fy * fy * 2.f * ay + dm12 * fx * fy * ax);
        float dby = icz2 * (dm22 * fy * fy * 2.f * by + dm12 * fx * fy * bx);
        dcz += -2.f * icz * (dm11 * m11 + dm12 * m12 + dm22 * m22);
        // ---- A2 = cz n'_x / (fx Nd), B2 = cz n'_y / (fy Nd), det0 = detR su sv Nd / cz
        float dNd = 0.f;
        dcz += (G[G_A2] * A2 + G[G_B2] * B2) * icz;
        const float dncx = G[G_A2] * cz * iNd / fx;
        const float dncy = G[G_B2] * cz * iNd / fy;
        dNd += -(G[G_A2] * A2 + G[G_B2] * B2) * iNd;
        const float kdet = detR * su * sv * icz;     // det0 / Nd
        dNd += ddet0 * kdet;
        gsu += ddet0 * detR * sv * Nd * icz;
        gsv += ddet0 * detR * su * Nd * icz;
        dcz += -ddet0 * det0 * icz;
        float dn[3], dcv[3];
        for (int k = 0; k < 3; ++k) {
            dn[k] = dncx * Rc[k] + dncy * Rc[3 + k] + dNd * cmo[k];   // n' = R n, Nd = n.(c - o)
            dcv[k] = dNd * nrm[k];
        }
        // ---- a = t'_u - m t'_uz, b = t'_v - m t'_vz ; p = f m + c
        float dtuc[3] = {dax, day, -(dax * mx + day * my)};
        float dtvc[3] = {dbx, dby, -(dbx * mx + dby * my)};
        float dmx = -(dax * tuc[2] + dbx * tvc[2]) + fx * G[G_PX];
        float dmy = -(day * tuc[2] + dby * tvc[2]) + fy * G[G_PY];
        // depth channel = c'_z
        dcz += G[G_CH + 11];
        float dcp[3] = {dmx * icz, dmy * icz, dcz - (dmx * mx + dmy * my) * icz};
        for (int k = 0; k < 3; ++k) {
            dcv[k] += Rc[k] * dcp[0] + Rc[3 + k] * dcp[1] + Rc[6 + k] * dcp[2];
            const float dtu = Rc[k] * dtuc[0] + Rc[3 + k] * dtuc[1] + Rc[6 + k] * dtuc[2];
            const float dtv = Rc[k] * dtvc[0] + Rc[3 + k] * dtvc[1] + Rc[6 + k] * dtvc[2];
            // t_u = su R[:,0], t_v = sv R[:,1]
            gsu += dtu * Rq[k * 3 + 0];
            gsv += dtv * Rq[k * 3 + 1];
            gRq[k * 3 + 0] += su * dtu;
            gRq[k * 3 + 1] += sv * dtv;
        }
        // ---- shading (Eq. ibl) and the AOV channels; the view direction as
        // the forward forms it
        const float ox = -(Rc[0] * cam.t[0] + Rc[3] * cam.t[1] + Rc[6] * cam.t[2]);
        const float oy = -(Rc[1] * cam.t[0] + Rc[4] * cam.t[1] + Rc[7] * cam.t[2]);
        const float oz = -(Rc[2] * cam.t[0] + Rc[5] * cam.t[1] + Rc[8] * cam.t[2]);
        const float wv[3] = {ox - c[0], oy - c[1], oz - c[2]};
        const float iwl = rsqrtf(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
        const float wo[3] = {wv[0] * iwl, wv[1] * iwl, wv[2] * iwl};
        const bool back = (flags & SS_FLAG_FLIPPED) != 0;
        const float fs = back ? -1.f : 1.f;
        const float ns[3] = {fs * nrm[0], fs * nrm[1], fs * nrm[2]};
        const float mup = ns[0] * wo[0] + ns[1] * wo[1] + ns[2] * wo[2];
        const float mu = fminf(fmaxf(mup, 0.f), 1.f);
        const float refl[3] = {2.f * mup * ns[0] - wo[0], 2.f * mup * ns[1] - wo[1], 2.f * mup * ns[2] - wo[2]};
        float dns[3] = {G[G_CH + 8], G[G_CH + 9], G[G_CH + 10]};
        for (int k = 0; k < 3; ++k) grho[k] += G[G_CH + 3 + k];
        grough += G[G_CH + 6];
        gmetal += G[G_CH + 7];
        const float dcol[3] = {G[G_CH + 0], G[G_CH + 1], G[G_CH + 2]};
        if (dcol[0] != 0.f || dcol[1] != 0.f || dcol[2] != 0.f) {
            float ur, vr;
            dir_to_uv(refl[0], refl[1], refl[2], ur, vr);
            const float Ld[3] = {back ? LdB[0] : LdF[0], back ? LdB[1] : LdF[1], back ? LdB[2] : LdF[2]};
            const ss_taps t0 = bilinear_taps(ur, vr, W0, H0, true), t1 = bilinear_taps(ur, vr, W1, H1, true);
            const lk3 S0 = lookup3(spec + o0, t0, W0, H0), S1 = lookup3(spec + o1, t1, W1, H1);
            ss_taps lt = bilinear_taps(mu, rcl, lutn, lutn, false);
            float be[2], dbe_mu[2], dbe_r[2];
            for (int z = 0; z < 2; ++z) {
                const float a0 = LUT[lt.i00 * 2 + z], a1 = LUT[lt.i01 * 2 + z], a2 = LUT[lt.i10 * 2 + z],
                            a3 = LUT[lt.i11 * 2 + z];
                be[z] = (1.f - lt.fy) * ((1.f - lt.fx) * a0 + lt.fx * a1) + lt.fy * ((1.f - lt.fx) * a2 + lt.fx * a3);
                dbe_mu[z] = (float)lutn * ((1.f - lt.fy) * (a1 - a0) + lt.fy * (a3 - a2));
                dbe_r[z] = (float)lutn * ((1.f - lt.fx) * (a2 - a0) + lt.fx * (a3 - a1));
            }
            float dLs[3], dbe1 = 0.f, dbe2 = 0.f, dlf = 0.f;
            for (int k = 0; k < 3; ++k) {
                const float F0 = 0.04f * (1.f - metal) + rho[k] * metal;
                const float kd = (1.f - F0) * (1.f - metal);
                const float Ls = (1.f - lf) * S0.v[k] + lf * S1.v[k];
                // col = kd rho Ld + Ls (F0 be1 + be2)
                const float dkd = dcol[k] * rho[k] * Ld[k];
                grho[k] += dcol[k] * kd * Ld[k];
                const float dLd = dcol[k] * kd * rho[k];
                if (back) gLdB[k] += dLd;
                else gLdF[k] += dLd;
                dLs[k] = dcol[k] * (F0 * be[0] + be[1]);
                float dF0 = dcol[k] * Ls * be[0];
                dbe1 += dcol[k] * Ls * F0;
                dbe2 += dcol[k] * Ls;
                dF0 += -dkd * (1.f - metal);
                gmetal += -dkd * (1.f - F0);
                grho[k] += dF0 * metal;
                gmetal += dF0 * (rho[k] - 0.04f);
                dlf += dLs[k] * (S1.v[k] - S0.v[k]);
            }
            // roughness: LUT row and level coordinate (both clamped to [0, 1])
            if (rough > 0.f && rough < 1.f) grough += dbe1 * dbe_r[0] + dbe2 * dbe_r[1] + dlf * (float)(nL - 1);
            float dmu = dbe1 * dbe_mu[0] + dbe2 * dbe_mu[1];
            float dmup = (mup > 0.f && mup < 1.f) ? dmu : 0.f;
            // specular texels into the workspace's RGBA accumulators (irradiance
            // texels first, then the specular stack)
            if (d_spec) {
                const int64_t sb = scene * ws.env_texels + (int64_t)IW * IH;   // the scene's first specular texel
                scatter_to(sink, sb + o0 / 3, t0, dLs, 1.f - lf);
                scatter_to(sink, sb + o1 / 3, t1, dLs, lf);
            }
            // reflected direction: Ls(uv(refl))
            float gur = 0.f, gvr = 0.f;
            for (int k = 0; k < 3; ++k) {
                gur += dLs[k] * ((1.f - lf) * S0.du[k] + lf * S1.du[k]);
                gvr += dLs[k] * ((1.f - lf) * S0.dv[k] + lf * S1.dv[k]);
            }
            float drefl[3];
            const float irl = rsqrtf(refl[0] * refl[0] + refl[1] * refl[1] + refl[2] * refl[2]);
            const float rn[3] = {refl[0] * irl, refl[1] * irl, refl[2] * irl};
            float drn[3];
            uv_grad(rn, gur, gvr, drn);
            // through the normalisation of refl (|refl| = 1 up to rounding)
            const float rd = drn[0] * rn[0] + drn[1] * rn[1] + drn[2] * rn[2];
            for (int k = 0; k < 3; ++k) drefl[k] = (drn[k] - rn[k] * rd) * irl;
            // refl = 2 mup ns - wo, mup = ns.wo
            float dwo[3];
            const float rdn = drefl[0] * ns[0] + drefl[1] * ns[1] + drefl[2] * ns[2];
            dmup += 2.f * rdn;
            for (int k = 0; k < 3; ++k) {
                dns[k] += 2.f * mup * drefl[k] + dmup * wo[k];
                dwo[k] = -drefl[k] + dmup * ns[k];
            }
            // wo = normalize(o - c)
            const float wd = dwo[0] * wo[0] + dwo[1] * wo[1] + dwo[2] * wo[2];
            for (int k = 0; k < 3; ++k) dcv[k] += -(dwo[k] - wo[k] * wd) * iwl;
        }
        for (int k = 0; k < 3; ++k) dn[k] += fs * dns[k];
        for (int k = 0; k < 3; ++k) {
            gRq[k * 3 + 2] += dn[k];
            gc[k] += dcv[k];
        }
    }
    if (ssg) {
        if (A.g.screen_grad_norm && ssg_norm != 0.f) A.g.screen_grad_norm[i] += ssg_norm;
        if (A.g.screen_grad_views && ssg_views != 0.f) A.g.screen_grad_views[i] += ssg_views;
    }
    if (!any_view) return;
    // ---- irradiance: once per side, from the view sums
    {
        float gRn[3] = {0.f, 0.f, 0.f};
        const ss_env_sink* sk = d_irr ? &sink : nullptr;
        irr_side_adjoint(irr, IW, IH, nrm, 1.f, gLdF, sk, scene * ws.env_texels, gRn);
        irr_side_adjoint(irr, IW, IH, nrm, -1.f, gLdB, sk, scene * ws.env_texels, gRn);
        for (int k = 0; k < 3; ++k) gRq[k * 3 + 2] += gRn[k];
    }
    // ---- R(q / |q|) -> q (linear in the summed dL/dR)
    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    const float* d = gRq;
    const float gw = 2.f * (-z * d[1] + y * d[2] + z * d[3] - x * d[5] - y * d[6] + x * d[7]);
    const float gx = 2.f * (y * d[1] + z * d[2] + y * d[3] - 2.f * x * d[4] - w * d[5] + z * d[6] + w * d[7] - 2.f * x * d[8]);
    const float gy = 2.f * (-2.f * y * d[0] + x * d[1] + w * d[2] + x * d[3] + z * d[5] - w * d[6] + z * d[7] - 2.f * y * d[8]);
    const float gz = 2.f * (-2.f * z * d[0] - w * d[1] + x * d[2] + w * d[3] - 2.f * z * d[4] + y * d[5] + x * d[6] + y * d[7]);
    const float dotq = gw * w + gx * x + gy * y + gz * z;
    const ss_surfel_grads& g = A.g;
    if (g.pos)
        for (int k = 0; k < 3; ++k) g.pos[i * 3 + k] += gc[k];
    if (g.quat) {
        g.quat[i * 4 + 0] += (gw - w * dotq) * qn;
        g.quat[i * 4 + 1] += (gx - x * dotq) * qn;
        g.quat[i * 4 + 2] += (gy - y * dotq) * qn;
        g.quat[i * 4 + 3] += (gz - z * dotq) * qn;
    }
    if (g.log_scale) {
        g.log_scale[i * 2 + 0] += gsu * su;
        g.log_scale[i * 2 + 1] += gsv * sv;
    }
    if (g.albedo)
        for (int k = 0; k < 3; ++k) g.albedo[i * 3 + k] += grho[k];
    if (g.roughness) g.roughness[i] += grough;
    if (g.metallic) g.metallic[i] += gmetal;
}

// One CTA per contiguous block of surfels (each thread one surfel at a time);
// three CTAs per SM leave 170 registers a thread (1.85 -> 1.81 ms against
// four CTAs at 128 registers, which spilled ~280 bytes a thread).
template <bool DET>
__global__ void __launch_bounds__(128, 3) project_bwd_kernel(ss_ws_view ws, ss_bwd_args A, int64_t n_surfels,
                                                            int64_t per_block) {
    const ss_layout* L = ws.layout;
    const int64_t i0 = blockIdx.x * per_block;
    if (i0 >= n_surfels) return;
    const int64_t i1 = min(n_surfels, i0 + per_block);
    auto scene_of = [&](int64_t i) {
        int lo = 0, hi = L->n_scenes - 1;
        while (lo < hi) {
            int m = (lo + hi + 1) >> 1;
            if (L->scene_begin[m] <= i) lo = m;
            else hi = m - 1;
        }
        return lo;
    };
    const int scene = scene_of(i0);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        pbwd_surfel<DET>(ws, A, i, i < L->scene_begin[scene + 1] ? scene : scene_of(i));
}

// Add the RGBA accumulators into the caller's env-map gradients (RGB); in
// the deterministic mode they hold fixed-point integers of scale 2^k.
__global__ void env_acc_flush_kernel(const float4* acc, int64_t texels, int64_t irr_tex, int64_t total,
                                     float* d_irr, float* d_spec, const unsigned int* det_maxbits, int vmax,
                                     int cbits) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int64_t sc = i / texels, k = i % texels;
    float4 v;
    if (det_maxbits) {
        const long long* x = reinterpret_cast<const long long*>(acc) + i * (2 * SS_ACC_STRIDE);
        const int e = -ss_det_env_exponent(*det_maxbits, vmax, cbits);
        v = make_float4((float)ldexp((double)x[0], e), (float)ldexp((double)x[1], e), (float)ldexp((double)x[2], e),
                        0.f);
    } else {
        v = acc[i * SS_ACC_STRIDE];
    }
    if (v.x == 0.f && v.y == 0.f && v.z == 0.f) return;
    float* d = k < irr_tex ? (d_irr ? d_irr + (sc * irr_tex + k) * 3 : nullptr)
                           : (d_spec ? d_spec + (sc * (texels - irr_tex) + (k - irr_tex)) * 3 : nullptr);
    if (!d) return;
    d[0] += v.x;
    d[1] += v.y;
    d[2] += v.z;
}

void ss_launch_project_bwd(const ss_ws_view& ws, const ss_layout& L, const ss_bwd_args& a, cudaStream_t st) {
    int64_t n = L.scene_begin[L.n_scenes];
    if (n <= 0 || L.total_records <= 0) return;
    const int64_t per_block = a.f.p.pbwd_block ? a.f.p.pbwd_block : 128;   // surfels per CTA (all their views)
    const unsigned blocks = (unsigned)((n + per_block - 1) / per_block);
    ss_note_launch();
    if (ws.det_cap) project_bwd_kernel<true><<<blocks, 128, 0, st>>>(ws, a, n, per_block);
    else project_bwd_kernel<false><<<blocks, 128, 0, st>>>(ws, a, n, per_block);
    if ((a.genv.irr || a.genv.spec) && ws.env_acc) {
        const int64_t total = ws.env_texels * L.n_scenes;
        ss_note_launch();
        env_acc_flush_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            ws.env_acc, ws.env_texels, (int64_t)a.f.ed.irr_width * a.f.ed.irr_height, total, a.genv.irr, a.genv.spec,
            ws.det_cap ? ws.det_maxbits : nullptr, a.det_vmax, a.det_cbits);
    }
}
