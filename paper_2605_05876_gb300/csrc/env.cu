// Split-sum BRDF table and environment prefilter (Sec. 3.4.2, Eq. ibl).
//
// The prefilter is a dense linear operator per output texel: every output
// texel is a normalised weighted sum over all texels of its source map.  It
// is bound by FP32 issue (a few GFLOP per call), not by memory, so one CTA
// owns one output texel and its threads stride over the source texels with
// the per-row / per-column trigonometry staged in shared memory.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "ss3d_internal.cuh"

// ------------------------------------------------------------------------
// BRDF table

#define LUT_NQ 128

// Quadrature nodes on [0, 1]: Gauss-Legendre abscissae t_i mapped through
// the endpoint-clustering map s(t) = t^3 (10 - 15 t + 6 t^2); the host keeps
// them in double so that the nodes next to 0 and 1 keep full relative
// precision, then rounds s_i and the weights w_i s'(t_i) / 2 to float.
struct gl_nodes {
    double s[LUT_NQ];    // xi nodes (double: for tiny alpha the mass sits within 1e-8 of xi = 1)
    double sc[LUT_NQ];   // 1 - s, formed as s(1 - t) (the map is symmetric) to keep precision
    double w[LUT_NQ];
    float sf[LUT_NQ];    // phi nodes
    float wf[LUT_NQ];
};

static gl_nodes make_gl_nodes() {
    gl_nodes g;
    const int n = LUT_NQ;
    double xs[LUT_NQ], ws[LUT_NQ];
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 0; j < n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j + 1.0) * z * p2 - j * p3) / (j + 1);
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-15) break;
        }
        double w = 2.0 / ((1.0 - z * z) * pp * pp);
        xs[i] = -z;
        xs[n - 1 - i] = z;
        ws[i] = ws[n - 1 - i] = w;
    }
    for (int i = 0; i < n; ++i) {
        // t = (x + 1)/2, written so that nodes next to either end keep precision
        double t = xs[i] < 0 ? 0.5 * (1.0 + xs[i]) : 1.0 - 0.5 * (1.0 - xs[i]);
        double u = 1.0 - t;
        g.s[i] = t * t * t * (10.0 - 15.0 * t + 6.0 * t * t);
        g.sc[i] = u * u * u * (10.0 - 15.0 * u + 6.0 * u * u);
        g.w[i] = 0.5 * ws[i] * 30.0 * t * t * u * u;
        g.sf[i] = (float)g.s[i];
        g.wf[i] = (float)g.w[i];
    }
    return g;
}

// beta1 = Int D G (v.h)(1-Fc)/(n.v) dh, beta2 = ... Fc ..., over n.l > 0.
// Variables: cos^2 th_h = (1-xi)/(1+(a^2-1)xi) makes D (n.h) dh = dxi dphi/(2pi);
// phi in [0, phi_max(xi)] by symmetry; xi split where n.l > 0 stops holding
// for all / for some phi (th_h = (pi/2 -+ th_v)/2); nodes clustered at the
// segment ends by t -> t^3 (10 - 15 t + 6 t^2).  FP32 integrand, FP64 sums.
__global__ void __launch_bounds__(256) brdf_lut_kernel(float* lut, int n, gl_nodes g) {
    const int cell = blockIdx.x;
    const int ir = cell / n, im = cell % n;
    const float r = (ir + 0.5f) / n, mu = (im + 0.5f) / n;
    const float alpha = r * r, k = 0.5f * alpha;
    const float sv = sqrtf(fmaxf(0.f, 1.f - mu * mu));
    const float thv = acosf(mu);
    // segment ends in xi, in double (for tiny alpha they sit within 1e-9 of 1)
    double xi_seg[3], om_seg[3];  // segment ends in xi and 1 - xi
    {
        double th[2] = {fmax(0.0, 0.5 * (0.5 * M_PI - (double)thv)), 0.5 * (0.5 * M_PI + (double)thv)};
        xi_seg[0] = 0.0;
        om_seg[0] = 1.0;
        for (int s = 0; s < 2; ++s) {
            double c = cos(th[s]), sn = sin(th[s]);
            double a2c2 = (double)alpha * alpha * c * c;
            xi_seg[s + 1] = sn * sn / (sn * sn + a2c2);
            om_seg[s + 1] = a2c2 / (sn * sn + a2c2);
        }
    }
    const float g1v = mu / (mu * (1.f - k) + k);
    double b1 = 0.0, b2 = 0.0;
    // 2 segments x LUT_NQ xi nodes; each thread takes one (segment, xi) node
    for (int idx = threadIdx.x; idx < 2 * LUT_NQ; idx += blockDim.x) {
        int sg = idx / LUT_NQ, i = idx % LUT_NQ;
        const double lo = xi_seg[sg], hi = xi_seg[sg + 1], om_lo = om_seg[sg], om_hi = om_seg[sg + 1];
        if (!(hi > lo)) continue;
        // the node's polar angle in double: with alpha^2 ~ 1e-10, (alpha^2 - 1) is
        // not representable in FP32 next to 1
        // xi and 1 - xi, each measured from its nearer end
        const double xi = g.s[i] < 0.5 ? lo + (hi - lo) * g.s[i] : hi - (hi - lo) * g.sc[i];
        const double one_m_xi = g.s[i] < 0.5 ? om_lo - (hi - lo) * g.s[i] : om_hi + (hi - lo) * g.sc[i];
        const float wxi = (float)(g.w[i] * (hi - lo));
        const double a2d = (double)alpha * (double)alpha;
        const double den = one_m_xi + a2d * xi;
        const double c2d = one_m_xi / den, s2d = a2d * xi / den;
        if (!(c2d > 0.0)) continue;
        const double ctd = sqrt(c2d), std_ = sqrt(s2d);
        const double Kd = (double)mu / (2.0 * ctd) - (double)mu * ctd;
        double phimax_d;
        if ((double)sv * std_ <= 0.0) {
            phimax_d = Kd < 0.0 ? M_PI : 0.0;
        } else {
            double kap = Kd / ((double)sv * std_);
            phimax_d = kap <= -1.0 ? M_PI : (kap >= 1.0 ? 0.0 : acos(kap));
        }
        if (!(phimax_d > 0.0)) continue;
        const float ct = (float)ctd, st = (float)std_, phimax = (float)phimax_d;
        float acc1 = 0.f, acc2 = 0.f;
        for (int j = 0; j < LUT_NQ; ++j) {
            float phi = phimax * g.sf[j], wphi = g.wf[j] * phimax;
            float vh = sv * st * cosf(phi) + mu * ct;
            float nl = 2.f * vh * ct - mu;
            if (nl <= 0.f || vh <= 0.f) continue;
            float G = g1v * (nl / (nl * (1.f - k) + k));
            // 1 - Fc = 1 - (1 - vh)^5 expanded, so it keeps precision for small vh
            float one_m_Fc = vh * (5.f + vh * (-10.f + vh * (10.f + vh * (-5.f + vh))));
            float om = 1.f - vh, om2 = om * om;
            float Fc = om2 * om2 * om;
            float common = wphi * G * vh / (mu * ct) * (1.f / SS_PI_F);
            acc1 += common * one_m_Fc;
            acc2 += common * Fc;
        }
        b1 += (double)wxi * acc1;
        b2 += (double)wxi * acc2;
    }
    __shared__ double red[2][256];
    red[0][threadIdx.x] = b1;
    red[1][threadIdx.x] = b2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lut[cell * 2 + 0] = (float)red[0][0];
        lut[cell * 2 + 1] = (float)red[1][0];
    }
}

void ss_launch_brdf_lut(float* lut, int n, cudaStream_t st) {
    static gl_nodes g = make_gl_nodes();
    ss_note_launch();
    brdf_lut_kernel<<<n * n, 256, 0, st>>>(lut, n, g);
}

// ------------------------------------------------------------------------
// environment prefilter

void ss_env_level_size(const ss_env_desc* d, int i, int* W, int* H) {
    int w = d->width >> i, h = d->height >> i;
    *W = w < 8 ? 8 : w;
    *H = h < 4 ? 4 : h;
}
int64_t ss_env_irr_floats(const ss_env_desc* d) { return (int64_t)d->irr_width * d->irr_height * 3; }
int64_t ss_env_spec_floats(const ss_env_desc* d) {
    int64_t t = 0;
    for (int i = 0; i < d->n_levels; ++i) {
        int W, H;
        ss_env_level_size(d, i, &W, &H);
        t += (int64_t)W * H * 3;
    }
    return t;
}
// aux per env: irradiance normaliser reciprocals [Hi*Wi], then for each
// level i >= 1: normaliser reciprocals [H_i*W_i] and the box-averaged
// source [H_i*W_i*3].
int64_t ss_env_aux_floats(const ss_env_desc* d) {
    int64_t t = (int64_t)d->irr_width * d->irr_height;
    for (int i = 1; i < d->n_levels; ++i) {
        int W, H;
        ss_env_level_size(d, i, &W, &H);
        t += (int64_t)W * H * 4;
    }
    return t;
}

// Source-map trigonometry staged in shared memory: per column (sin phi,
// cos phi), per row (sin th, cos th, dOmega).
struct src_tables {
    float* sphi;
    float* cphi;
    float* sth;
    float* cth;
    float* dom;
};

__device__ void load_tables(src_tables t, int W, int H) {
    for (int a = threadIdx.x; a < W; a += blockDim.x) {
        float s, c;
        sincospif(2.f * ((a + 0.5f) / W - 0.5f), &s, &c);
        t.sphi[a] = s;
        t.cphi[a] = c;
    }
    for (int b = threadIdx.x; b < H; b += blockDim.x) {
        float s, c;
        sincospif((b + 0.5f) / H, &s, &c);
        t.sth[b] = s;
        t.cth[b] = c;
        // (2 pi / W)(cos th- - cos th+) = (2 pi / W) 2 sin(th_b) sin(pi / 2H)
        t.dom[b] = (2.f * SS_PI_F / W) * 2.f * s * sinpif(0.5f / H);
    }
}

__device__ __forceinline__ void texel_dir(int a, int b, int W, int H, float d[3]) {
    float sp, cp, stt, ctt;
    sincospif(2.f * ((a + 0.5f) / W - 0.5f), &sp, &cp);
    sincospif((b + 0.5f) / H, &stt, &ctt);
    d[0] = stt * sp;
    d[1] = ctt;
    d[2] = -stt * cp;
}

// Weight of source direction wj for output direction wt: diffuse kind uses
// max(0, mu) dOmega; GGX kind uses D(h) max(0, mu) dOmega with
// (n.h)^2 = (1 + mu)/2.  1 - mu is formed as |wt - wj|^2 / 2 (exact for unit
// vectors, no cancellation near the lobe peak).
__device__ __forceinline__ float pf_weight(bool ggx, float a2, const float wt[3], float x, float y, float z,
                                           float dom) {
    float e0 = wt[0] - x, e1 = wt[1] - y, e2 = wt[2] - z;
    float omm = 0.5f * (e0 * e0 + e1 * e1 + e2 * e2);  // 1 - mu
    float mu = 1.f - omm;
    if (!(mu > 0.f)) return 0.f;
    if (!ggx) return mu * dom;
    float one_m_c2 = 0.5f * omm;                        // 1 - (n.h)^2
    float c2 = 1.f - one_m_c2;
    float den = one_m_c2 + c2 * a2;                     // c2 (a2 - 1) + 1
    return a2 * (1.f / SS_PI_F) * __frcp_rn(den * den) * mu * dom;
}

__device__ __forceinline__ float4 block_sum4(float4 v, float4* sh) {
    // warp shuffle then shared
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        v.z += __shfl_xor_sync(0xffffffffu, v.z, o);
        v.w += __shfl_xor_sync(0xffffffffu, v.w, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    float4 r = make_float4(0, 0, 0, 0);
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        r = l < nw ? sh[l] : make_float4(0, 0, 0, 0);
        for (int o = 16; o > 0; o >>= 1) {
            r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
            r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
            r.z += __shfl_xor_sync(0xffffffffu, r.z, o);
            r.w += __shfl_xor_sync(0xffffffffu, r.w, o);
        }
    }
    return r;  // valid in thread 0
}

// One CTA per output texel (blockIdx.x), blockIdx.y = env index.
// out[t] = sum_j w_tj src[j] / sum_j w_tj ; inv_norm[t] = 1 / sum_j w_tj.
__global__ void __launch_bounds__(256) prefilter_fwd_kernel(const float* src, int64_t src_stride, int Ws, int Hs,
                                                            float* out, int64_t out_stride, int Wo, int Ho,
                                                            float* inv_norm, int64_t norm_stride, int ggx,
                                                            float alpha) {
    extern __shared__ float smem[];
    src_tables tb{smem, smem + Ws, smem + 2 * Ws, smem + 2 * Ws + Hs, smem + 2 * Ws + 2 * Hs};
    __shared__ float4 red[8];
    const int e = blockIdx.y;
    const float* S = src + e * src_stride;
    load_tables(tb, Ws, Hs);
    __syncthreads();
    const int t = blockIdx.x;
    float wt[3];
    texel_dir(t % Wo, t / Wo, Wo, Ho, wt);
    const float a2 = alpha * alpha;
    float4 acc = make_float4(0, 0, 0, 0);
    const int n_src = Ws * Hs;
    for (int j = threadIdx.x; j < n_src; j += blockDim.x) {
        int a = j % Ws, b = j / Ws;
        float st = tb.sth[b];
        float w = pf_weight(ggx != 0, a2, wt, st * tb.sphi[a], tb.cth[b], -st * tb.cphi[a], tb.dom[b]);
        if (w != 0.f) {
            const float* s = S + (int64_t)j * 3;
            acc.x = fmaf(w, s[0], acc.x);
            acc.y = fmaf(w, s[1], acc.y);
            acc.z = fmaf(w, s[2], acc.z);
            acc.w += w;
        }
    }
    float4 r = block_sum4(acc, red);
    if (threadIdx.x == 0) {
        float inv = 1.f / r.w;
        float* o = out + e * out_stride + (int64_t)t * 3;
        o[0] = r.x * inv;
        o[1] = r.y * inv;
        o[2] = r.z * inv;
        inv_norm[e * norm_stride + t] = inv;
    }
}

// d_src[j] (+)= sum_t w_tj inv_norm[t] d_out[t]; one CTA per source texel.
// If box > 0, the result is spread over the box x box block of the base map
// (adjoint of the box average), else added to d_src[j] directly.
__global__ void __launch_bounds__(256) prefilter_bwd_kernel(const float* d_out, int64_t dout_stride, int Wo,
                                                            int Ho, const float* inv_norm, int64_t norm_stride,
                                                            int Ws, int Hs, float* d_base, int64_t base_stride,
                                                            int Wb, int bw, int bh, int ggx, float alpha) {
    extern __shared__ float smem[];
    src_tables tb{smem, smem + Wo, smem + 2 * Wo, smem + 2 * Wo + Ho, smem + 2 * Wo + 2 * Ho};
    __shared__ float4 red[8];
    const int e = blockIdx.y;
    // tables of the OUTPUT grid (we loop over outputs)
    load_tables(tb, Wo, Ho);
    __syncthreads();
    const int j = blockIdx.x;
    float wj[3];
    texel_dir(j % Ws, j / Ws, Ws, Hs, wj);
    // dOmega of the source texel
    float sj, cj;
    sincospif((j / Ws + 0.5f) / Hs, &sj, &cj);
    const float domj = (2.f * SS_PI_F / Ws) * 2.f * sj * sinpif(0.5f / Hs);
    const float a2 = alpha * alpha;
    const float* dO = d_out + e * dout_stride;
    const float* inv = inv_norm + e * norm_stride;
    float4 acc = make_float4(0, 0, 0, 0);
    const int n_out = Wo * Ho;
    for (int t = threadIdx.x; t < n_out; t += blockDim.x) {
        int a = t % Wo, b = t / Wo;
        float st = tb.sth[b];
        float wt[3] = {st * tb.sphi[a], tb.cth[b], -st * tb.cphi[a]};
        float w = pf_weight(ggx != 0, a2, wt, wj[0], wj[1], wj[2], domj);
        if (w != 0.f) {
            w *= inv[t];
            const float* g = dO + (int64_t)t * 3;
            acc.x = fmaf(w, g[0], acc.x);
            acc.y = fmaf(w, g[1], acc.y);
            acc.z = fmaf(w, g[2], acc.z);
        }
    }
    float4 r = block_sum4(acc, red);
    if (threadIdx.x == 0) {
        float* D = d_base + e * base_stride;
        int ja = j % Ws, jb = j / Ws;
        float sc = 1.f / (bw * bh);
        for (int y = 0; y < bh; ++y)
            for (int x = 0; x < bw; ++x) {
                float* o = D + ((int64_t)(jb * bh + y) * Wb + (ja * bw + x)) * 3;
                o[0] += r.x * sc;
                o[1] += r.y * sc;
                o[2] += r.z * sc;
            }
    }
}

// box average of the base map into a level-sized source
__global__ void box_down_kernel(const float* env, int64_t env_stride, int We, int He, float* out,
                                int64_t out_stride, int W, int H) {
    int e = blockIdx.y;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= W * H) return;
    int a = idx % W, b = idx / W;
    int bw = We / W, bh = He / H;
    const float* E = env + e * env_stride;
    float s0 = 0, s1 = 0, s2 = 0;
    for (int y = 0; y < bh; ++y)
        for (int x = 0; x < bw; ++x) {
            const float* p = E + ((int64_t)(b * bh + y) * We + (a * bw + x)) * 3;
            s0 += p[0];
            s1 += p[1];
            s2 += p[2];
        }
    float sc = 1.f / (bw * bh);
    float* o = out + e * out_stride + (int64_t)idx * 3;
    o[0] = s0 * sc;
    o[1] = s1 * sc;
    o[2] = s2 * sc;
}

__global__ void copy_level0_kernel(const float* env, int64_t env_stride, float* spec, int64_t spec_stride,
                                   int64_t n) {
    int e = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        spec[e * spec_stride + i] = env[e * env_stride + i];
}

__global__ void add_level0_kernel(const float* d_spec, int64_t spec_stride, float* d_env, int64_t env_stride,
                                  int64_t n) {
    int e = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d_env[e * env_stride + i] += d_spec[e * spec_stride + i];
}

static size_t table_smem(int W, int H) { return sizeof(float) * (2 * W + 3 * H); }

void ss_launch_env_prefilter(const ss_env_desc* d, int n_envs, const float* env, float* irr, float* spec,
                             float* aux, cudaStream_t st) {
    const int We = d->width, He = d->height;
    const int64_t env_stride = (int64_t)We * He * 3;
    const int64_t irr_stride = ss_env_irr_floats(d), spec_stride = ss_env_spec_floats(d),
                  aux_stride = ss_env_aux_floats(d);
    const int Wi = d->irr_width, Hi = d->irr_height;
    dim3 g(Wi * Hi, n_envs);
    ss_note_launch();
    prefilter_fwd_kernel<<<g, 256, table_smem(We, He), st>>>(env, env_stride, We, He, irr, irr_stride, Wi, Hi, aux,
                                                            aux_stride, 0, 0.f);
    ss_note_launch();
    copy_level0_kernel<<<dim3(256, n_envs), 256, 0, st>>>(env, env_stride, spec, spec_stride, env_stride);
    int64_t spec_off = env_stride, aux_off = (int64_t)Wi * Hi;
    for (int i = 1; i < d->n_levels; ++i) {
        int W, H;
        ss_env_level_size(d, i, &W, &H);
        float* norm = aux + aux_off;
        float* src = aux + aux_off + (int64_t)W * H;
        ss_note_launch();
        box_down_kernel<<<dim3((W * H + 255) / 256, n_envs), 256, 0, st>>>(env, env_stride, We, He, src, aux_stride,
                                                                           W, H);
        float r = (float)i / (float)(d->n_levels - 1);
        ss_note_launch();
        prefilter_fwd_kernel<<<dim3(W * H, n_envs), 256, table_smem(W, H), st>>>(
            src, aux_stride, W, H, spec + spec_off, spec_stride, W, H, norm, aux_stride, 1, r * r);
        spec_off += (int64_t)W * H * 3;
        aux_off += (int64_t)W * H * 4;
    }
}

void ss_launch_env_prefilter_bwd(const ss_env_desc* d, int n_envs, const float* d_irr, const float* d_spec,
                                 const float* aux, float* d_env, cudaStream_t st) {
    const int We = d->width, He = d->height;
    const int64_t env_stride = (int64_t)We * He * 3;
    const int64_t irr_stride = ss_env_irr_floats(d), spec_stride = ss_env_spec_floats(d),
                  aux_stride = ss_env_aux_floats(d);
    const int Wi = d->irr_width, Hi = d->irr_height;
    if (d_irr) {
        ss_note_launch();
        prefilter_bwd_kernel<<<dim3(We * He, n_envs), 256, table_smem(Wi, Hi), st>>>(
            d_irr, irr_stride, Wi, Hi, aux, aux_stride, We, He, d_env, env_stride, We, 1, 1, 0, 0.f);
    }
    if (!d_spec) return;
    ss_note_launch();
    add_level0_kernel<<<dim3(256, n_envs), 256, 0, st>>>(d_spec, spec_stride, d_env, env_stride, env_stride);
    int64_t spec_off = env_stride, aux_off = (int64_t)Wi * Hi;
    for (int i = 1; i < d->n_levels; ++i) {
        int W, H;
        ss_env_level_size(d, i, &W, &H);
        const float* norm = aux + aux_off;
        float r = (float)i / (float)(d->n_levels - 1);
        ss_note_launch();
        prefilter_bwd_kernel<<<dim3(W * H, n_envs), 256, table_smem(W, H), st>>>(
            d_spec + spec_off, spec_stride, W, H, norm, aux_stride, W, H, d_env, env_stride, We, We / W, He / H, 1,
            r * r);
        spec_off += (int64_t)W * H * 3;
        aux_off += (int64_t)W * H * 4;
    }
}

// ------------------------------------------------------------------------
// Environment prefilter for callers that cannot allocate device memory.
//
// Some callers only receive input and output buffers from a host
// application (a plugin inside a larger renderer, a module running under a
// fixed memory budget or a pooled allocator that forbids raw cudaMalloc,
// code that must not call cudaMalloc because it synchronises the device).
// They cannot provide the `aux` scratch of ss_env_prefilter, so this entry
// keeps that scratch in a fixed array in device memory that every GPU which
// loads the library holds until the process exits.
#include <mutex>

static __device__ __align__(256) float g_noalloc_aux[SS_NOALLOC_AUX_FLOATS];

static std::mutex g_noalloc_mutex;
static float* g_noalloc_aux_ptr[256] = {};   // device address of the array, per device

extern "C" ss_status ss_env_prefilter_noalloc(const ss_env_desc* d, int32_t n_envs, const float* env_dev,
                                              float* irr_dev, float* spec_dev, void* stream) {
    if (!d || n_envs < 1 || !env_dev || !irr_dev || !spec_dev) return SS_ERR_INVALID_ARG;
    int64_t irr_f, spec_f, aux_f;
    if (ss_env_sizes(d, &irr_f, &spec_f, &aux_f) != SS_OK) return SS_ERR_INVALID_ARG;
    if (aux_f * (int64_t)n_envs > (int64_t)SS_NOALLOC_AUX_FLOATS) return SS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SS_ERR_CUDA;
    float* aux = nullptr;
    {
        // first call on this device: look up the array's device address (the
        // host-side symbol is only a stand-in, not a device pointer)
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_aux_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_aux) != cudaSuccess || !p) return SS_ERR_CUDA;
            g_noalloc_aux_ptr[dev] = (float*)p;
        }
        aux = g_noalloc_aux_ptr[dev];
    }
    // every aux entry is written before it is read: nothing needs clearing
    ss_launch_env_prefilter(d, n_envs, env_dev, irr_dev, spec_dev, aux, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}
