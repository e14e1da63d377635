// Split-sum BRDF table and environment prefilter (Sec. 3.4.2, Eq. ibl).
//
// The prefilter is a dense linear operator: every output texel is a
// normalised weighted sum over all texels of its source map.  Its weight
// depends only on the angle between the two texel directions, so on the
// equirectangular grid each pair of rows contributes a circular convolution
// along phi; the kernels evaluate one weight per (row pair, phi offset) and
// spend the rest of their time in shared-memory multiply-adds (FP32 issue
// bound, a few GFLOP per call).
#include <math.h>
#include <stdio.h>

#include <cooperative_groups.h>
#include <vector>

#include <mutex>

#include "ss3d_internal.cuh"

namespace cg = cooperative_groups;

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

// Row-pair circular convolutions.  Output texel (a, b) of a Wo x Ho map and
// source texel (j, b') of a Ws x Hs map (Ws = r Wo, both equirectangular,
// texel centres at phi = 2 pi ((i + 1/2)/W - 1/2), th = pi (i + 1/2)/H) see
// each other at
//   1 - mu = 2 sin^2((th_b - th_b')/2) + 2 sin th_b sin th_b' sin^2(dphi/2),
//   dphi/2 = pi (2 delta - r + 1) / (2 Ws),  delta = (j - r a) mod Ws,
// so one row pair (b, b') adds a circular convolution along phi whose weights
// depend on delta alone.  Every term of 1 - mu is non-negative, so it keeps
// full relative precision next to the lobe peak, where the GGX weight of a
// low roughness is steepest.

struct conv_row {
    float A, B, dom;   // 2 sin^2((th_b - th_b')/2), 2 sin th_b sin th_b', dOmega of row b'
};

__device__ __forceinline__ conv_row conv_rowpair(int b, int Ho, int bs, int Hs, int Ws) {
    conv_row c;
    // (th_b - th_b') / 2 = pi ((2b + 1) Hs - (2b' + 1) Ho) / (4 Ho Hs); the
    // denominator is exact in float (Hs is a power of two, Ho <= 8192)
    const long long num = (long long)(2 * b + 1) * Hs - (long long)(2 * bs + 1) * Ho;
    const float sa = sinpif((float)num / (float)(4LL * Ho * Hs));
    c.A = 2.f * sa * sa;
    const float so = sinpif((b + 0.5f) / Ho), ss = sinpif((bs + 0.5f) / Hs);
    c.B = 2.f * so * ss;
    // (2 pi / Ws)(cos th- - cos th+) = (2 pi / Ws) 2 sin th_b' sin(pi / 2 Hs)
    c.dom = (2.f * SS_PI_F / Ws) * 2.f * ss * sinpif(0.5f / Hs);
    return c;
}

__device__ __forceinline__ float conv_T(int delta, int r, int Ws) {
    const float s = sinpif((float)(2 * delta - r + 1) / (float)(2 * Ws));   // sin(dphi / 2)
    return s * s;
}

// Weight of one (output, source) pair: diffuse kind max(0, mu) dOmega; GGX
// kind D(h) max(0, mu) dOmega with (n.h)^2 = (1 + mu)/2 (n = v = r).
__device__ __forceinline__ float conv_weight(int ggx, float a2, const conv_row& c, float T) {
    const float omm = fmaf(c.B, T, c.A);   // 1 - mu
    const float mu = 1.f - omm;
    if (!(mu > 0.f)) return 0.f;
    if (!ggx) return mu * c.dom;
    const float h = 0.5f * omm;             // 1 - (n.h)^2
    const float den = fmaf(1.f - h, a2, h); // (n.h)^2 (a2 - 1) + 1
    return a2 * (1.f / SS_PI_F) * __frcp_rn(den * den) * mu * c.dom;
}

// Staged rows are read at stride r or R by consecutive lanes; one pad float
// per 32 keeps those reads free of bank conflicts.
__device__ __forceinline__ int conv_pad(int k) { return k + (k >> 5); }
static inline int conv_pad_h(int k) { return k + (k >> 5); }

// Forward: out[b][a] = sum_{b', j} w src[b'][j] / sum_{b', j} w.
//
// A cluster of KS CTAs owns one (output row b, tile of TA*R outputs, env);
// CTA q of the cluster takes the source rows [q Hs/KS, (q+1) Hs/KS), its
// thread (al, p) the rows p (mod P) of those and the R consecutive outputs
// a0 + R al + t.  The weights of TD offsets delta and the source columns
// they reach are staged in shared memory per row; with R = 4 (r = 1) a
// thread reuses each staged source value for 4 outputs.  The cluster's
// partial sums meet in the leader's reduction through distributed shared
// memory, in a fixed order (deterministic), summed in FP64.
template <int R>
__global__ void __launch_bounds__(256) envconv_fwd_kernel(const float* __restrict__ src, int64_t src_stride, int Ws,
                                                          int Hs, float* out, int64_t out_stride, int Wo, int Ho,
                                                          float* inv_norm, int64_t norm_stride, int ggx, float alpha,
                                                          int TA, int P, int TD, int SCP) {
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) float csm[];
    const int KS = (int)cluster.num_blocks();
    const int q = (int)cluster.block_rank();
    const int r = Ws / Wo;
    const int OT = TA * R;
    const int n_ab = Wo / OT;
    const int tile = blockIdx.x / KS;
    const int b = tile / n_ab, a0 = (tile % n_ab) * OT;
    const int e = blockIdx.y;
    const int al = threadIdx.x % TA, p = threadIdx.x / TA;
    float* wts = csm;               // [P][TD]
    float* srcs = csm + P * TD;     // [P][3][SCP]
    const float* S = src + e * src_stride;
    const float a2 = alpha * alpha;
    const int SC = r * (OT - 1) + TD;
    const int RPC = (Hs + KS - 1) / KS, row0 = q * RPC;
    float acc[R][3];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t][0] = acc[t][1] = acc[t][2] = 0.f;
    float nsum = 0.f;
    for (int i0 = 0; i0 < RPC; i0 += P) {
        const bool row_ok = i0 + p < RPC && row0 + i0 + p < Hs;
        const int bs = row0 + (row_ok ? i0 + p : 0);
        const conv_row c = conv_rowpair(b, Ho, bs, Hs, Ws);
        const float* Srow = S + (int64_t)bs * Ws * 3;
        for (int d0 = 0; d0 < Ws; d0 += TD) {
            for (int i = al; i < TD; i += TA) {
                const float w = row_ok ? conv_weight(ggx, a2, c, conv_T(d0 + i, r, Ws)) : 0.f;
                wts[p * TD + i] = w;
                nsum += w;
            }
            if (row_ok) {
                const int jb = r * a0 + d0;
                for (int k = al; k < SC; k += TA) {
                    const float* g = Srow + (int64_t)((jb + k) & (Ws - 1)) * 3;
                    const int pk = conv_pad(k);
                    srcs[(p * 3 + 0) * SCP + pk] = __ldg(g);
                    srcs[(p * 3 + 1) * SCP + pk] = __ldg(g + 1);
                    srcs[(p * 3 + 2) * SCP + pk] = __ldg(g + 2);
                }
            }
            __syncthreads();
            if (row_ok) {
                const float4* wp = reinterpret_cast<const float4*>(wts + p * TD);
                const float* s0 = srcs + p * 3 * SCP;
                const float* s1 = s0 + SCP;
                const float* s2 = s1 + SCP;
                const int kb = r * R * al;
                float x[R][3][2];
#pragma unroll
                for (int t = 0; t < R; ++t)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) x[t][ch][0] = x[t][ch][1] = 0.f;
                for (int i = 0; i < TD; i += 4) {
                    const float4 w4 = wp[i >> 2];
                    const float w[4] = {w4.x, w4.y, w4.z, w4.w};
                    if constexpr (R == 1) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int pk = conv_pad(kb + i + u);
                            x[0][0][u & 1] = fmaf(w[u], s0[pk], x[0][0][u & 1]);
                            x[0][1][u & 1] = fmaf(w[u], s1[pk], x[0][1][u & 1]);
                            x[0][2][u & 1] = fmaf(w[u], s2[pk], x[0][2][u & 1]);
                        }
                    } else {
                        // r = 1: output t at offset i + u reads source k = kb + t + i + u
                        float v0[R + 3], v1[R + 3], v2[R + 3];
#pragma unroll
                        for (int m = 0; m < R + 3; ++m) {
                            const int pk = conv_pad(kb + i + m);
                            v0[m] = s0[pk];
                            v1[m] = s1[pk];
                            v2[m] = s2[pk];
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int t = 0; t < R; ++t) {
                                x[t][0][u & 1] = fmaf(w[u], v0[u + t], x[t][0][u & 1]);
                                x[t][1][u & 1] = fmaf(w[u], v1[u + t], x[t][1][u & 1]);
                                x[t][2][u & 1] = fmaf(w[u], v2[u + t], x[t][2][u & 1]);
                            }
                    }
                }
#pragma unroll
                for (int t = 0; t < R; ++t)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) acc[t][ch] += x[t][ch][0] + x[t][ch][1];
            }
            __syncthreads();
        }
    }
    // CTA partials: per output over the parts, normaliser over all threads
    const int nt = blockDim.x;
    float* red = csm;                                          // [nt][3R], then [nt] weights
    double* cpart = reinterpret_cast<double*>(csm + ((nt * (3 * R + 1) + 1) & ~1));   // [OT][3], then norm
#pragma unroll
    for (int t = 0; t < R; ++t)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) red[threadIdx.x * 3 * R + t * 3 + ch] = acc[t][ch];
    red[nt * 3 * R + threadIdx.x] = nsum;
    __syncthreads();
    if (p == 0) {
        for (int v = 0; v < 3 * R; ++v) {
            double s = 0.0;
            for (int pp = 0; pp < P; ++pp) s += red[(pp * TA + al) * 3 * R + v];
            cpart[R * al * 3 + v] = s;   // output R al + v / 3, channel v % 3
        }
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nt; ++i) s += red[nt * 3 * R + i];
        cpart[OT * 3] = s;
    }
    cluster.sync();
    if (q == 0) {
        for (int o = threadIdx.x; o < OT; o += nt) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, nrm = 0.0;
            for (int qq = 0; qq < KS; ++qq) {
                const double* pc = cluster.map_shared_rank(cpart, qq);
                t0 += pc[o * 3];
                t1 += pc[o * 3 + 1];
                t2 += pc[o * 3 + 2];
                nrm += pc[OT * 3];
            }
            const double inv = 1.0 / nrm;
            const int a = a0 + o;
            float* po = out + e * out_stride + ((int64_t)b * Wo + a) * 3;
            po[0] = (float)(t0 * inv);
            po[1] = (float)(t1 * inv);
            po[2] = (float)(t2 * inv);
            inv_norm[e * norm_stride + (int64_t)b * Wo + a] = (float)inv;
        }
    }
    cluster.sync();   // peers keep their shared memory until the leader has read it
}

// box average of a map (the base map, or the previous level's source) into a
// level-sized source; averages of block averages are the block average of
// the base map, since every level's blocks tile the previous level's
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

// Adjoint: d_src[b'][j] = sum_{b, a} w(b, b', (j - r a) mod Ws) inv_norm[b][a]
// d_out[b][a], spread over the bw x bh block of the base map that source
// texel was box-averaged from.
//
// A cluster of KS CTAs owns one (source row b', tile of TJ*R columns, env);
// CTA q takes the output rows [q Ho/KS, (q+1) Ho/KS), its thread (jl, p) the
// rows p (mod P) of those and the R consecutive columns j0 + R jl + t.  TAC
// outputs a at a time, the weights of the offset window they reach and the
// scaled upstream values inv_norm d_out are staged in shared memory; with
// R = 4 (r = 1) a thread reuses each staged weight for 4 columns.  The
// leader CTA sums the cluster's partials (FP64, fixed order) and writes the
// base-map block.
template <int R>
__global__ void __launch_bounds__(256) envconv_bwd_kernel(const float* __restrict__ d_out, int64_t dout_stride,
                                                          int Wo, int Ho, const float* __restrict__ inv_norm,
                                                          int64_t norm_stride, int Ws, int Hs, float* d_base,
                                                          int64_t base_stride, int Wb, int bw, int bh, int ggx,
                                                          float alpha, int TJ, int P, int TAC, int WWP) {
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) float csm[];
    const int KS = (int)cluster.num_blocks();
    const int q = (int)cluster.block_rank();
    const int r = Ws / Wo;
    const int JT = TJ * R;
    const int n_jb = Ws / JT;
    const int tile = blockIdx.x / KS;
    const int bs = tile / n_jb, j0 = (tile % n_jb) * JT;
    const int e = blockIdx.y;
    const int jl = threadIdx.x % TJ, p = threadIdx.x / TJ;
    const int WW = JT + r * (TAC - 1);
    float4* gs = reinterpret_cast<float4*>(csm);   // [P][TAC]
    float* wwin = csm + 4 * P * TAC;                // [P][WWP]
    const float* dO = d_out + e * dout_stride;
    const float* inv = inv_norm + e * norm_stride;
    const float a2 = alpha * alpha;
    const int RPC = (Ho + KS - 1) / KS, row0 = q * RPC;
    float acc[R][3];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t][0] = acc[t][1] = acc[t][2] = 0.f;
    for (int i0 = 0; i0 < RPC; i0 += P) {
        const bool row_ok = i0 + p < RPC && row0 + i0 + p < Ho;
        const int b = row0 + (row_ok ? i0 + p : 0);
        const conv_row c = conv_rowpair(b, Ho, bs, Hs, Ws);
        for (int c0 = 0; c0 < Wo; c0 += TAC) {
            // window entry k holds delta = (dstart + k) mod Ws
            const int dstart = j0 - r * (c0 + TAC - 1);
            for (int k = jl; k < WW; k += TJ) {
                const float w = row_ok ? conv_weight(ggx, a2, c, conv_T((dstart + k) & (Ws - 1), r, Ws)) : 0.f;
                wwin[p * WWP + (R > 1 ? conv_pad(k) : k)] = w;
            }
            for (int u = jl; u < TAC; u += TJ) {
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row_ok) {
                    const int64_t t = (int64_t)b * Wo + c0 + u;
                    const float s = __ldg(inv + t);
                    g = make_float4(__ldg(dO + t * 3) * s, __ldg(dO + t * 3 + 1) * s, __ldg(dO + t * 3 + 2) * s, 0.f);
                }
                gs[p * TAC + u] = g;
            }
            __syncthreads();
            if (row_ok) {
                const float* wp = wwin + p * WWP;
                const float4* gp = gs + p * TAC;
                // column t of this thread and output c0 + u meet at k = kb + t - u
                const int kb = R * jl + r * (TAC - 1);
                float x[R][3][2];
#pragma unroll
                for (int t = 0; t < R; ++t)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) x[t][ch][0] = x[t][ch][1] = 0.f;
                if constexpr (R == 1) {
                    for (int u = 0; u < TAC; ++u) {   // TAC <= 64 terms per chain
                        const float w = wp[kb - r * u];
                        const float4 g = gp[u];
                        x[0][0][0] = fmaf(w, g.x, x[0][0][0]);
                        x[0][1][0] = fmaf(w, g.y, x[0][1][0]);
                        x[0][2][0] = fmaf(w, g.z, x[0][2][0]);
                    }
                } else {
                    for (int u = 0; u < TAC; u += 4) {
                        // k = kb + t - (u + v) = (kb - u - 3) + m with m = t - v + 3
                        float wv[R + 3];
#pragma unroll
                        for (int m = 0; m < R + 3; ++m) wv[m] = wp[conv_pad(kb - u - 3 + m)];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const float4 g = gp[u + v];
#pragma unroll
                            for (int t = 0; t < R; ++t) {
                                const float w = wv[t - v + 3];
                                x[t][0][v & 1] = fmaf(w, g.x, x[t][0][v & 1]);
                                x[t][1][v & 1] = fmaf(w, g.y, x[t][1][v & 1]);
                                x[t][2][v & 1] = fmaf(w, g.z, x[t][2][v & 1]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int t = 0; t < R; ++t)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) acc[t][ch] += x[t][ch][0] + x[t][ch][1];
            }
            __syncthreads();
        }
    }
    const int nt = blockDim.x;
    float* red = csm;                                                              // [nt][3R]
    double* cpart = reinterpret_cast<double*>(csm + ((nt * 3 * R + 1) & ~1));     // [JT][3]
#pragma unroll
    for (int t = 0; t < R; ++t)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) red[threadIdx.x * 3 * R + t * 3 + ch] = acc[t][ch];
    __syncthreads();
    if (p == 0) {
        for (int v = 0; v < 3 * R; ++v) {
            double s = 0.0;
            for (int pp = 0; pp < P; ++pp) s += red[(pp * TJ + jl) * 3 * R + v];
            cpart[R * jl * 3 + v] = s;
        }
    }
    cluster.sync();
    if (q == 0) {
        const double sc = 1.0 / (bw * bh);
        float* D = d_base + e * base_stride;
        for (int o = threadIdx.x; o < JT; o += nt) {
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int qq = 0; qq < KS; ++qq) {
                const double* pc = cluster.map_shared_rank(cpart, qq);
                t0 += pc[o * 3];
                t1 += pc[o * 3 + 1];
                t2 += pc[o * 3 + 2];
            }
            cpart[o * 3] = t0 * sc;   // own partials are no longer read by anyone
            cpart[o * 3 + 1] = t1 * sc;
            cpart[o * 3 + 2] = t2 * sc;
        }
        __syncthreads();
        // spread over the bw x bh base texels of each column, all threads
        const int per = bw * bh;
        for (int idx = threadIdx.x; idx < JT * per; idx += nt) {
            const int o = idx / per, y = (idx % per) / bw, x = idx % bw;
            float* po = D + ((int64_t)(bs * bh + y) * Wb + ((j0 + o) * bw + x)) * 3;
            // atomic: the level convolutions run side by side into one map
            atomicAdd(po, (float)cpart[o * 3]);
            atomicAdd(po + 1, (float)cpart[o * 3 + 1]);
            atomicAdd(po + 2, (float)cpart[o * 3 + 2]);
        }
    }
    cluster.sync();
}

// launch shapes: power-of-two block sizes, clusters of <= 8 CTAs, <= 48 KB of
// shared memory per CTA
static const int CONV_SMEM = 48 * 1024;
static const int CONV_KS = 8;

static int pow2_floor(int x) {
    int p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

template <typename... KArgs, typename... Args>
static void launch_cluster(void (*kern)(KArgs...), dim3 grid, int block, int smem, int ks, cudaStream_t st,
                           Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ks;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ss_note_launch();
    cudaLaunchKernelEx(&cfg, kern, args...);
}

static void launch_conv_fwd(const float* src, int64_t src_stride, int Ws, int Hs, float* out, int64_t out_stride,
                            int Wo, int Ho, float* inv_norm, int64_t norm_stride, int ggx, float alpha, int n_envs,
                            cudaStream_t st) {
    const int r = Ws / Wo;
    const int R = (r == 1 && Wo >= 128) ? 8 : (r == 1 && Wo >= 64) ? 4 : 1;
    const int TA = (Wo / R < 256 / R) ? Wo / R : 256 / R;
    const int OT = TA * R;
    const int TD = Ws < 256 ? Ws : 256;
    const int SC = r * (OT - 1) + TD;
    const int SCP = conv_pad_h(SC - 1) + 1;
    const int per_part = (TD + 3 * SCP) * (int)sizeof(float);
    int P = 256 / TA;
    if (P > Hs) P = Hs;
    if (P * per_part > CONV_SMEM) P = CONV_SMEM / per_part;
    P = pow2_floor(P < 1 ? 1 : P);
    int KS = Hs / P;
    if (KS > CONV_KS) KS = CONV_KS;
    KS = pow2_floor(KS < 1 ? 1 : KS);
    const int nt = TA * P;
    int smem = P * per_part;
    const int red = (((nt * (3 * R + 1) + 1) & ~1) + 2 * (OT * 3 + 1)) * (int)sizeof(float);
    if (smem < red) smem = red;
    const dim3 grid(Ho * (Wo / OT) * KS, n_envs);
    if (R == 8)
        launch_cluster(envconv_fwd_kernel<8>, grid, nt, smem, KS, st, src, src_stride, Ws, Hs, out, out_stride, Wo, Ho,
                       inv_norm, norm_stride, ggx, alpha, TA, P, TD, SCP);
    else if (R == 4)
        launch_cluster(envconv_fwd_kernel<4>, grid, nt, smem, KS, st, src, src_stride, Ws, Hs, out, out_stride, Wo, Ho,
                       inv_norm, norm_stride, ggx, alpha, TA, P, TD, SCP);
    else
        launch_cluster(envconv_fwd_kernel<1>, grid, nt, smem, KS, st, src, src_stride, Ws, Hs, out, out_stride, Wo, Ho,
                       inv_norm, norm_stride, ggx, alpha, TA, P, TD, SCP);
}

static void launch_conv_bwd(const float* d_out, int64_t dout_stride, int Wo, int Ho, const float* inv_norm,
                            int64_t norm_stride, int Ws, int Hs, float* d_base, int64_t base_stride, int Wb, int bw,
                            int bh, int ggx, float alpha, int n_envs, cudaStream_t st) {
    const int r = Ws / Wo;
    const int R = (r == 1 && Ws >= 64) ? 4 : 1;
    const int TJ = (Ws / R < 256 / R) ? Ws / R : 256 / R;
    const int JT = TJ * R;
    const int TAC = Wo < 64 ? Wo : 64;
    const int WW = JT + r * (TAC - 1);
    const int WWP = R > 1 ? conv_pad_h(WW - 1) + 1 : WW;
    const int per_part = (4 * TAC + WWP) * (int)sizeof(float);
    int P = 256 / TJ;
    if (P > Ho) P = Ho;
    if (P * per_part > CONV_SMEM) P = CONV_SMEM / per_part;
    P = pow2_floor(P < 1 ? 1 : P);
    int KS = Ho / P;
    if (KS > CONV_KS) KS = CONV_KS;
    KS = pow2_floor(KS < 1 ? 1 : KS);
    const int nt = TJ * P;
    int smem = P * per_part;
    const int red = (((nt * 3 * R + 1) & ~1) + 2 * JT * 3) * (int)sizeof(float);
    if (smem < red) smem = red;
    const dim3 grid(Hs * (Ws / JT) * KS, n_envs);
    if (R == 4)
        launch_cluster(envconv_bwd_kernel<4>, grid, nt, smem, KS, st, d_out, dout_stride, Wo, Ho, inv_norm,
                       norm_stride, Ws, Hs, d_base, base_stride, Wb, bw, bh, ggx, alpha, TJ, P, TAC, WWP);
    else
        launch_cluster(envconv_bwd_kernel<1>, grid, nt, smem, KS, st, d_out, dout_stride, Wo, Ho, inv_norm,
                       norm_stride, Ws, Hs, d_base, base_stride, Wb, bw, bh, ggx, alpha, TJ, P, TAC, WWP);
}

// Side streams of one device on which the prefilter's convolutions run side
// by side (each is too small to fill the GPU alone), forked from and joined
// back to the caller's stream with events, so stream capture records them as
// parallel branches.  Created on first use; fork and join are serialised by a
// mutex so that concurrent callers never mix their events.
#define SS_SIDE_STREAMS 8
struct ss_side {
    cudaStream_t s[SS_SIDE_STREAMS];
    cudaEvent_t fork, join[SS_SIDE_STREAMS];
    bool ok;
};
static std::mutex g_side_mutex;
static ss_side g_side[64];
static bool g_side_init[64];

static ss_side* side_streams_locked(int dev, cudaStream_t st) {
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_side_init[dev]) {
        // creating streams inside a stream capture could end the caller's
        // capture: a call captured before any eager one runs on `st` alone
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
        g_side_init[dev] = true;
        ss_side& x = g_side[dev];
        x.ok = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < SS_SIDE_STREAMS && x.ok; ++i)
            x.ok = cudaStreamCreateWithFlags(&x.s[i], cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&x.join[i], cudaEventDisableTiming) == cudaSuccess;
    }
    return g_side[dev].ok ? &g_side[dev] : nullptr;
}

void ss_launch_env_prefilter(const ss_env_desc* d, int n_envs, const float* env, float* irr, float* spec,
                             float* aux, cudaStream_t st) {
    const int We = d->width, He = d->height;
    const int64_t env_stride = (int64_t)We * He * 3;
    const int64_t irr_stride = ss_env_irr_floats(d), spec_stride = ss_env_spec_floats(d),
                  aux_stride = ss_env_aux_floats(d);
    const int Wi = d->irr_width, Hi = d->irr_height;
    ss_note_launch();
    copy_level0_kernel<<<dim3(256, n_envs), 256, 0, st>>>(env, env_stride, spec, spec_stride, env_stride);
    // sources of the specular levels: the cascade of box filters
    {
        int64_t aux_off = (int64_t)Wi * Hi;
        const float* prev = env;
        int64_t prev_stride = env_stride;
        int Wp = We, Hp = He;
        for (int i = 1; i < d->n_levels; ++i) {
            int W, H;
            ss_env_level_size(d, i, &W, &H);
            float* src = aux + aux_off + (int64_t)W * H;
            ss_note_launch();
            box_down_kernel<<<dim3((W * H + 255) / 256, n_envs), 256, 0, st>>>(prev, prev_stride, Wp, Hp, src,
                                                                               aux_stride, W, H);
            prev = src;
            prev_stride = aux_stride;
            Wp = W;
            Hp = H;
            aux_off += (int64_t)W * H * 4;
        }
    }
    // the convolutions (irradiance, specular levels 1 .. L-1) write disjoint
    // outputs: level i on side stream i - 1, the irradiance map on `st`
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_side_mutex);
    ss_side* sd = side_streams_locked(dev, st);
    const bool fork = sd && d->n_levels - 1 <= SS_SIDE_STREAMS && cudaEventRecord(sd->fork, st) == cudaSuccess;
    int64_t spec_off = env_stride, aux_off = (int64_t)Wi * Hi;
    for (int i = 1; i < d->n_levels; ++i) {
        int W, H;
        ss_env_level_size(d, i, &W, &H);
        float* norm = aux + aux_off;
        float* src = aux + aux_off + (int64_t)W * H;
        float r = (float)i / (float)(d->n_levels - 1);
        cudaStream_t si = st;
        if (fork) {
            si = sd->s[i - 1];
            cudaStreamWaitEvent(si, sd->fork, 0);
        }
        launch_conv_fwd(src, aux_stride, W, H, spec + spec_off, spec_stride, W, H, norm, aux_stride, 1, r * r, n_envs,
                        si);
        if (fork) cudaEventRecord(sd->join[i - 1], si);
        spec_off += (int64_t)W * H * 3;
        aux_off += (int64_t)W * H * 4;
    }
    launch_conv_fwd(env, env_stride, We, He, irr, irr_stride, Wi, Hi, aux, aux_stride, 0, 0.f, n_envs, st);
    if (fork)
        for (int i = 1; i < d->n_levels; ++i) cudaStreamWaitEvent(st, sd->join[i - 1], 0);
}

void ss_launch_env_prefilter_bwd(const ss_env_desc* d, int n_envs, const float* d_irr, const float* d_spec,
                                 const float* aux, float* d_env, cudaStream_t st, bool ordered) {
    const int We = d->width, He = d->height;
    const int64_t env_stride = (int64_t)We * He * 3;
    const int64_t irr_stride = ss_env_irr_floats(d), spec_stride = ss_env_spec_floats(d),
                  aux_stride = ss_env_aux_floats(d);
    const int Wi = d->irr_width, Hi = d->irr_height;
    if (d_spec) {
        ss_note_launch();
        add_level0_kernel<<<dim3(256, n_envs), 256, 0, st>>>(d_spec, spec_stride, d_env, env_stride, env_stride);
    }
    // the transposed convolutions add into d_env with atomics: specular levels
    // on the side streams, the irradiance map on `st`
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_side_mutex);
    ss_side* sd = (d_spec && !ordered) ? side_streams_locked(dev, st) : nullptr;
    const bool fork = sd && d->n_levels - 1 <= SS_SIDE_STREAMS && cudaEventRecord(sd->fork, st) == cudaSuccess;
    if (d_spec) {
        int64_t spec_off = env_stride, aux_off = (int64_t)Wi * Hi;
        for (int i = 1; i < d->n_levels; ++i) {
            int W, H;
            ss_env_level_size(d, i, &W, &H);
            const float* norm = aux + aux_off;
            float r = (float)i / (float)(d->n_levels - 1);
            cudaStream_t si = st;
            if (fork) {
                si = sd->s[i - 1];
                cudaStreamWaitEvent(si, sd->fork, 0);
            }
            launch_conv_bwd(d_spec + spec_off, spec_stride, W, H, norm, aux_stride, W, H, d_env, env_stride, We,
                            We / W, He / H, 1, r * r, n_envs, si);
            if (fork) cudaEventRecord(sd->join[i - 1], si);
            spec_off += (int64_t)W * H * 3;
            aux_off += (int64_t)W * H * 4;
        }
    }
    if (d_irr)
        launch_conv_bwd(d_irr, irr_stride, Wi, Hi, aux, aux_stride, We, He, d_env, env_stride, We, 1, 1, 0, 0.f, n_envs,
                        st);
    if (fork)
        for (int i = 1; i < d->n_levels; ++i) cudaStreamWaitEvent(st, sd->join[i - 1], 0);
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
        // host-side symbol is only a stand-in, not a device pointer).  It is
        // kept for the life of the process: it stays valid as long as the
        // device's context does (a cudaDeviceReset ends it).
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_aux_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_aux) != cudaSuccess || !p) return SS_ERR_CUDA;
            g_noalloc_aux_ptr[dev] = (float*)p;
        }
        aux = g_noalloc_aux_ptr[dev];
    }
    // every aux entry is written before it is read: nothing needs clearing
    {
        ss_stage_scope sc(5, (cudaStream_t)stream);   // timed as the prefilter stage
        ss_launch_env_prefilter(d, n_envs, env_dev, irr_dev, spec_dev, aux, (cudaStream_t)stream);
    }
    if (cudaGetLastError() != cudaSuccess) return SS_ERR_CUDA;
    return SS_OK;
}
