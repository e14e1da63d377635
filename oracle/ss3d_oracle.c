/*
 * FP64 CPU oracle for the 3D Surface Splatting (3DSS) renderer -- TEST
 * INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  It shares
 * no code with the CUDA path; both read the same seeded inputs.
 *
 * This file holds the parts of the oracle that are loops over pixels or
 * texels (plain C, double precision, OpenMP over independent outputs):
 *
 *   oref_brdf_lut         split-sum BRDF table (beta1, beta2) of Sec. 3.4.2,
 *                         Eq. ibl, by Gauss-Legendre quadrature;
 *   oref_env_prefilter    diffuse irradiance map and roughness-indexed
 *                         specular levels (Sec. 3.4.2 "pre-convolved diffuse
 *                         environment map", "pre-filtered specular radiance
 *                         ... at a MIP level determined by the roughness");
 *   oref_env_adjoint      the transpose of that linear operator;
 *   oref_fragments        per-pixel discrete decisions of Algorithm 1: which
 *                         surfels cover a pixel (Eq. rho2 / Eq. mip_weight
 *                         cutoff), their order by z_start (Sec. 3.2.1) and the
 *                         surface layer each belongs to, capped at
 *                         K_max layers (App. A "Maximum layer count").
 *
 * The differentiable values (weights, Shepard sums, coverage, compositing)
 * are computed from these decisions in oracle/model.py with PyTorch FP64.
 *
 * Readings where the paper is silent (equirect convention, level sizes,
 * normalised prefilter sums, GGX/Smith forms) are restated next to each
 * function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Equirectangular convention.  Direction d <-> (phi = atan2(d_x, -d_z),
 * theta = acos(d_y)); texel (a, b) of a W x H map has its centre at
 * u = (a + 0.5) / W, v = (b + 0.5) / H with phi = 2 pi (u - 1/2),
 * theta = pi v.  Its solid angle is (2 pi / W)(cos th_b^- - cos th_b^+). */

static void texel_dir(int a, int b, int W, int H, double d[3]) {
    double phi = 2.0 * M_PI * ((a + 0.5) / W - 0.5);
    double th = M_PI * (b + 0.5) / H;
    d[0] = sin(th) * sin(phi);
    d[1] = cos(th);
    d[2] = -sin(th) * cos(phi);
}

static double texel_solid_angle(int b, int W, int H) {
    double t0 = M_PI * b / H, t1 = M_PI * (b + 1) / H;
    return (2.0 * M_PI / W) * (cos(t0) - cos(t1));
}

/* GGX normal distribution D(h) as a function of c2 = (n.h)^2, alpha = r^2. */
static double ggx_D(double c2, double alpha) {
    double a2 = alpha * alpha;
    double den = c2 * (a2 - 1.0) + 1.0;
    return a2 / (M_PI * den * den);
}

/* Smith-Schlick G1 with k = alpha / 2. */
static double smith_G1(double x, double k) { return x / (x * (1.0 - k) + k); }

/* ------------------------------------------------------------------------ */
/* Split-sum BRDF table (Eq. ibl: F0 beta1 + beta2).  For view v with
 * n.v = mu and roughness r (alpha = r^2):
 *   beta1 = Int D(h) G(v,l) (v.h) (1 - Fc) / (n.v) dh,
 *   beta2 = Int D(h) G(v,l) (v.h) Fc / (n.v) dh,   Fc = (1 - v.h)^5,
 * over half vectors h with n.l > 0, l = 2 (v.h) h - v.  (This is the
 * Cook-Torrance specular integral  Int f (n.l) dl  split by Schlick's
 * Fresnel F = F0 (1 - Fc) + Fc, after the change of variable dl = 4 (v.h) dh.)
 *
 * Quadrature: substitute cos^2 th_h = (1 - xi) / (1 + (alpha^2 - 1) xi), under
 * which D(h) (n.h) dh = dxi dphi / (2 pi); the integrand over the unit square
 * is then G (v.h) F-term / ((n.v)(n.h)) / (2 pi).  It is even in phi, so phi
 * runs over [0, phi_max(xi)] (phi_max: where n.l changes sign) and the result
 * is doubled.  With th_v = acos(mu), n.l > 0 holds for every phi when
 * th_h < (pi/2 - th_v)/2 and for none when th_h > (pi/2 + th_v)/2 (at
 * phi = pi and 0, n.l = cos(th_v +- 2 th_h)), so the xi range is split at
 * those two angles.  Each 1D integral uses Gauss-Legendre on nodes clustered
 * at both ends by t -> t^3 (10 - 15 t + 6 t^2), which absorbs the endpoint
 * behaviour (converges to ~1e-8 at nq = 128).
 *
 * oref_brdf_eval evaluates m arbitrary (mu, r) pairs into out[m][2];
 * oref_brdf_lut fills lut[(ir * n + im) * 2 + {0,1}] at the cell centres
 * r = (ir+0.5)/n, mu = (im+0.5)/n.
 */
static double smoother(double t, double* dt) {
    *dt = 30.0 * t * t * (1.0 - t) * (1.0 - t);
    return t * t * t * (10.0 - 15.0 * t + 6.0 * t * t);
}

static double xi_of_theta(double th, double alpha) {
    double c2 = cos(th) * cos(th);
    return (1.0 - c2) / (1.0 - c2 + alpha * alpha * c2);
}

static void brdf_integral(double mu, double r, int nq, const double* gl_x, const double* gl_w,
                          double* b1_out, double* b2_out) {
    double alpha = r * r, k = alpha / 2.0;
    double sv = sqrt(1.0 - mu * mu); /* v = (sv, 0, mu) */
    double thv = acos(mu);
    double th1 = 0.5 * (0.5 * M_PI - thv), th2 = 0.5 * (0.5 * M_PI + thv);
    double seg[3] = {0.0, xi_of_theta(th1 > 0.0 ? th1 : 0.0, alpha), xi_of_theta(th2, alpha)};
    double b1 = 0.0, b2 = 0.0;
    for (int sgi = 0; sgi < 2; ++sgi) {
        double lo = seg[sgi], hi = seg[sgi + 1];
        if (!(hi > lo)) continue;
        for (int i = 0; i < nq; ++i) {
            double dti, ti = smoother(0.5 * (gl_x[i] + 1.0), &dti);
            double xi = lo + (hi - lo) * ti, wxi = 0.5 * gl_w[i] * (hi - lo) * dti;
            double c2 = (1.0 - xi) / (1.0 + (alpha * alpha - 1.0) * xi);
            if (c2 <= 0.0) continue;
            double ct = sqrt(c2), st = sqrt(fmax(0.0, 1.0 - c2));
            /* n.l > 0  <=>  2 (v.h) ct > mu  <=>  sv st cos(phi) > mu/(2ct) - mu ct */
            double K = mu / (2.0 * ct) - mu * ct;
            double phimax;
            if (sv * st <= 0.0) {
                phimax = (K < 0.0) ? M_PI : 0.0;
            } else {
                double kap = K / (sv * st);
                phimax = (kap <= -1.0) ? M_PI : (kap >= 1.0 ? 0.0 : acos(kap));
            }
            if (phimax <= 0.0) continue;
            for (int j = 0; j < nq; ++j) {
                double dtj, tj = smoother(0.5 * (gl_x[j] + 1.0), &dtj);
                double phi = phimax * tj, wphi = 0.5 * gl_w[j] * phimax * dtj;
                double vh = sv * st * cos(phi) + mu * ct; /* h = (st cos phi, st sin phi, ct) */
                double nl = 2.0 * vh * ct - mu;
                if (nl <= 0.0 || vh <= 0.0) continue;
                double G = smith_G1(mu, k) * smith_G1(nl, k);
                double Fc = pow(1.0 - vh, 5.0);
                double common = G * vh / (mu * ct) / (2.0 * M_PI) * 2.0; /* x2: phi symmetry */
                b1 += wxi * wphi * common * (1.0 - Fc);
                b2 += wxi * wphi * common * Fc;
            }
        }
    }
    *b1_out = b1;
    *b2_out = b2;
}

void oref_brdf_eval(int m, const double* mu, const double* r, int nq, const double* gl_x,
                    const double* gl_w, double* out) {
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < m; ++i) brdf_integral(mu[i], r[i], nq, gl_x, gl_w, out + 2 * i, out + 2 * i + 1);
}

void oref_brdf_lut(int n, int nq, const double* gl_x, const double* gl_w, double* lut) {
#pragma omp parallel for schedule(dynamic)
    for (int cell = 0; cell < n * n; ++cell) {
        int ir = cell / n, im = cell % n;
        brdf_integral((im + 0.5) / n, (ir + 0.5) / n, nq, gl_x, gl_w, lut + 2 * cell, lut + 2 * cell + 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Environment prefilter (the "pre-convolved diffuse environment map" and the
 * roughness-indexed specular levels of Sec. 3.4.2).
 *
 * Irradiance (Wi x Hi): L_d(n_t) = sum_j L_j max(0, n_t.w_j) dW_j
 *                                  / sum_j max(0, n_t.w_j) dW_j
 * over all base texels j (a constant map is a fixed point).
 *
 * Specular levels i = 0..L-1, roughness r_i = i/(L-1), size
 * (max(We>>i, 8), max(He>>i, 4)).  Level 0 is the base map.  Level i >= 1:
 * the source S is the base map box-averaged to the level's size; with the
 * split-sum assumption n = v = w_t, h_j = normalize(w_t + w_j), n.h_j squared
 * is (1 + w_t.w_j) / 2, and
 *   L_i(w_t) = sum_j S_j D(h_j) max(0, w_t.w_j) dW_j / sum_j D(h_j) max(0, w_t.w_j) dW_j.
 *
 * spec_out holds the levels one after the other, each [H_i][W_i][3].
 * Both are linear in the base map; oref_env_adjoint applies the transpose.
 */
static void level_size(int i, int We, int He, int* W, int* H) {
    int w = We >> i, h = He >> i;
    *W = w < 8 ? 8 : w;
    *H = h < 4 ? 4 : h;
}

long long oref_spec_levels_size(int We, int He, int L) {
    long long tot = 0;
    for (int i = 0; i < L; ++i) {
        int W, H;
        level_size(i, We, He, &W, &H);
        tot += (long long)W * H * 3;
    }
    return tot;
}

/* Box average of the base map to (W, H): plain mean of each block. */
static void box_down(const double* env, int We, int He, int W, int H, double* out) {
    int bw = We / W, bh = He / H;
    for (int b = 0; b < H; ++b)
        for (int a = 0; a < W; ++a)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int y = 0; y < bh; ++y)
                    for (int x = 0; x < bw; ++x) s += env[((b * bh + y) * We + (a * bw + x)) * 3 + c];
                out[(b * W + a) * 3 + c] = s / (bw * bh);
            }
}

static void box_down_adjoint(const double* d_small, int W, int H, int We, int He, double* d_env) {
    int bw = We / W, bh = He / H;
    for (int b = 0; b < H; ++b)
        for (int a = 0; a < W; ++a)
            for (int c = 0; c < 3; ++c) {
                double g = d_small[(b * W + a) * 3 + c] / (bw * bh);
                for (int y = 0; y < bh; ++y)
                    for (int x = 0; x < bw; ++x) d_env[((b * bh + y) * We + (a * bw + x)) * 3 + c] += g;
            }
}

/* weight of source texel j (direction wj, solid angle dW) for output
 * direction wt: diffuse (kind 0) or GGX with alpha (kind 1). */
static double pf_weight(int kind, double alpha, const double* wt, const double* wj, double dW) {
    double mu = wt[0] * wj[0] + wt[1] * wj[1] + wt[2] * wj[2];
    if (mu <= 0.0) return 0.0;
    if (kind == 0) return mu * dW;
    double c2 = 0.5 * (1.0 + mu);
    return ggx_D(c2, alpha) * mu * dW;
}

/* out[t] = sum_j w_tj src[j] / sum_j w_tj  (forward) */
static void pf_apply(int kind, double alpha, const double* src, int Ws, int Hs, double* out, int Wo,
                     int Ho) {
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < Wo * Ho; ++t) {
        double wt[3], wj[3];
        texel_dir(t % Wo, t / Wo, Wo, Ho, wt);
        double acc[3] = {0, 0, 0}, norm = 0.0;
        for (int j = 0; j < Ws * Hs; ++j) {
            texel_dir(j % Ws, j / Ws, Ws, Hs, wj);
            double w = pf_weight(kind, alpha, wt, wj, texel_solid_angle(j / Ws, Ws, Hs));
            if (w == 0.0) continue;
            norm += w;
            for (int c = 0; c < 3; ++c) acc[c] += w * src[j * 3 + c];
        }
        for (int c = 0; c < 3; ++c) out[t * 3 + c] = acc[c] / norm;
    }
}

/* d_src[j] += sum_t w_tj / norm_t d_out[t]  (transpose of pf_apply) */
static void pf_adjoint(int kind, double alpha, const double* d_out, int Wo, int Ho, double* d_src,
                       int Ws, int Hs) {
    double* norm = (double*)calloc((size_t)Wo * Ho, sizeof(double));
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < Wo * Ho; ++t) {
        double wt[3], wj[3], s = 0.0;
        texel_dir(t % Wo, t / Wo, Wo, Ho, wt);
        for (int j = 0; j < Ws * Hs; ++j) {
            texel_dir(j % Ws, j / Ws, Ws, Hs, wj);
            s += pf_weight(kind, alpha, wt, wj, texel_solid_angle(j / Ws, Ws, Hs));
        }
        norm[t] = s;
    }
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < Ws * Hs; ++j) {
        double wt[3], wj[3];
        texel_dir(j % Ws, j / Ws, Ws, Hs, wj);
        double dW = texel_solid_angle(j / Ws, Ws, Hs);
        double acc[3] = {0, 0, 0};
        for (int t = 0; t < Wo * Ho; ++t) {
            texel_dir(t % Wo, t / Wo, Wo, Ho, wt);
            double w = pf_weight(kind, alpha, wt, wj, dW);
            if (w == 0.0) continue;
            for (int c = 0; c < 3; ++c) acc[c] += w / norm[t] * d_out[t * 3 + c];
        }
        for (int c = 0; c < 3; ++c) d_src[j * 3 + c] += acc[c];
    }
    free(norm);
}

void oref_env_prefilter(const double* env, int We, int He, int Wi, int Hi, int L, double* irr,
                        double* spec) {
    pf_apply(0, 0.0, env, We, He, irr, Wi, Hi);
    long long off = 0;
    for (int i = 0; i < L; ++i) {
        int W, H;
        level_size(i, We, He, &W, &H);
        if (i == 0) {
            memcpy(spec, env, sizeof(double) * (size_t)We * He * 3);
        } else {
            double r = (double)i / (L - 1);
            double* src = (double*)malloc(sizeof(double) * (size_t)W * H * 3);
            box_down(env, We, He, W, H, src);
            pf_apply(1, r * r, src, W, H, spec + off, W, H);
            free(src);
        }
        off += (long long)W * H * 3;
    }
}

/* d_env += P^T (d_irr, d_spec) */
void oref_env_adjoint(const double* d_irr, const double* d_spec, int We, int He, int Wi, int Hi,
                      int L, double* d_env) {
    pf_adjoint(0, 0.0, d_irr, Wi, Hi, d_env, We, He);
    long long off = 0;
    for (int i = 0; i < L; ++i) {
        int W, H;
        level_size(i, We, He, &W, &H);
        if (i == 0) {
            for (long long k = 0; k < (long long)We * He * 3; ++k) d_env[k] += d_spec[k];
        } else {
            double r = (double)i / (L - 1);
            double* d_src = (double*)calloc((size_t)W * H * 3, sizeof(double));
            pf_adjoint(1, r * r, d_spec + off, W, H, d_src, W, H);
            box_down_adjoint(d_src, W, H, We, He, d_env);
            free(d_src);
        }
        off += (long long)W * H * 3;
    }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel decisions of Algorithm 1.
 *
 * Surfel i (already transformed for this view) is given by the three used
 * rows T1, T2, T4 of its T-matrix (Sec. 3.1: T = P S with
 * S = [t'_u t'_v 0 c']; column 3 of S is zero so each row is a 3-vector over
 * (t'_u, t'_v, c')), its centre-precomputed inverse MIP covariance
 * (Sigma^-1_uu, Sigma^-1_uv, Sigma^-1_vv) (Eq. mip_weight), its depth interval
 * [z_start, z_end] (Sec. 3.2.1), a validity flag and its support rectangle
 * [x_lo, x_hi] x [y_lo, y_hi] in continuous pixel coordinates (built in
 * model.py from the T-matrix rows, App. A).
 *
 * For a pixel centre (x, y) the ray is the intersection of the planes
 * h_x = (-1, 0, 0, x) and h_y = (0, -1, 0, y) (Sec. 3.1).  Pulled back through
 * T they become k = x T4 - T1 and l = y T4 - T2 (coefficients over (u, v, 1));
 * the hit in the surfel plane is the common zero of both, i.e. the
 * homogeneous point s = k x l, (u, v) = (s0, s1) / s2, provided the hit is
 * in front of the camera (depth T4.(u, v, 1) > 0).
 *
 * A surfel covers the pixel iff the pixel centre lies in its support
 * rectangle and rho2_mip < r_cut^2 (Algorithm 1; pp_sigma >= 0 selects the
 * per-pixel MIP filter, see hit_rho2).  Covering surfels are
 * visited in ascending (z_start, index) order and grouped by Algorithm 1: a
 * new layer starts when the open layer has weight and z_start > z_max_end;
 * layers after the K_max-th are discarded.
 *
 * Outputs per pixel: number of kept layers, and the kept fragments
 * (pixel, surfel, layer) in visiting order.  Decision margins let tests set
 * aside pixels whose decisions are within rounding of flipping:
 * margin[0] = min |rho2_mip - r^2| / r^2 over hits inside the rectangle,
 * margin[1] = min |z_start - z_max_end| / z_max_end over grouping tests,
 * margin[2] = min distance (px) from the pixel centre to a rectangle edge
 *             over surfels that pass the rho2 test.
 *
 * Two-call protocol: call with frag_offset == NULL to get per-pixel
 * fragment counts (frag_count) and the total (returned); then call again with
 * frag_offset = exclusive prefix sum of frag_count and output arrays of the
 * total size.
 */
typedef struct {
    double zs, ze;
    int idx;
} frag_t;

/* Pixels outside a support rectangle by less than this (px) still count
 * toward the rectangle margin (a covering surfel there is a decision within
 * rounding of flipping). */
#define RECT_NEAR 0.01

static int frag_cmp(const void* a, const void* b) {
    const frag_t* x = (const frag_t*)a;
    const frag_t* y = (const frag_t*)b;
    if (x->zs < y->zs) return -1;
    if (x->zs > y->zs) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* rho2_mip of surfel i at pixel centre (x, y); returns 0 if there is no hit
 * in front of the camera.  With pp_sigma < 0 the MIP filter is the one
 * precomputed at the surfel centre (Sinv, Sec. 3.3.2, Eq. mip_weight).  With
 * pp_sigma >= 0 it is evaluated at the hit itself (the per-pixel Jacobian of
 * AA-2DGS that Sec. 3.3.1 describes and Sec. 4.4.2 ablates):
 * J = d(u,v)/d(x,y) of the intersection mapping at this pixel, by the
 * quotient rule on s = k x l (dk/dx = T4, dl/dy = T4), then
 * Sigma = I + sigma_f J J^T (Eq. mip_cov) and rho2 = u^T Sigma^-1 u; the
 * per-pixel n_f is then returned in *nf (else *nf is untouched). */
static int hit_rho2(const double* T, const double* Sinv, double x, double y, double pp_sigma, double* rho2,
                    double* nf) {
    const double* T1 = T;
    const double* T2 = T + 3;
    const double* T4 = T + 6;
    double k[3], l[3], s[3];
    for (int a = 0; a < 3; ++a) {
        k[a] = x * T4[a] - T1[a];
        l[a] = y * T4[a] - T2[a];
    }
    s[0] = k[1] * l[2] - k[2] * l[1];
    s[1] = k[2] * l[0] - k[0] * l[2];
    s[2] = k[0] * l[1] - k[1] * l[0];
    if (s[2] == 0.0) return 0;
    double u = s[0] / s[2], v = s[1] / s[2];
    double depth = T4[0] * u + T4[1] * v + T4[2];
    if (!(depth > 0.0)) return 0;
    if (pp_sigma < 0.0) {
        *rho2 = Sinv[0] * u * u + 2.0 * Sinv[1] * u * v + Sinv[2] * v * v;
        return 1;
    }
    double sx[3], sy[3];   /* ds/dx = T4 x l, ds/dy = k x T4 */
    sx[0] = T4[1] * l[2] - T4[2] * l[1];
    sx[1] = T4[2] * l[0] - T4[0] * l[2];
    sx[2] = T4[0] * l[1] - T4[1] * l[0];
    sy[0] = k[1] * T4[2] - k[2] * T4[1];
    sy[1] = k[2] * T4[0] - k[0] * T4[2];
    sy[2] = k[0] * T4[1] - k[1] * T4[0];
    double Juu = (sx[0] - u * sx[2]) / s[2], Juv = (sy[0] - u * sy[2]) / s[2];
    double Jvu = (sx[1] - v * sx[2]) / s[2], Jvv = (sy[1] - v * sy[2]) / s[2];
    double a = 1.0 + pp_sigma * (Juu * Juu + Juv * Juv);
    double b = pp_sigma * (Juu * Jvu + Juv * Jvv);
    double c = 1.0 + pp_sigma * (Jvu * Jvu + Jvv * Jvv);
    double det = a * c - b * b;
    *rho2 = (c * u * u - 2.0 * b * u * v + a * v * v) / det;
    if (nf) *nf = 1.0 / sqrt(det);
    return 1;
}

long long oref_fragments(int N, const double* T /* [N][9] */, const double* Sinv /* [N][3] */,
                         const double* zse /* [N][2] */, const uint8_t* valid,
                         const double* rect /* [N][4] x_lo, x_hi, y_lo, y_hi */, int W, int H,
                         double rcut2, int kmax, double pp_sigma, int npix, const int32_t* pix /* [npix] or NULL */,
                         int32_t* n_layers /* [P] */, double* margin /* [P][3] */,
                         int64_t* frag_count /* [P] */, const int64_t* frag_offset /* [P] */,
                         int32_t* frag_pix, int32_t* frag_sid, int32_t* frag_layer) {
    int P = pix ? npix : W * H;
    /* integer pixel ranges whose centres lie in each rectangle widened by
     * RECT_NEAR px (the pixels outside the rectangle proper only enter the
     * rectangle margin) */
    int32_t* bbox = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) {
        double lo[2] = {rect[i * 4 + 0] - RECT_NEAR, rect[i * 4 + 2] - RECT_NEAR},
               hi[2] = {rect[i * 4 + 1] + RECT_NEAR, rect[i * 4 + 3] + RECT_NEAR};
        int lim[2] = {W, H};
        for (int a = 0; a < 2; ++a) {
            double i0 = ceil(lo[a] - 0.5), i1 = floor(hi[a] - 0.5);
            if (i0 < 0) i0 = 0;
            if (i1 > lim[a] - 1) i1 = lim[a] - 1;
            if (!(i0 <= i1)) { i0 = 1; i1 = 0; } /* empty (also catches NaN) */
            bbox[i * 4 + 2 * a + 0] = (int32_t)i0;
            bbox[i * 4 + 2 * a + 1] = (int32_t)i1;
        }
    }
    /* candidate lists per image row: surfels whose range spans the row */
    int* row_start = (int*)calloc((size_t)H + 1, sizeof(int));
    for (int i = 0; i < N; ++i) {
        if (!valid[i]) continue;
        for (int y = bbox[i * 4 + 2]; y <= bbox[i * 4 + 3]; ++y) row_start[y + 1]++;
    }
    for (int y = 0; y < H; ++y) row_start[y + 1] += row_start[y];
    int* row_list = (int*)malloc(sizeof(int) * (size_t)(row_start[H] > 0 ? row_start[H] : 1));
    int* fill = (int*)calloc((size_t)H, sizeof(int));
    for (int i = 0; i < N; ++i) {
        if (!valid[i]) continue;
        for (int y = bbox[i * 4 + 2]; y <= bbox[i * 4 + 3]; ++y) row_list[row_start[y] + fill[y]++] = i;
    }
    free(fill);

    long long total = 0;
#pragma omp parallel reduction(+ : total)
    {
        int capf = 256;
        frag_t* fr = (frag_t*)malloc(sizeof(frag_t) * capf);
#pragma omp for schedule(dynamic, 64)
        for (int p = 0; p < P; ++p) {
            int pid = pix ? pix[p] : p;
            int px = pid % W, py = pid / W;
            double x = px + 0.5, y = py + 0.5;
            double m_cut = INFINITY, m_gap = INFINITY, m_box = INFINITY;
            int nf = 0;
            for (int c = row_start[py]; c < row_start[py + 1]; ++c) {
                int i = row_list[c];
                if (px < bbox[i * 4 + 0] || px > bbox[i * 4 + 1]) continue;
                double rho2;
                if (!hit_rho2(T + (size_t)i * 9, Sinv + (size_t)i * 3, x, y, pp_sigma, &rho2, NULL)) continue;
                const double* R = rect + (size_t)i * 4;
                /* signed distance of the pixel centre from the rectangle's edge (< 0 outside) */
                double d = fmin(fmin(x - R[0], R[1] - x), fmin(y - R[2], R[3] - y));
                if (!(d >= 0.0)) {   /* outside: a candidate only within rounding of the edge */
                    if (rho2 < rcut2 && -d < m_box) m_box = -d;
                    continue;
                }
                double m = fabs(rho2 - rcut2) / rcut2;
                if (m < m_cut) m_cut = m;
                if (!(rho2 < rcut2)) continue;
                if (d < m_box) m_box = d;
                if (nf == capf) {
                    capf *= 2;
                    fr = (frag_t*)realloc(fr, sizeof(frag_t) * capf);
                }
                fr[nf].zs = zse[i * 2 + 0];
                fr[nf].ze = zse[i * 2 + 1];
                fr[nf].idx = i;
                nf++;
            }
            qsort(fr, (size_t)nf, sizeof(frag_t), frag_cmp);
            /* Algorithm 1 over the sorted covering fragments; "layer >= 0"
             * means the open layer already holds weight. */
            int layer = -1;
            double zmax = 0.0;
            long long kept = 0;
            for (int f = 0; f < nf; ++f) {
                if (layer >= 0) {
                    /* an exact tie (equal interval ends, e.g. coplanar
                     * fronto-parallel surfels) is not near a flip */
                    double m = fabs(fr[f].zs - zmax) / fabs(zmax);
                    if (m > 0.0 && m < m_gap) m_gap = m;
                }
                if (layer < 0 || fr[f].zs > zmax) { /* gap: flush and open a new layer */
                    layer++;
                    zmax = 0.0;
                    if (layer >= kmax) break; /* layers after the K_max-th are discarded */
                }
                if (fr[f].ze > zmax) zmax = fr[f].ze;
                if (frag_offset) {
                    long long o = frag_offset[p] + kept;
                    frag_pix[o] = pid;
                    frag_sid[o] = fr[f].idx;
                    frag_layer[o] = layer;
                }
                kept++;
            }
            n_layers[p] = layer + 1 > kmax ? kmax : layer + 1;
            margin[p * 3 + 0] = m_cut;
            margin[p * 3 + 1] = m_gap;
            margin[p * 3 + 2] = m_box;
            frag_count[p] = kept;
            total += kept;
        }
        free(fr);
    }
    free(row_start);
    free(row_list);
    free(bbox);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Every surfel that may take part in the decisions of pixel `pid`: those
 * whose support rectangle, widened by `near` px, contains the pixel centre
 * and whose plane is hit in front of the camera.  For each: its index, rho2_mip
 * at the pixel centre, its depth interval and the signed distance (px) of the
 * pixel centre from the rectangle's edge (negative outside).  Fills at most
 * `cap` entries; returns how many there are (call again with a larger cap if
 * the return value exceeds it).  Tests use it to enumerate the outcomes of
 * decisions that sit within rounding of flipping. */
int oref_pixel_candidates(int N, const double* T, const double* Sinv, const double* zse, const uint8_t* valid,
                          const double* rect, int W, int pid, double near, double pp_sigma, int cap, int32_t* idx,
                          double* rho2_out, double* zs_out, double* ze_out, double* dist_out) {
    int px = pid % W, py = pid / W;
    double x = px + 0.5, y = py + 0.5;
    int n = 0;
    for (int i = 0; i < N; ++i) {
        if (!valid[i]) continue;
        const double* R = rect + (size_t)i * 4;
        double d = fmin(fmin(x - R[0], R[1] - x), fmin(y - R[2], R[3] - y));
        if (!(d > -near)) continue;
        double rho2;
        if (!hit_rho2(T + (size_t)i * 9, Sinv + (size_t)i * 3, x, y, pp_sigma, &rho2, NULL)) continue;
        if (n < cap) {
            idx[n] = i;
            rho2_out[n] = rho2;
            zs_out[n] = zse[i * 2 + 0];
            ze_out[n] = zse[i * 2 + 1];
            dist_out[n] = d;
        }
        n++;
    }
    return n;
}
