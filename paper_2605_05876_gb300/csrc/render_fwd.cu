// Forward render: projection + shading, tile binning, per-tile depth sort and
// the fused per-pixel rasteriser (Algorithm 1 with coverage compositing).
#include <math.h>

#include "ss3d_internal.cuh"
#include "raster_common.cuh"

// ------------------------------------------------------------------------
// projection (Sec. 3.1), centre-precomputed MIP filter (Sec. 3.3.2) and
// forward split-sum shading (Sec. 3.4.2) for one surfel and every view of its
// scene.  One thread per surfel: the 64 B of parameters are read once per
// batch and one 112 B record is written per view.

struct ss_env_ptrs {
    const float* irr;
    const float* spec;
    const float* lut;
};

__device__ __forceinline__ float3 tex3(const float* T, int i) { return make_float3(T[i * 3], T[i * 3 + 1], T[i * 3 + 2]); }

__device__ __forceinline__ float3 bilerp3(const float* T, ss_taps t) {
    float3 a = tex3(T, t.i00), b = tex3(T, t.i01), c = tex3(T, t.i10), d = tex3(T, t.i11);
    float w00 = (1.f - t.fx) * (1.f - t.fy), w01 = t.fx * (1.f - t.fy), w10 = (1.f - t.fx) * t.fy, w11 = t.fx * t.fy;
    return make_float3(w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x, w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y,
                       w00 * a.z + w01 * b.z + w10 * c.z + w11 * d.z);
}

// level offsets of the specular stack (floats)
__device__ __forceinline__ int64_t spec_level_off(const ss_env_desc& ed, int i, int& W, int& H) {
    int64_t off = 0;
    for (int k = 0; k < i; ++k) {
        int w = max(ed.width >> k, 8), h = max(ed.height >> k, 4);
        off += (int64_t)w * h * 3;
    }
    W = max(ed.width >> i, 8);
    H = max(ed.height >> i, 4);
    return off;
}

// One thread per (surfel, view) record: blockIdx.y is the view, blockIdx.x
// runs over its scene's surfels (blocks past the scene's count return).
__global__ void __launch_bounds__(256, 4) project_kernel(ss_ws_view ws, ss_fwd_args a, int64_t n_total) {
    const ss_layout* L = ws.layout;
    const int vthis = blockIdx.y;
    const ss_view_layout& vl0 = L->v[vthis];
    const int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ws.grad_rec && a.with_backward && a.p.zero_grad_in_forward) {
        // clear this block's gradient rows for the backward: the block's
        // records are consecutive, so its rows are one span of float4s
        // (rows of SS_NGRAD floats, 256-byte aligned base); evict-first
        // stores, so the rows do not push the surfels and the prefiltered
        // maps, which every view's blocks read again, out of L2
        const int64_t b0 = blockIdx.x * (int64_t)blockDim.x;
        const int64_t nrow = min((int64_t)blockDim.x, (int64_t)vl0.n_surfels - b0);
        if (nrow > 0) {
            float4* g = reinterpret_cast<float4*>(ws.grad_rec + (vl0.rec_off + b0) * SS_NGRAD);
            const int n4 = (int)nrow * (SS_NGRAD / 4);
            for (int k = threadIdx.x; k < n4; k += blockDim.x) __stcs(&g[k], make_float4(0.f, 0.f, 0.f, 0.f));
        }
    }
    if (li >= vl0.n_surfels) return;
    const int64_t i = vl0.surfel_begin + li;
    const int scene = vl0.scene;
    const float* P = a.s.pos + i * 3;
    float c0 = P[0], c1 = P[1], c2 = P[2];
    float4 q = *reinterpret_cast<const float4*>(a.s.quat + i * 4);
    float2 ls = *reinterpret_cast<const float2*>(a.s.log_scale + i * 2);
    float rho0 = a.s.albedo[i * 3], rho1 = a.s.albedo[i * 3 + 1], rho2 = a.s.albedo[i * 3 + 2];
    float rough = a.s.roughness[i], metal = a.s.metallic[i];
    bool finite = isfinite(c0) && isfinite(c1) && isfinite(c2) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) &&
                  isfinite(q.w) && isfinite(ls.x) && isfinite(ls.y) && isfinite(rho0) && isfinite(rho1) &&
                  isfinite(rho2) && isfinite(rough) && isfinite(metal) &&
                  (q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w) > 0.f;
    if (!finite) atomicOr(ws.status, SS_ERR_NONFINITE);
    float Rq[9];
    quat_rot(q.x, q.y, q.z, q.w, Rq);
    const float su = expf(ls.x), sv = expf(ls.y);
    const float tu[3] = {su * Rq[0], su * Rq[3], su * Rq[6]};
    const float tv[3] = {sv * Rq[1], sv * Rq[4], sv * Rq[7]};
    const float nrm[3] = {Rq[2], Rq[5], Rq[8]};
    const float rc = a.p.r_cut, rc2 = rc * rc;
    const int nL = a.ed.n_levels;
    const int64_t irr_stride = (int64_t)a.ed.irr_width * a.ed.irr_height * 3;
    int64_t spec_stride = 0;
    {
        int W, H;
        spec_stride = spec_level_off(a.ed, nL, W, H);
    }
    const float* irr = a.env.irr + scene * irr_stride;
    const float* spec = a.env.spec + scene * spec_stride;
    const int lutn = a.p.lut_n;

    {
        const int v = vthis;
        const ss_view_layout& vl = vl0;
        const ss_camera& cam = a.cams[v];
        const int64_t local = i - vl.surfel_begin;
        ss_rec rec;
        uint32_t flags = 0;
        // camera-space centre in double-float, camera-space tangents in FP32
        dfl cx_ = df_dot3_add(cam.R[0], cam.R[1], cam.R[2], c0, c1, c2, cam.t[0]);
        dfl cy_ = df_dot3_add(cam.R[3], cam.R[4], cam.R[5], c0, c1, c2, cam.t[1]);
        dfl cz_ = df_dot3_add(cam.R[6], cam.R[7], cam.R[8], c0, c1, c2, cam.t[2]);
        float tuc[3], tvc[3];
        for (int r = 0; r < 3; ++r) {
            tuc[r] = cam.R[r * 3] * tu[0] + cam.R[r * 3 + 1] * tu[1] + cam.R[r * 3 + 2] * tu[2];
            tvc[r] = cam.R[r * 3] * tv[0] + cam.R[r * 3 + 1] * tv[1] + cam.R[r * 3 + 2] * tv[2];
        }
        const float cz = cz_.hi + cz_.lo;
        const float eps = rc * sqrtf(tuc[2] * tuc[2] + tvc[2] * tvc[2]);   // Sec. 3.1 depth extent
        const float zs = __fadd_rn(__fsub_rn(cz_.hi, eps), cz_.lo);
        const float ze = __fadd_rn(__fadd_rn(cz_.hi, eps), cz_.lo);
        // centre in pixels (double-float): p = f c'_xy / c'_z + c
        dfl mx = df_div(cx_, cz_), my = df_div(cy_, cz_);
        dfl px = df_add_f(df_mul_f(mx, cam.fx), cam.cx);
        dfl py = df_add_f(df_mul_f(my, cam.fy), cam.cy);
        const float mxf = mx.hi, myf = my.hi;
        const float fx = cam.fx, fy = cam.fy;
        // screen-plane parts of the tangents: a = t'_u - m t'_uz, b = t'_v - m t'_vz
        const float ax = __fmaf_rn(-mxf, tuc[2], tuc[0]), ay = __fmaf_rn(-myf, tuc[2], tuc[1]);
        const float bx = __fmaf_rn(-mxf, tvc[2], tvc[0]), by = __fmaf_rn(-myf, tvc[2], tvc[1]);
        // N_d = n . (c - o), o = -R^-1 t the camera centre: the signed distance of the
        // camera from the surfel plane.  It is the one ill-conditioned quantity for
        // nearly edge-on surfels, so it is formed in double-float from the quaternion,
        // n = (2(xz+wy), 2(yz-wx), w^2-x^2-y^2+z^2) / |q|^2.
        const float Nd = ss_plane_distance(q, c0, c1, c2, ws.vgeo[v].o_hi, ws.vgeo[v].o_lo);
        const float ncx = cam.R[0] * nrm[0] + cam.R[1] * nrm[1] + cam.R[2] * nrm[2];   // n' = R n
        const float ncy = cam.R[3] * nrm[0] + cam.R[4] * nrm[1] + cam.R[5] * nrm[2];
        // (t'_u x t'_v) . c'/c'_z = det R s_u s_v N_d / c'_z
        const float det0 = ws.vgeo[v].detR * su * sv * Nd / cz;
        bool valid = finite && (zs > a.p.z_near) && (Nd != 0.f) && isfinite(Nd);
        // perspective denominator: s2 = c'_z / depth(hit) = 1 + (n'_x dx/fx + n'_y dy/fy) c'_z / N_d
        // (n' = R^-T n is the camera-space plane normal; R n differs from it by rounding only)
        const float A2 = cz * ncx / (fx * Nd), B2 = cz * ncy / (fy * Nd);
        // M M^T (M = d(x,y)/d(u,v) at the centre) and the filtered screen covariance
        const float icz = 1.f / cz, icz2 = icz * icz;
        const float fx2 = fx * fx, fy2 = fy * fy;
        const float m11 = fx2 * (ax * ax + bx * bx) * icz2;
        const float m12 = fx * fy * (ax * ay + bx * by) * icz2;
        const float m22 = fy2 * (ay * ay + by * by) * icz2;
        const float sdg = fx * fy * det0 * icz2;     // det M
        const float detG = sdg * sdg;
        const float sig = a.p.sigma_f;
        const float Dn = detG + sig * (m11 + m22) + sig * sig;   // det(M M^T + sig I)
        const float nf = sqrtf(detG / Dn);                        // Eq. mip_eval: sqrt(|I| / |Sigma_mip|)
        // Qs = (M M^T + sig I)^-1 = [[m22 + sig, -m12], [-m12, m11 + sig]] / Dn, factor P^T P = Qs
        const float qa = (m22 + sig) / Dn, qb = -m12 / Dn, qc = (m11 + sig) / Dn;
        float P00, P01, P10, P11;
        if (qa >= qc) {   // q = (l00 dx + l01 dy)^2 + (l11 dy)^2, det Qs = 1/Dn
            float l00 = sqrtf(qa);
            P00 = l00; P01 = qb / l00; P10 = 0.f; P11 = rsqrtf(Dn) / l00;
        } else {          // q = (l11 dy + l10 dx)^2 + (l00 dx)^2
            float l11 = sqrtf(qc);
            P00 = qb / l11; P01 = l11; P10 = rsqrtf(Dn) / l11; P11 = 0.f;
        }
        // support rectangle (centred pixel offsets): exact bounds of the projected r_cut
        // disc (dual conic, App. A) U r_cut bounds of the EWA ellipse M M^T + sig I, +1 px
        const float C00 = fx2 * (ax * ax + bx * bx), C02 = fx * (ax * tuc[2] + bx * tvc[2]);
        const float C11 = fy2 * (ay * ay + by * by), C12 = fy * (ay * tuc[2] + by * tvc[2]);
        const float C22 = tuc[2] * tuc[2] + tvc[2] * tvc[2] - cz * cz / rc2;
        float lo[2], hi[2];
        {
            const float Caa[2] = {C00, C11}, Ca2[2] = {C02, C12}, Maa[2] = {m11, m22};
            for (int ax_ = 0; ax_ < 2; ++ax_) {
                float dsc = sqrtf(fmaxf(Ca2[ax_] * Ca2[ax_] - Caa[ax_] * C22, 0.f));
                float r0 = (Ca2[ax_] + dsc) / C22, r1 = (Ca2[ax_] - dsc) / C22;
                float ext = rc * sqrtf(Maa[ax_] + sig);
                lo[ax_] = fminf(fminf(r0, r1), -ext) - 1.f;
                hi[ax_] = fmaxf(fmaxf(r0, r1), ext) + 1.f;
            }
        }
        valid = valid && (C22 < 0.f) && isfinite(nf) && isfinite(A2) && isfinite(B2);
        int i0 = (int)ceilf(px.hi + lo[0] - 0.5f), i1 = (int)floorf(px.hi + hi[0] - 0.5f);
        int j0 = (int)ceilf(py.hi + lo[1] - 0.5f), j1 = (int)floorf(py.hi + hi[1] - 0.5f);
        i0 = max(i0, 0); j0 = max(j0, 0);
        i1 = min(i1, vl.width - 1); j1 = min(j1, vl.height - 1);
        valid = valid && (i0 <= i1) && (j0 <= j1) && isfinite(px.hi) && isfinite(py.hi);
        if (valid) {
            // does the exact filtered support {d^T Qs d < r^2 s2(d)^2} stay inside the
            // rectangle?  It is the ellipse (d - dc)^T Q2 (d - dc) < kap with
            // Q2 = Qs - r^2 g g^T, g = (A2, B2), dc = r^2 Q2^-1 g, kap = r^2 + r^2 g.dc
            const float q00 = qa - rc2 * A2 * A2, q01 = qb - rc2 * A2 * B2, q11 = qc - rc2 * B2 * B2;
            const float dq = q00 * q11 - q01 * q01;
            bool inside = (q00 > 0.f) && (dq > 0.f);
            if (inside) {
                const float i00 = q11 / dq, i01 = -q01 / dq, i11 = q00 / dq;
                const float dcx = rc2 * (i00 * A2 + i01 * B2), dcy = rc2 * (i01 * A2 + i11 * B2);
                const float kap = rc2 * (1.f + A2 * dcx + B2 * dcy);
                const float hx = sqrtf(fmaxf(kap * i00, 0.f)), hy = sqrtf(fmaxf(kap * i11, 0.f));
                inside = (dcx - hx > lo[0] + 0.25f) && (dcx + hx < hi[0] - 0.25f) && (dcy - hy > lo[1] + 0.25f) &&
                         (dcy + hy < hi[1] - 0.25f);
            }
            if (!inside) flags |= SS_FLAG_RECT_TEST;
            flags |= SS_FLAG_VALID;
        }
        // forward shading (Eq. ibl): one pre-shaded colour per surfel and view
        const float ox = -(cam.R[0] * cam.t[0] + cam.R[3] * cam.t[1] + cam.R[6] * cam.t[2]);
        const float oy = -(cam.R[1] * cam.t[0] + cam.R[4] * cam.t[1] + cam.R[7] * cam.t[2]);
        const float oz = -(cam.R[2] * cam.t[0] + cam.R[5] * cam.t[1] + cam.R[8] * cam.t[2]);
        float wo[3] = {ox - c0, oy - c1, oz - c2};
        {
            float inv = rsqrtf(wo[0] * wo[0] + wo[1] * wo[1] + wo[2] * wo[2]);
            wo[0] *= inv; wo[1] *= inv; wo[2] *= inv;
        }
        float ns[3] = {nrm[0], nrm[1], nrm[2]};
        float facing = ns[0] * wo[0] + ns[1] * wo[1] + ns[2] * wo[2];
        if (facing < 0.f) {
            ns[0] = -ns[0]; ns[1] = -ns[1]; ns[2] = -ns[2];
            facing = -facing;
            flags |= SS_FLAG_FLIPPED;
        }
        const float mu = fminf(fmaxf(facing, 0.f), 1.f);
        const float refl[3] = {2.f * facing * ns[0] - wo[0], 2.f * facing * ns[1] - wo[1], 2.f * facing * ns[2] - wo[2]};
        float3 col = make_float3(0.f, 0.f, 0.f);
        if (valid) {
            float u, vv;
            dir_to_uv(ns[0], ns[1], ns[2], u, vv);
            float3 Ld = bilerp3(irr, bilinear_taps(u, vv, a.ed.irr_width, a.ed.irr_height, true));
            dir_to_uv(refl[0], refl[1], refl[2], u, vv);
            float lc = fminf(fmaxf(rough, 0.f), 1.f) * (float)(nL - 1);
            int l0 = min((int)floorf(lc), nL - 1), l1 = min(l0 + 1, nL - 1);
            float lf = lc - (float)l0;
            int W0, H0, W1, H1;
            int64_t o0 = spec_level_off(a.ed, l0, W0, H0), o1 = spec_level_off(a.ed, l1, W1, H1);
            float3 s0 = bilerp3(spec + o0, bilinear_taps(u, vv, W0, H0, true));
            float3 s1 = bilerp3(spec + o1, bilinear_taps(u, vv, W1, H1, true));
            float3 Ls = make_float3((1.f - lf) * s0.x + lf * s1.x, (1.f - lf) * s0.y + lf * s1.y,
                                    (1.f - lf) * s0.z + lf * s1.z);
            ss_taps lt = bilinear_taps(mu, fminf(fmaxf(rough, 0.f), 1.f), lutn, lutn, false);
            const float* LUT = a.env.lut;
            float w00 = (1.f - lt.fx) * (1.f - lt.fy), w01 = lt.fx * (1.f - lt.fy), w10 = (1.f - lt.fx) * lt.fy,
                  w11 = lt.fx * lt.fy;
            float be1 = w00 * LUT[lt.i00 * 2] + w01 * LUT[lt.i01 * 2] + w10 * LUT[lt.i10 * 2] + w11 * LUT[lt.i11 * 2];
            float be2 = w00 * LUT[lt.i00 * 2 + 1] + w01 * LUT[lt.i01 * 2 + 1] + w10 * LUT[lt.i10 * 2 + 1] +
                        w11 * LUT[lt.i11 * 2 + 1];
            const float rho[3] = {rho0, rho1, rho2};
            float cc[3];
            const float Lda[3] = {Ld.x, Ld.y, Ld.z}, Lsa[3] = {Ls.x, Ls.y, Ls.z};
            for (int k = 0; k < 3; ++k) {
                float F0 = 0.04f * (1.f - metal) + rho[k] * metal;
                float kd = (1.f - F0) * (1.f - metal);
                cc[k] = kd * rho[k] * Lda[k] + Lsa[k] * (F0 * be1 + be2);
            }
            col = make_float3(cc[0], cc[1], cc[2]);
        }
        if (a.p.mip_mode == 2) {
            // per-pixel MIP filter: the raster needs J0 = M^-1 = d(u,v)/d(x,y) at the
            // centre, adj(M) / det M with det M = sdg (formed from N_d in double-float,
            // so it stays accurate for nearly edge-on surfels), and |det J0| =
            // 1 / |sdg| in place of n_f (which is per pixel there); the exact support
            // is not the centre quadratic's, so the support rectangle is always tested
            const float k = 1.f / (cz * sdg);
            rec.r0 = make_float4(fy * by * k, -fx * bx * k, -fy * ay * k, fx * ax * k);
            rec.r1 = make_float4(A2, B2, 1.f, 1.f / fabsf(sdg));
            if (valid) flags |= SS_FLAG_RECT_TEST;
        } else {
            rec.r0 = make_float4(P00, P01, P10, P11);
            rec.r1 = make_float4(A2, B2, 1.f, nf);
        }
        rec.r2 = make_float4(px.hi, py.hi, px.lo, py.lo);
        rec.r3 = make_float4(zs, ze, __uint_as_float(valid ? pack16(i0, i1) : 0xffffu),
                             __uint_as_float(valid ? pack16(j0, j1) : 0xffffu));
        rec.r4 = make_float4(col.x, col.y, col.z, __uint_as_float(flags));
        rec.r5 = make_float4(rho0, rho1, rho2, rough);
        rec.r6 = make_float4(metal, ns[0], ns[1], ns[2]);
        ws.rec[vl.rec_off + local] = rec;
        if (valid) {
            // bin counts: the record's rank in the bins of its first four tiles
            // (kept for the scatter, which then needs no atomics for them),
            // plain counts for the rest
            const int tx0 = i0 >> a.ts.tw_log2, tx1 = i1 >> a.ts.tw_log2, ty0 = j0 >> a.ts.th_log2,
                      ty1 = j1 >> a.ts.th_log2;
            const int ntx = tx1 - tx0 + 1, nt = ntx * (ty1 - ty0 + 1);
            uint32_t rk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nt) {
                    const int t = vl.tile_off + (ty0 + q / ntx) * vl.tiles_x + tx0 + q % ntx;
                    rk[q] = atomicAdd(&ws.tile_count[(size_t)t * SS_CNT_STRIDE], 1u);
                }
            for (int q = 4; q < nt; ++q) {
                const int t = vl.tile_off + (ty0 + q / ntx) * vl.tiles_x + tx0 + q % ntx;
                atomicAdd(&ws.tile_cursor[(size_t)t * SS_CNT_STRIDE], 1u);
            }
            ws.inst_rank[vl.rec_off + local] = make_uint4(rk[0], rk[1], rk[2], rk[3]);
        }
    }
}

void ss_launch_project(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st) {
    int64_t n = L.scene_begin[L.n_scenes];
    if (n <= 0) return;
    int64_t nmax = 0;   // the largest scene's surfels: the grid's x extent
    for (int v = 0; v < L.n_views; ++v) nmax = nmax > L.v[v].n_surfels ? nmax : L.v[v].n_surfels;
    if (nmax <= 0) return;
    ss_note_launch();
    project_kernel<<<dim3((unsigned)((nmax + 255) / 256), (unsigned)L.n_views), 256, 0, st>>>(ws, a, n);
}

// ------------------------------------------------------------------------
// binning: exclusive scan of tile counts, scatter of (z_start, id) keys,
// per-tile sort by (z_start, id) (Sec. 3.2.1: sort key z_start; ties by id)

__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t* cnt, const uint32_t* extra, uint32_t* start, int n,
                                                    int* status,
                                                    int64_t cap, unsigned long long* stats) {
    // The running total is kept in 64 bits: a batch with 2^32 or more
    // instances must be reported, not wrapped.  Tile starts past the 32-bit
    // range (or past the capacity) are stored clamped to the capacity, so
    // those tiles read as empty and the scatter places none of their keys.
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long lim = (unsigned long long)cap;   // cap <= 0xffffffff (host-checked)
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < n ? cnt[(size_t)i * SS_CNT_STRIDE] + extra[(size_t)i * SS_CNT_STRIDE] : 0u;
        uint32_t x = v;   // a prefix of at most 1024 tile counts; counts per tile stay far below 2^22
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const unsigned long long excl = carry + (w > 0 ? wsum[w - 1] : 0u) + x - v;
        if (i < n) start[i] = (uint32_t)(excl < lim ? excl : lim);
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        start[n] = (uint32_t)(carry < lim ? carry : lim);
        stats[0] = carry;
        if (carry > lim) atomicOr(status, SS_ERR_CAPACITY);
    }
}

// Block masks.  For an instance of a record in a tile, bit b (8 x 4 block
// b = (b & 1, b >> 1) of the 16 x 16 tile) is set when the record's support
// rectangle overlaps the block and -- except for the per-pixel MIP filter,
// whose support is not the centre quadratic's -- the exact support can reach
// one of the block's pixel centres (ss_conic_box_may_cover, with the centre relative
// to the tile formed exactly as the rasteriser's staging forms it).  The
// rasterisers stage a record for a block only when its bit is set, so the
// per-pixel tests they run are unchanged.  The scatter kernel, which streams
// the records, computes the masks of each record's first four tiles; the sort
// kernel reads them back for the sorted instances (instances past a record's
// fourth tile keep the rectangle test alone).
// (block b of a tile of 2^bxl blocks across sits at (8 (b mod 2^bxl), 4 (b >> bxl)))
__device__ __forceinline__ uint32_t rect_block_bits(uint32_t rx, uint32_t ry, int x0, int y0, int bxl, int bpt) {
    const int i0 = (int)(rx & 0xffff), i1 = (int)(rx >> 16), j0 = (int)(ry & 0xffff), j1 = (int)(ry >> 16);
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b >= bpt) break;
        const int gx0 = x0 + 8 * (b & ((1 << bxl) - 1)), gy0 = y0 + 4 * (b >> bxl);
        if (i0 <= gx0 + 7 && i1 >= gx0 && j0 <= gy0 + 3 && j1 >= gy0) m |= 1u << b;
    }
    return m;
}

// Blocks whose pixel-centre box misses the bounding box of the surfel's
// exact support {f < t} are cleared (t_pre: a margin at least the per-pixel
// test's rounding bound for any block of the record, so that only blocks
// without a covering pixel are cleared).
__device__ __forceinline__ uint32_t exact_block_bits(uint32_t m, const ss_conic& q, float t_pre, float4 r2, int x0,
                                                     int y0, int bxl) {
    if (!q.pd) return m;
    const float prx = __fadd_rn(__fsub_rn(r2.x, (float)x0), r2.z);
    const float pry = __fadd_rn(__fsub_rn(r2.y, (float)y0), r2.w);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (!((m >> b) & 1u)) continue;
        const float dxb = (float)(8 * (b & ((1 << bxl) - 1))) - prx, dyb = (float)(4 * (b >> bxl)) - pry;
        if (!ss_conic_aabb_meets(q, t_pre, dxb + 0.5f, dxb + 7.5f, dyb + 0.5f, dyb + 3.5f)) m &= ~(1u << b);
    }
    return m;
}

// the block mask of a sorted instance (key) in tile (x0, y0): from the
// scatter's per-record masks, or the rectangle test past the fourth tile
__device__ __forceinline__ uint32_t block_mask_of(const ss_ws_view& ws, const ss_tile_shape& ts,
                                                  unsigned long long key, int x0, int y0) {
    const uint32_t r = (uint32_t)(key & 0xffffffffull);
    const uint2 bm = __ldg(ws.rec_bmask + r);
    const int tx0 = (int)(bm.y & 0xfff), ty0 = (int)((bm.y >> 12) & 0xfff), ntx = (int)(bm.y >> 24);
    const int q = ((y0 >> ts.th_log2) - ty0) * ntx + ((x0 >> ts.tw_log2) - tx0);
    if (q < 4) return (bm.x >> (8 * q)) & 0xffu;
    const float4 r3 = __ldg(&ws.rec[r].r3);
    return rect_block_bits(__float_as_uint(r3.z), __float_as_uint(r3.w), x0, y0, ts.bx_log2, ts.bpt);
}

// One thread per record: its keys go to the bins of the tiles its support
// rectangle covers, at the ranks the projection took in the bins of its
// first four tiles; instances past those take positions behind the first-
// four instances of their bin by counting the bin's cursor down.
__global__ void __launch_bounds__(256) scatter_kernel(ss_ws_view ws, int64_t total_records, float rc2, int exact,
                                                      ss_tile_shape ts) {
    const ss_layout* L = ws.layout;
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= total_records) return;
    const uint32_t flags = __float_as_uint(ws.rec[r].r4.w);
    const float4 r3 = ws.rec[r].r3;
    const uint4 rk = ws.inst_rank[r];
    if (!(flags & SS_FLAG_VALID)) return;
    const float4 P = ws.rec[r].r0, r1 = ws.rec[r].r1, r2 = ws.rec[r].r2;
    int v = 0;
    {
        int lo = 0, hi = L->n_views - 1;
        while (lo < hi) {
            int m = (lo + hi + 1) >> 1;
            if (L->v[m].rec_off <= r) lo = m;
            else hi = m - 1;
        }
        v = lo;
    }
    const ss_view_layout& vl = L->v[v];
    const uint32_t rx = __float_as_uint(r3.z), ry = __float_as_uint(r3.w);
    const int tx0 = (int)(rx & 0xffff) >> ts.tw_log2, tx1 = (int)(rx >> 16) >> ts.tw_log2;
    const int ty0 = (int)(ry & 0xffff) >> ts.th_log2, ty1 = (int)(ry >> 16) >> ts.th_log2;
    const int bxl = ts.bx_log2, bpt = ts.bpt;
    const int ntx = tx1 - tx0 + 1, nt = ntx * (ty1 - ty0 + 1);
    // low half: the batch-wide record index (ties of z_start in one tile, which
    // belongs to one view, are broken by surfel index all the same)
    const unsigned long long key = ((unsigned long long)__float_as_uint(r3.x) << 32) | (uint32_t)r;
    const uint32_t rks[4] = {rk.x, rk.y, rk.z, rk.w};
    uint32_t masks = 0;
    // per-record part of the exact-support test, and a margin bound over every
    // pixel-centre offset the record's rectangle allows
    const ss_conic cq = ss_conic_of(P, r1.x, r1.y, rc2);
    float t_pre = 0.f;
    {
        const float cx = r2.x + r2.z, cy = r2.y + r2.w;   // centre (pixels)
        const float ex = fmaxf(fabsf((float)(rx & 0xffff) - 8.f - cx), fabsf((float)(rx >> 16) + 9.f - cx));
        const float ey = fmaxf(fabsf((float)(ry & 0xffff) - 4.f - cy), fabsf((float)(ry >> 16) + 5.f - cy));
        t_pre = 2.f * ss_box_margin(cq, ex, ey);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (q < nt) {
            const int tx = tx0 + q % ntx, ty = ty0 + q / ntx;
            const int t = vl.tile_off + ty * vl.tiles_x + tx;
            const uint64_t p = (uint64_t)ws.tile_start[t] + rks[q];
            if ((int64_t)p < ws.max_instances) ws.keys[p] = key;
            const int ox = tx << ts.tw_log2, oy = ty << ts.th_log2;
            uint32_t m = rect_block_bits(rx, ry, ox, oy, bxl, bpt);
            if (exact && m) m = exact_block_bits(m, cq, t_pre, r2, ox, oy, bxl);
            masks |= m << (8 * q);
        }
    ws.rec_bmask[r] = make_uint2(masks, (uint32_t)tx0 | ((uint32_t)ty0 << 12) | ((uint32_t)min(ntx, 255) << 24));
    for (int q = 4; q < nt; ++q) {
        const int t = vl.tile_off + (ty0 + q / ntx) * vl.tiles_x + tx0 + q % ntx;
        const uint32_t k = atomicSub(&ws.tile_cursor[(size_t)t * SS_CNT_STRIDE], 1u) - 1u;
        const uint64_t p = (uint64_t)ws.tile_start[t] + ws.tile_count[(size_t)t * SS_CNT_STRIDE] + k;
        if ((int64_t)p < ws.max_instances) ws.keys[p] = key;
    }
}

#define SORT_THREADS 256
#define SORT_KPL 32                              // keys per thread, held in registers
#define SORT_CAP (SORT_THREADS * SORT_KPL)       // keys sorted by one CTA at once (8192)

// Bitonic sort of N (a power of two, N <= SORT_CAP) keys held in registers:
// thread t holds positions t*KPL .. t*KPL + KPL - 1.  Compare-exchange
// distances j < KPL stay inside a thread, KPL <= j < 32 KPL go across the
// lanes of a warp by shuffles, and only j >= 32 KPL across warps through
// shared memory (laid out [k][thread], so that every access is conflict-free).
__device__ __forceinline__ void cmpx(unsigned long long& a, unsigned long long& b, bool up) {
    const bool sw = (a > b) == up;
    const unsigned long long lo = sw ? b : a, hi = sw ? a : b;
    a = lo;
    b = hi;
}

template <int KPL>
__device__ void bitonic_regs(unsigned long long (&x)[KPL], int N, unsigned long long* xs) {
    const int t = threadIdx.x, lane = t & 31;
    // whole warps take part (the shuffles need every lane); lanes past N hold padding
    const bool active = (t & ~31) * KPL < N;
    for (int size = 2; size <= N; size <<= 1) {
        // across warps
        for (int j = size >> 1; j >= 32 * KPL; j >>= 1) {
            if (active) {
#pragma unroll
                for (int k = 0; k < KPL; ++k) xs[k * SORT_THREADS + t] = x[k];
            }
            __syncthreads();
            if (active) {
                const int pt = t ^ (j / KPL);
                const bool up = ((t * KPL) & size) == 0, lower = (t & (j / KPL)) == 0;
#pragma unroll
                for (int k = 0; k < KPL; ++k) {
                    const unsigned long long y = xs[k * SORT_THREADS + pt];
                    const bool keep_min = lower == up;
                    x[k] = keep_min ? (y < x[k] ? y : x[k]) : (y > x[k] ? y : x[k]);
                }
            }
            __syncthreads();
        }
        if (!active) continue;
        // across the lanes of a warp
        for (int j = min(size >> 1, 16 * KPL); j >= KPL; j >>= 1) {
            const int m = j / KPL;
            const bool up = ((t * KPL) & size) == 0, lower = (lane & m) == 0;
            const bool keep_min = lower == up;
#pragma unroll
            for (int k = 0; k < KPL; ++k) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[k], m);
                x[k] = keep_min ? (y < x[k] ? y : x[k]) : (y > x[k] ? y : x[k]);
            }
        }
        // inside the thread
#pragma unroll
        for (int j = KPL / 2; j >= 1; j >>= 1) {
            if (j < size) {
#pragma unroll
                for (int k = 0; k < KPL; ++k)
                    if ((k & j) == 0) cmpx(x[k], x[k | j], ((t * KPL + k) & size) == 0);
            }
        }
    }
}

// merge two sorted runs A[0,na) and B[0,nb) into out, all threads of the CTA
__device__ void merge_runs(const unsigned long long* A, int na, const unsigned long long* B, int nb,
                           unsigned long long* out) {
    const int n = na + nb;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    int d0 = min(n, (int)threadIdx.x * per), d1 = min(n, d0 + per);
    if (d0 >= d1) return;
    // merge path: find i in A with i + j = d0
    int lo = max(0, d0 - nb), hi = min(d0, na);
    while (lo < hi) {
        int m = (lo + hi) >> 1;
        if (A[m] < B[d0 - 1 - m]) lo = m + 1;
        else hi = m;
    }
    int ia = lo, ib = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        bool takeA = ib >= nb || (ia < na && A[ia] < B[ib]);
        out[d] = takeA ? A[ia++] : B[ib++];
    }
}

// Sort one chunk of m keys (N = the power of two >= m, N <= SORT_THREADS * KPL)
// in registers, KPL per thread, and store it.
template <int KPL>
__device__ __noinline__ void sort_chunk(unsigned long long* K, int m, int N, unsigned long long* xs) {
    const int base = threadIdx.x * KPL;
    unsigned long long x[KPL];
#pragma unroll
    for (int k = 0; k < KPL; ++k) x[k] = base + k < m ? K[base + k] : ~0ull;
    bitonic_regs<KPL>(x, N, xs);
    __syncthreads();   // every thread's reads of this chunk are done before the stores
#pragma unroll
    for (int k = 0; k < KPL; ++k)
        if (base + k < m) K[base + k] = x[k];
    __syncthreads();
}

// block masks of n sorted keys, all threads of the CTA (coalesced key reads);
// each thread counts the bits of the masks it wrote (candidates per block)
__device__ __forceinline__ void gather_masks(const ss_ws_view& ws, const ss_tile_shape& ts, const unsigned long long* K,
                                             uint8_t* BM, int n, int x0, int y0, uint32_t (&cnt)[8]) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t m = block_mask_of(ws, ts, K[i], x0, y0);
        BM[i] = (uint8_t)m;
#pragma unroll
        for (int b = 0; b < 8; ++b) cnt[b] += (m >> b) & 1u;
    }
}

// the tile's candidates per block (the threads' counts summed) -> cand_cnt
__device__ __forceinline__ void store_block_counts(const ss_ws_view& ws, int t, const uint32_t (&cnt)[8]) {
    __shared__ uint32_t tot[8];
    if (threadIdx.x < 8) tot[threadIdx.x] = 0u;
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[b]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&tot[b], v);
    }
    __syncthreads();
    if (threadIdx.x < 8) ws.cand_cnt[(int64_t)t * 8 + threadIdx.x] = tot[threadIdx.x];
}

// SMALL: the tiles of at most SORT_SMALL keys (4 or 8 per thread: 16 KB of
// shared memory, so 4 CTAs share an SM); the others in a launch of their own
// with room for SORT_CAP keys.  Each launch skips the other's tiles.
#define SORT_SMALL (SORT_THREADS * 8)
template <bool SMALL>
__global__ void __launch_bounds__(SORT_THREADS, SMALL ? 4 : 2) tile_sort_kernel(ss_ws_view ws, int total_tiles,
                                                                              ss_tile_shape ts) {
    extern __shared__ unsigned long long xs[];
    const int t = blockIdx.x;
    const int64_t cap = ws.max_instances;
    int64_t b = ws.tile_start[t], e = ws.tile_start[t + 1];
    if (e > cap) e = cap;
    if ((e - b <= SORT_SMALL) != SMALL) return;   // the other launch's tile
    uint32_t cnt[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // candidates per block (the mask bits)
    if (b >= e) {
        if (threadIdx.x < 8) ws.cand_cnt[(int64_t)t * 8 + threadIdx.x] = 0u;
        return;
    }
    const int n = (int)(e - b);
    unsigned long long* K = ws.keys + b;
    uint8_t* BM = ws.bmask + b;
    int x0, y0;   // tile origin (pixels)
    {
        const ss_layout* L = ws.layout;
        const ss_view_layout& vl = L->v[find_view_tile(L, t)];
        const int lt = t - vl.tile_off;
        x0 = (lt % vl.tiles_x) << ts.tw_log2;
        y0 = (lt / vl.tiles_x) << ts.th_log2;
    }
    if (n == 1) {
        gather_masks(ws, ts, K, BM, 1, x0, y0, cnt);
        store_block_counts(ws, t, cnt);
        return;
    }
    unsigned long long* Alt = ws.keys_alt + b;
    // chunks of SORT_CAP sorted in registers, with as many keys per thread as
    // spread the chunk over all threads (fewer sequential steps per thread)
    for (int c0 = 0; c0 < n; c0 += SORT_CAP) {
        const int m = min(SORT_CAP, n - c0);
        int N = 2;
        while (N < m) N <<= 1;
        if (N <= SORT_THREADS * 4) sort_chunk<4>(K + c0, m, N, xs);
        else if (SMALL || N <= SORT_THREADS * 8) sort_chunk<8>(K + c0, m, N, xs);
        else if (N <= SORT_THREADS * 16) sort_chunk<16>(K + c0, m, N, xs);
        else sort_chunk<SORT_KPL>(K + c0, m, N, xs);
    }
    if (n <= SORT_CAP) {
        gather_masks(ws, ts, K, BM, n, x0, y0, cnt);
        store_block_counts(ws, t, cnt);
        return;
    }
    // pairwise merges in global memory, ping-pong between K and Alt
    unsigned long long *src = K, *dst = Alt;
    for (int w = SORT_CAP; w < n; w <<= 1) {
        for (int lo = 0; lo < n; lo += 2 * w) {
            int na = min(w, n - lo), nb = min(w, max(0, n - lo - w));
            if (nb == 0) {
                for (int i = threadIdx.x; i < na; i += blockDim.x) dst[lo + i] = src[lo + i];
            } else {
                merge_runs(src + lo, na, src + lo + w, nb, dst + lo);
            }
        }
        __syncthreads();
        unsigned long long* tmp = src;
        src = dst;
        dst = tmp;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long k = src[i];
        if (src != K) K[i] = k;
        const uint32_t m = block_mask_of(ws, ts, k, x0, y0);
        BM[i] = (uint8_t)m;
#pragma unroll
        for (int bb = 0; bb < 8; ++bb) cnt[bb] += (m >> bb) & 1u;
    }
    store_block_counts(ws, t, cnt);
}

void ss_launch_bin_sort(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st) {
    ss_note_launch();
    scan_kernel<<<1, 1024, 0, st>>>(ws.tile_count, ws.tile_cursor, ws.tile_start, L.total_tiles, ws.status,
                                    ws.max_instances,
                                    ws.stats);
    if (L.total_records > 0) {
        ss_note_launch();
        scatter_kernel<<<(unsigned)((L.total_records + 255) / 256), 256, 0, st>>>(
            ws, L.total_records, a.p.r_cut * a.p.r_cut, a.p.mip_mode == 2 ? 0 : 1, a.ts);
    }
    static std::atomic<unsigned long long> optin{0};
    ss_smem_optin(tile_sort_kernel<false>, SORT_CAP * (int)sizeof(unsigned long long), optin);
    ss_note_launch();
    tile_sort_kernel<true><<<L.total_tiles, SORT_THREADS, SORT_SMALL * sizeof(unsigned long long), st>>>(
        ws, L.total_tiles, a.ts);
    ss_note_launch();
    tile_sort_kernel<false><<<L.total_tiles, SORT_THREADS, SORT_CAP * sizeof(unsigned long long), st>>>(
        ws, L.total_tiles, a.ts);
    // each (tile, block)'s list starts at the prefix sum of the candidate counts
    ss_launch_scan_u32(ws.cand_cnt, (int64_t)L.total_tiles * 8, ws.cand_off, ws.scan_tmp,
                       (unsigned long long)ws.cand_cap, ws.status, ws.stats + 10, st);
}

// ------------------------------------------------------------------------
// per-pixel rasteriser (Algorithm 1, Eq. alpha, Eq. compositing)
//
// One warp per 8 x 4 pixel block of a tile; every warp streams the tile's
// z_start-sorted list on its own (raster_common.cuh), so a warp with little
// work never waits for a busy one, and a warp whose 32 pixels have all
// reached K_max layers stops reading the list.  The kernel is persistent:
// as many warps as fit on the device take (tile, block) items from a queue
// in item order, so no warp slot idles while items are left.

// POOL: layers past dense_layers go to pool slots (an instance of its own, so
// that the all-dense one carries none of that code)
template <bool STATS, bool PP, bool CONS, bool POOL, int RWPB_FWD>
__device__ __forceinline__ void raster_fwd_block(const ss_ws_view& ws, const ss_fwd_args& a, const int gw,
                                                 unsigned char* fwd_smem) {
    ss_wstage* Wst = reinterpret_cast<ss_wstage*>(fwd_smem);   // [RWPB_FWD warps][stage depth]
    const ss_layout* L = ws.layout;
    const int lw = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = gw / a.ts.bpt, warp = gw - tile * a.ts.bpt;    // bpt blocks per tile
    const int view = find_view_tile(L, tile);
    const ss_view_layout& vl = L->v[view];
    const int lt = tile - vl.tile_off;
    const int tx = lt % vl.tiles_x, ty = lt / vl.tiles_x;
    const int x0 = tx << a.ts.tw_log2, y0 = ty << a.ts.th_log2;
    const int wx0 = 8 * (warp & ((1 << a.ts.bx_log2) - 1)), wy0 = 4 * (warp >> a.ts.bx_log2);   // 8 x 4 block
    const int lx = wx0 + (lane & 7), ly = wy0 + (lane >> 3);
    const int px = x0 + lx, py = y0 + ly;
    const bool inside = px < vl.width && py < vl.height;
    const float xl = (float)lx + 0.5f, yl = (float)ly + 0.5f;
    const float rc2 = a.p.r_cut * a.p.r_cut;
    const float kw = a.p.gamma * (0.5f / SS_PI_F);
    const int kmax = a.p.k_max;
    const int64_t gpix = vl.pixel_off + (int64_t)py * vl.width + px;
    const int64_t P = L->total_pixels;
    unsigned n_lane = 0, n_rect = 0, n_frag = 0, n_staged = 0, n_cov = 0;

    float C[SS_NCH];
#pragma unroll
    for (int c = 0; c < SS_NCH; ++c) C[c] = 0.f;
    float out[SS_NCH];
#pragma unroll
    for (int c = 0; c < SS_NCH; ++c) out[c] = 0.f;
    float Wg = 0.f, zmax = 0.f, Tb = 1.f, Acov = 0.f;
    int K = 0;
    bool done = !inside;
    // depth-consolidation term (Eq. cons_loss): per open layer its first
    // fragment's depth z_r and the shifted sums sum w (z - z_r), sum w (z - z_r)^2
    // (a well-conditioned variance); per pixel the running sums of the
    // composited layers' w_i and w_i z_i and the term itself.  Layer means
    // increase with the layer index (layers are separated by depth gaps and a
    // fragment's depth lies in its interval), so sum_{i<j} w_i w_j |z_i - z_j|
    // = sum_j w_j (z_j S_j - M_j) with S_j, M_j those sums over i < j.
    float zr = 0.f, Dz = 0.f, Dz2 = 0.f, Sb = 0.f, Mb = 0.f, Lp = 0.f;
    const int lsr = ws.ls_rows;
    // layers past dense_layers: the pixel's first pool slot and the last one taken
    uint32_t first_slot = SS_NO_SLOT, last_slot = SS_NO_SLOT;

    auto flush = [&]() {
        const float invW = 1.f / Wg;
        float hat[SS_NCH];
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) hat[c] = C[c] * invW;
        const float nl = sqrtf(C[8] * C[8] + C[9] * C[9] + C[10] * C[10]);
        const float inl = nl > 0.f ? 1.f / nl : 0.f;
        hat[8] = C[8] * inl; hat[9] = C[9] * inl; hat[10] = C[10] * inl;   // renormalised normal
        const float al = -expm1f(-kw * Wg);                                   // Eq. alpha
        const float tw = Tb * al;
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) out[c] = fmaf(tw, hat[c], out[c]);  // Eq. compositing
        if (CONS) {
            const float zk = C[11] * invW, mdz = Dz * invW;
            const float var = fmaf(Dz2, invW, -mdz * mdz);
            Lp = fmaf(tw, fmaf(zk, Sb, -Mb), Lp);
            Lp = fmaf(tw * tw, var, Lp);
            Sb += tw;
            Mb = fmaf(tw, zk, Mb);
        }
        if (a.with_backward) {
            if (!POOL || K < ws.dense_layers) {   // the dense planes (every pixel has a place)
                float* ls = ws.layer_state + (int64_t)K * lsr * P + gpix;
#pragma unroll
                for (int c = 0; c < SS_NCH; ++c) ls[c * P] = C[c];
                ls[12 * P] = Wg;
                if (CONS) {
                    ls[13 * P] = Dz;
                    ls[14 * P] = Dz2;
                    ls[15 * P] = zr;
                }
            } else {   // a pool slot, linked from the previous layer's slot or the pixel's first-slot word
                const unsigned long long t = atomicAdd(ws.stats + 9, 1ull);   // (ss_stats.pool_layers)
                const uint32_t slot = t < (unsigned long long)ws.pool_cap ? (uint32_t)t : SS_NO_SLOT;
                if (slot == SS_NO_SLOT) atomicOr(ws.status, SS_ERR_CAPACITY);
                if (K == ws.dense_layers) first_slot = slot;
                else if (last_slot != SS_NO_SLOT)
                    ws.layer_pool[(int64_t)last_slot * ws.pool_stride + lsr] = __uint_as_float(slot);
                last_slot = slot;
                if (slot != SS_NO_SLOT) {
                    float4* q = reinterpret_cast<float4*>(ws.layer_pool + (int64_t)slot * ws.pool_stride);
                    const float nx = __uint_as_float(SS_NO_SLOT);   // the chain ends here until a next layer
                    q[0] = make_float4(C[0], C[1], C[2], C[3]);
                    q[1] = make_float4(C[4], C[5], C[6], C[7]);
                    q[2] = make_float4(C[8], C[9], C[10], C[11]);
                    if (CONS) {
                        q[3] = make_float4(Wg, Dz, Dz2, zr);
                        q[4] = make_float4(nx, 0.f, 0.f, 0.f);
                    } else {
                        q[3] = make_float4(Wg, nx, 0.f, 0.f);
                    }
                }
            }
        }
        Acov = fmaf(Tb, al, Acov);
        Tb *= expf(-kw * Wg);
        ++K;
#pragma unroll
        for (int c = 0; c < SS_NCH; ++c) C[c] = 0.f;
        Wg = 0.f;
        zmax = 0.f;
        Dz = Dz2 = 0.f;
        if (K >= kmax) done = true;
    };

    const int64_t cap = ws.max_instances;
    int64_t beg = ws.tile_start[tile], end = ws.tile_start[tile + 1];
    if (end > cap) end = cap;
    if (beg > end) beg = end;
    const ss_rec* recs = ws.rec;   // keys hold batch-wide record indices
    // the backward pass's fragment list: (record, coverage word) of every
    // staged surfel that covers a pixel of this block, in list order;
    // the block's lists (candidates, covering entries) start at cand_off[tile * 8 + block]; a block
    // whose lists would pass the capacity is not rendered (the scan flagged SS_ERR_CAPACITY)
    const int64_t loff = ws.cand_off[(int64_t)tile * 8 + warp];
    const bool fits = (int64_t)ws.cand_off[(int64_t)tile * 8 + warp + 1] <= ws.cand_cap &&
                      ws.cand_off[(int64_t)tile * 8 + warp + 1] != 0xffffffffu;
    if (!fits) end = beg;
    uint2* clist = ws.cover_list ? ws.cover_list + loff : nullptr;
    uint32_t* alist = clist ? ws.cover_adv + loff : nullptr;
    uint32_t n_list = 0;
    ss_wstage* Wb = Wst + (a.p.stage_depth ? a.p.stage_depth : 2) * lw;
    // pass 1: the records whose support rectangle meets the block, in list
    // order, into the warp's candidate list (four chunks of keys in flight)
    uint32_t* cand = ws.cand_list + loff;
    int n_cand = 0;
    for (int64_t j0 = beg; j0 < end; j0 += 128) {
        ss_chunk c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = fetch_chunk(ws.keys, ws.bmask, j0 + 32 * u + lane, end);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool ov = c[u].live && ((c[u].bm >> warp) & 1u);
            const uint32_t m = __ballot_sync(0xffffffffu, ov);
            if (ov) cand[n_cand + __popc(m & ((1u << lane) - 1u))] = c[u].id;
            n_cand += __popc(m);
        }
    }
    __syncwarp();
    // pass 2: the candidates 32 at a time through a ring of D staging buffers
    // (chunks c+1 .. c+D-1 in flight while chunk c is processed)
    const int D = a.p.stage_depth ? a.p.stage_depth : 2;
    for (int j = 0; j + 1 < D; ++j) {   // prologue: the first D - 1 chunks
        const bool act = 32 * j + lane < n_cand;
        stage_ids(Wb[j], recs, act ? cand[32 * j + lane] : 0u, lane, act);
    }
    int buf = 0;
    // record indices of the next chunk to issue, read one iteration ahead
    uint32_t idn = 32 * (D - 1) + lane < n_cand ? cand[32 * (D - 1) + lane] : 0u;
    for (int b0 = 0; b0 < n_cand; b0 += 32) {
        if (__all_sync(0xffffffffu, done)) break;   // every pixel of the block has K_max layers
        {   // chunk b0 + 32 (D - 1) into the buffer processed last (one copy group, maybe empty)
            const int c0 = b0 + 32 * (D - 1);
            const int ib = buf + D - 1 >= D ? buf - 1 : buf + D - 1;
            stage_ids(Wb[ib], recs, idn, lane, c0 + lane < n_cand);
            idn = c0 + 32 + lane < n_cand ? cand[c0 + 32 + lane] : 0u;
        }
        if (b0 + 32 * D + lane < n_cand) {   // ask L2 for the records a chunk beyond the ring
            const char* pr = reinterpret_cast<const char*>(recs + cand[b0 + 32 * D + lane]);
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pr));
            asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pr + sizeof(ss_rec) - 1));
        }
        ss_wstage& W = Wb[buf];
        const int n = min(32, n_cand - b0);
        stage_finish(W, n, lane, (float)x0, (float)y0, D - 1);
        uint32_t my_mask = 0, my_adv = 0;
        uint32_t advc = 0;   // the slots whose fragment opened a layer at this lane's pixel
        // staged surfels whose exact support can reach a pixel centre of the block
        // (the block bit only says that the support's bounding box does; the
        // per-pixel filter's support is not the centre quadratic's: no test)
        bool may = false;
        if (lane < n) {
            const float4 g1 = W.h1[lane];
            const float bx = (float)wx0 - g1.z, by = (float)wy0 - g1.w;
            may = PP || ss_conic_box_may_cover(ss_conic_of(W.h0[lane], g1.x, g1.y, rc2), bx + 0.5f, bx + 7.5f,
                                                by + 0.5f, by + 3.5f);
        }
        for (uint32_t live = __ballot_sync(0xffffffffu, may); live; live &= live - 1) {
            const int s = __ffs(live) - 1;
            const float4 h0 = W.h0[s], h1 = W.h1[s], h2 = W.h2[s];
            float rho2, nf;
            bool cg;
            if constexpr (PP) {
                const ss_hit_pp h = ss_pixel_test_pp(h0, h1, fabsf(h2.z), xl - h1.z, yl - h1.w, rc2, a.p.sigma_f);
                rho2 = h.rho2;
                nf = h.nf;
                cg = h.cover && inside;
            } else {
                const ss_hit h = ss_pixel_test(h0, h1, xl - h1.z, yl - h1.w, rc2);
                rho2 = __fdividef(h.q, h.t);
                nf = fabsf(h2.z);
                cg = h.cover && inside;   // geometric coverage (support and cutoff)
            }
            if (STATS && inside) {
                const uint2 rr = make_uint2(__float_as_uint(W.zr[s].z), __float_as_uint(W.zr[s].w));
                ++n_lane;
                n_rect += in_rect(rr.x, rr.y, px, py) ? 1u : 0u;
            }
            if (cg && h2.z < 0.f) {   // support rectangle may clip this surfel
                const uint2 rr = make_uint2(__float_as_uint(W.zr[s].z), __float_as_uint(W.zr[s].w));
                cg = in_rect(rr.x, rr.y, px, py);
            }
            const uint32_t cm = __ballot_sync(0xffffffffu, cg);
            my_mask = lane == s ? cm : my_mask;
            if (cg && !done) {
                if (STATS) ++n_frag;
                const float w = nf * __expf(-0.5f * rho2);   // Eq. mip_weight (Eq. mip_eval per pixel)
                if (Wg > 0.f && h2.x > zmax) {   // gap: new layer (kept for the backward's replay)
                    advc |= 1u << s;
                    flush();
                }
                if (!done) {
                    zmax = fmaxf(zmax, h2.y);
                    const float4 c0v = W.c0[s], c1v = W.c1[s], c2v = W.c2[s];
                    C[0] = fmaf(w, c0v.x, C[0]); C[1] = fmaf(w, c0v.y, C[1]); C[2] = fmaf(w, c0v.z, C[2]);
                    C[3] = fmaf(w, c1v.x, C[3]); C[4] = fmaf(w, c1v.y, C[4]); C[5] = fmaf(w, c1v.z, C[5]);
                    C[6] = fmaf(w, c1v.w, C[6]); C[7] = fmaf(w, c2v.x, C[7]); C[8] = fmaf(w, c2v.y, C[8]);
                    C[9] = fmaf(w, c2v.z, C[9]); C[10] = fmaf(w, c2v.w, C[10]);
                    const float zc = 0.5f * (h2.x + h2.y);
                    C[11] = fmaf(w, zc, C[11]);
                    if (CONS) {
                        if (Wg == 0.f) zr = zc;   // the layer's first fragment
                        const float dz = zc - zr;
                        Dz = fmaf(w, dz, Dz);
                        Dz2 = fmaf(w * dz, dz, Dz2);
                    }
                    Wg += w;
                }
            }
        }
        if (clist) {   // slot s's layer-opening word: bit p of pixel p's advc, for the slots with one
            for (uint32_t any = __reduce_or_sync(0xffffffffu, advc); any; any &= any - 1) {
                const int s = __ffs(any) - 1;
                const uint32_t am = __ballot_sync(0xffffffffu, (advc >> s) & 1u);
                my_adv = lane == s ? am : my_adv;
            }
        }
        if (STATS) {   // warp-uniform counts, kept by lane 0
            n_staged += n;
            n_cov += __popc(__ballot_sync(0xffffffffu, lane < n && my_mask != 0u));
        }
        if (clist) {
            const bool keep = lane < n && my_mask != 0u;
            const uint32_t km = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const uint32_t e = n_list + __popc(km & ((1u << lane) - 1u));
                clist[e] = make_uint2(W.id[lane], my_mask);
                alist[e] = my_adv;
            }
            n_list += __popc(km);
        }
        buf = buf + 1 == D ? 0 : buf + 1;
        __syncwarp();
    }
    cp_async_wait0();   // copies of chunks an early exit left unread
    if (clist && lane == 0) ws.cover_count[(int64_t)tile * 8 + warp] = n_list;
    if (!done && Wg > 0.f) flush();
    if (STATS) {
        unsigned long long v[4] = {n_rect, n_lane, n_frag, (unsigned)K * (inside ? 1u : 0u)};
        for (int q = 0; q < 4; ++q) {
            unsigned long long x = v[q];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0 && x) atomicAdd(ws.stats + 1 + q, x);
        }
        if (lane == 0 && n_staged) atomicAdd(ws.stats + 6, (unsigned long long)n_staged);
        if (lane == 0 && n_cov) atomicAdd(ws.stats + 7, (unsigned long long)n_cov);
    }
    if (!inside) return;
    float4 o;
    o.x = fmaf(Tb, a.p.bg[0], out[0]);
    o.y = fmaf(Tb, a.p.bg[1], out[1]);
    o.z = fmaf(Tb, a.p.bg[2], out[2]);
    o.w = Acov;
    reinterpret_cast<float4*>(a.out_rgba)[gpix] = o;
    if (a.out_aov) {
#pragma unroll
        for (int c = 0; c < SS_N_AOV; ++c) a.out_aov[c * P + gpix] = out[3 + c];
        if (CONS) a.out_aov[SS_N_AOV * P + gpix] = Lp;
    }
    if (a.with_backward) {
        ws.pix_state[gpix] = __int_as_float(K);
        ws.pix_state[P + gpix] = Tb;
        ws.pix_state[2 * P + gpix] = __uint_as_float(first_slot);
    }
}

// 28 warps per SM (at most 72 registers a thread): more resident warps hide
// more of the staging and shared-memory latency (6.52 -> 6.39 ms against 24)
template <bool STATS, bool PP, bool CONS, bool POOL, int RWPB_FWD>
__global__ void __launch_bounds__(32 * RWPB_FWD, 28 / RWPB_FWD) raster_fwd_kernel(ss_ws_view ws, ss_fwd_args a,
                                                                                  int n_items) {
    extern __shared__ __align__(16) unsigned char fwd_smem[];
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(ws.work + 0, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        raster_fwd_block<STATS, PP, CONS, POOL, RWPB_FWD>(ws, a, item, fwd_smem);
        __syncwarp();
    }
}

template <bool STATS, bool PP, bool CONS, bool POOL, int W>
static void launch_raster_fwd(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st) {
    const int D = a.p.stage_depth ? a.p.stage_depth : 2;
    const int smem = D * W * (int)sizeof(ss_wstage);
    // opt in once for the deepest ring; resident CTAs depend on the depth
    static std::atomic<unsigned long long> optin{0}, resident[4];
    ss_smem_optin(raster_fwd_kernel<STATS, PP, CONS, POOL, W>, 3 * W * (int)sizeof(ss_wstage), optin);
    const int n_items = (int)(L.total_tiles * L.bpt);
    const int ctas = ss_resident_ctas(raster_fwd_kernel<STATS, PP, CONS, POOL, W>, 32 * W, smem, resident[D]);
    const int grid = max(1, min(ctas > 0 ? ctas : 1, (n_items + W - 1) / W));
    raster_fwd_kernel<STATS, PP, CONS, POOL, W><<<grid, 32 * W, smem, st>>>(ws, a, n_items);
}

template <bool STATS, bool PP, bool CONS, bool POOL>
static void launch_raster_fwd_w2(int w, const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a,
                                 cudaStream_t st) {
    if (w == 1) launch_raster_fwd<STATS, PP, CONS, POOL, 1>(ws, L, a, st);
    else if (w == 2) launch_raster_fwd<STATS, PP, CONS, POOL, 2>(ws, L, a, st);
    else launch_raster_fwd<STATS, PP, CONS, POOL, 4>(ws, L, a, st);
}

template <bool STATS, bool PP, bool CONS>
static void launch_raster_fwd_w(int w, const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a,
                                cudaStream_t st) {
    if (a.with_backward && ws.dense_layers < a.p.k_max) launch_raster_fwd_w2<STATS, PP, CONS, true>(w, ws, L, a, st);
    else launch_raster_fwd_w2<STATS, PP, CONS, false>(w, ws, L, a, st);
}

template <bool STATS>
static void launch_raster_fwd_mode(int w, const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a,
                                   cudaStream_t st) {
    if (a.p.mip_mode == 2) launch_raster_fwd_w<STATS, true, false>(w, ws, L, a, st);   // (no cons with mode 2)
    else if (a.p.cons) launch_raster_fwd_w<STATS, false, true>(w, ws, L, a, st);
    else launch_raster_fwd_w<STATS, false, false>(w, ws, L, a, st);
}

void ss_launch_raster_fwd(const ss_ws_view& ws, const ss_layout& L, const ss_fwd_args& a, cudaStream_t st) {
    if (L.total_tiles <= 0) return;
    ss_note_launch();
    const int w = a.p.fwd_warps ? a.p.fwd_warps : RWPB_FWD_DEFAULT;
    if (a.p.collect_stats) launch_raster_fwd_mode<true>(w, ws, L, a, st);
    else launch_raster_fwd_mode<false>(w, ws, L, a, st);
}

// ------------------------------------------------------------------------
// box filter of an RGBA image by an integer factor (supersampled reference)

__global__ void box_downsample_kernel(const float4* __restrict__ in, int W, int H, int f, float4* __restrict__ out) {
    const int Wo = W / f, Ho = H / f;
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= (int64_t)Wo * Ho) return;
    const int xo = (int)(o % Wo), yo = (int)(o / Wo);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < f; ++j)
        for (int i = 0; i < f; ++i) {
            const float4 v = in[(int64_t)(yo * f + j) * W + xo * f + i];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
    const float k = 1.f / (float)(f * f);
    out[o] = make_float4(acc.x * k, acc.y * k, acc.z * k, acc.w * k);
}

void ss_launch_box_downsample(const float* in, int W, int H, int f, float* out, cudaStream_t st) {
    const int64_t n = (int64_t)(W / f) * (H / f);
    if (n <= 0) return;
    ss_note_launch();
    box_downsample_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4*>(in), W, H, f,
                                                                       reinterpret_cast<float4*>(out));
}
