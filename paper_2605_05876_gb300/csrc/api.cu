// C ABI entry points (include/ss3d.h): argument checks, batch layout,
// workspace carving and the launch sequences.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <math.h>
#include <string.h>

#include <vector>

#include "ss3d_internal.cuh"

// ------------------------------------------------------------------------
// stage timing (host side): events recorded around each stage launch while a
// profile is open
namespace {
struct prof_rec {
    int stage;
    cudaEvent_t a, b;
};
struct profiler {
    bool on = false;
    std::vector<prof_rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
};
profiler g_prof;

}  // namespace

int ss_stage_open(int stage, cudaStream_t st) {
    if (!g_prof.on) return -1;
    prof_rec r{stage, g_prof.take(), g_prof.take()};
    cudaEventRecord(r.a, st);
    g_prof.recs.push_back(r);
    return (int)g_prof.recs.size() - 1;
}

void ss_stage_close(int handle, cudaStream_t st) {
    if (handle >= 0 && handle < (int)g_prof.recs.size()) cudaEventRecord(g_prof.recs[handle].b, st);
}

static std::atomic<long long> g_launches{0};
void ss_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" ss_status ss_launch_count(int64_t* out) {
    if (!out) return SS_ERR_INVALID_ARG;
    *out = (int64_t)g_launches.load(std::memory_order_relaxed);
    return SS_OK;
}

extern "C" ss_status ss_stream_capture_id(void* stream, uint64_t* id) {
    if (!id) return SS_ERR_INVALID_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    unsigned long long cid = 0;
    if (cudaStreamGetCaptureInfo((cudaStream_t)stream, &cs, &cid) != cudaSuccess) return SS_ERR_CUDA;
    *id = cs == cudaStreamCaptureStatusActive ? (uint64_t)cid : 0;
    return SS_OK;
}

extern "C" ss_status ss_profile_begin(void) {
    g_prof.on = true;
    for (auto& r : g_prof.recs) {
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.recs.clear();
    return SS_OK;
}

extern "C" ss_status ss_profile_end(ss_stage_times* out) {
    if (!out) return SS_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    ss_status st = SS_OK;
    for (auto& r : g_prof.recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) st = SS_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) st = SS_ERR_CUDA;
        out->ms[r.stage] += ms;
        out->launches[r.stage] += 1;
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.recs.clear();
    g_prof.on = false;
    return st;
}

#define CK(x)                                      \
    do {                                           \
        if ((x) != cudaSuccess) return SS_ERR_CUDA; \
    } while (0)

static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// launch shapes: only the values with a compiled kernel instance
static ss_status check_knobs(const ss_render_params* p) {
    if (!(p->fwd_warps == 0 || p->fwd_warps == 1 || p->fwd_warps == 2 || p->fwd_warps == 4)) return SS_ERR_INVALID_ARG;
    if (!(p->bwd_warps == 0 || p->bwd_warps == 2 || p->bwd_warps == 4 || p->bwd_warps == 8)) return SS_ERR_INVALID_ARG;
    if (!(p->pbwd_block == 0 || (p->pbwd_block >= 32 && p->pbwd_block <= 1024))) return SS_ERR_INVALID_ARG;
    if (p->screen_grad != 0 && p->screen_grad != 1) return SS_ERR_INVALID_ARG;
    if (p->mip_mode < 0 || p->mip_mode > 2) return SS_ERR_INVALID_ARG;
    if (p->cons != 0 && p->cons != 1) return SS_ERR_INVALID_ARG;
    if (p->cons && (p->mip_mode == 2 || !p->write_aov)) return SS_ERR_INVALID_ARG;
    // a tile is a whole number of 8 x 4 blocks, at most 8 of them
    const int tw = p->tile_w ? p->tile_w : SS_TILE, th = p->tile_h ? p->tile_h : SS_TILE;
    if (!(tw == 8 || tw == 16 || tw == 32) || !(th == 4 || th == 8 || th == 16 || th == 32)) return SS_ERR_INVALID_ARG;
    if ((tw / 8) * (th / 4) > 8) return SS_ERR_INVALID_ARG;
    if (p->stage_depth < 0 || p->stage_depth > 3) return SS_ERR_INVALID_ARG;
    if (p->deterministic != 0 && p->deterministic != 1) return SS_ERR_INVALID_ARG;
    if (p->det_rows < 0 || p->det_rows > 0xffffffffll) return SS_ERR_INVALID_ARG;
    if (p->dense_layers < 0 || p->dense_layers > p->k_max) return SS_ERR_INVALID_ARG;
    if (p->layer_pool < 0 || p->layer_pool > 0xffffffffll) return SS_ERR_INVALID_ARG;
    if (p->max_candidates < 0 || p->max_candidates > 0xffffffffll) return SS_ERR_INVALID_ARG;
    if (p->zero_grad_in_forward != 0 && p->zero_grad_in_forward != 1) return SS_ERR_INVALID_ARG;
    return SS_OK;
}

extern "C" void ss_default_params(ss_render_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->r_cut = 3.f;
    p->sigma_f = 0.5f;
    p->gamma = 6.28318530717958647692f;
    p->k_max = 16;
    p->z_near = 0.01f;
    p->write_aov = 1;
    p->lut_n = 128;
    p->max_instances = 0;
}

extern "C" const char* ss_error_string(ss_status s) {
    if (s == SS_OK) return "ok";
    if (s & SS_ERR_INVALID_ARG) return "invalid argument";
    if (s & SS_ERR_WORKSPACE) return "workspace too small";
    if (s & SS_ERR_CAPACITY) return "instance capacity exceeded";
    if (s & SS_ERR_TIMEOUT) return "device wait timed out";
    if (s & SS_ERR_NONFINITE) return "non-finite surfel parameter";
    if (s & SS_ERR_CUDA) return "CUDA runtime error";
    return "unknown status";
}

// ------------------------------------------------------------------------
// batch layout

static ss_status build_layout(const ss_batch_desc* b, const ss_render_params* p, ss_layout* L) {
    if (!b || !p || !L) return SS_ERR_INVALID_ARG;
    if (check_knobs(p)) return SS_ERR_INVALID_ARG;
    if (b->n_scenes < 1 || b->n_scenes > SS_MAX_SCENES) return SS_ERR_INVALID_ARG;
    if (b->n_views < 1 || b->n_views > SS_MAX_VIEWS) return SS_ERR_INVALID_ARG;
    if (!b->scene_offsets_host || !b->cams_host) return SS_ERR_INVALID_ARG;
    if (p->k_max < 1 || p->k_max > SS_KMAX_LIMIT) return SS_ERR_INVALID_ARG;
    if (!(p->r_cut > 0.f) || !(p->sigma_f >= 0.f) || !(p->gamma > 0.f) || p->lut_n < 2) return SS_ERR_INVALID_ARG;
    memset(L, 0, sizeof(*L));
    L->n_views = b->n_views;
    L->n_scenes = b->n_scenes;
    L->k_max = p->k_max;
    {
        const int tw = p->tile_w ? p->tile_w : SS_TILE, th = p->tile_h ? p->tile_h : SS_TILE;
        L->tw_log2 = 31 - __builtin_clz((unsigned)tw);
        L->th_log2 = 31 - __builtin_clz((unsigned)th);
        L->bx = tw / 8;
        L->bx_log2 = L->tw_log2 - 3;
        L->bpt = (tw / 8) * (th / 4);
    }
    for (int s = 0; s <= b->n_scenes; ++s) {
        L->scene_begin[s] = b->scene_offsets_host[s];
        if (s > 0 && L->scene_begin[s] < L->scene_begin[s - 1]) return SS_ERR_INVALID_ARG;
    }
    if (L->scene_begin[0] != 0) return SS_ERR_INVALID_ARG;
    for (int s = 0; s <= SS_MAX_SCENES; ++s) L->scene_view_begin[s] = b->n_views;
    int prev_scene = -1;
    int64_t pix = 0, rec = 0;
    int tiles = 0;
    for (int v = 0; v < b->n_views; ++v) {
        const ss_camera& c = b->cams_host[v];
        if (c.scene < 0 || c.scene >= b->n_scenes || c.scene < prev_scene) return SS_ERR_INVALID_ARG;
        if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768) return SS_ERR_INVALID_ARG;
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) return SS_ERR_INVALID_ARG;
        for (int s = prev_scene + 1; s <= c.scene; ++s) L->scene_view_begin[s] = v;
        prev_scene = c.scene;
        ss_view_layout& vl = L->v[v];
        vl.scene = c.scene;
        vl.width = c.width;
        vl.height = c.height;
        vl.tiles_x = (c.width + (1 << L->tw_log2) - 1) >> L->tw_log2;
        vl.tiles_y = (c.height + (1 << L->th_log2) - 1) >> L->th_log2;
        // (tile, block) items are numbered tile * 8 + block in 32-bit integers
        if ((int64_t)tiles + (int64_t)vl.tiles_x * vl.tiles_y > SS_MAX_TILES) return SS_ERR_INVALID_ARG;
        vl.tile_off = tiles;
        vl.pixel_off = pix;
        vl.rec_off = rec;
        vl.surfel_begin = L->scene_begin[c.scene];
        int64_t ns = L->scene_begin[c.scene + 1] - L->scene_begin[c.scene];
        if (ns > 0x7fffffffll) return SS_ERR_INVALID_ARG;
        vl.n_surfels = (int32_t)ns;
        tiles += vl.tiles_x * vl.tiles_y;
        pix += (int64_t)c.width * c.height;
        rec += ns;
    }
    for (int s = prev_scene + 1; s <= SS_MAX_SCENES; ++s) L->scene_view_begin[s] = b->n_views;
    // record indices are 32-bit in the instance keys and the block lists, and
    // 0xffffffff marks an unused row
    if (rec > SS_MAX_RECORDS) return SS_ERR_INVALID_ARG;
    L->total_tiles = tiles;
    L->total_pixels = pix;
    L->total_records = rec;
    return SS_OK;
}

struct ws_plan {
    size_t status, layout, vgeo, rec, rank, rbm, tc, ts, tcur, keys, keys_alt, bmask, cand, ccnt, coff, stmp, layer,
        pool, pix, grad, masks, madv, mcount, env_acc, jac, total;
    int64_t cand_cap;
    int64_t env_texels;   // irradiance + specular texels of one scene (0: no env-gradient scratch)
    // deterministic backward
    size_t d_icnt, d_coff, d_rows, d_rid, d_rcnt, d_roff, d_rcur, d_rlist, d_scan;
    int64_t det_cap;
};

// entries of the per-(tile, block) candidate and cover lists: max_candidates,
// or (blocks per tile) x max_instances
static int64_t cand_capacity(const ss_layout& L, const ss_render_params& p) {
    const int64_t c = p.max_candidates ? p.max_candidates : (int64_t)L.bpt * p.max_instances;
    return c < 0xffffffffll ? c : 0xffffffffll;
}

// layers per pixel in the dense planes (dense_layers; 0 = all k_max)
static int dense_layers(const ss_render_params& p) { return p.dense_layers > 0 ? p.dense_layers : p.k_max; }

// rows of the deterministic backward: det_rows, or (blocks per tile) x max_instances
static int64_t det_capacity(const ss_layout& L, const ss_render_params& p) {
    if (!p.deterministic) return 0;
    const int64_t c = p.det_rows ? p.det_rows : (int64_t)L.bpt * p.max_instances;
    return c < 0xffffffffll ? (c > 0 ? c : 1) : 0xffffffffll;
}

static ws_plan plan_ws(const ss_layout& L, const ss_render_params& p, int with_bwd, const ss_env_desc* ed) {
    ws_plan w;
    w.env_texels = (with_bwd && ed) ? (ss_env_irr_floats(ed) + ss_env_spec_floats(ed)) / 3 : 0;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    w.status = take(256);
    w.layout = take(sizeof(ss_layout));
    w.vgeo = take(sizeof(ss_view_geo) * SS_MAX_VIEWS);
    w.rec = take(sizeof(ss_rec) * (size_t)L.total_records);
    w.rank = take(sizeof(uint4) * (size_t)L.total_records);
    w.rbm = take(sizeof(uint2) * (size_t)L.total_records);
    w.tc = take(sizeof(uint32_t) * SS_CNT_STRIDE * (size_t)L.total_tiles);
    w.ts = take(sizeof(uint32_t) * ((size_t)L.total_tiles + 1));
    w.tcur = take(sizeof(uint32_t) * SS_CNT_STRIDE * (size_t)L.total_tiles);
    w.keys = take(sizeof(unsigned long long) * (size_t)p.max_instances);
    w.keys_alt = take(sizeof(unsigned long long) * (size_t)p.max_instances);
    w.bmask = take(sizeof(uint8_t) * (size_t)p.max_instances);
    w.cand_cap = cand_capacity(L, p);
    w.cand = take(sizeof(uint32_t) * (size_t)w.cand_cap);
    w.ccnt = take(sizeof(uint32_t) * 8 * (size_t)L.total_tiles);
    w.coff = take(sizeof(uint32_t) * (8 * (size_t)L.total_tiles + 1));
    w.stmp = take(sizeof(unsigned long long) * (size_t)(ss_det_scan_blocks(8 * (int64_t)L.total_tiles) + 1));
    if (with_bwd) {
        w.layer = take(sizeof(float) * (size_t)dense_layers(p) * (p.cons ? 16 : 13) * (size_t)L.total_pixels);
        w.pool = dense_layers(p) < p.k_max ? take(sizeof(float) * (p.cons ? 20 : 16) * (size_t)p.layer_pool) : 0;
        w.pix = take(sizeof(float) * 3 * (size_t)L.total_pixels);
        w.grad = take(sizeof(float) * SS_NGRAD * (size_t)L.total_records);
        w.masks = take(sizeof(uint2) * (size_t)w.cand_cap);
        w.madv = take(sizeof(uint32_t) * (size_t)w.cand_cap);
        w.mcount = take(sizeof(uint32_t) * 8 * (size_t)L.total_tiles);
        w.env_acc = take(sizeof(float4) * SS_ACC_STRIDE * (size_t)w.env_texels * (size_t)L.n_scenes);
        w.jac = p.screen_grad ? take(sizeof(float4) * 4 * (size_t)L.total_records) : 0;
    } else {
        w.layer = w.pool = w.pix = w.grad = w.masks = w.madv = w.mcount = w.env_acc = w.jac = 0;
    }
    w.det_cap = with_bwd ? det_capacity(L, p) : 0;
    if (w.det_cap) {
        const int64_t items = (int64_t)L.total_tiles * L.bpt, R = L.total_records;
        w.d_icnt = take(sizeof(uint32_t) * (size_t)items);
        w.d_coff = take(sizeof(uint32_t) * (size_t)(items + 1));
        w.d_rows = take(sizeof(float) * SS_NGRAD * (size_t)w.det_cap);
        w.d_rid = take(sizeof(uint32_t) * (size_t)w.det_cap);
        w.d_rcnt = take(sizeof(uint32_t) * (size_t)R);
        w.d_roff = take(sizeof(uint32_t) * (size_t)(R + 1));
        w.d_rcur = take(sizeof(uint32_t) * (size_t)R);
        w.d_rlist = take(sizeof(uint32_t) * (size_t)w.det_cap);
        const int64_t nb = ss_det_scan_blocks(items > R ? items : R);
        w.d_scan = take(sizeof(unsigned long long) * (size_t)(nb + 1));
    } else {
        w.d_icnt = w.d_coff = w.d_rows = w.d_rid = w.d_rcnt = w.d_roff = w.d_rcur = w.d_rlist = w.d_scan = 0;
    }
    w.total = o;
    return w;
}

static ss_ws_view carve(void* ws, const ws_plan& w, const ss_render_params& p, int with_bwd) {
    char* b = (char*)ws;
    ss_ws_view v;
    v.status = (int*)(b + w.status);
    v.stats = (unsigned long long*)(b + w.status + SS_STATS_OFFSET);
    v.work = (unsigned int*)(b + w.status + SS_WORK_OFFSET);
    v.layout = (ss_layout*)(b + w.layout);
    v.vgeo = (ss_view_geo*)(b + w.vgeo);
    v.rec = (ss_rec*)(b + w.rec);
    v.inst_rank = (uint4*)(b + w.rank);
    v.rec_bmask = (uint2*)(b + w.rbm);
    v.tile_count = (uint32_t*)(b + w.tc);
    v.tile_start = (uint32_t*)(b + w.ts);
    v.tile_cursor = (uint32_t*)(b + w.tcur);
    v.keys = (unsigned long long*)(b + w.keys);
    v.keys_alt = (unsigned long long*)(b + w.keys_alt);
    v.bmask = (uint8_t*)(b + w.bmask);
    v.cand_list = (uint32_t*)(b + w.cand);
    v.cand_cnt = (uint32_t*)(b + w.ccnt);
    v.cand_off = (uint32_t*)(b + w.coff);
    v.scan_tmp = (unsigned long long*)(b + w.stmp);
    v.cand_cap = w.cand_cap;
    v.layer_state = with_bwd ? (float*)(b + w.layer) : nullptr;
    v.ls_rows = p.cons ? 16 : 13;
    v.dense_layers = dense_layers(p);
    v.pool_stride = p.cons ? 20 : 16;
    v.pool_cap = (with_bwd && v.dense_layers < p.k_max) ? p.layer_pool : 0;
    v.layer_pool = (with_bwd && w.pool) ? (float*)(b + w.pool) : nullptr;
    v.pix_state = with_bwd ? (float*)(b + w.pix) : nullptr;
    v.grad_rec = with_bwd ? (float*)(b + w.grad) : nullptr;
    v.cover_list = with_bwd ? (uint2*)(b + w.masks) : nullptr;
    v.cover_adv = with_bwd ? (uint32_t*)(b + w.madv) : nullptr;
    v.cover_count = with_bwd ? (uint32_t*)(b + w.mcount) : nullptr;
    v.env_acc = (with_bwd && w.env_texels) ? (float4*)(b + w.env_acc) : nullptr;
    v.ssg_jac = (with_bwd && p.screen_grad) ? (float4*)(b + w.jac) : nullptr;
    v.env_texels = w.env_texels;
    v.max_instances = p.max_instances;
    v.det_cap = with_bwd ? w.det_cap : 0;
    v.det_icnt = v.det_cap ? (uint32_t*)(b + w.d_icnt) : nullptr;
    v.det_coff = v.det_cap ? (uint32_t*)(b + w.d_coff) : nullptr;
    v.det_rows = v.det_cap ? (float*)(b + w.d_rows) : nullptr;
    v.det_rid = v.det_cap ? (uint32_t*)(b + w.d_rid) : nullptr;
    v.det_rcnt = v.det_cap ? (uint32_t*)(b + w.d_rcnt) : nullptr;
    v.det_roff = v.det_cap ? (uint32_t*)(b + w.d_roff) : nullptr;
    v.det_rcur = v.det_cap ? (uint32_t*)(b + w.d_rcur) : nullptr;
    v.det_rlist = v.det_cap ? (uint32_t*)(b + w.d_rlist) : nullptr;
    v.det_scan = v.det_cap ? (unsigned long long*)(b + w.d_scan) : nullptr;
    v.det_maxbits = (unsigned int*)(b + w.status + SS_DET_OFFSET);
    return v;
}

// camera centre o = -R^-1 t (double-float) and det R of every view, in FP64
__global__ void view_geo_kernel(const ss_camera* cams, ss_view_geo* out, int n_views) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    const ss_camera& c = cams[v];
    double R[9], t[3] = {c.t[0], c.t[1], c.t[2]};
    for (int k = 0; k < 9; ++k) R[k] = c.R[k];
    double A[9];  // adjugate
    A[0] = R[4] * R[8] - R[5] * R[7]; A[1] = R[2] * R[7] - R[1] * R[8]; A[2] = R[1] * R[5] - R[2] * R[4];
    A[3] = R[5] * R[6] - R[3] * R[8]; A[4] = R[0] * R[8] - R[2] * R[6]; A[5] = R[2] * R[3] - R[0] * R[5];
    A[6] = R[3] * R[7] - R[4] * R[6]; A[7] = R[1] * R[6] - R[0] * R[7]; A[8] = R[0] * R[4] - R[1] * R[3];
    double det = R[0] * A[0] + R[1] * A[3] + R[2] * A[6];
    ss_view_geo g;
    for (int r = 0; r < 3; ++r) {
        double o = -(A[r * 3] * t[0] + A[r * 3 + 1] * t[1] + A[r * 3 + 2] * t[2]) / det;
        g.o_hi[r] = (float)o;
        g.o_lo[r] = (float)(o - (double)g.o_hi[r]);
    }
    g.detR = (float)det;
    g.pad_ = 0.f;
    out[v] = g;
}

__global__ void set_layout_kernel(ss_layout* dst, ss_layout src) {
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(ss_layout) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

static bool env_desc_ok(const ss_env_desc* d);

extern "C" ss_status ss_workspace_size(const ss_batch_desc* b, const ss_render_params* p, const ss_env_desc* ed,
                                       int32_t with_backward, size_t* bytes) {
    if (!bytes || !p || p->max_instances <= 0 || p->max_instances > 0xffffffffll) return SS_ERR_INVALID_ARG;
    if (check_knobs(p)) return SS_ERR_INVALID_ARG;
    ss_layout L;   // on the stack: entry points may be called from several threads
    ss_status st = build_layout(b, p, &L);
    if (st) return st;
    if (ed && !env_desc_ok(ed)) return SS_ERR_INVALID_ARG;
    *bytes = plan_ws(L, *p, with_backward, ed).total;
    return SS_OK;
}

// ------------------------------------------------------------------------
// BRDF table and environment

extern "C" ss_status ss_read_stats(void* ws, ss_stats* out, void* stream) {
    if (!ws || !out) return SS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out, (char*)ws + SS_STATS_OFFSET, sizeof(ss_stats), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SS_OK;
}

extern "C" ss_status ss_brdf_lut(float* lut_dev, int32_t n, void* stream) {
    if (!lut_dev || n < 4 || n > 1024) return SS_ERR_INVALID_ARG;
    ss_launch_brdf_lut(lut_dev, n, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return SS_OK;
}

static bool env_desc_ok(const ss_env_desc* d) {
    if (!d) return false;
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    return pow2(d->width) && pow2(d->height) && d->width >= 8 && d->height >= 4 && d->width <= 16384 &&
           d->height <= 8192 && d->n_levels >= 1 && d->n_levels <= 16 && d->irr_width >= 1 && d->irr_height >= 1 &&
           d->irr_width <= d->width && pow2(d->irr_width) && d->irr_height <= 512;
}

extern "C" ss_status ss_env_sizes(const ss_env_desc* d, int64_t* irr_floats, int64_t* spec_floats,
                                  int64_t* aux_floats) {
    if (!env_desc_ok(d)) return SS_ERR_INVALID_ARG;
    if (irr_floats) *irr_floats = ss_env_irr_floats(d);
    if (spec_floats) *spec_floats = ss_env_spec_floats(d);
    if (aux_floats) *aux_floats = ss_env_aux_floats(d);
    return SS_OK;
}

extern "C" ss_status ss_env_prefilter(const ss_env_desc* d, int32_t n_envs, const float* env_dev, float* irr_dev,
                                      float* spec_dev, float* aux_dev, void* stream) {
    if (!env_desc_ok(d) || n_envs < 1 || !env_dev || !irr_dev || !spec_dev || !aux_dev) return SS_ERR_INVALID_ARG;
    if (d->n_levels < 2 && d->n_levels != 1) return SS_ERR_INVALID_ARG;
    {
        ss_stage_scope sc(5, (cudaStream_t)stream);
        ss_launch_env_prefilter(d, n_envs, env_dev, irr_dev, spec_dev, aux_dev, (cudaStream_t)stream);
    }
    CK(cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status ss_env_prefilter_backward(const ss_env_desc* d, int32_t n_envs, const float* d_irr_dev,
                                               const float* d_spec_dev, const float* aux_dev, float* d_env_dev,
                                               void* stream) {
    if (!env_desc_ok(d) || n_envs < 1 || !aux_dev || !d_env_dev) return SS_ERR_INVALID_ARG;
    {
        ss_stage_scope sc(6, (cudaStream_t)stream);
        ss_launch_env_prefilter_bwd(d, n_envs, d_irr_dev, d_spec_dev, aux_dev, d_env_dev, (cudaStream_t)stream);
    }
    CK(cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status ss_env_prefilter_backward_ordered(const ss_env_desc* d, int32_t n_envs, const float* d_irr_dev,
                                                       const float* d_spec_dev, const float* aux_dev,
                                                       float* d_env_dev, void* stream) {
    if (!env_desc_ok(d) || n_envs < 1 || !aux_dev || !d_env_dev) return SS_ERR_INVALID_ARG;
    {
        ss_stage_scope sc(6, (cudaStream_t)stream);
        ss_launch_env_prefilter_bwd(d, n_envs, d_irr_dev, d_spec_dev, aux_dev, d_env_dev, (cudaStream_t)stream, true);
    }
    CK(cudaGetLastError());
    return SS_OK;
}

// ------------------------------------------------------------------------
// render

static ss_status check_render_args(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                                   const ss_env_desc* ed, const ss_env_maps* env, void* ws) {
    if (!b || !s || !p || !ed || !env || !ws || !b->cams_dev) return SS_ERR_INVALID_ARG;
    if (!s->pos || !s->quat || !s->log_scale || !s->albedo || !s->roughness || !s->metallic) return SS_ERR_INVALID_ARG;
    if (!env->irr || !env->spec || !env->lut || !env_desc_ok(ed)) return SS_ERR_INVALID_ARG;
    if (((uintptr_t)s->quat & 15) || ((uintptr_t)s->log_scale & 7) || ((uintptr_t)ws & 255)) return SS_ERR_INVALID_ARG;
    if (p->max_instances <= 0 || p->max_instances > 0xffffffffll) return SS_ERR_INVALID_ARG;
    return check_knobs(p);
}

static ss_status forward_core(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                              const ss_env_desc* ed, const ss_env_maps* env, float* out_rgba, float* out_aov,
                              void* ws, size_t ws_bytes, int with_bwd, int stop_after_count, cudaStream_t st,
                              ss_layout& L, ss_ws_view& W) {
    ss_status e = check_render_args(b, s, p, ed, env, ws);
    if (e) return e;
    e = build_layout(b, p, &L);
    if (e) return e;
    ws_plan plan = plan_ws(L, *p, with_bwd, ed);
    if (ws_bytes < plan.total) return SS_ERR_WORKSPACE;
    W = carve(ws, plan, *p, with_bwd);
    ss_fwd_args a;
    a.s = *s;
    a.p = *p;
    a.ts = {L.tw_log2, L.th_log2, L.bx_log2, L.bpt};
    if (p->mip_mode == 1) a.p.sigma_f = 0.f;   // no MIP filter: Sigma_mip = I, n_f = 1
    a.ed = *ed;
    a.env = *env;
    a.cams = b->cams_dev;
    a.out_rgba = out_rgba;
    a.out_aov = p->write_aov ? out_aov : nullptr;
    a.with_backward = with_bwd;
    CK(cudaMemsetAsync(W.status, 0, 256, st));   // status word and work counters
    ss_note_launch();
    set_layout_kernel<<<1, 256, 0, st>>>(W.layout, L);
    ss_note_launch();
    view_geo_kernel<<<(L.n_views + 63) / 64, 64, 0, st>>>(b->cams_dev, W.vgeo, L.n_views);
    CK(cudaMemsetAsync(W.tile_count, 0, sizeof(uint32_t) * SS_CNT_STRIDE * (size_t)L.total_tiles, st));
    CK(cudaMemsetAsync(W.tile_cursor, 0, sizeof(uint32_t) * SS_CNT_STRIDE * (size_t)L.total_tiles, st));
    {
        ss_stage_scope sc(0, st);
        ss_launch_project(W, L, a, st);
    }
    {
        ss_stage_scope sc(1, st);
        ss_launch_bin_sort(W, L, a, st);  // for a count, the scatter is bounded by capacity 1
    }
    if (stop_after_count) {
        CK(cudaGetLastError());
        return SS_OK;
    }
    {
        ss_stage_scope sc(2, st);
        ss_launch_raster_fwd(W, L, a, st);
    }
    CK(cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status ss_render_forward(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                                       const ss_env_desc* ed, const ss_env_maps* env, float* out_rgba_dev,
                                       float* out_aov_dev, void* ws, size_t ws_bytes, void* stream) {
    if (!out_rgba_dev || (p && p->write_aov && !out_aov_dev)) return SS_ERR_INVALID_ARG;
    ss_layout L;
    ss_ws_view W;
    // the workspace decides whether backward state is kept: use the larger plan if it fits
    int with_bwd = 0;
    if (b && p && p->max_instances > 0) {
        ss_layout Lt;
        if (build_layout(b, p, &Lt) == SS_OK && ws_bytes >= plan_ws(Lt, *p, 1, ed).total) with_bwd = 1;
    }
    return forward_core(b, s, p, ed, env, out_rgba_dev, out_aov_dev, ws, ws_bytes, with_bwd, 0,
                        (cudaStream_t)stream, L, W);
}

extern "C" ss_status ss_count_instances(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                                        const ss_env_desc* ed, const ss_env_maps* env, void* ws, size_t ws_bytes,
                                        int64_t* count, void* stream) {
    if (!count || !p) return SS_ERR_INVALID_ARG;
    ss_render_params q = *p;
    q.max_instances = 1;
    ss_layout L;
    ss_ws_view W;
    cudaStream_t st = (cudaStream_t)stream;
    ss_status e = forward_core(b, s, &q, ed, env, nullptr, nullptr, ws, ws_bytes, 0, 1, st, L, W);
    if (e) return e;
    // the scan's 64-bit total (the 32-bit tile starts are clamped to the capacity)
    unsigned long long total = 0;
    CK(cudaMemcpyAsync(&total, W.stats, sizeof(total), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *count = (int64_t)total;
    return SS_OK;
}

extern "C" ss_status ss_render_backward(const ss_batch_desc* b, const ss_surfels* s, const ss_render_params* p,
                                        const ss_env_desc* ed, const ss_env_maps* env, const float* out_rgba_dev,
                                        const float* out_aov_dev, const float* d_rgba_dev, const float* d_aov_dev,
                                        ss_surfel_grads* g, ss_env_map_grads* genv, void* ws, size_t ws_bytes,
                                        void* stream) {
    ss_status e = check_render_args(b, s, p, ed, env, ws);
    if (e) return e;
    if (!out_rgba_dev || !d_rgba_dev || !g) return SS_ERR_INVALID_ARG;
    // the densification statistic needs its per-record scratch in the workspace
    if ((g->screen_grad_norm || g->screen_grad_views) && !p->screen_grad) return SS_ERR_INVALID_ARG;
    if (p->mip_mode == 2) return SS_ERR_INVALID_ARG;   // the per-pixel MIP filter is forward-only
    if (p->cons && !d_aov_dev) return SS_ERR_INVALID_ARG;   // its upstream gradient is d_aov's tenth plane
    if (p->write_aov && d_aov_dev && !out_aov_dev) return SS_ERR_INVALID_ARG;
    ss_layout L;   // on the stack: entry points may be called from several threads
    e = build_layout(b, p, &L);
    if (e) return e;
    ws_plan plan = plan_ws(L, *p, 1, ed);
    if (ws_bytes < plan.total) return SS_ERR_WORKSPACE;
    ss_ws_view W = carve(ws, plan, *p, 1);
    cudaStream_t st = (cudaStream_t)stream;
    ss_bwd_args a;
    a.f.s = *s;
    a.f.p = *p;
    a.f.ts = {L.tw_log2, L.th_log2, L.bx_log2, L.bpt};
    if (p->mip_mode == 1) a.f.p.sigma_f = 0.f;
    a.f.ed = *ed;
    a.f.env = *env;
    a.f.cams = b->cams_dev;
    a.f.out_rgba = nullptr;
    a.f.out_aov = nullptr;
    a.f.with_backward = 1;
    a.out_rgba = out_rgba_dev;
    a.out_aov = p->write_aov ? out_aov_dev : nullptr;
    a.d_rgba = d_rgba_dev;
    a.d_aov = p->write_aov ? d_aov_dev : nullptr;
    a.g = *g;
    ss_env_map_grads ge = {nullptr, nullptr};
    a.genv = genv ? *genv : ge;
    // deterministic mode: the most views of a scene, and log2 of a bound on the
    // contributions one env texel can receive (every surfel side's irradiance
    // taps and every record's specular taps: 8 each)
    a.det_vmax = 1;
    a.det_cbits = 1;
    if (W.det_cap) {
        int vmax = 1;
        for (int sc = 0; sc < L.n_scenes; ++sc) vmax = std::max(vmax, L.scene_view_begin[sc + 1] - L.scene_view_begin[sc]);
        const double contrib = 8.0 * ((double)L.scene_begin[L.n_scenes] + (double)L.total_records) + 1.0;
        a.det_vmax = vmax;
        a.det_cbits = (int)std::ceil(std::log2(contrib));
        if (a.det_cbits > 40) return SS_ERR_INVALID_ARG;   // the fixed-point sums would keep too few bits
    }
    // the per-record gradient rows start at zero: cleared here, or by the
    // projection pass of the forward that preceded this call
    if (!p->zero_grad_in_forward)
        CK(cudaMemsetAsync(W.grad_rec, 0, sizeof(float) * SS_NGRAD * (size_t)L.total_records, st));
    if (a.genv.irr || a.genv.spec)
        CK(cudaMemsetAsync(W.env_acc, 0, sizeof(float4) * SS_ACC_STRIDE * (size_t)W.env_texels * (size_t)L.n_scenes,
                           st));
    CK(cudaMemsetAsync(W.work + 1, 0, sizeof(unsigned int), st));   // backward work-queue head
    if (W.det_cap) {
        CK(cudaMemsetAsync(W.det_rid, 0xff, sizeof(uint32_t) * (size_t)W.det_cap, st));
        CK(cudaMemsetAsync(W.det_rcnt, 0, sizeof(uint32_t) * (size_t)L.total_records, st));
        CK(cudaMemsetAsync(W.det_rcur, 0, sizeof(uint32_t) * (size_t)L.total_records, st));
        CK(cudaMemsetAsync(W.det_maxbits, 0, sizeof(unsigned int), st));
    }
    {
        ss_stage_scope sc(8, st);
        ss_launch_screen_grad_jac(W, L, a, st);
    }
    {
        ss_stage_scope sc(3, st);
        if (W.det_cap) ss_launch_det_item_offsets(W, L, st);
        ss_launch_raster_bwd(W, L, a, st);
        if (W.det_cap) {
            const bool ssg = W.ssg_jac && (a.g.screen_grad_norm || a.g.screen_grad_views);
            ss_launch_det_record_sums(W, L, (p->cons || a.d_aov) ? 21 : 12, ssg, st);
            ss_launch_det_env_bound(W, L, st);
        }
    }
    {
        ss_stage_scope sc(4, st);
        ss_launch_project_bwd(W, L, a, st);
    }
    CK(cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status ss_box_downsample(const float* in_dev, int32_t width, int32_t height, int32_t factor,
                                       float* out_dev, void* stream) {
    if (!in_dev || !out_dev || factor < 1 || factor > 16 || width < 1 || height < 1 || width % factor ||
        height % factor)
        return SS_ERR_INVALID_ARG;
    ss_launch_box_downsample(in_dev, width, height, factor, out_dev, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status ss_read_status(void* ws, void* stream) {
    if (!ws) return SS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    CK(cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return (ss_status)v;
}
