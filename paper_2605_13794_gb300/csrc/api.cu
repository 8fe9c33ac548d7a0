// api.cu -- host side of the C ABI declared in gsblitz.h: argument checks,
// workspace layout, and the order of kernel launches for each call.
#include <math.h>
#include <atomic>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "gs_internal.cuh"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                                                                       \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);                                                   \
    } while (0)

struct Layout {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        size_t o = off;
        off += count * sizeof(T);
        return o;
    }
};

struct Offsets {
    size_t cand_g, cand_mask, gate_g, gate_mask, rec_first, cgrad, rec_g, rec_cam, rd0, rd1, rd2, rect, tt, inst_off, clampm, rgrad, dkey, tile_cnt, tile_cur, tile_last;
    size_t tkey0, tkey1, tval0, tval1, slots, imp_slots, ranges, n_contrib, T_final, imp_w, imp_a, sel_cum, sel_bsum;
    size_t selk0, selk1, selv0, selv1, loss_maps, loss_partial, lb_status, rx_status, red_partial,
        ctr, d_cams, d_adam_step, d_adam_coef;
    size_t mkey0, mkey1, mval0, mval1, mcum, mbsum, mrx_status, mlb, mhist, mctr;
    size_t total;
    size_t lb_words, rx_words, red_words, loss_partial_words;
};

Offsets plan(const gs_capacity &c)
{
    Offsets o;
    Layout L;
    const size_t N = (size_t)c.max_gaussians, R = (size_t)c.max_records, I = (size_t)c.max_instances;
    const size_t T = (size_t)c.max_tiles, P = (size_t)c.max_pixels;
    o.cand_g = L.take<uint32_t>(N);
    o.cand_mask = L.take<unsigned long long>(N);
    o.gate_g = L.take<uint32_t>(N);
    o.gate_mask = L.take<unsigned long long>(N);
    o.rec_first = L.take<uint32_t>(N);
    const bool fwd_only = (c.flags & GS_CAP_FORWARD_ONLY) != 0;
    o.cgrad = L.take<float>(fwd_only ? 0 : R * gs::kGradRow);
    o.rec_g = L.take<uint32_t>(R);
    o.rec_cam = L.take<uint16_t>(R);
    o.rd0 = L.take<float4>(R);
    o.rd1 = L.take<float4>(R);
    o.rd2 = L.take<float4>(R);
    o.rect = L.take<uint2>(R);
    o.tt = L.take<uint32_t>(R);
    o.inst_off = L.take<uint32_t>(R);
    o.clampm = L.take<uint8_t>(R);
    o.rgrad = L.take<float>(fwd_only ? 0 : R * gs::kSlotFloats);
    o.dkey = L.take<uint32_t>(R);
    o.tkey0 = L.take<uint32_t>(I);
    o.tkey1 = L.take<uint32_t>(I);
    o.tval0 = L.take<uint32_t>(I);
    o.tval1 = L.take<uint32_t>(I);
    o.slots = L.take<float>(fwd_only ? 0 : I * gs::kSlotFloats);
    o.imp_slots = L.take<float2>(I); // importance (w, a) per instance
    o.ranges = L.take<uint2>(T);
    o.tile_cnt = L.take<uint32_t>(T);
    o.tile_cur = L.take<uint32_t>(T);
    o.tile_last = L.take<uint32_t>(T);
    o.n_contrib = L.take<uint32_t>(P);
    o.T_final = L.take<float>(P);
    o.imp_w = L.take<float>(R);
    o.imp_a = L.take<uint32_t>(R);
    o.sel_cum = L.take<double>(R);
    o.sel_bsum = L.take<unsigned long long>(R / 4096 + 2);
    o.selk0 = L.take<uint32_t>(R);
    o.selk1 = L.take<uint32_t>(R);
    o.selv0 = L.take<uint32_t>(R);
    o.selv1 = L.take<uint32_t>(R);
    o.loss_maps = L.take<float>(fwd_only ? 0 : P * 3 * 3); // per pixel and channel: F0, F1, F2 (planar)
    o.loss_partial_words = fwd_only ? 0 : 2 * 3 * (P / 1024 + 65536);
    o.loss_partial = L.take<float>(o.loss_partial_words);
    // look-back words: one per chunk of the smallest chunked pass (the
    // projection's candidates) plus the ticket, and the binning's two regions
    // (records of its count pass, tiles of its tile scan)
    const size_t nb = (N > R ? N : R) / 64 + 2;
    o.lb_words = nb + 1 + T / 1024 + 4;
    o.lb_status = L.take<unsigned long long>(o.lb_words);
    const size_t items = (R > I ? R : I);
    // the histograms, then the look-back state of up to four passes, for the
    // smallest (1024-key) blocks
    o.rx_words = gs::kRxHistWords + 4 * ((items / (gs::kSortThreads * 4) + 1) * 256 + 1);
    o.rx_status = L.take<uint32_t>(o.rx_words);
    o.red_words = R / 128 + 2;
    o.red_partial = L.take<float>(o.red_words);
    o.ctr = L.take<gs::DevCounters>(1);
    o.d_cams = L.take<gs::CamTable>(1);
    o.d_adam_step = L.take<int>(1);
    o.d_adam_coef = L.take<float>(2 * GS_MAX_ADAM_GROUPS);
    const size_t NM = (c.flags & GS_CAP_MODEL_OPS) ? N : 0; // model-level scratch
    o.mkey0 = L.take<uint32_t>(NM);
    o.mkey1 = L.take<uint32_t>(NM);
    o.mval0 = L.take<uint32_t>(NM);
    o.mval1 = L.take<uint32_t>(NM);
    o.mcum = L.take<double>(NM);
    o.mbsum = L.take<double>(NM ? NM / 4096 + 2 : 0);
    o.mrx_status = L.take<uint32_t>(NM ? (NM / (gs::kSortThreads * 8) + 1) * 256 + 1 : 0);
    o.mlb = L.take<unsigned long long>(NM ? NM / 256 + 3 : 0);
    o.mhist = L.take<uint32_t>(4 * 256);
    o.mctr = L.take<gs::DevCounters>(1);
    o.total = (L.off + 255) & ~(size_t)255;
    return o;
}

int check_cap(const gs_capacity *c)
{
    if (!c) return fail(GS_ERR_INVALID_ARG, "capacity is NULL");
    if (c->max_gaussians < 0 || c->max_records < 0 || c->max_instances < 0 || c->max_tiles < 0 || c->max_pixels < 0)
        return fail(GS_ERR_INVALID_ARG, "negative capacity");
    if (c->max_cameras < 1 || c->max_cameras > GS_MAX_CAMERAS)
        return fail(GS_ERR_INVALID_ARG, "max_cameras must be in [1, %d]", GS_MAX_CAMERAS);
    if (c->max_instances >= (1ll << 30) || c->max_records >= (1ll << 30))
        return fail(GS_ERR_INVALID_ARG, "max_instances and max_records must be below 2^30");
    if (c->max_gaussians >= (1ll << 32) - 1) return fail(GS_ERR_INVALID_ARG, "max_gaussians must be below 2^32 - 1");
    return GS_OK;
}

std::atomic<long long> g_launches{0};

} // namespace

void gs::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int gs::report_error(int code, const char *msg)
{
    return fail(code, "%s", msg);
}

static cudaError_t kt_release(gs_workspace *ws)
{
    cudaError_t e = cudaSuccess, e2;
    for (int k = 0; k < GS_KT_COUNT; k++)
        for (int i = 0; i < gs_workspace::kTimedPairs; i++)
            for (int h = 0; h < 2; h++)
                if (ws->kt.ev[k][i][h]) {
                    if ((e2 = cudaEventDestroy(ws->kt.ev[k][i][h])) != cudaSuccess) e = e2;
                    ws->kt.ev[k][i][h] = nullptr;
                }
    ws->kt.on = 0;
    return e;
}

// Records one event of a timed launch: an ordinary record on an eager stream,
// an event node (cudaEventRecordExternal) under stream capture, which every
// replay of the graph records again.
static void kt_record(cudaEvent_t ev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return;
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else if (cs == cudaStreamCaptureStatusNone)
        cudaEventRecord(ev, st);
}

void gs::kt_begin(gs_workspace *ws, int id, cudaStream_t st)
{
    if (!ws->kt.on || !((ws->kt.mask >> id) & 1u)) return;
    ws->kt.launches[id]++;
    if (ws->kt.used[id] >= gs_workspace::kTimedPairs) return;
    kt_record(ws->kt.ev[id][ws->kt.used[id]][0], st);
}

void gs::kt_end(gs_workspace *ws, int id, cudaStream_t st)
{
    if (!ws->kt.on || !((ws->kt.mask >> id) & 1u) || ws->kt.used[id] >= gs_workspace::kTimedPairs) return;
    kt_record(ws->kt.ev[id][ws->kt.used[id]][1], st);
    ws->kt.used[id]++;
}

struct gs_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

int64_t gs_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void gs_default_params(gs_render_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->tile_w = GS_TILE;
    p->tile_h = GS_TILE;
    p->lod_enable = 0;
    p->lod_Lmax = 5;
    p->cull_enable = 0;
    p->alpha_min = 1.f / 255.f;
    p->alpha_max = 0.99f;
    p->T_min = 1e-4f;
    p->dilation = 0.3f;
    p->znear = 0.2f;
    p->fov_clamp = 1.3f;
    p->lod_d0 = 1600.f;
    p->lod_f = 2.f;
    p->eps_score = 1e-6f;
    p->vis_mass = 0.99f;
}

const char *gs_last_error(void) { return g_err; }

int64_t gs_workspace_bytes(const gs_capacity *cap)
{
    if (check_cap(cap) != GS_OK) return -1;
    return (int64_t)plan(*cap).total;
}

int gs_workspace_create(const gs_capacity *cap, gs_workspace **out)
{
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_cap(cap);
    if (rc != GS_OK) return rc;
    Offsets o = plan(*cap);
    gs_workspace *ws = new (std::nothrow) gs_workspace();
    if (!ws) return fail(GS_ERR_OOM, "host allocation failed");
    ws->cap = *cap;
    ws->sort_items = 0; // by the size of each sort
    ws->sel_spin_limit = gs::kSpinLimit;
    cudaGetDevice(&ws->device);
    if (cudaDeviceGetAttribute(&ws->sm_count, cudaDevAttrMultiProcessorCount, ws->device) != cudaSuccess ||
        ws->sm_count < 1)
        ws->sm_count = 152;
    cudaError_t e = cudaMalloc(&ws->base, o.total);
    if (e != cudaSuccess) {
        delete ws;
        cudaGetLastError();
        return fail(GS_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", o.total, cudaGetErrorString(e));
    }
    ws->bytes = o.total;
    char *b = (char *)ws->base;
    ws->cand_g = (uint32_t *)(b + o.cand_g);
    ws->cand_mask = (unsigned long long *)(b + o.cand_mask);
    ws->gate_g = (uint32_t *)(b + o.gate_g);
    ws->gate_mask = (unsigned long long *)(b + o.gate_mask);
    ws->rec_first = (uint32_t *)(b + o.rec_first);
    ws->cgrad = (float *)(b + o.cgrad);
    ws->rec_g = (uint32_t *)(b + o.rec_g);
    ws->rec_cam = (uint16_t *)(b + o.rec_cam);
    ws->rd0 = (float4 *)(b + o.rd0);
    ws->rd1 = (float4 *)(b + o.rd1);
    ws->rd2 = (float4 *)(b + o.rd2);
    ws->rect = (uint2 *)(b + o.rect);
    ws->tt = (uint32_t *)(b + o.tt);
    ws->inst_off = (uint32_t *)(b + o.inst_off);
    ws->clampm = (uint8_t *)(b + o.clampm);
    ws->rgrad = (float *)(b + o.rgrad);
    ws->dkey = (uint32_t *)(b + o.dkey);
    ws->tile_cnt = (uint32_t *)(b + o.tile_cnt);
    ws->tile_cur = (uint32_t *)(b + o.tile_cur);
    ws->tile_last = (uint32_t *)(b + o.tile_last);
    ws->tkey[0] = (uint32_t *)(b + o.tkey0); ws->tkey[1] = (uint32_t *)(b + o.tkey1);
    ws->tval[0] = (uint32_t *)(b + o.tval0); ws->tval[1] = (uint32_t *)(b + o.tval1);
    ws->slots = (float *)(b + o.slots);
    ws->imp_slots = (float2 *)(b + o.imp_slots);
    ws->ranges = (uint2 *)(b + o.ranges);
    ws->n_contrib = (uint32_t *)(b + o.n_contrib);
    ws->T_final = (float *)(b + o.T_final);
    ws->imp_w = (float *)(b + o.imp_w);
    ws->imp_a = (uint32_t *)(b + o.imp_a);
    ws->sel_cum = (double *)(b + o.sel_cum);
    ws->sel_bsum = (unsigned long long *)(b + o.sel_bsum);
    ws->selk[0] = (uint32_t *)(b + o.selk0); ws->selk[1] = (uint32_t *)(b + o.selk1);
    ws->selv[0] = (uint32_t *)(b + o.selv0); ws->selv[1] = (uint32_t *)(b + o.selv1);
    ws->loss_maps = (float *)(b + o.loss_maps);
    ws->loss_partial = (float *)(b + o.loss_partial);
    ws->loss_partial_words = o.loss_partial_words;
    ws->lb_status = (unsigned long long *)(b + o.lb_status);
    ws->lb_words = o.lb_words;
    ws->rx_status = (uint32_t *)(b + o.rx_status);
    ws->rx_words = o.rx_words;
    ws->rx_hist = ws->rx_status; // the first kRxHistWords words
    ws->red_partial = (float *)(b + o.red_partial);
    ws->red_words = o.red_words;
    ws->ctr = (gs::DevCounters *)(b + o.ctr);
    ws->d_cams = (gs::CamTable *)(b + o.d_cams);
    ws->d_adam_step = (int *)(b + o.d_adam_step);
    ws->d_adam_coef = (float *)(b + o.d_adam_coef);
    ws->mkey[0] = (uint32_t *)(b + o.mkey0); ws->mkey[1] = (uint32_t *)(b + o.mkey1);
    ws->mval[0] = (uint32_t *)(b + o.mval0); ws->mval[1] = (uint32_t *)(b + o.mval1);
    ws->mcum = (double *)(b + o.mcum);
    ws->mbsum = (double *)(b + o.mbsum);
    ws->mrx_status = (uint32_t *)(b + o.mrx_status);
    ws->mlb = (unsigned long long *)(b + o.mlb);
    ws->mhist = (uint32_t *)(b + o.mhist);
    ws->mctr = (gs::DevCounters *)(b + o.mctr);
    e = cudaMemset(ws->ctr, 0, sizeof(gs::DevCounters));
    if (e == cudaSuccess) e = cudaMemset(ws->d_cams, 0, sizeof(gs::CamTable));
    if (e == cudaSuccess) e = cudaMemset(ws->d_adam_step, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ws->mctr, 0, sizeof(gs::DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost(&ws->h_stage, gs_workspace::kStageSlots * sizeof(gs::CamTable));
    for (int k = 0; e == cudaSuccess && k < gs_workspace::kStageSlots; k++) {
        e = cudaEventCreateWithFlags(&ws->stage_ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) ws->stage_ev[k] = nullptr;
    }
    if (e != cudaSuccess) {
        gs_workspace_destroy(ws);
        return cuda_fail(e, "gs_workspace_create");
    }
    *out = ws;
    return GS_OK;
}

int gs_kernel_timing(gs_workspace *ws, int32_t kernels)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_kernel_timing: null workspace");
    if (kernels & ~GS_KT_ALL) return fail(GS_ERR_INVALID_ARG, "gs_kernel_timing: unknown kernel bits 0x%x", kernels);
    const int enable = kernels != 0;
    // the events live as long as the workspace: a graph captured with timing on
    // holds event nodes that name them
    if (enable && !ws->kt.ev[0][0][0]) {
        for (int k = 0; k < GS_KT_COUNT; k++)
            for (int i = 0; i < gs_workspace::kTimedPairs; i++)
                for (int h = 0; h < 2; h++) {
                    const cudaError_t e = cudaEventCreate(&ws->kt.ev[k][i][h]);
                    if (e != cudaSuccess) {
                        kt_release(ws);
                        return cuda_fail(e, "gs_kernel_timing");
                    }
                }
    }
    for (int k = 0; k < GS_KT_COUNT; k++) {
        ws->kt.used[k] = 0;
        ws->kt.launches[k] = 0;
    }
    ws->kt.on = enable;
    ws->kt.mask = (unsigned)kernels;
    return GS_OK;
}

int gs_kernel_time(gs_workspace *ws, int32_t kernel, double *total_ms, int64_t *launches)
{
    if (!ws || !total_ms || !launches || kernel < 0 || kernel >= GS_KT_COUNT)
        return fail(GS_ERR_INVALID_ARG, "gs_kernel_time: bad arguments");
    *total_ms = 0.0;
    *launches = 0;
    if (!ws->kt.on) return GS_OK;
    for (int i = 0; i < ws->kt.used[kernel]; i++) {
        cudaError_t e = cudaEventSynchronize(ws->kt.ev[kernel][i][1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ws->kt.ev[kernel][i][0], ws->kt.ev[kernel][i][1]);
        if (e != cudaSuccess) return cuda_fail(e, "gs_kernel_time");
        *total_ms += ms;
    }
    *launches = ws->kt.used[kernel];
    return GS_OK;
}

int gs_workspace_destroy(gs_workspace *ws)
{
    if (!ws) return GS_OK;
    cudaError_t e = kt_release(ws), e2;
    for (int k = 0; k < gs_workspace::kStageSlots; k++)
        if (ws->stage_ev[k] && (e2 = cudaEventDestroy(ws->stage_ev[k])) != cudaSuccess) e = e2;
    if (ws->h_stage && (e2 = cudaFreeHost(ws->h_stage)) != cudaSuccess) e = e2;
    if (ws->lazy.hist && (e2 = cudaFree(ws->lazy.hist)) != cudaSuccess) e = e2;
    if (ws->base && (e2 = cudaFree(ws->base)) != cudaSuccess) e = e2;
    delete ws;
    if (e != cudaSuccess) return cuda_fail(e, "gs_workspace_destroy");
    return GS_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int gs_workspace_set_sort_chunk(gs_workspace *ws, int32_t keys_per_block)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_workspace_set_sort_chunk: NULL workspace");
    if (keys_per_block != 0 && keys_per_block != 1024 && keys_per_block != 2048 && keys_per_block != 4096)
        return fail(GS_ERR_INVALID_ARG, "gs_workspace_set_sort_chunk: keys_per_block must be 0, 1024, 2048 or 4096");
    ws->sort_items = keys_per_block / gs::kSortThreads;
    return GS_OK;
}

int gs_workspace_set_spin_limit(gs_workspace *ws, uint64_t spins)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_workspace_set_spin_limit: NULL workspace");
    ws->sel_spin_limit = spins == 0 ? gs::kSpinLimit : (unsigned long long)spins;
    return GS_OK;
}

static int check_tile_shape(const gs_render_params *p, const char *who)
{
    if (gs::tile_shape_id(p->tile_w, p->tile_h) < 0)
        return fail(GS_ERR_INVALID_ARG, "%s: tile %dx%d not one of 16x16, 32x8, 8x32, 32x16, 16x8, 8x16", who, p->tile_w,
                    p->tile_h);
    return GS_OK;
}

int gs_upload_cameras(gs_workspace *ws, const gs_camera *cams, int32_t n_cams, const gs_render_params *params,
                      gs_stream stream)
{
    if (!ws || !cams || !params) return fail(GS_ERR_INVALID_ARG, "gs_upload_cameras: NULL argument");
    if (n_cams < 1 || n_cams > ws->cap.max_cameras)
        return fail(GS_ERR_INVALID_ARG, "gs_upload_cameras: n_cams %d outside [1, %d]", n_cams,
                    ws->cap.max_cameras);
    int rc = check_tile_shape(params, "gs_upload_cameras");
    if (rc != GS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs), "gs_upload_cameras");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(GS_ERR_INVALID_ARG, "gs_upload_cameras: upload outside stream capture (the graph reads the "
                                        "uploaded table; capture gs_preprocess_uploaded instead)");
    const int tw = params->tile_w, th = params->tile_h;
    gs::CamTable ct;
    memset(&ct, 0, sizeof(ct));
    ct.n = n_cams;
    ct.tile_w = tw;
    ct.tile_h = th;
    long long tiles = 0, pix = 0;
    for (int c = 0; c < n_cams; c++) {
        const gs_camera &s = cams[c];
        if (s.width <= 0 || s.height <= 0 || s.width > 65535 * 8 || s.height > 65535 * 8)
            return fail(GS_ERR_INVALID_ARG, "gs_upload_cameras: camera %d has size %dx%d", c, s.width, s.height);
        if (!(s.fx > 0.f) || !(s.fy > 0.f)) return fail(GS_ERR_INVALID_ARG, "gs_upload_cameras: camera %d focal", c);
        gs::CamInfo &d = ct.c[c];
        memcpy(d.R, s.R, sizeof(d.R));
        memcpy(d.t, s.t, sizeof(d.t));
        d.fx = s.fx; d.fy = s.fy; d.cx = s.cx; d.cy = s.cy;
        memcpy(d.campos, s.campos, sizeof(d.campos));
        d.width = s.width; d.height = s.height;
        d.tiles_x = (s.width + tw - 1) / tw;
        d.tiles_y = (s.height + th - 1) / th;
        if (d.tiles_x > 65535 || d.tiles_y > 65535)
            return fail(GS_ERR_INVALID_ARG, "gs_upload_cameras: camera %d has more than 65535 tiles a side", c);
        d.tile_base = (int)tiles;
        d.pix_base = pix;
        {
            const double lx = (double)params->fov_clamp * s.width / (2.0 * s.fx);
            const double ly = (double)params->fov_clamp * s.height / (2.0 * s.fy);
            d.jbound = (float)(1.001 * ((double)s.fx * s.fx * (1 + lx * lx) + (double)s.fy * s.fy * (1 + ly * ly)));
        }
        tiles += (long long)d.tiles_x * d.tiles_y;
        pix += (long long)s.width * s.height;
    }
    if (tiles > ws->cap.max_tiles) return fail(GS_ERR_CAPACITY, "gs_upload_cameras: %lld tiles > max_tiles", tiles);
    if (pix > ws->cap.max_pixels) return fail(GS_ERR_CAPACITY, "gs_upload_cameras: %lld pixels > max_pixels", pix);
    ct.total_tiles = (int)tiles;
    // stage in the next pinned slot once the copy that last read it has run
    const int k = ws->stage_next;
    if (ws->stage_pending[k]) CK(cudaEventSynchronize(ws->stage_ev[k]), "gs_upload_cameras(stage)");
    ws->stage_pending[k] = false;
    memcpy(&ws->h_stage[k], &ct, sizeof(ct));
    CK(cudaMemcpyAsync(ws->d_cams, &ws->h_stage[k], sizeof(ct), cudaMemcpyHostToDevice, st), "gs_upload_cameras");
    CK(cudaEventRecord(ws->stage_ev[k], st), "gs_upload_cameras");
    ws->stage_pending[k] = true;
    ws->stage_next = (k + 1) % gs_workspace::kStageSlots;
    ws->cams = ct;
    ws->up_fov_clamp = params->fov_clamp;
    ws->have_upload = 1;
    ws->have_preprocess = 0;
    ws->have_binning = 0;
    ws->have_compact = 0;
    ws->imp_ready = 0;
    return GS_OK;
}

int gs_preprocess_uploaded(gs_workspace *ws, const gs_gaussians *g, const uint32_t *cull,
                           const gs_render_params *params, gs_stream stream)
{
    if (!ws || !g || !params) return fail(GS_ERR_INVALID_ARG, "gs_preprocess_uploaded: NULL argument");
    if (!ws->have_upload) return fail(GS_ERR_INVALID_ARG, "gs_preprocess_uploaded: no gs_upload_cameras yet");
    if (params->tile_w != ws->cams.tile_w || params->tile_h != ws->cams.tile_h ||
        params->fov_clamp != ws->up_fov_clamp)
        return fail(GS_ERR_INVALID_ARG, "gs_preprocess_uploaded: tile shape and fov_clamp must be those of the upload");
    if (g->n < 0 || g->n > ws->cap.max_gaussians)
        return fail(GS_ERR_CAPACITY, "gs_preprocess: n = %lld exceeds max_gaussians %lld", (long long)g->n,
                    (long long)ws->cap.max_gaussians);
    if (g->n > 0 && (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->sh))
        return fail(GS_ERR_INVALID_ARG, "gs_preprocess: NULL Gaussian array");
    if (!aligned16(g->mean) || !aligned16(g->log_scale) || !aligned16(g->quat) || !aligned16(g->opacity_logit) ||
        !aligned16(g->sh))
        return fail(GS_ERR_INVALID_ARG, "gs_preprocess: Gaussian arrays must be 16-byte aligned");
    if (params->cull_enable < GS_CULL_OFF || params->cull_enable > GS_CULL_MARK)
        return fail(GS_ERR_INVALID_ARG, "gs_preprocess: cull_enable must be GS_CULL_OFF, GS_CULL_DROP or GS_CULL_MARK");
    if (params->cull_enable && !cull) return fail(GS_ERR_INVALID_ARG, "gs_preprocess: cull_enable needs a cull array");
    if (params->lod_enable && (params->lod_Lmax < 0 || params->lod_Lmax > gs::kMaxLod || !(params->lod_f > 1.f) ||
                               !(params->lod_d0 > 0.f)))
        return fail(GS_ERR_INVALID_ARG, "gs_preprocess: LOD gate needs 0 <= lod_Lmax <= %d, lod_f > 1, lod_d0 > 0",
                    gs::kMaxLod);
    gs::RenderConsts rc;
    memcpy(rc.bg, params->bg, sizeof(rc.bg));
    rc.alpha_min = params->alpha_min; rc.alpha_max = params->alpha_max; rc.T_min = params->T_min;
    rc.dilation = params->dilation; rc.znear = params->znear; rc.fov_clamp = params->fov_clamp;
    rc.lod_d0 = params->lod_d0; rc.lod_f = params->lod_f;
    rc.lod_enable = params->lod_enable; rc.lod_Lmax = params->lod_Lmax; rc.cull_enable = params->cull_enable;
    rc.eps_score = params->eps_score; rc.vis_mass = params->vis_mass;
    // round(log_f(d0 / d)) >= l  <=>  d <= d0 f^(0.5 - l)  (half away from zero, l >= 1)
    for (int l = 0; l <= gs::kMaxLod; l++) {
        const double thr = (double)params->lod_d0 * pow((double)params->lod_f, 0.5 - l);
        rc.lod_thr2[l] = l == 0 ? INFINITY : (float)(thr * thr);
    }
    ws->rc = rc;
    ws->g = *g;
    ws->have_preprocess = 1;
    ws->have_binning = 0;
    ws->have_compact = 0;
    ws->imp_ready = 0;
    CK(gs::launch_preprocess(ws, (cudaStream_t)stream, cull), "gs_preprocess");
    return GS_OK;
}

int gs_preprocess(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams, int32_t n_cams,
                  const uint32_t *cull, const gs_render_params *params, gs_stream stream)
{
    if (!ws || !g || !cams || !params) return fail(GS_ERR_INVALID_ARG, "gs_preprocess: NULL argument");
    int rc = gs_upload_cameras(ws, cams, n_cams, params, stream);
    if (rc != GS_OK) return rc;
    return gs_preprocess_uploaded(ws, g, cull, params, stream);
}

int gs_bin_sort(gs_workspace *ws, gs_stream stream)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_bin_sort: NULL workspace");
    if (!ws->have_preprocess) return fail(GS_ERR_INVALID_ARG, "gs_bin_sort: no preprocess on this workspace");
    cudaStream_t st = (cudaStream_t)stream;
    // the instance counters, then tile counts, ranges, scatter and the
    // per-tile depth sort (the final order: camera, tile, depth bits, record)
    CK(cudaMemsetAsync(&ws->ctr->n_instances, 0, sizeof(unsigned long long), st), "gs_bin_sort");
    CK(cudaMemsetAsync(&ws->ctr->instances_needed, 0, sizeof(unsigned long long), st), "gs_bin_sort");
    CK(gs::launch_bin(ws, st), "gs_bin_sort");
    ws->tile_buf = 0;
    ws->have_binning = 1;
    ws->imp_ready = 0;
    return GS_OK;
}

int gs_render_fwd(gs_workspace *ws, float *rgb_out, float *T_out, gs_stream stream)
{
    if (!ws || !rgb_out) return fail(GS_ERR_INVALID_ARG, "gs_render_fwd: NULL argument");
    if (!ws->have_binning) return fail(GS_ERR_INVALID_ARG, "gs_render_fwd: call gs_bin_sort first");
    CK(gs::launch_render_fwd(ws, (cudaStream_t)stream, rgb_out, T_out), "gs_render_fwd");
    return GS_OK;
}

int gs_render_fwd_importance(gs_workspace *ws, float *rgb_out, float *T_out, gs_stream stream)
{
    if (!ws || !rgb_out) return fail(GS_ERR_INVALID_ARG, "gs_render_fwd_importance: NULL argument");
    if (!ws->have_binning) return fail(GS_ERR_INVALID_ARG, "gs_render_fwd_importance: call gs_bin_sort first");
    CK(gs::launch_render_fwd_importance(ws, (cudaStream_t)stream, rgb_out, T_out), "gs_render_fwd_importance");
    CK(gs::launch_importance_reduce(ws, (cudaStream_t)stream), "gs_render_fwd_importance(reduce)");
    ws->imp_ready = 1;
    return GS_OK;
}

int gs_render_bwd(gs_workspace *ws, const gs_gaussians *g, const float *dL_drgb, const gs_gaussian_grads *grads,
                  int32_t accumulate, float *absgrad, float scale_reg_beta, float *scale_reg_value, gs_stream stream)
{
    if (ws && (ws->cap.flags & GS_CAP_FORWARD_ONLY))
        return fail(GS_ERR_INVALID_ARG, "gs_render_bwd: the workspace was created GS_CAP_FORWARD_ONLY");
    if (!ws || !g || !dL_drgb || !grads) return fail(GS_ERR_INVALID_ARG, "gs_render_bwd: NULL argument");
    if (!ws->have_binning) return fail(GS_ERR_INVALID_ARG, "gs_render_bwd: call gs_bin_sort and gs_render_fwd first");
    if (g->n != ws->g.n) return fail(GS_ERR_INVALID_ARG, "gs_render_bwd: Gaussian count differs from preprocess");
    if (g->n > 0 && (!grads->mean || !grads->log_scale || !grads->quat || !grads->opacity_logit || !grads->sh))
        return fail(GS_ERR_INVALID_ARG, "gs_render_bwd: NULL gradient array");
    cudaStream_t st = (cudaStream_t)stream;
    CK(gs::launch_render_bwd(ws, st, dL_drgb), "gs_render_bwd(raster)");
    CK(gs::launch_reduce_slots(ws, st), "gs_render_bwd(reduce)");
    CK(gs::launch_preprocess_bwd(ws, st, *g, *grads, accumulate, absgrad, scale_reg_beta, scale_reg_value, nullptr),
       "gs_render_bwd(preprocess)");
    return GS_OK;
}

int gs_render_bwd_compact(gs_workspace *ws, const gs_gaussians *g, const float *dL_drgb, float *absgrad,
                          float scale_reg_beta, float *scale_reg_value, gs_stream stream)
{
    if (ws && (ws->cap.flags & GS_CAP_FORWARD_ONLY))
        return fail(GS_ERR_INVALID_ARG, "gs_render_bwd_compact: the workspace was created GS_CAP_FORWARD_ONLY");
    if (!ws || !g || !dL_drgb) return fail(GS_ERR_INVALID_ARG, "gs_render_bwd_compact: NULL argument");
    if (!ws->have_binning)
        return fail(GS_ERR_INVALID_ARG, "gs_render_bwd_compact: call gs_bin_sort and gs_render_fwd first");
    if (g->n != ws->g.n) return fail(GS_ERR_INVALID_ARG, "gs_render_bwd_compact: Gaussian count differs from preprocess");
    cudaStream_t st = (cudaStream_t)stream;
    gs_gaussian_grads none;
    memset(&none, 0, sizeof(none));
    CK(gs::launch_render_bwd(ws, st, dL_drgb), "gs_render_bwd_compact(raster)");
    CK(gs::launch_reduce_slots(ws, st), "gs_render_bwd_compact(reduce)");
    CK(gs::launch_preprocess_bwd(ws, st, *g, none, 0, absgrad, scale_reg_beta, scale_reg_value, ws->cgrad),
       "gs_render_bwd_compact(preprocess)");
    ws->have_compact = 1;
    return GS_OK;
}

int gs_adam_step_compact(gs_workspace *ws, const gs_gaussians *g, const gs_gaussian_grads *m,
                         const gs_gaussian_grads *v, const float lr[5], float beta1, float beta2, float eps,
                         int32_t step, gs_stream stream)
{
    if (ws && (ws->cap.flags & GS_CAP_FORWARD_ONLY))
        return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: the workspace was created GS_CAP_FORWARD_ONLY");
    if (!ws || !g || !m || !v || !lr) return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: NULL argument");
    if (!ws->have_compact)
        return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: no gs_render_bwd_compact since the last preprocess");
    if (g->n != ws->g.n) return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: Gaussian count differs from preprocess");
    if (step < 0) return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: step is >= 1, or 0 for one past the device counter");
    if (g->n > 0 && (!m->mean || !m->log_scale || !m->quat || !m->opacity_logit || !m->sh || !v->mean ||
                     !v->log_scale || !v->quat || !v->opacity_logit || !v->sh))
        return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: NULL moment array");
    if (ws->lazy.enabled &&
        (m->mean != ws->lazy.m.mean || v->mean != ws->lazy.v.mean || beta1 != ws->lazy.b1 || beta2 != ws->lazy.b2 ||
         eps != ws->lazy.eps))
        return fail(GS_ERR_INVALID_ARG, "gs_adam_step_compact: moments and betas must be those of gs_adam_lazy_enable");
    gs_gaussian_grads param;
    param.mean = const_cast<float *>(g->mean);
    param.log_scale = const_cast<float *>(g->log_scale);
    param.quat = const_cast<float *>(g->quat);
    param.opacity_logit = const_cast<float *>(g->opacity_logit);
    param.sh = const_cast<float *>(g->sh);
    CK(gs::launch_adam_sparse(ws, (cudaStream_t)stream, param, *m, *v, g->n, lr, beta1, beta2, eps, step),
       "gs_adam_step_compact");
    return GS_OK;
}

int gs_adam_lazy_enable(gs_workspace *ws, const gs_gaussian_grads *m, const gs_gaussian_grads *v, int32_t *last_step,
                        float *drift, float beta1, float beta2, float eps, int32_t max_steps)
{
    if (!ws || !m || !v || !last_step || !drift) return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_enable: NULL argument");
    if (ws->cap.flags & GS_CAP_FORWARD_ONLY)
        return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_enable: the workspace was created GS_CAP_FORWARD_ONLY");
    if (!m->mean || !m->log_scale || !m->quat || !m->opacity_logit || !m->sh || !v->mean || !v->log_scale ||
        !v->quat || !v->opacity_logit || !v->sh)
        return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_enable: NULL moment array");
    if (!aligned16(m->mean) || !aligned16(m->log_scale) || !aligned16(m->quat) || !aligned16(m->opacity_logit) ||
        !aligned16(m->sh) || !aligned16(v->mean) || !aligned16(v->log_scale) || !aligned16(v->quat) ||
        !aligned16(v->opacity_logit) || !aligned16(v->sh))
        return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_enable: moment arrays must be 16-byte aligned");
    const double r = (double)beta1 / sqrt((double)beta2);
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 > 0.f && beta2 < 1.f && r < 1.0))
        return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_enable: needs 0 <= beta1 < sqrt(beta2) < 1");
    if (max_steps < 1) return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_enable: max_steps < 1");
    if (ws->lazy.hist) {
        cudaFree(ws->lazy.hist);
        ws->lazy.hist = nullptr;
    }
    cudaError_t e = cudaMalloc(&ws->lazy.hist, (size_t)(max_steps + 1) * 10 * sizeof(float));
    if (e != cudaSuccess) {
        ws->lazy.hist = nullptr;
        ws->lazy.enabled = 0;
        cudaGetLastError();
        return fail(GS_ERR_OOM, "gs_adam_lazy_enable: cudaMalloc of the step history failed");
    }
    ws->lazy.max_steps = max_steps;
    ws->lazy.m = *m;
    ws->lazy.v = *v;
    ws->lazy.last = last_step;
    ws->lazy.drift = drift;
    ws->lazy.b1 = beta1; ws->lazy.b2 = beta2; ws->lazy.eps = eps;
    ws->lazy.drift_factor = (float)(1.01 * r / (1.0 - r));
    ws->lazy.enabled = 1;
    return GS_OK;
}

int gs_adam_lazy_disable(gs_workspace *ws)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_adam_lazy_disable: NULL workspace");
    if (ws->lazy.hist) cudaFree(ws->lazy.hist);
    memset(&ws->lazy, 0, sizeof(ws->lazy));
    return GS_OK;
}

int gs_adam_flush(gs_workspace *ws, const gs_gaussians *g, gs_stream stream)
{
    if (!ws || !g) return fail(GS_ERR_INVALID_ARG, "gs_adam_flush: NULL argument");
    if (!ws->lazy.enabled) return GS_OK;
    if (g->n < 0 || g->n > ws->cap.max_gaussians) return fail(GS_ERR_CAPACITY, "gs_adam_flush: n > max_gaussians");
    if (!aligned16(g->mean) || !aligned16(g->log_scale) || !aligned16(g->quat) || !aligned16(g->opacity_logit) ||
        !aligned16(g->sh))
        return fail(GS_ERR_INVALID_ARG, "gs_adam_flush: parameter arrays must be 16-byte aligned");
    CK(gs::launch_lazy_flush(ws, (cudaStream_t)stream, *g), "gs_adam_flush");
    return GS_OK;
}

int gs_render_bwd_adam(gs_workspace *ws, const gs_gaussians *g, const float *dL_drgb, const gs_gaussian_grads *m,
                       const gs_gaussian_grads *v, const float lr[5], float beta1, float beta2, float eps,
                       int32_t step, float *absgrad, float scale_reg_beta, float *scale_reg_value, gs_stream stream)
{
    int rc = gs_render_bwd_compact(ws, g, dL_drgb, absgrad, scale_reg_beta, scale_reg_value, stream);
    if (rc != GS_OK) return rc;
    return gs_adam_step_compact(ws, g, m, v, lr, beta1, beta2, eps, step, stream);
}

int gs_importance(gs_workspace *ws, float *w, uint32_t *a, float *s_accum, uint32_t *crad_accum,
                  uint32_t *cvis_accum, uint32_t *cull_out, gs_stream stream)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_importance: NULL workspace");
    if (!ws->have_binning) return fail(GS_ERR_INVALID_ARG, "gs_importance: call gs_bin_sort first");
    CK(gs::launch_importance(ws, (cudaStream_t)stream, w, a, s_accum, crad_accum, cvis_accum, cull_out),
       "gs_importance");
    return GS_OK;
}

int gs_photometric_loss(gs_workspace *ws, const float *image, const float *target, int32_t batch, int32_t height,
                        int32_t width, float lambda, float *loss_out, float *dL_dimage, gs_stream stream)
{
    if (ws && (ws->cap.flags & GS_CAP_FORWARD_ONLY))
        return fail(GS_ERR_INVALID_ARG, "gs_photometric_loss: the workspace was created GS_CAP_FORWARD_ONLY");
    if (!ws || !image || !target || !loss_out || !dL_dimage)
        return fail(GS_ERR_INVALID_ARG, "gs_photometric_loss: NULL argument");
    if (batch < 1 || height < 1 || width < 1) return fail(GS_ERR_INVALID_ARG, "gs_photometric_loss: empty batch");
    const long long px = (long long)batch * height * width;
    if (px > ws->cap.max_pixels)
        return fail(GS_ERR_CAPACITY, "gs_photometric_loss: batch*H*W = %lld exceeds max_pixels", px);
    const long long blocks = (long long)((width + 31) / 32) * ((height + 31) / 32) * batch * 3;
    if (2 * blocks > (long long)ws->loss_partial_words)
        return fail(GS_ERR_CAPACITY, "gs_photometric_loss: image too large for the workspace's partial sums");
    CK(gs::launch_loss(ws, (cudaStream_t)stream, image, target, batch, height, width, lambda, loss_out, dL_dimage),
       "gs_photometric_loss");
    return GS_OK;
}

int gs_adam_step(const gs_adam_group *groups, int32_t n_groups, int32_t step, gs_stream stream)
{
    if (!groups || n_groups < 1 || n_groups > GS_MAX_ADAM_GROUPS)
        return fail(GS_ERR_INVALID_ARG, "gs_adam_step: 1..%d groups required", GS_MAX_ADAM_GROUPS);
    if (step < 1) return fail(GS_ERR_INVALID_ARG, "gs_adam_step: step counts from 1");
    for (int k = 0; k < n_groups; k++) {
        const gs_adam_group &gr = groups[k];
        if (gr.n < 0 || (gr.n > 0 && (!gr.param || !gr.grad || !gr.m || !gr.v)))
            return fail(GS_ERR_INVALID_ARG, "gs_adam_step: group %d invalid", k);
    }
    CK(gs::launch_adam(groups, n_groups, step, (cudaStream_t)stream), "gs_adam_step");
    return GS_OK;
}

static int model_ops_check(gs_workspace *ws, int64_t n, const char *who)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "%s: NULL workspace", who);
    if (!(ws->cap.flags & GS_CAP_MODEL_OPS))
        return fail(GS_ERR_INVALID_ARG, "%s: the workspace was created without GS_CAP_MODEL_OPS", who);
    if (n < 0 || n > ws->cap.max_gaussians)
        return fail(GS_ERR_CAPACITY, "%s: n = %lld outside [0, max_gaussians = %lld]", who, (long long)n,
                    (long long)ws->cap.max_gaussians);
    return GS_OK;
}

static bool model_ok(const gs_model *m)
{
    return m && m->mean && m->log_scale && m->quat && m->opacity_logit && m->sh;
}

int gs_prune_sample(gs_workspace *ws, const float *s, const float *expo, int64_t n, int64_t k, uint32_t *keep_bits,
                    gs_stream stream)
{
    int rc = model_ops_check(ws, n, "gs_prune_sample");
    if (rc != GS_OK) return rc;
    if (n > 0 && (!s || !expo || !keep_bits)) return fail(GS_ERR_INVALID_ARG, "gs_prune_sample: NULL argument");
    if (k < 0) return fail(GS_ERR_INVALID_ARG, "gs_prune_sample: k < 0");
    if (n == 0) return GS_OK;
    CK(gs::launch_prune_sample(ws, (cudaStream_t)stream, s, expo, n, k, keep_bits), "gs_prune_sample");
    return GS_OK;
}

int gs_prune_mass(gs_workspace *ws, const float *s, int64_t n, float mass, uint32_t *keep_bits, gs_stream stream)
{
    int rc = model_ops_check(ws, n, "gs_prune_mass");
    if (rc != GS_OK) return rc;
    if (n > 0 && (!s || !keep_bits)) return fail(GS_ERR_INVALID_ARG, "gs_prune_mass: NULL argument");
    if (!(mass > 0.f) || mass > 1.f) return fail(GS_ERR_INVALID_ARG, "gs_prune_mass: mass must be in (0, 1]");
    if (n == 0) return GS_OK;
    CK(gs::launch_prune_mass(ws, (cudaStream_t)stream, s, n, mass, keep_bits), "gs_prune_mass");
    return GS_OK;
}

int gs_compact(gs_workspace *ws, const gs_model *src, const uint32_t *keep_bits, gs_model *dst, int64_t dst_capacity,
               int64_t *n_out, gs_stream stream)
{
    if (!src) return fail(GS_ERR_INVALID_ARG, "gs_compact: NULL src");
    int rc = model_ops_check(ws, src->n, "gs_compact");
    if (rc != GS_OK) return rc;
    if (!n_out || !keep_bits || (src->n > 0 && (!model_ok(src) || !model_ok(dst))))
        return fail(GS_ERR_INVALID_ARG, "gs_compact: NULL argument");
    if (src->mean == dst->mean) return fail(GS_ERR_INVALID_ARG, "gs_compact: src and dst overlap");
    CK(gs::launch_compact(ws, (cudaStream_t)stream, *src, keep_bits, *dst, dst_capacity, (long long *)n_out),
       "gs_compact");
    return GS_OK;
}

int gs_densify(gs_workspace *ws, const gs_model *src, const float *absgrad, const uint32_t *denom,
               const uint32_t *cvis, const uint32_t *crad, const float *noise, const gs_densify_params *params,
               gs_model *dst, int64_t dst_capacity, int64_t *n_out, gs_stream stream)
{
    if (!src || !params) return fail(GS_ERR_INVALID_ARG, "gs_densify: NULL argument");
    int rc = model_ops_check(ws, src->n, "gs_densify");
    if (rc != GS_OK) return rc;
    if (!n_out || (src->n > 0 && (!model_ok(src) || !model_ok(dst) || !absgrad || !denom || !cvis || !crad || !noise)))
        return fail(GS_ERR_INVALID_ARG, "gs_densify: NULL argument");
    if (src->mean == dst->mean) return fail(GS_ERR_INVALID_ARG, "gs_densify: src and dst overlap");
    if (!(params->min_opacity > 0.f && params->min_opacity < 1.f) || !(params->dense_scale > 0.f) ||
        !(params->split_shrink > 0.f) || params->n_levels < 1 || params->n_levels > 256)
        return fail(GS_ERR_INVALID_ARG, "gs_densify: parameters out of range");
    CK(gs::launch_densify(ws, (cudaStream_t)stream, *src, absgrad, denom, cvis, crad, noise, *params, *dst,
                          dst_capacity, (long long *)n_out),
       "gs_densify");
    return GS_OK;
}

int gs_count_views(gs_workspace *ws, uint32_t *counts, gs_stream stream)
{
    if (!ws || !counts) return fail(GS_ERR_INVALID_ARG, "gs_count_views: NULL argument");
    if (!ws->have_preprocess) return fail(GS_ERR_INVALID_ARG, "gs_count_views: no preprocess on this workspace");
    CK(gs::launch_count_views(ws, (cudaStream_t)stream, counts), "gs_count_views");
    return GS_OK;
}

int gs_graph_capture_begin(gs_stream stream)
{
    if (!stream) return fail(GS_ERR_INVALID_ARG, "gs_graph_capture_begin: the legacy NULL stream cannot be captured");
    CK(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal), "gs_graph_capture_begin");
    return GS_OK;
}

int gs_graph_capture_end(gs_stream stream, gs_graph **out)
{
    if (!out) return fail(GS_ERR_INVALID_ARG, "gs_graph_capture_end: out is NULL");
    *out = nullptr;
    if (!stream) return fail(GS_ERR_INVALID_ARG, "gs_graph_capture_end: the legacy NULL stream cannot be captured");
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture((cudaStream_t)stream, &g), "gs_graph_capture_end");
    cudaGraphExec_t x = nullptr;
    // per-node priorities: each kernel keeps the priority of the stream it was captured from
    cudaError_t e = cudaGraphInstantiateWithFlags(&x, g, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "gs_graph_capture_end(instantiate)");
    }
    gs_graph *h = new (std::nothrow) gs_graph{g, x};
    if (!h) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return fail(GS_ERR_OOM, "host allocation failed");
    }
    *out = h;
    return GS_OK;
}

int gs_graph_launch(gs_graph *graph, gs_stream stream)
{
    if (!graph) return fail(GS_ERR_INVALID_ARG, "gs_graph_launch: NULL graph");
    CK(cudaGraphLaunch(graph->exec, (cudaStream_t)stream), "gs_graph_launch");
    return GS_OK;
}

int gs_graph_destroy(gs_graph *graph)
{
    if (!graph) return GS_OK;
    cudaError_t e1 = cudaGraphExecDestroy(graph->exec), e2 = cudaGraphDestroy(graph->graph);
    delete graph;
    CK(e1, "gs_graph_destroy");
    CK(e2, "gs_graph_destroy");
    return GS_OK;
}

int gs_sync_status(gs_workspace *ws, gs_stream stream)
{
    gs_counts c;
    int rc = gs_workspace_counts(ws, &c, stream);
    if (rc != GS_OK) return rc;
    int merr[2] = {0, 0}; // error word of the model-level calls
    CK(cudaMemcpy(merr, &ws->mctr->error, sizeof(merr), cudaMemcpyDeviceToHost), "gs_sync_status");
    if (merr[0]) return fail(merr[0], "device error %d in a model-level call (site %d)", merr[0], merr[1]);
    if (c.error)
        return fail(c.error, "device error %d at site %d (records needed %lld of %lld, instances needed %lld of %lld)",
                    c.error, c.error_site, (long long)c.records_needed, (long long)ws->cap.max_records,
                    (long long)c.instances_needed, (long long)ws->cap.max_instances);
    return GS_OK;
}

int gs_workspace_counts(gs_workspace *ws, gs_counts *out, gs_stream stream)
{
    if (!ws || !out) return fail(GS_ERR_INVALID_ARG, "gs_workspace_counts: NULL argument");
    gs::DevCounters d;
    CK(cudaMemcpyAsync(&d, ws->ctr, sizeof(d), cudaMemcpyDeviceToHost, (cudaStream_t)stream), "gs_workspace_counts");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "gs_workspace_counts");
    out->n_records = (int64_t)d.n_records;
    out->n_instances = (int64_t)d.n_instances;
    out->n_visible = (int64_t)d.n_visible;
    out->records_needed = (int64_t)d.records_needed;
    out->instances_needed = (int64_t)d.instances_needed;
    out->error = d.error;
    out->error_site = d.error_site;
    out->fragments = (int64_t)d.fragments;
    out->composited = (int64_t)d.composited;
    out->n_candidates = (int64_t)d.n_candidates;
    return GS_OK;
}

int gs_clear_error(gs_workspace *ws, gs_stream stream)
{
    if (!ws) return fail(GS_ERR_INVALID_ARG, "gs_clear_error: NULL workspace");
    CK(cudaMemsetAsync(&ws->ctr->error, 0, 2 * sizeof(int), (cudaStream_t)stream), "gs_clear_error");
    CK(cudaMemsetAsync(&ws->mctr->error, 0, 2 * sizeof(int), (cudaStream_t)stream), "gs_clear_error");
    return GS_OK;
}

int gs_workspace_buffer(gs_workspace *ws, int32_t which, void **ptr, int64_t *count)
{
    if (!ws || !ptr || !count) return fail(GS_ERR_INVALID_ARG, "gs_workspace_buffer: NULL argument");
    const gs_capacity &c = ws->cap;
    switch (which) {
    case GS_BUF_REC_GAUSSIAN: *ptr = ws->rec_g; *count = c.max_records; break;
    case GS_BUF_REC_CAMERA: *ptr = ws->rec_cam; *count = c.max_records; break;
    case GS_BUF_REC_RECT: *ptr = ws->rect; *count = c.max_records; break;
    case GS_BUF_REC_TILES: *ptr = ws->tt; *count = c.max_records; break;
    case GS_BUF_REC_DEPTH: *ptr = ws->dkey; *count = c.max_records; break;
    case GS_BUF_REC_XY_CONIC: *ptr = ws->rd0; *count = c.max_records; break;
    case GS_BUF_REC_C_OPAC_RG: *ptr = ws->rd1; *count = c.max_records; break;
    case GS_BUF_REC_B_LO: *ptr = ws->rd2; *count = c.max_records; break;
    case GS_BUF_SORTED_VALUES: *ptr = ws->tval[ws->tile_buf]; *count = c.max_instances; break;
    case GS_BUF_TILE_RANGES: *ptr = ws->ranges; *count = c.max_tiles; break;
    case GS_BUF_N_CONTRIB: *ptr = ws->n_contrib; *count = c.max_pixels; break;
    default: return fail(GS_ERR_INVALID_ARG, "gs_workspace_buffer: unknown buffer %d", which);
    }
    return GS_OK;
}

} // extern "C"
