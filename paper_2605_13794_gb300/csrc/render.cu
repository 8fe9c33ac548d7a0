// render.cu -- per-tile compositing (App. A, Eq. for C(p) and T_i), its
// adjoint, and the instrumented colourless sweep of the importance pass
// (Sec. 3.2, Fig. 2).
//
// One 256-thread block per 16x16 tile; each thread owns one pixel.  The tile's
// depth-ordered list is staged through shared memory in batches; every
// pixel walks the same entry at the same time, so per-Gaussian quantities are
// block reductions rather than per-pixel global atomics.  The backward and
// the importance sweep write one gradient/score slot per (record, tile) --
// slot index = the record's first instance + the tile's position inside the
// record's rectangle -- and a later per-record pass sums a record's slots in
// a fixed order, so results are bit-reproducible run to run.
#include "gs_internal.cuh"

namespace gs {

// Pixel-to-thread map: warp w covers an 8x4 pixel block of the tile.
__device__ __forceinline__ void pixel_of_thread(int tid, int &lx, int &ly)
{
    const int w = tid >> 5, l = tid & 31;
    lx = (w & 1) * 8 + (l & 7);
    ly = (w >> 1) * 4 + (l >> 3);
}

// Gaussian exponent at pixel offset (dx, dy) with explicitly rounded
// operations, so the forward, backward and importance kernels take the same
// skip decisions bit for bit.
__device__ __forceinline__ float gs_power(float A, float B, float C, float dx, float dy)
{
    const float q = __fmaf_rn(__fmul_rn(C, dy), dy, __fmul_rn(__fmul_rn(A, dx), dx));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(__fmul_rn(B, dx), dy));
}

__device__ __forceinline__ float gs_alpha(float o, float power, float alpha_max)
{
    return fminf(alpha_max, __fmul_rn(o, __expf(power)));
}

// ---- forward --------------------------------------------------------------

__global__ void __launch_bounds__(256) render_fwd_kernel(const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ vals,
                                                         const float4 *__restrict__ rd0,
                                                         const float4 *__restrict__ rd1,
                                                         const float *__restrict__ rd2, CamTable ct, RenderConsts rc,
                                                         float *__restrict__ rgb_out, float *__restrict__ T_out,
                                                         float *__restrict__ T_ws, uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s0[256];
    __shared__ float4 s1[256];
    __shared__ float s2[256];
    const int tile = blockIdx.x;
    const int c = camera_of_tile(ct, tile);
    const CamInfo &cam = ct.c[c];
    const int lt = tile - cam.tile_base;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    int lx, ly;
    pixel_of_thread(threadIdx.x, lx, ly);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < cam.width && py < cam.height;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    const int start = (int)rg.x, end = (int)rg.y;

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t contrib = 0, last = 0;
    bool done = !inside;
    for (int b = start; b < end; b += 256) {
        if (__syncthreads_count(done) == 256) break;
        const int s = b + threadIdx.x;
        if (s < end) {
            const uint32_t r = vals[s];
            s0[threadIdx.x] = rd0[r];
            s1[threadIdx.x] = rd1[r];
            s2[threadIdx.x] = rd2[r];
        }
        __syncthreads();
        const int cnt = min(256, end - b);
        for (int j = 0; j < cnt && !done; j++) {
            contrib++;
            const float4 p0 = s0[j];
            const float dx = __fsub_rn(pxf, p0.x), dy = __fsub_rn(pyf, p0.y);
            const float power = gs_power(p0.z, p0.w, s1[j].x, dx, dy);
            if (power > 0.f) continue;
            const float4 p1 = s1[j];
            const float alpha = gs_alpha(p1.y, power, rc.alpha_max);
            if (alpha < rc.alpha_min) continue;
            const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (test_T < rc.T_min) { done = true; continue; }
            const float wgt = alpha * T;
            C0 = fmaf(wgt, p1.z, C0);
            C1 = fmaf(wgt, p1.w, C1);
            C2 = fmaf(wgt, s2[j], C2);
            T = test_T;
            last = contrib;
        }
    }
    if (inside) {
        const long long pix = (long long)py * cam.width + px;
        const long long np = (long long)cam.width * cam.height;
        float *img = rgb_out + 3 * cam.pix_base;
        img[pix] = C0 + T * rc.bg[0];
        img[np + pix] = C1 + T * rc.bg[1];
        img[2 * np + pix] = C2 + T * rc.bg[2];
        const long long gp = cam.pix_base + pix;
        if (T_out) T_out[gp] = T;
        T_ws[gp] = T;
        n_contrib[gp] = last;
    }
}

cudaError_t launch_render_fwd(gs_workspace *ws, cudaStream_t st, float *rgb, float *T_out)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    render_fwd_kernel<<<ws->cams.total_tiles, 256, 0, st>>>(ws->ranges, ws->tval[ws->tile_buf], ws->rd0, ws->rd1,
                                                            ws->rd2, ws->cams, ws->rc, rgb, T_out, ws->T_final,
                                                            ws->n_contrib);
    note_launch();
    return cudaGetLastError();
}

// ---- backward ---------------------------------------------------------------

constexpr int kBwdBatch = 32;

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Slot of (record r, tile (tx, ty)): first instance of r + position of the
// tile inside r's rectangle (row-major, the order of emission).
__device__ __forceinline__ unsigned long long slot_of(const uint32_t *inst_off, const uint2 *rect, uint32_t r, int tx,
                                                      int ty)
{
    int x0, y0, x1, y1;
    unpack_rect(rect[r], x0, y0, x1, y1);
    return (unsigned long long)inst_off[r] + (unsigned long long)((ty - y0) * (x1 - x0) + (tx - x0));
}

struct BwdRenderArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float4 *rd0, *rd1;
    const float *rd2;
    const uint32_t *inst_off;
    const uint2 *rect;
    const float *T_final;
    const uint32_t *n_contrib;
    const float *dL_drgb;
    float *slots;
};

__global__ void __launch_bounds__(256) render_bwd_kernel(BwdRenderArgs a, CamTable ct, RenderConsts rc)
{
    __shared__ float4 s0[kBwdBatch];
    __shared__ float4 s1[kBwdBatch];
    __shared__ float s2[kBwdBatch];
    __shared__ unsigned long long s_slot[kBwdBatch];
    __shared__ float s_red[8][kBwdBatch][kSlotFloats];
    __shared__ int s_max;
    const int tile = blockIdx.x;
    const int c = camera_of_tile(ct, tile);
    const CamInfo &cam = ct.c[c];
    const int lt = tile - cam.tile_base;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    int lx, ly;
    pixel_of_thread(threadIdx.x, lx, ly);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < cam.width && py < cam.height;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 rg = a.ranges[tile];
    const int start = (int)rg.x, end = (int)rg.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    int nc = 0;
    if (inside) {
        const long long pix = (long long)py * cam.width + px;
        const long long np = (long long)cam.width * cam.height;
        const float *gimg = a.dL_drgb + 3 * cam.pix_base;
        g0 = gimg[pix]; g1 = gimg[np + pix]; g2 = gimg[2 * np + pix];
        T = a.T_final[cam.pix_base + pix];
        nc = (int)a.n_contrib[cam.pix_base + pix];
    }
    const float Tfin = T;
    const float gbg = g0 * rc.bg[0] + g1 * rc.bg[1] + g2 * rc.bg[2];
    float S0 = 0.f, S1 = 0.f, S2 = 0.f; // sum over later fragments of alpha T c

    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, nc);
    __syncthreads();
    const int last = start + s_max;
    // entries after the last contribution of every pixel carry zero gradient
    for (int s = last + threadIdx.x; s < end; s += 256) {
        const unsigned long long slot = slot_of(a.inst_off, a.rect, a.vals[s], tx, ty);
        float *dst = a.slots + slot * kSlotFloats;
#pragma unroll
        for (int k = 0; k < kSlotFloats; k++) dst[k] = 0.f;
    }
    for (int hi = last; hi > start; hi -= kBwdBatch) {
        const int lo = max(start, hi - kBwdBatch);
        const int cnt = hi - lo;
        if (threadIdx.x < cnt) {
            const uint32_t r = a.vals[lo + threadIdx.x];
            s0[threadIdx.x] = a.rd0[r];
            s1[threadIdx.x] = a.rd1[r];
            s2[threadIdx.x] = a.rd2[r];
            s_slot[threadIdx.x] = slot_of(a.inst_off, a.rect, r, tx, ty);
        }
        __syncthreads();
        for (int jj = cnt - 1; jj >= 0; jj--) {
            const int j = lo + jj - start; // position in the tile list
            float v[kSlotFloats];
#pragma unroll
            for (int k = 0; k < kSlotFloats; k++) v[k] = 0.f;
            bool act = false;
            if (j < nc) {
                const float4 p0 = s0[jj], p1 = s1[jj];
                const float dx = __fsub_rn(pxf, p0.x), dy = __fsub_rn(pyf, p0.y);
                const float power = gs_power(p0.z, p0.w, p1.x, dx, dy);
                if (power <= 0.f) {
                    const float G = __expf(power);
                    const float og = __fmul_rn(p1.y, G);
                    const float alpha = fminf(rc.alpha_max, og);
                    if (alpha >= rc.alpha_min) {
                        act = true;
                        const float cb = s2[jj];
                        const float oma = 1.f - alpha;
                        const float inv = 1.f / oma;
                        const float Tj = T * inv; // transmittance in front of this fragment
                        const float aT = alpha * Tj;
                        v[6] = aT * g0; v[7] = aT * g1; v[8] = aT * g2;
                        float dalpha = g0 * (Tj * p1.z - S0 * inv) + g1 * (Tj * p1.w - S1 * inv) +
                                       g2 * (Tj * cb - S2 * inv) - Tfin * gbg * inv;
                        S0 = fmaf(aT, p1.z, S0);
                        S1 = fmaf(aT, p1.w, S1);
                        S2 = fmaf(aT, cb, S2);
                        T = Tj;
                        if (og < rc.alpha_max) {
                            v[5] = G * dalpha;
                            const float dpow = G * p1.y * dalpha;
                            v[0] = dpow * (p0.z * dx + p0.w * dy);
                            v[1] = dpow * (p1.x * dy + p0.w * dx);
                            v[2] = -0.5f * dpow * dx * dx;
                            v[3] = -dpow * dx * dy;
                            v[4] = -0.5f * dpow * dy * dy;
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, act)) {
#pragma unroll
                for (int k = 0; k < kSlotFloats; k++) v[k] = warp_sum_f(v[k]);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < kSlotFloats; k++) s_red[warp][jj][k] = v[k];
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < cnt * kSlotFloats; idx += 256) {
            const int jj = idx / kSlotFloats, k = idx - jj * kSlotFloats;
            float sum = 0.f;
#pragma unroll
            for (int w = 0; w < 8; w++) sum += s_red[w][jj][k];
            a.slots[s_slot[jj] * kSlotFloats + k] = sum;
        }
        __syncthreads();
    }
}

cudaError_t launch_render_bwd(gs_workspace *ws, cudaStream_t st, const float *dL_drgb)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    BwdRenderArgs a;
    a.ranges = ws->ranges; a.vals = ws->tval[ws->tile_buf]; a.rd0 = ws->rd0; a.rd1 = ws->rd1; a.rd2 = ws->rd2;
    a.inst_off = ws->inst_off; a.rect = ws->rect; a.T_final = ws->T_final; a.n_contrib = ws->n_contrib;
    a.dL_drgb = dL_drgb; a.slots = ws->slots;
    render_bwd_kernel<<<ws->cams.total_tiles, 256, 0, st>>>(a, ws->cams, ws->rc);
    note_launch();
    return cudaGetLastError();
}

// ---- importance sweep (colourless forward) -------------------------------------

constexpr int kImpBatch = 64;

struct ImpArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float4 *rd0, *rd1;
    const uint32_t *inst_off;
    const uint2 *rect;
    float *slots; // [I][2]: alpha-weight (float), composited pixels (uint32 bits)
};

__global__ void __launch_bounds__(256) importance_raster_kernel(ImpArgs a, CamTable ct, RenderConsts rc)
{
    __shared__ float4 s0[kImpBatch];
    __shared__ float2 s1[kImpBatch];
    __shared__ unsigned long long s_slot[kImpBatch];
    __shared__ float s_w[8][kImpBatch];
    __shared__ uint32_t s_a[8][kImpBatch];
    const int tile = blockIdx.x;
    const int c = camera_of_tile(ct, tile);
    const CamInfo &cam = ct.c[c];
    const int lt = tile - cam.tile_base;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    int lx, ly;
    pixel_of_thread(threadIdx.x, lx, ly);
    const int px = tx * kTile + lx, py = ty * kTile + ly;
    const bool inside = px < cam.width && py < cam.height;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 rg = a.ranges[tile];
    const int start = (int)rg.x, end = (int)rg.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float T = 1.f;
    bool done = !inside;
    int b = start;
    for (; b < end; b += kImpBatch) {
        if (__syncthreads_count(done) == 256) break;
        const int cnt = min(kImpBatch, end - b);
        if (threadIdx.x < cnt) {
            const uint32_t r = a.vals[b + threadIdx.x];
            s0[threadIdx.x] = a.rd0[r];
            const float4 p1 = a.rd1[r];
            s1[threadIdx.x] = make_float2(p1.x, p1.y);
            s_slot[threadIdx.x] = slot_of(a.inst_off, a.rect, r, tx, ty);
        }
        __syncthreads();
        for (int j = 0; j < cnt; j++) {
            float wv = 0.f;
            uint32_t av = 0;
            if (!done) {
                const float4 p0 = s0[j];
                const float2 p1 = s1[j];
                const float dx = __fsub_rn(pxf, p0.x), dy = __fsub_rn(pyf, p0.y);
                const float power = gs_power(p0.z, p0.w, p1.x, dx, dy);
                if (power <= 0.f) {
                    const float alpha = gs_alpha(p1.y, power, rc.alpha_max);
                    if (alpha >= rc.alpha_min) {
                        const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
                        if (test_T < rc.T_min) {
                            done = true;
                        } else {
                            wv = alpha * T;
                            av = 1;
                            T = test_T;
                        }
                    }
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, av);
            if (bal) wv = warp_sum_f(wv);
            if (lane == 0) { s_w[warp][j] = wv; s_a[warp][j] = __popc(bal); }
        }
        __syncthreads();
        if (threadIdx.x < cnt) {
            float ws = 0.f;
            uint32_t as = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) { ws += s_w[w][threadIdx.x]; as += s_a[w][threadIdx.x]; }
            float2 out = make_float2(ws, __uint_as_float(as));
            reinterpret_cast<float2 *>(a.slots)[s_slot[threadIdx.x]] = out;
        }
    }
    // entries never reached (every pixel of the tile had stopped)
    for (int s = b + threadIdx.x; s < end; s += 256) {
        const unsigned long long slot = slot_of(a.inst_off, a.rect, a.vals[s], tx, ty);
        reinterpret_cast<float2 *>(a.slots)[slot] = make_float2(0.f, 0.f);
    }
}

cudaError_t launch_importance_raster(gs_workspace *ws, cudaStream_t st)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    ImpArgs a;
    a.ranges = ws->ranges; a.vals = ws->tval[ws->tile_buf]; a.rd0 = ws->rd0; a.rd1 = ws->rd1;
    a.inst_off = ws->inst_off; a.rect = ws->rect; a.slots = ws->slots;
    importance_raster_kernel<<<ws->cams.total_tiles, 256, 0, st>>>(a, ws->cams, ws->rc);
    note_launch();
    return cudaGetLastError();
}

} // namespace gs
