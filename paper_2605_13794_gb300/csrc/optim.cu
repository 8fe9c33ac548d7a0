// optim.cu -- photometric loss of Eq. 4 (L1 + lambda (1 - SSIM)) with its
// gradient, and the Adam step (Kingma and Ba) of standard 3DGS training.
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5, separable), C1 = 0.01^2,
// C2 = 0.03^2 and zero padding.  Pass 1 blurs x, y, x^2, y^2, xy over a tile
// with a 5-pixel halo, forms the SSIM map and the three coefficient maps its
// gradient needs; pass 2 blurs those maps (the window is symmetric, so the
// adjoint of the blur is the blur) and assembles dL/dx.  The per-tile sums of
// SSIM and |x - y| are added in 64-bit fixed point (exact, so independent of
// the order of the blocks).
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

constexpr int kLT = 32;           // output tile edge
constexpr int kHalo = 5;          // window radius
constexpr int kLTH = kLT + 2 * kHalo;

struct Win {
    float w[11];
};

__device__ __forceinline__ float ld_zero(const float *p, int H, int W, int y, int x)
{
    return (y >= 0 && y < H && x >= 0 && x < W) ? p[(long long)y * W + x] : 0.f;
}

// The two 11-tap passes run as sliding windows in registers: a thread
// produces kHSeg consecutive outputs of a row from kHSeg + 10 inputs (or kVSeg
// outputs of a column), so each shared-memory value is read once per thread
// rather than once per tap.  Maps travel in pairs as FP32x2 values -- (x, y),
// (x^2, y^2) in the forward, (F0, F1) in the backward -- so one packed FMA
// advances two maps.
constexpr int kHSeg = 8;                 // horizontal outputs per thread (42 rows x 4 segments)
constexpr int kVSeg = 4;                 // vertical outputs per thread (32 columns x 8 segments)
constexpr int kLTP = kLTH + 1;           // padded row of the staged tile
// staging: warp w loads rows w, w + 8, ... of the tile with its halo, lane l
// columns l and l + 32
constexpr int kStageRows = (kLTH + 7) / 8;
static_assert(kLTH <= 64, "two columns per lane cover a staged row");

__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }

// grid: (tiles_x, tiles_y, batch * 3).  F: the three coefficient maps of the
// SSIM gradient of each plane, planar: F[(plane * 3 + m) * H * W + pixel].
__global__ void __launch_bounds__(256, 4) ssim_fwd_kernel(const float *img, const float *tgt, int H, int W, Win win,
                                                       float C1, float C2, float *F, unsigned long long *acc)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ float2 sxy[kLTH][kLTP];
    __shared__ float2 hb01[kLTH][kLT + 1], hb23[kLTH][kLT + 1];
    __shared__ float hb4[kLTH][kLT + 1];
    __shared__ float red[2][8];
    const int plane = blockIdx.z;
    const float *x = img + (long long)plane * H * W;
    const float *y = tgt + (long long)plane * H * W;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    {
        // every load of the thread issued before the first store
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        float2 buf[kStageRows][2];
#pragma unroll
        for (int q = 0; q < kStageRows; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = warp + 8 * q, c = lane + 32 * h;
                const int gy = oy + r - kHalo, gx = ox + c - kHalo;
                buf[q][h] = r < kLTH && c < kLTH ? make_float2(ld_zero(x, H, W, gy, gx), ld_zero(y, H, W, gy, gx))
                                                 : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int q = 0; q < kStageRows; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = warp + 8 * q, c = lane + 32 * h;
                if (r < kLTH && c < kLTH) sxy[r][c] = buf[q][h];
            }
    }
    __syncthreads();
    // horizontal blur of (x, y), (x^2, y^2) and xy: 42 rows x (32 / kHSeg) segments,
    // consecutive threads on consecutive rows (no bank conflicts)
    // input by input: each input's products x^2, y^2 and xy are formed once and
    // added to the kHSeg outputs whose window holds it
    for (int wi = threadIdx.x; wi < kLTH * (kLT / kHSeg); wi += 256) {
        const int r = wi % kLTH, c0 = (wi / kLTH) * kHSeg;
        float2 a01[kHSeg], a23[kHSeg];
        float a4[kHSeg];
#pragma unroll
        for (int o = 0; o < kHSeg; o++) { a01[o] = f2s(0.f); a23[o] = f2s(0.f); a4[o] = 0.f; }
#pragma unroll
        for (int j = 0; j < kHSeg + 10; j++) {
            const float2 vj = sxy[r][c0 + j];
            const float2 sj = __fmul2_rn(vj, vj);
            const float xj = vj.x * vj.y;
#pragma unroll
            for (int o = 0; o < kHSeg; o++) {
                const int t = j - o;
                if (t >= 0 && t < 11) {
                    const float2 wt = f2s(win.w[t]);
                    a01[o] = __ffma2_rn(wt, vj, a01[o]);
                    a23[o] = __ffma2_rn(wt, sj, a23[o]);
                    a4[o] = fmaf(wt.x, xj, a4[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kHSeg; o++) { hb01[r][c0 + o] = a01[o]; hb23[r][c0 + o] = a23[o]; hb4[r][c0 + o] = a4[o]; }
    }
    __syncthreads();
    // vertical blur and the SSIM terms: 32 columns x (32 / kVSeg) segments
    float ssum = 0.f, l1sum = 0.f;
    {
        const int c = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * kVSeg;
        float2 m01[kVSeg], m23[kVSeg];
        float m4[kVSeg];
#pragma unroll
        for (int o = 0; o < kVSeg; o++) { m01[o] = f2s(0.f); m23[o] = f2s(0.f); m4[o] = 0.f; }
#pragma unroll
        for (int j = 0; j < kVSeg + 10; j++) {
            const float2 v01 = hb01[r0 + j][c], v23 = hb23[r0 + j][c];
            const float v4 = hb4[r0 + j][c];
#pragma unroll
            for (int o = 0; o < kVSeg; o++) {
                const int t = j - o;
                if (t >= 0 && t < 11) {
                    const float2 wt = f2s(win.w[t]);
                    m01[o] = __ffma2_rn(wt, v01, m01[o]);
                    m23[o] = __ffma2_rn(wt, v23, m23[o]);
                    m4[o] = fmaf(wt.x, v4, m4[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kVSeg; o++) {
            const int r = r0 + o;
            const int gy = oy + r, gx = ox + c;
            if (gy >= H || gx >= W) continue;
            const float mx = m01[o].x, my = m01[o].y, exx = m23[o].x, eyy = m23[o].y, exy = m4[o];
            const float sxx = exx - mx * mx, syy = eyy - my * my, sxy_ = exy - mx * my;
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy_ + C2;
            const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
            const float iB = 1.f / (B1 * B2); // 1 / B1 = B2 iB, 1 / B2 = B1 iB
            const float S = A1 * A2 * iB;
            const float dmx = 2.f * my * A2 * iB - S * 2.f * mx * (B2 * iB);
            const float dsxx = -S * (B1 * iB);
            const float dsxy = 2.f * A1 * iB;
            const long long hw = (long long)H * W, p = (long long)gy * W + gx;
            float *Fp = F + 3 * (long long)plane * hw + p;
            Fp[0] = dmx - 2.f * mx * dsxx - my * dsxy;
            Fp[hw] = dsxx;
            Fp[2 * hw] = dsxy;
            ssum += S;
            const float2 px = sxy[r + kHalo][c + kHalo];
            l1sum += fabsf(px.x - px.y);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        l1sum += __shfl_xor_sync(0xffffffffu, l1sum, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ssum; red[1][threadIdx.x >> 5] = l1sum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < 8; w++) { a += red[0][w]; b += red[1][w]; }
        // the view's sums in 64-bit fixed point (24 fractional bits): integer
        // atomics add exactly, so the totals do not depend on block order
        const int view = blockIdx.z / 3;
        atomicAdd(&acc[2 * view], (unsigned long long)__float2ll_rn(a * 16777216.f));
        atomicAdd(&acc[2 * view + 1], (unsigned long long)__float2ll_rn(b * 16777216.f));
    }
}

// The loss from the views' fixed-point sums (SSIM, L1) of ssim_fwd_kernel,
// zeroed before it in the same call.
__device__ __forceinline__ float loss_from_sums(const unsigned long long *acc, int batch, int H, int W, float lambda)
{
    const double npx = 3.0 * H * W, unit = 1.0 / 16777216.0;
    double loss = 0.0;
    for (int b = 0; b < batch; b++) {
        const double ssim = (double)(long long)acc[2 * b] * unit, l1 = (double)(long long)acc[2 * b + 1] * unit;
        loss += ((1.0 - lambda) * l1 / npx + lambda * (1.0 - ssim / npx)) / batch;
    }
    return (float)loss;
}

// s_l1 = (1 - lambda) / (3 H W batch), s_ssim = lambda / (3 H W batch): the
// weights of the two mean terms of the batch's loss.  The first thread also
// writes the loss: the forward's sums are complete once this kernel runs.
__global__ void __launch_bounds__(256, 4) ssim_bwd_kernel(const float *img, const float *tgt, int H, int W, Win win,
                                                       const float *F, float s_l1, float s_ssim, float *dL,
                                                       const unsigned long long *acc, int batch, float lambda,
                                                       float *loss_out)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    if ((blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *loss_out = loss_from_sums(acc, batch, H, W, lambda);
    __shared__ float2 sf01[kLTH][kLTP];
    __shared__ float sf2[kLTH][kLTP];
    __shared__ float2 hb01[kLTH][kLT + 1];
    __shared__ float hb2[kLTH][kLT + 1];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    const long long hw = (long long)H * W;
    const float *Fp = F + 3 * (long long)plane * hw;
    // the image and target at this thread's outputs, in flight with the staging loads
    const int c = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * kVSeg;
    float xo[kVSeg], yo[kVSeg];
#pragma unroll
    for (int o = 0; o < kVSeg; o++) {
        const int gy = oy + r0 + o, gx = ox + c;
        const bool in = gy < H && gx < W;
        const long long p = (long long)plane * H * W + (long long)gy * W + gx;
        xo[o] = in ? img[p] : 0.f;
        yo[o] = in ? tgt[p] : 0.f;
    }
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        float2 b01[kStageRows][2];
        float b2[kStageRows][2];
#pragma unroll
        for (int q = 0; q < kStageRows; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = warp + 8 * q, cc = lane + 32 * h;
                const int gy = oy + r - kHalo, gx = ox + cc - kHalo;
                const bool in = r < kLTH && cc < kLTH && gy >= 0 && gy < H && gx >= 0 && gx < W;
                const long long p = (long long)gy * W + gx;
                b01[q][h] = in ? make_float2(Fp[p], Fp[hw + p]) : make_float2(0.f, 0.f);
                b2[q][h] = in ? Fp[2 * hw + p] : 0.f;
            }
#pragma unroll
        for (int q = 0; q < kStageRows; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = warp + 8 * q, cc = lane + 32 * h;
                if (r < kLTH && cc < kLTH) {
                    sf01[r][cc] = b01[q][h];
                    sf2[r][cc] = b2[q][h];
                }
            }
    }
    __syncthreads();
    for (int wi = threadIdx.x; wi < kLTH * (kLT / kHSeg); wi += 256) {
        const int r = wi % kLTH, c0 = (wi / kLTH) * kHSeg;
        float2 v01[kHSeg + 10];
        float v2[kHSeg + 10];
#pragma unroll
        for (int j = 0; j < kHSeg + 10; j++) { v01[j] = sf01[r][c0 + j]; v2[j] = sf2[r][c0 + j]; }
#pragma unroll
        for (int o = 0; o < kHSeg; o++) {
            float2 a01 = f2s(0.f);
            float a2 = 0.f;
#pragma unroll
            for (int t = 0; t < 11; t++) {
                a01 = __ffma2_rn(f2s(win.w[t]), v01[o + t], a01);
                a2 = fmaf(win.w[t], v2[o + t], a2);
            }
            hb01[r][c0 + o] = a01;
            hb2[r][c0 + o] = a2;
        }
    }
    __syncthreads();
    float2 b01[kVSeg];
    float b2[kVSeg];
#pragma unroll
    for (int o = 0; o < kVSeg; o++) { b01[o] = f2s(0.f); b2[o] = 0.f; }
#pragma unroll
    for (int j = 0; j < kVSeg + 10; j++) {
        const float2 v01 = hb01[r0 + j][c];
        const float v2 = hb2[r0 + j][c];
#pragma unroll
        for (int o = 0; o < kVSeg; o++) {
            const int t = j - o;
            if (t >= 0 && t < 11) {
                b01[o] = __ffma2_rn(f2s(win.w[t]), v01, b01[o]);
                b2[o] = fmaf(win.w[t], v2, b2[o]);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < kVSeg; o++) {
        const int gy = oy + r0 + o, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        const long long p = (long long)plane * H * W + (long long)gy * W + gx;
        const float xv = xo[o], yv = yo[o];
        const float dssim = b01[o].x + 2.f * xv * b01[o].y + yv * b2[o];
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dL[p] = s_l1 * sgn - s_ssim * dssim;
    }
}

cudaError_t launch_loss(gs_workspace *ws, cudaStream_t st, const float *img, const float *tgt, int B, int H, int W,
                        float lambda, float *loss_out, float *dL)
{
    Win win;
    double g[11], sum = 0.0;
    for (int k = 0; k < 11; k++) { g[k] = exp(-((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5)); sum += g[k]; }
    for (int k = 0; k < 11; k++) win.w[k] = (float)(g[k] / sum);
    const dim3 grid((W + kLT - 1) / kLT, (H + kLT - 1) / kLT, B * 3);
    float *maps = ws->loss_maps; // three planes per image plane
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(ws->loss_partial); // [B][2]
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * (size_t)B * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    kt_begin(ws, GS_KT_SSIM_FWD, st);
    launch_pdl(ssim_fwd_kernel, grid, 256, 0, st, img, tgt, H, W, win, 0.01f * 0.01f, 0.03f * 0.03f, maps, acc);
    kt_end(ws, GS_KT_SSIM_FWD, st);
    note_launch();
    kt_begin(ws, GS_KT_SSIM_BWD, st);
    const double wsum = 3.0 * H * W * B; // SSIM and L1 are means over channels, pixels and views
    launch_pdl(ssim_bwd_kernel, grid, 256, 0, st, img, tgt, H, W, win, maps, (float)((1.0 - lambda) / wsum),
               (float)(lambda / wsum), dL, (const unsigned long long *)acc, B, lambda, loss_out);
    kt_end(ws, GS_KT_SSIM_BWD, st);
    note_launch();
    return cudaGetLastError();
}

// ---- Adam -------------------------------------------------------------------

// b^t by binary powering: the same IEEE operations in the same order on the
// host and the device, so both compute bit-identical bias corrections (kept
// out of line so that no caller fuses its result into a multiply-add).
__host__ __device__ __noinline__ double powi(double b, int t)
{
    double r = 1.0;
    while (t > 0) {
        if (t & 1) r *= b;
        b *= b;
        t >>= 1;
    }
    return r;
}

struct AdamTable {
    int n;
    unsigned block_start[GS_MAX_ADAM_GROUPS + 1]; // first block of each group
    long long count[GS_MAX_ADAM_GROUPS];
    int vec[GS_MAX_ADAM_GROUPS];                  // all four arrays 16-byte aligned
    float *p[GS_MAX_ADAM_GROUPS];
    const float *g[GS_MAX_ADAM_GROUPS];
    float *m[GS_MAX_ADAM_GROUPS];
    float *v[GS_MAX_ADAM_GROUPS];
    // sparse gradient source (fused backward): element e of the group belongs to
    // Gaussian e / per_g; its gradient is cgrad[rec_first[gauss] * 59 + col + e % per_g],
    // or 0 when rec_first[gauss] == ~0 (no record this step)
    const uint32_t *rec_first[GS_MAX_ADAM_GROUPS];
    const float *cgrad;
    int col[GS_MAX_ADAM_GROUPS], per_g[GS_MAX_ADAM_GROUPS];
    float lr_c[GS_MAX_ADAM_GROUPS];   // lr / (1 - beta1^t)
    float ibc2[GS_MAX_ADAM_GROUPS];   // 1 / sqrt(1 - beta2^t)
    const float *coef;                // device [2][GS_MAX_ADAM_GROUPS]: lr_c, ibc2 (replaces the two above)
    float b1[GS_MAX_ADAM_GROUPS], b2[GS_MAX_ADAM_GROUPS], eps[GS_MAX_ADAM_GROUPS];
};

constexpr int kAdamPerThread = 4;  // float4 chunks per thread
constexpr int kAdamBlockElems = 256 * 4 * kAdamPerThread;

// m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;  p <- p - lr_c m / (sqrt(v) ibc2 + eps)
// with lr_c = lr / (1 - b1^t), ibc2 = 1 / sqrt(1 - b2^t) (bias correction folded in).
__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float b1, float b2, float lr_c,
                                         float ibc2, float eps)
{
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p = fmaf(-lr_c * m, rcp_approx(fmaf(sqrt_approx(v), ibc2, eps)), p);
}

// Gradient of element e of a group with PER elements per Gaussian taken from
// the compact rows: 0 unless Gaussian e / PER has a record.
template <int PER>
__device__ __forceinline__ float sparse_grad(const uint32_t *rec_first, const float *cgrad, int col, long long e)
{
    const long long gauss = (long long)((unsigned long long)e / (unsigned)PER);
    const uint32_t rh = rec_first[gauss];
    return rh == 0xffffffffu ? 0.f : cgrad[(long long)rh * kGradRow + col + (e - gauss * PER)];
}

template <int PER>
__device__ __forceinline__ float4 sparse_grad4(const uint32_t *rec_first, const float *cgrad, int col, long long e)
{
    if (PER % 4 == 0) { // the chunk lies in one Gaussian's row: one lookup
        const long long gauss = (long long)((unsigned long long)e / (unsigned)PER);
        const uint32_t rh = rec_first[gauss];
        if (rh == 0xffffffffu) return make_float4(0.f, 0.f, 0.f, 0.f);
        const float *row = cgrad + (long long)rh * kGradRow + col + (e - gauss * PER);
        return make_float4(row[0], row[1], row[2], row[3]);
    }
    return make_float4(sparse_grad<PER>(rec_first, cgrad, col, e), sparse_grad<PER>(rec_first, cgrad, col, e + 1),
                       sparse_grad<PER>(rec_first, cgrad, col, e + 2), sparse_grad<PER>(rec_first, cgrad, col, e + 3));
}

// One block's range of one group.  PER == 0: dense gradient array; PER > 0:
// gradients from the compact rows, PER elements per Gaussian.
template <int PER>
__device__ __forceinline__ void adam_block(const AdamTable &t, int gi, long long base)
{
    const long long n = t.count[gi];
    const float b1 = t.b1[gi], b2 = t.b2[gi], eps = t.eps[gi];
    const float lr_c = t.coef ? t.coef[gi] : t.lr_c[gi];
    const float ibc2 = t.coef ? t.coef[GS_MAX_ADAM_GROUPS + gi] : t.ibc2[gi];
    float *P = t.p[gi], *M = t.m[gi], *V = t.v[gi];
    const float *G = t.g[gi];
    const uint32_t *rf = t.rec_first[gi];
    const float *cg = t.cgrad;
    const int col = t.col[gi];
    if (t.vec[gi]) {
        float4 pv[kAdamPerThread], gv[kAdamPerThread], mv[kAdamPerThread], vv[kAdamPerThread];
        // every streaming load of this thread first ...
#pragma unroll
        for (int k = 0; k < kAdamPerThread; k++) {
            const long long e = base + 4ll * (threadIdx.x + 256 * k);
            if (e + 3 < n) {
                pv[k] = __ldcs(reinterpret_cast<const float4 *>(P + e));
                mv[k] = __ldcs(reinterpret_cast<const float4 *>(M + e));
                vv[k] = __ldcs(reinterpret_cast<const float4 *>(V + e));
                if (PER == 0) gv[k] = __ldcs(reinterpret_cast<const float4 *>(G + e));
            }
        }
        // ... then the (mostly empty) compact-row lookups
        if (PER > 0) {
#pragma unroll
            for (int k = 0; k < kAdamPerThread; k++) {
                const long long e = base + 4ll * (threadIdx.x + 256 * k);
                if (e + 3 < n) gv[k] = sparse_grad4<(PER > 0 ? PER : 1)>(rf, cg, col, e);
            }
        }
#pragma unroll
        for (int k = 0; k < kAdamPerThread; k++) {
            const long long e = base + 4ll * (threadIdx.x + 256 * k);
            if (e + 3 < n) {
                adam_one(pv[k].x, gv[k].x, mv[k].x, vv[k].x, b1, b2, lr_c, ibc2, eps);
                adam_one(pv[k].y, gv[k].y, mv[k].y, vv[k].y, b1, b2, lr_c, ibc2, eps);
                adam_one(pv[k].z, gv[k].z, mv[k].z, vv[k].z, b1, b2, lr_c, ibc2, eps);
                adam_one(pv[k].w, gv[k].w, mv[k].w, vv[k].w, b1, b2, lr_c, ibc2, eps);
                __stcs(reinterpret_cast<float4 *>(P + e), pv[k]);
                __stcs(reinterpret_cast<float4 *>(M + e), mv[k]);
                __stcs(reinterpret_cast<float4 *>(V + e), vv[k]);
            } else {
                for (long long q = e; q < n && q < e + 4; q++)
                    adam_one(P[q], PER == 0 ? G[q] : sparse_grad<(PER > 0 ? PER : 1)>(rf, cg, col, q), M[q], V[q],
                             b1, b2, lr_c, ibc2, eps);
            }
        }
    } else {
        for (int k = 0; k < 4 * kAdamPerThread; k++) {
            const long long q = base + threadIdx.x + 256ll * k;
            if (q < n)
                adam_one(P[q], PER == 0 ? G[q] : sparse_grad<(PER > 0 ? PER : 1)>(rf, cg, col, q), M[q], V[q], b1,
                         b2, lr_c, ibc2, eps);
        }
    }
}

// One block range per group; the group's gradient source is resolved once per
// block.  Streaming: 28 bytes of HBM traffic per parameter with a dense
// gradient, 24 with the compact rows.
__global__ void __launch_bounds__(256) adam_kernel(AdamTable t)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    int gi = 0;
    while (blockIdx.x >= t.block_start[gi + 1]) gi++;
    const long long base = (long long)(blockIdx.x - t.block_start[gi]) * kAdamBlockElems;
    if (!t.rec_first[gi]) { adam_block<0>(t, gi, base); return; }
    switch (t.per_g[gi]) {
    case 48: adam_block<48>(t, gi, base); break;
    case 4: adam_block<4>(t, gi, base); break;
    case 3: adam_block<3>(t, gi, base); break;
    default: adam_block<1>(t, gi, base); break;
    }
}

static cudaError_t run_adam(AdamTable &t, int n_groups, cudaStream_t st)
{
    for (int k = n_groups; k < GS_MAX_ADAM_GROUPS; k++) t.block_start[k + 1] = t.block_start[k];
    if (t.block_start[n_groups] == 0) return cudaSuccess;
    launch_pdl(adam_kernel, t.block_start[n_groups], 256, 0, st, t);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adam(const gs_adam_group *groups, int n_groups, int step, cudaStream_t st)
{
    AdamTable t;
    t.n = n_groups;
    t.cgrad = nullptr;
    t.coef = nullptr;
    t.block_start[0] = 0;
    auto al16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    for (int k = 0; k < n_groups; k++) {
        const gs_adam_group &g = groups[k];
        const long long blocks = (g.n + kAdamBlockElems - 1) / kAdamBlockElems;
        t.block_start[k + 1] = t.block_start[k] + (unsigned)blocks;
        t.count[k] = g.n;
        t.vec[k] = al16(g.param) && al16(g.grad) && al16(g.m) && al16(g.v);
        t.p[k] = g.param; t.g[k] = g.grad; t.m[k] = g.m; t.v[k] = g.v;
        t.lr_c[k] = (float)((double)g.lr / (1.0 - powi((double)g.beta1, step)));
        t.ibc2[k] = (float)(1.0 / sqrt(1.0 - powi((double)g.beta2, step)));
        t.b1[k] = g.beta1; t.b2[k] = g.beta2; t.eps[k] = g.eps;
        t.rec_first[k] = nullptr; t.col[k] = 0; t.per_g[k] = 1;
    }
    return run_adam(t, n_groups, st);
}

struct AdamCoefArgs {
    float lr[5];
    float b1, b2;
    int step; // > 0: this step; 0: one past the device counter
};

// Step number and bias-corrected coefficients on the device, so a captured
// optimizer step advances its own counter on every replay.  With deferred
// steps enabled the coefficients of every step are also kept (hist), so a
// Gaussian brought up to date later replays exactly the steps it missed.
__global__ void adam_coef_kernel(AdamCoefArgs a, int *d_step, float *coef, float *hist, int max_steps,
                                 DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    if (threadIdx.x != 0) return;
    const int t = a.step > 0 ? a.step : *d_step + 1;
    *d_step = t;
    const double c1 = 1.0 - powi((double)a.b1, t), c2 = 1.0 - powi((double)a.b2, t);
    for (int k = 0; k < 5; k++) {
        coef[k] = (float)((double)a.lr[k] / c1);
        coef[GS_MAX_ADAM_GROUPS + k] = (float)(1.0 / sqrt(c2));
    }
    if (hist) {
        if (t > max_steps) {
            set_error(ctr, GS_ERR_CAPACITY, kSiteModel);
            return;
        }
        for (int k = 0; k < 5; k++) {
            hist[10 * t + k] = coef[k];
            hist[10 * t + 5 + k] = coef[GS_MAX_ADAM_GROUPS + k];
        }
    }
}

// ---- deferred zero-gradient steps ------------------------------------------------
//
// Dense Adam moves every parameter every step, also those without a gradient
// (m and v decay, p follows the momentum).  With deferred steps a Gaussian's
// p, m, v are kept as of the step in last[i] and brought up to date only
// when it is next used: before its projection (preprocess), before its next
// gradient step, or by a flush.  Bringing it up to date replays exactly the
// zero-gradient steps it missed, through adam_one with the coefficients of
// each step, so every value equals dense Adam's bit for bit.  While it waits,
// drift[i] bounds how far its mean (Euclidean, summed over the axes) and its
// largest log-scale can still move: every further zero-gradient step moves a
// parameter by lr_c(t) |m| b1^j / ((sqrt(v) b2^(j/2)) ibc2 + eps) <=
// lr_c(last) |m| / (sqrt(v) + eps) r^j, r = b1 / sqrt(b2) < 1, so the total is
// at most lr_c(last) |m| / (sqrt(v) + eps) r / (1 - r) (drift_factor adds 1 %
// for the approximate square root and reciprocal).  The view gate widens its
// tests by these bounds, and the projection decides exactly on the
// up-to-date values.

struct LazyArgs {
    float *p[5], *m[5], *v[5];
    int32_t *last;
    float *drift;      // [2][n]: bounds on the further drift of the mean and of the largest log-scale
    long long n;       // Gaussians
    const float *hist;
    const int *d_step;
    float b1, b2, eps, drift_factor;
};


__device__ __forceinline__ int group_len(int k) { return k == 4 ? 48 : k == 3 ? 1 : k == 2 ? 4 : 3; }

// The deferred steps run element-parallel.  A first kernel gives each
// (Gaussian, parameter) pair one thread, which replays that parameter's missed
// zero-gradient steps (and takes the gradient step): it reads last[i] and
// never writes it, so the threads of one Gaussian need no ordering.  A second
// kernel, one thread per Gaussian, then moves last[i] to the current step and
// recomputes the drift bounds from the moments now stored.  Items: every
// Gaussian (flush), the gate's candidates (catch-up, before projecting them) or
// the Gaussians with a record (the gradient step).  A parameter whose m and v
// are both +0 is a fixed point of the zero-gradient step (m and v stay +0, p
// moves by (-lr m) / (sqrt(v) ibc2 + eps) = -0), so its replay is skipped and,
// without a gradient step, it is not written at all.
enum LazyMode { kLazyAll = 0, kLazyCandidates = 1, kLazyGrad = 2 };
// kLazyCandidates runs over the list of the candidates that are behind (the
// catch-up list), in the order a selection pass appended them: each
// Gaussian's replay is independent of the others, so the order is immaterial.

struct LazyItems {
    const uint32_t *cand_g;    // kLazyCandidates: the catch-up list (Gaussians of the gate's candidates that are behind)
    const uint32_t *rec_g;     // kLazyGrad: Gaussian of each record (a Gaussian's records contiguous)
    const uint32_t *rec_first; // kLazyGrad: first record of each Gaussian
    const float *cgrad;        // kLazyGrad: compact gradient rows at the first record
    const DevCounters *ctr;    // sizes of the device lists
    long long n;               // kLazyAll: Gaussians
};

template <int MODE> __device__ __forceinline__ unsigned long long lazy_count(const LazyItems &it)
{
    return MODE == kLazyAll ? (unsigned long long)it.n
                            : MODE == kLazyCandidates ? it.ctr->n_catchup : it.ctr->n_records;
}

// item j -> Gaussian i; false for a record that is not its Gaussian's first
template <int MODE> __device__ __forceinline__ bool lazy_item(const LazyItems &it, unsigned long long j, long long &i)
{
    if (MODE == kLazyAll) { i = (long long)j; return true; }
    if (MODE == kLazyCandidates) { i = it.cand_g[j]; return true; }
    const uint32_t gi = it.rec_g[j];
    if (j > 0 && it.rec_g[j - 1] == gi) return false;
    i = gi;
    return true;
}

// Parameter element idx of group k of Gaussian i: from its step `from` to step
// t (kLazyGrad: the zero-gradient steps to t - 1, then the gradient step t).
template <int MODE>
__device__ __forceinline__ void lazy_param(const LazyArgs &a, int k, long long idx, int from, int t, float grad)
{
    const int to = MODE == kLazyGrad ? t - 1 : t;
    float mv = a.m[k][idx], vv = a.v[k][idx];
    const bool zero = (__float_as_uint(mv) | __float_as_uint(vv)) == 0u;
    if (zero && MODE != kLazyGrad) return;
    float pv = a.p[k][idx];
    if (!zero)
        for (int s = from + 1; s <= to; s++)
            adam_one(pv, 0.f, mv, vv, a.b1, a.b2, a.hist[10 * s + k], a.hist[10 * s + 5 + k], a.eps);
    if (MODE == kLazyGrad) adam_one(pv, grad, mv, vv, a.b1, a.b2, a.hist[10 * t + k], a.hist[10 * t + 5 + k], a.eps);
    a.p[k][idx] = pv; a.m[k][idx] = mv; a.v[k][idx] = vv;
}

// every Gaussian: each group's array of n * LEN floats (16-byte aligned) in
// float4 chunks, consecutive threads on consecutive chunks.  A chunk whose m
// and v are all +0 needs nothing, not even its Gaussians' steps.
template <int LEN>
__device__ __forceinline__ void lazy_all_group(const LazyArgs &a, int k, long long n, int t)
{
    const unsigned long long total = (unsigned long long)n * LEN, chunks = total / 4;
    const unsigned long long stride = gridDim.x * 256ull;
    float *P = a.p[k], *M = a.m[k], *V = a.v[k];
    for (unsigned long long c = blockIdx.x * 256ull + threadIdx.x; c < chunks; c += stride) {
        float4 m4 = reinterpret_cast<const float4 *>(M)[c], v4 = reinterpret_cast<const float4 *>(V)[c];
        float mv[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
        unsigned nz = 0;
#pragma unroll
        for (int u = 0; u < 4; u++) nz |= (__float_as_uint(mv[u]) | __float_as_uint(vv[u])) != 0u ? 1u << u : 0u;
        if (!nz) continue;
        int from[4];
        bool any = false;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            from[u] = a.last[(4 * c + u) / LEN];
            any = any || ((nz >> u) & 1u && from[u] < t);
        }
        if (!any) continue;
        const float4 p4 = reinterpret_cast<const float4 *>(P)[c];
        float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (!((nz >> u) & 1u)) continue;
            for (int s = from[u] + 1; s <= t; s++)
                adam_one(pv[u], 0.f, mv[u], vv[u], a.b1, a.b2, a.hist[10 * s + k], a.hist[10 * s + 5 + k], a.eps);
        }
        reinterpret_cast<float4 *>(P)[c] = make_float4(pv[0], pv[1], pv[2], pv[3]);
        reinterpret_cast<float4 *>(M)[c] = make_float4(mv[0], mv[1], mv[2], mv[3]);
        reinterpret_cast<float4 *>(V)[c] = make_float4(vv[0], vv[1], vv[2], vv[3]);
    }
    // the last total % 4 elements
    for (unsigned long long e = chunks * 4 + blockIdx.x * 256ull + threadIdx.x; e < total; e += stride) {
        const int from = a.last[e / LEN];
        if (from < t) lazy_param<kLazyAll>(a, k, (long long)e, from, t, 0.f);
    }
}

__global__ void __launch_bounds__(256) lazy_all_elem_kernel(LazyArgs a, long long n)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const int t = *a.d_step;
    lazy_all_group<3>(a, 0, n, t);   // mean
    lazy_all_group<3>(a, 1, n, t);   // log-scale
    lazy_all_group<4>(a, 2, n, t);   // quaternion
    lazy_all_group<1>(a, 3, n, t);   // opacity
    lazy_all_group<48>(a, 4, n, t);  // SH
}

// The Gaussians of a device list, 20 consecutive threads per Gaussian, one
// per unit of its row: the 48 SH coefficients as 12 float4, the quaternion as
// one float4 (both 16-byte aligned rows), and the 3 + 3 + 1 scalars of mean,
// log-scale and opacity.  Every component takes exactly lazy_param's steps.
// A record head j is its Gaussian's first record: its compact gradient row
// is row j.
constexpr int kLazyUnits = 20;
__device__ __forceinline__ void lazy_unit(int u, int &k, int &el, int &row)
{
    if (u < 12) { k = 4; el = 4 * u; row = 11 + el; }            // SH, float4
    else if (u == 12) { k = 2; el = 0; row = 6; }                  // quaternion, float4
    else if (u < 16) { k = 0; el = u - 13; row = el; }             // mean
    else if (u < 19) { k = 1; el = u - 16; row = 3 + el; }         // log-scale
    else { k = 3; el = 0; row = 10; }                              // opacity
}

// The gradient step of one unit (a float4 of SH or quaternion, or a scalar)
// of Gaussian i: the zero-gradient steps it missed, then step t with its
// gradient, exactly lazy_param's steps.  Every load it needs (last step,
// p, m, v, gradient) is issued before any is used, so a unit waits for memory
// once.
__device__ __forceinline__ void lazy_grad_unit(const LazyArgs &a, const float *grad, long long i, int u, int k,
                                               long long idx, int t)
{
    const int from = a.last[i];
    if (u > 12) { // a scalar
        float pv = a.p[k][idx], mv = a.m[k][idx], vv = a.v[k][idx];
        const float g = grad[0];
        if (from >= t) return;
        if ((__float_as_uint(mv) | __float_as_uint(vv)) != 0u)
            for (int s = from + 1; s <= t - 1; s++)
                adam_one(pv, 0.f, mv, vv, a.b1, a.b2, a.hist[10 * s + k], a.hist[10 * s + 5 + k], a.eps);
        adam_one(pv, g, mv, vv, a.b1, a.b2, a.hist[10 * t + k], a.hist[10 * t + 5 + k], a.eps);
        a.p[k][idx] = pv; a.m[k][idx] = mv; a.v[k][idx] = vv;
        return;
    }
    const float4 p4 = *reinterpret_cast<const float4 *>(a.p[k] + idx);
    const float4 m4 = *reinterpret_cast<const float4 *>(a.m[k] + idx);
    const float4 v4 = *reinterpret_cast<const float4 *>(a.v[k] + idx);
    const float g[4] = {grad[0], grad[1], grad[2], grad[3]};
    if (from >= t) return;
    float pv[4] = {p4.x, p4.y, p4.z, p4.w}, mv[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if ((__float_as_uint(mv[c]) | __float_as_uint(vv[c])) != 0u)
            for (int s = from + 1; s <= t - 1; s++)
                adam_one(pv[c], 0.f, mv[c], vv[c], a.b1, a.b2, a.hist[10 * s + k], a.hist[10 * s + 5 + k], a.eps);
        adam_one(pv[c], g[c], mv[c], vv[c], a.b1, a.b2, a.hist[10 * t + k], a.hist[10 * t + 5 + k], a.eps);
    }
    *reinterpret_cast<float4 *>(a.p[k] + idx) = make_float4(pv[0], pv[1], pv[2], pv[3]);
    *reinterpret_cast<float4 *>(a.m[k] + idx) = make_float4(mv[0], mv[1], mv[2], mv[3]);
    *reinterpret_cast<float4 *>(a.v[k] + idx) = make_float4(vv[0], vv[1], vv[2], vv[3]);
}

template <int MODE> __global__ void __launch_bounds__(256) lazy_list_vec_kernel(LazyArgs a, LazyItems it)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const int t = *a.d_step;
    const unsigned long long total = lazy_count<MODE>(it) * kLazyUnits;
    for (unsigned long long e = blockIdx.x * 256ull + threadIdx.x; e < total; e += gridDim.x * 256ull) {
        const unsigned long long j = e / kLazyUnits;
        const int u = (int)(e - j * kLazyUnits);
        long long i;
        if (!lazy_item<MODE>(it, j, i)) continue;
        int k, el, row;
        lazy_unit(u, k, el, row);
        const long long idx = i * group_len(k) + el;
        if (MODE == kLazyGrad) {
            lazy_grad_unit(a, it.cgrad + j * kGradRow + row, i, u, k, idx, t);
            continue;
        }
        const int from = a.last[i];
        if (from >= t) continue;
        // a catch-up (no gradient): only units with a moment that is not +0 move
        if (u > 12) { // a scalar
            lazy_param<MODE>(a, k, idx, from, t, 0.f);
            continue;
        }
        const float4 m4 = *reinterpret_cast<const float4 *>(a.m[k] + idx);
        const float4 v4 = *reinterpret_cast<const float4 *>(a.v[k] + idx);
        float mv[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
        bool zero[4], any = false;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            zero[c] = (__float_as_uint(mv[c]) | __float_as_uint(vv[c])) == 0u;
            any = any || !zero[c];
        }
        if (!any) continue; // every component a fixed point
        const float4 p4 = *reinterpret_cast<const float4 *>(a.p[k] + idx);
        float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (!zero[c])
                for (int s2 = from + 1; s2 <= t; s2++)
                    adam_one(pv[c], 0.f, mv[c], vv[c], a.b1, a.b2, a.hist[10 * s2 + k], a.hist[10 * s2 + 5 + k], a.eps);
        }
        *reinterpret_cast<float4 *>(a.p[k] + idx) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        *reinterpret_cast<float4 *>(a.m[k] + idx) = make_float4(mv[0], mv[1], mv[2], mv[3]);
        *reinterpret_cast<float4 *>(a.v[k] + idx) = make_float4(vv[0], vv[1], vv[2], vv[3]);
    }
}

// last[i] = t and the drift bounds of Gaussian i from its current moments
template <int MODE> __global__ void __launch_bounds__(256) lazy_fin_kernel(LazyArgs a, LazyItems it)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const int t = *a.d_step;
    const unsigned long long cnt = lazy_count<MODE>(it);
    for (unsigned long long j = blockIdx.x * 256ull + threadIdx.x; j < cnt; j += gridDim.x * 256ull) {
        long long i;
        if (!lazy_item<MODE>(it, j, i)) continue;
        if (a.last[i] >= t) continue;
        a.last[i] = t;
        float dm = 0.f, ds = 0.f;
#pragma unroll
        for (int l = 0; l < 3; l++) {
            dm += fabsf(a.m[0][3 * i + l]) / (sqrtf(a.v[0][3 * i + l]) + a.eps);
            ds = fmaxf(ds, fabsf(a.m[1][3 * i + l]) / (sqrtf(a.v[1][3 * i + l]) + a.eps));
        }
        a.drift[i] = t > 0 ? a.drift_factor * a.hist[10 * t] * dm : 0.f;
        a.drift[a.n + i] = t > 0 ? a.drift_factor * a.hist[10 * t + 1] * ds : 0.f;
    }
}

static LazyArgs lazy_args(gs_workspace *ws, const gs_gaussian_grads &param, long long n)
{
    LazyArgs a;
    a.n = n;
    float *P[5] = {param.mean, param.log_scale, param.quat, param.opacity_logit, param.sh};
    const gs_gaussian_grads &m = ws->lazy.m, &v = ws->lazy.v;
    float *M[5] = {m.mean, m.log_scale, m.quat, m.opacity_logit, m.sh};
    float *V[5] = {v.mean, v.log_scale, v.quat, v.opacity_logit, v.sh};
    for (int k = 0; k < 5; k++) { a.p[k] = P[k]; a.m[k] = M[k]; a.v[k] = V[k]; }
    a.last = ws->lazy.last;
    a.drift = ws->lazy.drift;
    a.hist = ws->lazy.hist;
    a.d_step = ws->d_adam_step;
    a.b1 = ws->lazy.b1; a.b2 = ws->lazy.b2; a.eps = ws->lazy.eps; a.drift_factor = ws->lazy.drift_factor;
    return a;
}

static gs_gaussian_grads params_of(const gs_gaussians &g)
{
    gs_gaussian_grads p;
    p.mean = const_cast<float *>(g.mean);
    p.log_scale = const_cast<float *>(g.log_scale);
    p.quat = const_cast<float *>(g.quat);
    p.opacity_logit = const_cast<float *>(g.opacity_logit);
    p.sh = const_cast<float *>(g.sh);
    return p;
}

static LazyItems lazy_items(gs_workspace *ws, long long n)
{
    LazyItems it;
    it.cand_g = ws->cand_g; it.rec_g = ws->rec_g; it.rec_first = ws->rec_first; it.cgrad = ws->cgrad;
    it.ctr = ws->ctr; it.n = n;
    return it;
}

// grid of up to 8 resident 256-thread blocks per SM, striding over `work` items
static unsigned lazy_grid(gs_workspace *ws, unsigned long long work)
{
    return (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>((work + 255) / 256,
                                                                                   8ull * ws->sm_count));
}

template <int MODE>
static cudaError_t launch_lazy_list(gs_workspace *ws, cudaStream_t st, const LazyArgs &a, unsigned long long cap)
{
    const LazyItems it = lazy_items(ws, 0);
    if (MODE == kLazyGrad) kt_begin(ws, GS_KT_ADAM_GRAD, st);
    launch_pdl(lazy_list_vec_kernel<MODE>, lazy_grid(ws, cap * kLazyUnits), 256, 0, st, a, it);
    if (MODE == kLazyGrad) kt_end(ws, GS_KT_ADAM_GRAD, st);
    note_launch();
    launch_pdl(lazy_fin_kernel<MODE>, lazy_grid(ws, cap), 256, 0, st, a, it);
    note_launch();
    return cudaGetLastError();
}

// The catch-up list: the gate's candidates whose p, m, v are behind the
// current step (in the steady state of a training run, few or none), appended
// with one atomic per warp.
__global__ void __launch_bounds__(256) lazy_select_kernel(const uint32_t *cand_g, const int32_t *last,
                                                          const int *d_step, uint32_t *list, DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const unsigned long long ncand = ctr->n_candidates;
    const int t = *d_step, lane = threadIdx.x & 31;
    for (unsigned long long j0 = (unsigned long long)blockIdx.x * 256 + (threadIdx.x & ~31u); j0 < ncand;
         j0 += (unsigned long long)gridDim.x * 256) {
        const unsigned long long j = j0 + lane;
        uint32_t i = 0;
        bool behind = false;
        if (j < ncand) {
            i = cand_g[j];
            behind = last[i] < t;
        }
        const unsigned b = __ballot_sync(0xffffffffu, behind);
        if (!b) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctr->n_catchup, (unsigned long long)__popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (behind) list[base + __popc(b & ((1u << lane) - 1u))] = i;
    }
}

cudaError_t launch_lazy_catchup(gs_workspace *ws, cudaStream_t st, const gs_gaussians &g)
{
    if (g.n == 0) return cudaSuccess;
    // the list goes to the gate's per-chunk candidate buffer ([n], free once gathered)
    launch_pdl(lazy_select_kernel, lazy_grid(ws, (unsigned long long)g.n), 256, 0, st, ws->cand_g, ws->lazy.last,
               ws->d_adam_step, ws->gate_g, ws->ctr);
    note_launch();
    LazyArgs a = lazy_args(ws, params_of(g), g.n);
    LazyItems it = lazy_items(ws, 0);
    it.cand_g = ws->gate_g;
    launch_pdl(lazy_list_vec_kernel<kLazyCandidates>, lazy_grid(ws, (unsigned long long)g.n * kLazyUnits), 256, 0,
               st, a, it);
    note_launch();
    launch_pdl(lazy_fin_kernel<kLazyCandidates>, lazy_grid(ws, (unsigned long long)g.n), 256, 0, st, a, it);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_lazy_flush(gs_workspace *ws, cudaStream_t st, const gs_gaussians &g)
{
    if (g.n == 0) return cudaSuccess;
    const LazyArgs a = lazy_args(ws, params_of(g), g.n);
    launch_pdl(lazy_all_elem_kernel, lazy_grid(ws, (unsigned long long)g.n * kGradRow), 256, 0, st, a, g.n);
    note_launch();
    launch_pdl(lazy_fin_kernel<kLazyAll>, lazy_grid(ws, (unsigned long long)g.n), 256, 0, st, a, lazy_items(ws, g.n));
    note_launch();
    return cudaGetLastError();
}

static cudaError_t launch_lazy_adam(gs_workspace *ws, cudaStream_t st, const gs_gaussian_grads &param, long long n)
{
    if (ws->cap.max_records == 0) return cudaSuccess;
    return launch_lazy_list<kLazyGrad>(ws, st, lazy_args(ws, param, n), (unsigned long long)ws->cap.max_records);
}

cudaError_t launch_adam_sparse(gs_workspace *ws, cudaStream_t st, const gs_gaussian_grads &param,
                               const gs_gaussian_grads &m, const gs_gaussian_grads &v, long long n,
                               const float lr[5], float beta1, float beta2, float eps, int step)
{
    AdamCoefArgs ca;
    for (int k = 0; k < 5; k++) ca.lr[k] = lr[k];
    ca.b1 = beta1; ca.b2 = beta2; ca.step = step;
    launch_pdl(adam_coef_kernel, 1, 32, 0, st, ca, ws->d_adam_step, ws->d_adam_coef, ws->lazy.hist, ws->lazy.max_steps,
                                       ws->ctr);
    note_launch();
    if (ws->lazy.enabled) return launch_lazy_adam(ws, st, param, n);
    AdamTable t;
    t.n = 5;
    t.cgrad = ws->cgrad;
    t.coef = ws->d_adam_coef;
    t.block_start[0] = 0;
    float *P[5] = {param.mean, param.log_scale, param.quat, param.opacity_logit, param.sh};
    float *M[5] = {m.mean, m.log_scale, m.quat, m.opacity_logit, m.sh};
    float *V[5] = {v.mean, v.log_scale, v.quat, v.opacity_logit, v.sh};
    const int per[5] = {3, 3, 4, 1, 48}, col[5] = {0, 3, 6, 10, 11};
    auto al16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
    for (int k = 0; k < 5; k++) {
        const long long cnt = n * per[k];
        t.block_start[k + 1] = t.block_start[k] + (unsigned)((cnt + kAdamBlockElems - 1) / kAdamBlockElems);
        t.count[k] = cnt;
        t.vec[k] = al16(P[k]) && al16(M[k]) && al16(V[k]);
        t.p[k] = P[k]; t.g[k] = nullptr; t.m[k] = M[k]; t.v[k] = V[k];
        t.rec_first[k] = ws->rec_first; t.col[k] = col[k]; t.per_g[k] = per[k];
        t.lr_c[k] = 0.f; t.ibc2[k] = 0.f;
        t.b1[k] = beta1; t.b2[k] = beta2; t.eps[k] = eps;
    }
    return run_adam(t, 5, st);
}

} // namespace gs
