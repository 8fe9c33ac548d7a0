// optim.cu -- photometric loss of Eq. 4 (L1 + lambda (1 - SSIM)) with its
// gradient, and the Adam step (Kingma and Ba) of standard 3DGS training.
//
// SSIM uses an 11x11 Gaussian window (sigma 1.5, separable), C1 = 0.01^2,
// C2 = 0.03^2 and zero padding.  Pass 1 blurs x, y, x^2, y^2, xy over a tile
// with a 5-pixel halo, forms the SSIM map and the three coefficient maps its
// gradient needs; pass 2 blurs those maps (the window is symmetric, so the
// adjoint of the blur is the blur) and assembles dL/dx.  Partial sums are
// reduced in a fixed order in FP64.
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
// rather than once per tap.
constexpr int kHSeg = 8;                 // horizontal outputs per thread (42 rows x 4 segments)
constexpr int kVSeg = 4;                 // vertical outputs per thread (32 columns x 8 segments)
constexpr int kLTP = kLTH + 1;           // padded row of the staged tile

// grid: (tiles_x, tiles_y, batch * 3)
__global__ void __launch_bounds__(256) ssim_fwd_kernel(const float *img, const float *tgt, int H, int W, Win win,
                                                       float C1, float C2, float *F /*[3][B*3][H][W]*/,
                                                       long long plane_stride_maps, float *partial)
{
    __shared__ float sx[kLTH][kLTP], sy[kLTH][kLTP];
    __shared__ float hb[5][kLTH][kLT + 1];
    __shared__ float red[2][8];
    const int plane = blockIdx.z;
    const float *x = img + (long long)plane * H * W;
    const float *y = tgt + (long long)plane * H * W;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    for (int k = threadIdx.x; k < kLTH * kLTH; k += 256) {
        const int r = k / kLTH, c = k % kLTH;
        sx[r][c] = ld_zero(x, H, W, oy + r - kHalo, ox + c - kHalo);
        sy[r][c] = ld_zero(y, H, W, oy + r - kHalo, ox + c - kHalo);
    }
    __syncthreads();
    // horizontal blur of x, y, x^2, y^2, xy: 42 rows x (32 / kHSeg) segments
    for (int wi = threadIdx.x; wi < kLTH * (kLT / kHSeg); wi += 256) {
        const int r = wi / (kLT / kHSeg), c0 = (wi % (kLT / kHSeg)) * kHSeg;
        float xv[kHSeg + 10], yv[kHSeg + 10];
#pragma unroll
        for (int j = 0; j < kHSeg + 10; j++) { xv[j] = sx[r][c0 + j]; yv[j] = sy[r][c0 + j]; }
#pragma unroll
        for (int o = 0; o < kHSeg; o++) {
            float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
#pragma unroll
            for (int t = 0; t < 11; t++) {
                const float xt = xv[o + t], yt = yv[o + t], wt = win.w[t];
                a0 += wt * xt; a1 += wt * yt; a2 += wt * xt * xt; a3 += wt * yt * yt; a4 += wt * xt * yt;
            }
            hb[0][r][c0 + o] = a0; hb[1][r][c0 + o] = a1; hb[2][r][c0 + o] = a2; hb[3][r][c0 + o] = a3;
            hb[4][r][c0 + o] = a4;
        }
    }
    __syncthreads();
    // vertical blur and the SSIM terms: 32 columns x (32 / kVSeg) segments
    float ssum = 0.f, l1sum = 0.f;
    {
        const int c = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * kVSeg;
        float m[5][kVSeg];
#pragma unroll
        for (int q = 0; q < 5; q++)
#pragma unroll
            for (int o = 0; o < kVSeg; o++) m[q][o] = 0.f;
#pragma unroll
        for (int j = 0; j < kVSeg + 10; j++) {
            float v[5];
#pragma unroll
            for (int q = 0; q < 5; q++) v[q] = hb[q][r0 + j][c];
#pragma unroll
            for (int o = 0; o < kVSeg; o++) {
                const int t = j - o;
                if (t >= 0 && t < 11) {
                    const float wt = win.w[t];
#pragma unroll
                    for (int q = 0; q < 5; q++) m[q][o] += wt * v[q];
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kVSeg; o++) {
            const int r = r0 + o;
            const int gy = oy + r, gx = ox + c;
            if (gy >= H || gx >= W) continue;
            const float mx = m[0][o], my = m[1][o], exx = m[2][o], eyy = m[3][o], exy = m[4][o];
            const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
            const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
            const float iB = 1.f / (B1 * B2);
            const float S = A1 * A2 * iB;
            const float dmx = 2.f * my * A2 * iB - S * 2.f * mx / B1;
            const float dsxx = -S / B2;
            const float dsxy = 2.f * A1 * iB;
            const long long p = (long long)plane * H * W + (long long)gy * W + gx;
            F[p] = dmx - 2.f * mx * dsxx - my * dsxy;
            F[plane_stride_maps + p] = dsxx;
            F[2 * plane_stride_maps + p] = dsxy;
            ssum += S;
            l1sum += fabsf(sx[r + kHalo][c + kHalo] - sy[r + kHalo][c + kHalo]);
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
        const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partial[2 * blk] = a;
        partial[2 * blk + 1] = b;
    }
}

__global__ void __launch_bounds__(256) ssim_bwd_kernel(const float *img, const float *tgt, int H, int W, Win win,
                                                       const float *F, long long plane_stride_maps, float lambda,
                                                       int batch, float *dL)
{
    __shared__ float sf[3][kLTH][kLTP];
    __shared__ float hb[3][kLTH][kLT + 1];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    for (int k = threadIdx.x; k < kLTH * kLTH; k += 256) {
        const int r = k / kLTH, c = k % kLTH;
        for (int m = 0; m < 3; m++)
            sf[m][r][c] = ld_zero(F + m * plane_stride_maps + (long long)plane * H * W, H, W, oy + r - kHalo,
                                  ox + c - kHalo);
    }
    __syncthreads();
    for (int wi = threadIdx.x; wi < kLTH * (kLT / kHSeg); wi += 256) {
        const int r = wi / (kLT / kHSeg), c0 = (wi % (kLT / kHSeg)) * kHSeg;
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float v[kHSeg + 10];
#pragma unroll
            for (int j = 0; j < kHSeg + 10; j++) v[j] = sf[m][r][c0 + j];
#pragma unroll
            for (int o = 0; o < kHSeg; o++) {
                float a = 0.f;
#pragma unroll
                for (int t = 0; t < 11; t++) a += win.w[t] * v[o + t];
                hb[m][r][c0 + o] = a;
            }
        }
    }
    __syncthreads();
    const float npx = 3.f * (float)H * (float)W; // SSIM and L1 are means over channels and pixels
    const int c = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * kVSeg;
    float b[3][kVSeg];
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int o = 0; o < kVSeg; o++) b[m][o] = 0.f;
#pragma unroll
    for (int j = 0; j < kVSeg + 10; j++) {
        float v[3];
#pragma unroll
        for (int m = 0; m < 3; m++) v[m] = hb[m][r0 + j][c];
#pragma unroll
        for (int o = 0; o < kVSeg; o++) {
            const int t = j - o;
            if (t >= 0 && t < 11) {
#pragma unroll
                for (int m = 0; m < 3; m++) b[m][o] += win.w[t] * v[m];
            }
        }
    }
#pragma unroll
    for (int o = 0; o < kVSeg; o++) {
        const int gy = oy + r0 + o, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        const long long p = (long long)plane * H * W + (long long)gy * W + gx;
        const float xv = img[p], yv = tgt[p];
        const float dssim = (b[0][o] + 2.f * xv * b[1][o] + yv * b[2][o]) / npx;
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dL[p] = ((1.f - lambda) * sgn / npx - lambda * dssim) / (float)batch;
    }
}

__global__ void loss_finalize_kernel(const float *partial, int blocks_per_view, int batch, int H, int W, float lambda,
                                     float *loss_out)
{
    __shared__ double s_s[256], s_l[256];
    double loss = 0.0;
    for (int b = 0; b < batch; b++) {
        double as = 0.0, al = 0.0;
        for (int k = threadIdx.x; k < blocks_per_view; k += 256) {
            const long long blk = (long long)b * blocks_per_view + k;
            as += (double)partial[2 * blk];
            al += (double)partial[2 * blk + 1];
        }
        s_s[threadIdx.x] = as;
        s_l[threadIdx.x] = al;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) { s_s[threadIdx.x] += s_s[threadIdx.x + o]; s_l[threadIdx.x] += s_l[threadIdx.x + o]; }
            __syncthreads();
        }
        const double npx = 3.0 * H * W;
        loss += ((1.0 - lambda) * s_l[0] / npx + lambda * (1.0 - s_s[0] / npx)) / batch;
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss_out = (float)loss;
}

cudaError_t launch_loss(gs_workspace *ws, cudaStream_t st, const float *img, const float *tgt, int B, int H, int W,
                        float lambda, float *loss_out, float *dL)
{
    Win win;
    double g[11], sum = 0.0;
    for (int k = 0; k < 11; k++) { g[k] = exp(-((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5)); sum += g[k]; }
    for (int k = 0; k < 11; k++) win.w[k] = (float)(g[k] / sum);
    const dim3 grid((W + kLT - 1) / kLT, (H + kLT - 1) / kLT, B * 3);
    const long long stride = (long long)B * 3 * H * W;
    ssim_fwd_kernel<<<grid, 256, 0, st>>>(img, tgt, H, W, win, 0.01f * 0.01f, 0.03f * 0.03f, ws->loss_maps, stride,
                                          ws->loss_partial);
    note_launch();
    ssim_bwd_kernel<<<grid, 256, 0, st>>>(img, tgt, H, W, win, ws->loss_maps, stride, lambda, B, dL);
    note_launch();
    const int bpv = (int)(grid.x * grid.y * 3);
    loss_finalize_kernel<<<1, 256, 0, st>>>(ws->loss_partial, bpv, B, H, W, lambda, loss_out);
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

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

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
    adam_kernel<<<t.block_start[n_groups], 256, 0, st>>>(t);
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
// optimizer step advances its own counter on every replay.
__global__ void adam_coef_kernel(AdamCoefArgs a, int *d_step, float *coef)
{
    if (threadIdx.x != 0) return;
    const int t = a.step > 0 ? a.step : *d_step + 1;
    *d_step = t;
    const double c1 = 1.0 - powi((double)a.b1, t), c2 = 1.0 - powi((double)a.b2, t);
    for (int k = 0; k < 5; k++) {
        coef[k] = (float)((double)a.lr[k] / c1);
        coef[GS_MAX_ADAM_GROUPS + k] = (float)(1.0 / sqrt(c2));
    }
}

cudaError_t launch_adam_sparse(gs_workspace *ws, cudaStream_t st, const gs_gaussian_grads &param,
                               const gs_gaussian_grads &m, const gs_gaussian_grads &v, long long n,
                               const float lr[5], float beta1, float beta2, float eps, int step)
{
    AdamCoefArgs ca;
    for (int k = 0; k < 5; k++) ca.lr[k] = lr[k];
    ca.b1 = beta1; ca.b2 = beta2; ca.step = step;
    adam_coef_kernel<<<1, 32, 0, st>>>(ca, ws->d_adam_step, ws->d_adam_coef);
    note_launch();
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
