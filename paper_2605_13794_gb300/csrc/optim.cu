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

// grid: (tiles_x, tiles_y, batch * 3)
__global__ void __launch_bounds__(256) ssim_fwd_kernel(const float *img, const float *tgt, int H, int W, Win win,
                                                       float C1, float C2, float *F /*[3][B*3][H][W]*/,
                                                       long long plane_stride_maps, float *partial)
{
    __shared__ float sx[kLTH][kLTH], sy[kLTH][kLTH];
    __shared__ float hb[5][kLTH][kLT];
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
    for (int k = threadIdx.x; k < kLTH * kLT; k += 256) {
        const int r = k / kLT, c = k % kLT;
        float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
#pragma unroll
        for (int t = 0; t < 11; t++) {
            const float xv = sx[r][c + t], yv = sy[r][c + t], wt = win.w[t];
            a0 += wt * xv; a1 += wt * yv; a2 += wt * xv * xv; a3 += wt * yv * yv; a4 += wt * xv * yv;
        }
        hb[0][r][c] = a0; hb[1][r][c] = a1; hb[2][r][c] = a2; hb[3][r][c] = a3; hb[4][r][c] = a4;
    }
    __syncthreads();
    float ssum = 0.f, l1sum = 0.f;
    for (int k = threadIdx.x; k < kLT * kLT; k += 256) {
        const int r = k / kLT, c = k % kLT;
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
#pragma unroll
        for (int t = 0; t < 11; t++) {
            const float wt = win.w[t];
            mx += wt * hb[0][r + t][c]; my += wt * hb[1][r + t][c];
            exx += wt * hb[2][r + t][c]; eyy += wt * hb[3][r + t][c]; exy += wt * hb[4][r + t][c];
        }
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
    __shared__ float sf[3][kLTH][kLTH];
    __shared__ float hb[3][kLTH][kLT];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    for (int k = threadIdx.x; k < kLTH * kLTH; k += 256) {
        const int r = k / kLTH, c = k % kLTH;
        for (int m = 0; m < 3; m++)
            sf[m][r][c] = ld_zero(F + m * plane_stride_maps + (long long)plane * H * W, H, W, oy + r - kHalo,
                                  ox + c - kHalo);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kLTH * kLT; k += 256) {
        const int r = k / kLT, c = k % kLT;
        float a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int t = 0; t < 11; t++) {
            const float wt = win.w[t];
            a0 += wt * sf[0][r][c + t]; a1 += wt * sf[1][r][c + t]; a2 += wt * sf[2][r][c + t];
        }
        hb[0][r][c] = a0; hb[1][r][c] = a1; hb[2][r][c] = a2;
    }
    __syncthreads();
    const float npx = 3.f * (float)H * (float)W; // SSIM and L1 are means over channels and pixels
    for (int k = threadIdx.x; k < kLT * kLT; k += 256) {
        const int r = k / kLT, c = k % kLT;
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float b0 = 0, b1 = 0, b2 = 0;
#pragma unroll
        for (int t = 0; t < 11; t++) {
            const float wt = win.w[t];
            b0 += wt * hb[0][r + t][c]; b1 += wt * hb[1][r + t][c]; b2 += wt * hb[2][r + t][c];
        }
        const long long p = (long long)plane * H * W + (long long)gy * W + gx;
        const float xv = img[p], yv = tgt[p];
        const float dssim = (b0 + 2.f * xv * b1 + yv * b2) / npx;
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

struct AdamTable {
    int n;
    long long start[GS_MAX_ADAM_GROUPS + 1];
    float *p[GS_MAX_ADAM_GROUPS];
    const float *g[GS_MAX_ADAM_GROUPS];
    float *m[GS_MAX_ADAM_GROUPS];
    float *v[GS_MAX_ADAM_GROUPS];
    float lr_c[GS_MAX_ADAM_GROUPS];   // lr / (1 - beta1^t)
    float ibc2[GS_MAX_ADAM_GROUPS];   // 1 / sqrt(1 - beta2^t)
    float b1[GS_MAX_ADAM_GROUPS], b2[GS_MAX_ADAM_GROUPS], eps[GS_MAX_ADAM_GROUPS];
};

__global__ void __launch_bounds__(256) adam_kernel(AdamTable t)
{
    const long long total = t.start[t.n];
    for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < total; k += (long long)gridDim.x * 256) {
        int gi = 0;
        while (k >= t.start[gi + 1]) gi++;
        const long long i = k - t.start[gi];
        const float g = t.g[gi][i];
        const float m = t.b1[gi] * t.m[gi][i] + (1.f - t.b1[gi]) * g;
        const float v = t.b2[gi] * t.v[gi][i] + (1.f - t.b2[gi]) * g * g;
        t.m[gi][i] = m;
        t.v[gi][i] = v;
        t.p[gi][i] -= t.lr_c[gi] * m / (sqrtf(v) * t.ibc2[gi] + t.eps[gi]);
    }
}

cudaError_t launch_adam(const gs_adam_group *groups, int n_groups, int step, cudaStream_t st)
{
    AdamTable t;
    t.n = n_groups;
    t.start[0] = 0;
    for (int k = 0; k < n_groups; k++) {
        const gs_adam_group &g = groups[k];
        t.start[k + 1] = t.start[k] + g.n;
        t.p[k] = g.param; t.g[k] = g.grad; t.m[k] = g.m; t.v[k] = g.v;
        t.lr_c[k] = (float)(g.lr / (1.0 - pow((double)g.beta1, step)));
        t.ibc2[k] = (float)(1.0 / sqrt(1.0 - pow((double)g.beta2, step)));
        t.b1[k] = g.beta1; t.b2[k] = g.beta2; t.eps[k] = g.eps;
    }
    if (t.start[n_groups] == 0) return cudaSuccess;
    long long blocks = (t.start[n_groups] + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(t);
    note_launch();
    return cudaGetLastError();
}

} // namespace gs
