// model.cu -- model-level operations over all Gaussians (Sec. 3.2, Sec. 3.3):
//   * the two simplification passes on the importance score s: Pass 1 keeps k
//     Gaussians by importance-weighted sampling without replacement (as
//     exponential clocks: Gaussian i fires at e_i / s_i with e_i ~ Exp(1)
//     given, the k earliest are kept), Pass 2 keeps the smallest prefix by
//     descending s carrying a fraction `mass` of the total;
//   * order-preserving compaction of the model by a keep bit array;
//   * density control: the averaged view-space positional gradient, reweighted
//     by phi_i = c^vis_i / (c^rad_i + eps), selects Gaussians; small ones are
//     cloned, large ones split into two children (LOD: a clone keeps its
//     parent's level, a split child takes the next finer one), low-opacity
//     ones removed; the new model is written in parent order.
// Keep decisions are integer results of FP32 arithmetic done identically on
// every call (no transcendental functions), and the selections use the
// stable radix sort, so results are deterministic.
#include <math.h>
#include <string.h>

#include "gs_internal.cuh"

namespace gs {

cudaError_t launch_radix_sort_scratch(cudaStream_t st, uint32_t *keys[2], uint32_t *vals[2],
                                      const unsigned long long *count, unsigned long long cap, int bits,
                                      bool vals_identity, uint32_t *status, uint32_t *hist, DevCounters *ctr,
                                      int &out_buf);
cudaError_t launch_mass_scan(cudaStream_t st, const uint32_t *sorted, const float *w, double *bsum, double *cum,
                             const DevCounters *ctr, unsigned long long cap);

// ---- selections ------------------------------------------------------------------

// Pass 1 keys: FP32 bits of e_i / s_i (positive, so the bits order as the
// values); s_i = 0 gives +inf and fires after every Gaussian with s > 0.
__global__ void sample_keys_kernel(const float *s, const float *expo, long long n, uint32_t *keys, DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i == 0) {
        ctr->n_records = (unsigned long long)n;
        ctr->error = 0;
    }
    if (i >= n) return;
    const float si = s[i];
    keys[i] = si > 0.f ? __float_as_uint(__fdiv_rn(expo[i], si)) : 0x7f800000u;
}

// Pass 2 keys: bit-complement of the FP32 bits of s (s >= 0), so ascending
// keys are descending s and s = 0 sorts last.
__global__ void mass_keys_kernel(const float *s, long long n, uint32_t *keys, DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i == 0) {
        ctr->n_records = (unsigned long long)n;
        ctr->error = 0;
    }
    if (i < n) keys[i] = ~__float_as_uint(s[i]);
}

__global__ void clear_bits_kernel(uint32_t *bits, long long words)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long k = (long long)blockIdx.x * 256 + threadIdx.x;
    if (k < words) bits[k] = 0u;
}

__global__ void keep_first_kernel(const uint32_t *sorted, long long n, long long k, uint32_t *keep)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long j = (long long)blockIdx.x * 256 + threadIdx.x;
    if (j >= n || j >= k) return;
    const uint32_t g = sorted[j];
    atomicOr(&keep[g >> 5], 1u << (g & 31));
}

__global__ void keep_mass_kernel(const uint32_t *sorted, const float *s, const double *cum, long long n, float mass,
                                 uint32_t *keep)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long j = (long long)blockIdx.x * 256 + threadIdx.x;
    if (j >= n) return;
    const uint32_t g = sorted[j];
    if (!(s[g] > 0.f)) return;
    const double excl = j > 0 ? cum[j - 1] : 0.0;
    if (excl < (double)mass * cum[n - 1]) atomicOr(&keep[g >> 5], 1u << (g & 31));
}

// ---- compaction and density control ------------------------------------------------

struct ModelRows {
    float *p[5];        // mean [n][3], log-scale [n][3], quat [n][4], opacity [n], SH [n][48]
    float *m[5], *v[5]; // Adam moments in the same layout (NULL: not carried)
    uint8_t *lod;       // may be NULL
};

__device__ constexpr int kRowLen[5] = {3, 3, 4, 1, 48};

struct ScatterArgs {
    ModelRows src, dst;
    long long n;
    long long dst_cap;
    const uint32_t *keep; // compaction; NULL: density control
    // density control
    const float *absgrad;
    const uint32_t *denom, *cvis, *crad;
    const float *noise;   // [n][2][3]
    float tau, eps, logit_min, log_dense, log_shrink;
    int max_level;
    unsigned long long *lb_status;
    long long *n_out;     // device
    DevCounters *ctr;
};

// 0 removed, 1 kept, 2 cloned, 3 split: FP32 quantities formed as the oracle
// forms them (its decision instance mirrors these operations).
__device__ __forceinline__ int densify_kind(const ScatterArgs &a, long long i)
{
    if (a.src.p[3][i] < a.logit_min) return 0;
    const uint32_t d = a.denom[i];
    const float grad = d > 0 ? __fdiv_rn(a.absgrad[i], (float)d) : 0.f;
    const float phi = __fdiv_rn((float)a.cvis[i], __fadd_rn((float)a.crad[i], a.eps));
    if (!(__fmul_rn(grad, phi) >= a.tau)) return 1;
    const float *ls = a.src.p[1] + 3 * i;
    return fmaxf(ls[0], fmaxf(ls[1], ls[2])) <= a.log_dense ? 2 : 3;
}

__device__ __forceinline__ void copy_row(const ModelRows &s, long long i, const ModelRows &d, long long o, bool moments)
{
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const int L = kRowLen[k];
        for (int e = 0; e < L; e++) d.p[k][o * L + e] = s.p[k][i * L + e];
        if (d.m[k]) for (int e = 0; e < L; e++) d.m[k][o * L + e] = moments && s.m[k] ? s.m[k][i * L + e] : 0.f;
        if (d.v[k]) for (int e = 0; e < L; e++) d.v[k][o * L + e] = moments && s.v[k] ? s.v[k][i * L + e] : 0.f;
    }
    if (d.lod) d.lod[o] = s.lod ? s.lod[i] : 0;
}

// One split child: mu + R(q) (s * z), log-scale - log(1.6), next finer level.
__device__ __forceinline__ void write_child(const ScatterArgs &a, long long i, long long o, int c)
{
    copy_row(a.src, i, a.dst, o, false);
    const float *q = a.src.p[2] + 4 * i;
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                           {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                           {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    const float *ls = a.src.p[1] + 3 * i;
    const float *zz = a.noise + 6 * i + 3 * c;
    const float l[3] = {expf(ls[0]) * zz[0], expf(ls[1]) * zz[1], expf(ls[2]) * zz[2]};
    for (int r = 0; r < 3; r++) {
        a.dst.p[0][3 * o + r] = a.src.p[0][3 * i + r] + (R[r][0] * l[0] + R[r][1] * l[1] + R[r][2] * l[2]);
        a.dst.p[1][3 * o + r] = ls[r] - a.log_shrink;
    }
    if (a.dst.lod) {
        const int lv = (a.src.lod ? (int)a.src.lod[i] : 0) + 1;
        a.dst.lod[o] = (uint8_t)(lv < a.max_level ? lv : a.max_level);
    }
}

// Ticket-ordered blocks of 256 Gaussians: each block counts its outputs,
// finds its offset by decoupled look-back and writes them in parent order.
__global__ void __launch_bounds__(256) model_scatter_kernel(ScatterArgs a)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ unsigned s_bid;
    __shared__ unsigned long long s_warp[8];
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) s_bid = atomicAdd((unsigned *)a.lb_status, 1u);
    __syncthreads();
    const unsigned bid = s_bid;
    const long long i = (long long)bid * 256 + threadIdx.x;
    int kind = 0;
    if (i < a.n) kind = a.keep ? (int)((a.keep[i >> 5] >> (i & 31)) & 1u) : densify_kind(a, i);
    const unsigned long long cnt = kind == 0 ? 0 : (kind == 1 ? 1 : 2);
    unsigned long long total;
    const unsigned long long excl = block_exclusive_scan_256<unsigned long long>(cnt, s_warp, total);
    if (threadIdx.x < 32) {
        const unsigned long long b = lookback_exclusive(a.lb_status + 1, bid, total, a.ctr, kSiteModel);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    const unsigned long long o = s_base + excl;
    const unsigned long long nblocks = ((unsigned long long)a.n + 255) / 256;
    if (bid == nblocks - 1 && threadIdx.x == 0) *a.n_out = (long long)(s_base + total);
    if (cnt == 0) return;
    if ((long long)(o + cnt) > a.dst_cap) {
        set_error(a.ctr, GS_ERR_CAPACITY, kSiteModel);
        return;
    }
    if (kind == 1) copy_row(a.src, i, a.dst, (long long)o, true);
    else if (kind == 2) {
        copy_row(a.src, i, a.dst, (long long)o, true);
        copy_row(a.src, i, a.dst, (long long)o + 1, false);
    } else {
        write_child(a, i, (long long)o, 0);
        write_child(a, i, (long long)o + 1, 1);
    }
}

// Views in which each Gaussian has a record (+= per Gaussian; records of a
// Gaussian are contiguous).
__global__ void count_views_kernel(const uint32_t *rec_g, const float4 *rd2, const DevCounters *ctr, uint32_t *counts)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const unsigned long long r = (unsigned long long)blockIdx.x * 256 + threadIdx.x;
    const unsigned long long nrec = ctr->n_records;
    if (r >= nrec || (r > 0 && rec_g[r - 1] == rec_g[r])) return;
    uint32_t views = 0;
    for (unsigned long long e = r; e < nrec && rec_g[e] == rec_g[r]; e++)
        views += rd2[e].w != 0.f ? 0u : 1u; // records marked culled (GS_CULL_MARK) are not rendered
    counts[rec_g[r]] += views;
}

// ---- launchers ------------------------------------------------------------------------

static cudaError_t sort_model_keys(gs_workspace *ws, cudaStream_t st, long long n, int &ob)
{
    return launch_radix_sort_scratch(st, ws->mkey, ws->mval, &ws->mctr->n_records, (unsigned long long)n, 32, true,
                                     ws->mrx_status, ws->mhist, ws->mctr, ob);
}

cudaError_t launch_prune_sample(gs_workspace *ws, cudaStream_t st, const float *s, const float *expo, long long n,
                                long long k, uint32_t *keep)
{
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const long long words = (n + 31) / 32;
    launch_pdl(sample_keys_kernel, blocks, 256, 0, st, s, expo, n, ws->mkey[0], ws->mctr);
    note_launch();
    launch_pdl(clear_bits_kernel, (unsigned)((words + 255) / 256), 256, 0, st, keep, words);
    note_launch();
    int ob = 0;
    cudaError_t e = sort_model_keys(ws, st, n, ob);
    if (e != cudaSuccess) return e;
    launch_pdl(keep_first_kernel, blocks, 256, 0, st, ws->mval[ob], n, k, keep);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prune_mass(gs_workspace *ws, cudaStream_t st, const float *s, long long n, float mass,
                              uint32_t *keep)
{
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const long long words = (n + 31) / 32;
    launch_pdl(mass_keys_kernel, blocks, 256, 0, st, s, n, ws->mkey[0], ws->mctr);
    note_launch();
    launch_pdl(clear_bits_kernel, (unsigned)((words + 255) / 256), 256, 0, st, keep, words);
    note_launch();
    int ob = 0;
    cudaError_t e = sort_model_keys(ws, st, n, ob);
    if (e != cudaSuccess) return e;
    if ((e = launch_mass_scan(st, ws->mval[ob], s, ws->mbsum, ws->mcum, ws->mctr, (unsigned long long)n)) !=
        cudaSuccess)
        return e;
    launch_pdl(keep_mass_kernel, blocks, 256, 0, st, ws->mval[ob], s, ws->mcum, n, mass, keep);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_model_scatter(gs_workspace *ws, cudaStream_t st, ScatterArgs &a)
{
    const unsigned long long blocks = ((unsigned long long)a.n + 255) / 256;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws->mlb, 0, (blocks + 1) * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.n_out, 0, sizeof(long long), st)) != cudaSuccess) return e;
    a.lb_status = ws->mlb;
    a.ctr = ws->mctr;
    if (blocks == 0) return cudaSuccess;
    launch_pdl(model_scatter_kernel, (unsigned)blocks, 256, 0, st, a);
    note_launch();
    return cudaGetLastError();
}

static ModelRows rows_of(const gs_model &m)
{
    ModelRows r;
    r.p[0] = m.mean; r.p[1] = m.log_scale; r.p[2] = m.quat; r.p[3] = m.opacity_logit; r.p[4] = m.sh;
    float *mm[5] = {m.m.mean, m.m.log_scale, m.m.quat, m.m.opacity_logit, m.m.sh};
    float *vv[5] = {m.v.mean, m.v.log_scale, m.v.quat, m.v.opacity_logit, m.v.sh};
    for (int k = 0; k < 5; k++) { r.m[k] = mm[k]; r.v[k] = vv[k]; }
    r.lod = m.lod;
    return r;
}

cudaError_t launch_compact(gs_workspace *ws, cudaStream_t st, const gs_model &src, const uint32_t *keep,
                           const gs_model &dst, long long dst_cap, long long *n_out)
{
    ScatterArgs a;
    memset(&a, 0, sizeof(a));
    a.src = rows_of(src);
    a.dst = rows_of(dst);
    a.n = src.n;
    a.dst_cap = dst_cap;
    a.keep = keep;
    a.n_out = n_out;
    return launch_model_scatter(ws, st, a);
}

cudaError_t launch_densify(gs_workspace *ws, cudaStream_t st, const gs_model &src, const float *absgrad,
                           const uint32_t *denom, const uint32_t *cvis, const uint32_t *crad, const float *noise,
                           const gs_densify_params &p, const gs_model &dst, long long dst_cap, long long *n_out)
{
    ScatterArgs a;
    memset(&a, 0, sizeof(a));
    a.src = rows_of(src);
    a.dst = rows_of(dst);
    a.n = src.n;
    a.dst_cap = dst_cap;
    a.keep = nullptr;
    a.absgrad = absgrad; a.denom = denom; a.cvis = cvis; a.crad = crad; a.noise = noise;
    // thresholds in the form the kernel compares, from FP64 (the oracle rounds them the same way)
    a.tau = p.grad_threshold;
    a.eps = p.eps;
    a.logit_min = (float)log((double)p.min_opacity / (1.0 - (double)p.min_opacity));
    a.log_dense = (float)log((double)p.dense_scale);
    a.log_shrink = (float)log((double)p.split_shrink);
    a.max_level = p.n_levels - 1;
    a.n_out = n_out;
    return launch_model_scatter(ws, st, a);
}

cudaError_t launch_count_views(gs_workspace *ws, cudaStream_t st, uint32_t *counts)
{
    const unsigned blocks = (unsigned)((ws->cap.max_records + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    launch_pdl(count_views_kernel, blocks, 256, 0, st, ws->rec_g, ws->rd2, ws->ctr, counts);
    note_launch();
    return cudaGetLastError();
}

} // namespace gs
