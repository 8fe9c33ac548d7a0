// select.cu -- importance-pass outputs (Sec. 3.2, Fig. 2; Sec. 3.3, Eq. 3).
//
// From the per-(record, tile) slots of the colourless sweep:
//   w_{i,v}, a_{i,v}             per record, summed over its tiles in order;
//   s_i += w/(a + eps) (a > 0), c^rad_i += 1   per Gaussian over its records;
//   c^vis_{i,v}: the smallest set of largest w carrying vis_mass of the view's
//   total w, ties toward the lower Gaussian index; Cull = 1 - c^vis.
// The selection sorts each view's records by w (descending, stable), takes an
// inclusive scan of w in 64-bit fixed point (32 fractional bits: exact, so
// the same in any association), and marks every entry whose exclusive prefix
// is still below vis_mass * total.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

cudaError_t launch_importance_raster(gs_workspace *ws, cudaStream_t st);

// w and a of each record.  A warp takes 8 consecutive records (whose slots
// are contiguous: a record's first instance follows record order); records of at most 32 tiles are summed by
// groups of 8 lanes, 4 records at a time (lanes strided over the record's
// slots, then a fixed shuffle tree over the group), larger ones by the whole
// warp each (lanes strided by 32, a fixed tree over 32 lanes).  Which way a
// record is summed depends only on its tile count: the same sums on every run.
constexpr int kImpLanes = 8, kImpRecs = 8;
constexpr uint32_t kImpBig = 4 * kImpLanes;
__global__ void __launch_bounds__(256) imp_reduce_kernel(const uint32_t *inst_off,
                                                         const uint32_t *tt, const float2 *slots, float *imp_w,
                                                         uint32_t *imp_a, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    constexpr int kGroups = 32 / kImpLanes;
    constexpr uint32_t kSkip = 0xffffffffu;
    const unsigned long long nrec = ctr->n_records, ninst = ctr->n_instances;
    const int lane = threadIdx.x & 31, sub = lane & (kImpLanes - 1), grp = lane / kImpLanes;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * 8;
    for (unsigned long long k0 = ((unsigned long long)blockIdx.x * 8 + (threadIdx.x >> 5)) * kImpRecs; k0 < nrec;
         k0 += nwarps * kImpRecs) {
        uint32_t r = 0, cnt = kSkip;
        unsigned long long off = 0;
        if (lane < kImpRecs && k0 + lane < nrec) {
            r = (uint32_t)(k0 + lane);
            off = inst_off[r];
            cnt = tt[r];
            if (off + cnt > ninst) cnt = 0; // capacity error already recorded: zero sums
        }
        const unsigned big = __ballot_sync(0xffffffffu, cnt != kSkip && cnt > kImpBig);
#pragma unroll
        for (int round = 0; round < kImpRecs / kGroups; round++) {
            const int src = round * kGroups + grp;
            const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
            const uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
            const unsigned long long o = __shfl_sync(0xffffffffu, off, src);
            const bool live = c <= kImpBig;
            float w = 0.f;
            uint32_t aa = 0;
            if (live)
                #pragma unroll 4 // the loads of four iterations in flight (the adds keep their order)
                for (uint32_t t = sub; t < c; t += kImpLanes) {
                    const float2 sl = slots[o + t];
                    w += sl.x;
                    aa += __float_as_uint(sl.y);
                }
#pragma unroll
            for (int x = kImpLanes / 2; x > 0; x >>= 1) {
                w += __shfl_xor_sync(0xffffffffu, w, x);
                aa += __shfl_xor_sync(0xffffffffu, aa, x);
            }
            if (live && sub == 0) {
                imp_w[rr] = w;
                imp_a[rr] = aa;
            }
        }
        for (unsigned rest = big; rest; rest &= rest - 1) {
            const int src = __ffs(rest) - 1;
            const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
            const uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
            const unsigned long long o = __shfl_sync(0xffffffffu, off, src);
            float w = 0.f;
            uint32_t aa = 0;
            #pragma unroll 4 // the loads of four iterations in flight (the adds keep their order)
            for (uint32_t t = lane; t < c; t += 32) {
                const float2 sl = slots[o + t];
                w += sl.x;
                aa += __float_as_uint(sl.y);
            }
            for (int x = 16; x > 0; x >>= 1) w += __shfl_xor_sync(0xffffffffu, w, x);
            aa = __reduce_add_sync(0xffffffffu, aa);
            if (lane == 0) {
                imp_w[rr] = w;
                imp_a[rr] = aa;
            }
        }
    }
}

struct ImpGaussArgs {
    const uint32_t *rec_g;
    const uint16_t *rec_cam;
    const float *imp_w;
    const uint32_t *imp_a;
    float *w_out;
    uint32_t *a_out;
    float *s_accum;
    uint32_t *crad;
    long long n;
    float eps;
    const DevCounters *ctr;
};

// One thread per Gaussian with records (the thread of its first record; a
// Gaussian's records are contiguous).
__global__ void __launch_bounds__(256) imp_gauss_kernel(ImpGaussArgs a)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const unsigned long long rh = (unsigned long long)blockIdx.x * 256 + threadIdx.x;
    const unsigned long long nrec = a.ctr->n_records;
    if (rh >= nrec || (rh > 0 && a.rec_g[rh - 1] == a.rec_g[rh])) return;
    const long long i = a.rec_g[rh];
    float s = 0.f;
    uint32_t nr = 0;
    for (unsigned long long r = rh; r < nrec && a.rec_g[r] == (uint32_t)i; r++, nr++) {
        const float w = a.imp_w[r];
        const uint32_t cnt = a.imp_a[r];
        if (cnt > 0) s += w / ((float)cnt + a.eps);
        const int c = a.rec_cam[r];
        if (a.w_out) a.w_out[(long long)c * a.n + i] = w;
        if (a.a_out) a.a_out[(long long)c * a.n + i] = cnt;
    }
    if (a.s_accum) a.s_accum[i] += s;
    if (a.crad) a.crad[i] += nr;
}

// keys = bit-complement of the FP32 bits of w (w >= 0), so ascending keys are
// descending w and w = 0 sorts last.
__global__ void sel_keys_kernel(const float *imp_w, uint32_t *keys, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const unsigned long long r = (unsigned long long)blockIdx.x * 256 + threadIdx.x;
    if (r < ctr->n_records) keys[r] = ~__float_as_uint(imp_w[r]);
}

__global__ void sel_camkeys_kernel(const uint32_t *vals, const uint16_t *rec_cam, uint32_t *keys,
                                   const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    if (ctr->error != 0) return; // a sort that gave up: its order is not a permutation
    const unsigned long long k = (unsigned long long)blockIdx.x * 256 + threadIdx.x;
    if (k < ctr->n_records) keys[k] = rec_cam[vals[k]];
}


// The mass of a record in the prefix sums: FP64, or 64-bit fixed point with 32
// fractional bits (exact and associative; a view's total alpha weight is at
// most its pixel count, so 64 bits hold every prefix of up to 64 views).
template <typename M> __device__ __forceinline__ M mass_of(float w);
template <> __device__ __forceinline__ double mass_of<double>(float w) { return (double)w; }
template <> __device__ __forceinline__ unsigned long long mass_of<unsigned long long>(float w)
{
    return __double2ull_rn((double)w * 4294967296.0);
}

// Per-block sums of w in sorted order (fixed association).
template <typename M>
__global__ void __launch_bounds__(256) sel_block_sum_kernel(const uint32_t *vals, const float *imp_w, M *bsum,
                                                            const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ M s[256];
    if (block_error(ctr)) return; // a sort that gave up: its order is not a permutation
    const unsigned long long n = ctr->n_records;
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile;
    M acc = 0;
    if (base < n) {
        for (int j = 0; j < kScanTile / 256; j++) {
            const unsigned long long k = base + (unsigned long long)threadIdx.x * (kScanTile / 256) + j;
            if (k < n) acc += mass_of<M>(imp_w[vals[k]]);
        }
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

// Inclusive scan of x over the block (blockDim.x a multiple of 32, <= 1024):
// shuffles within the warps, then over the warp totals.  Returns the
// block-inclusive value; s_w holds 32 scratch entries.
template <typename M> __device__ __forceinline__ M block_inclusive_scan(M x, M *s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const M y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        M t = lane < nw ? s_w[lane] : M(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const M y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < nw) s_w[lane] = t - s_w[lane]; // exclusive over the warps
    }
    __syncthreads();
    return s_w[warp] + x;
}

// Exclusive scan of the block sums in one block of 1024 threads: each thread
// a contiguous chunk, then a shuffle scan of the chunk sums (a fixed
// association).
constexpr int kBScanThreads = 1024;
template <typename M> __global__ void __launch_bounds__(kBScanThreads) sel_block_scan_kernel(M *bsum, int nblocks)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ M s_w[32];
    const int per = (nblocks + kBScanThreads - 1) / kBScanThreads;
    const int b0 = threadIdx.x * per;
    M acc = 0;
    for (int b = b0; b < b0 + per && b < nblocks; b++) acc += bsum[b];
    M run = block_inclusive_scan<M>(acc, s_w) - acc;
    for (int b = b0; b < b0 + per && b < nblocks; b++) { const M v = bsum[b]; bsum[b] = run; run += v; }
}

// Inclusive prefix of w in sorted order: cum[k].
template <typename M>
__global__ void __launch_bounds__(256) sel_scan_kernel(const uint32_t *vals, const float *imp_w, const M *boff,
                                                       M *cum, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ M s_w[32];
    if (block_error(ctr)) return; // a sort that gave up: its order is not a permutation
    const unsigned long long n = ctr->n_records;
    const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile;
    if (base >= n) return;
    constexpr int per = kScanTile / 256;
    M v[per];
    M acc = 0;
    for (int j = 0; j < per; j++) {
        const unsigned long long k = base + (unsigned long long)threadIdx.x * per + j;
        v[j] = k < n ? mass_of<M>(imp_w[vals[k]]) : M(0);
        acc += v[j];
    }
    M run = boff[blockIdx.x] + block_inclusive_scan<M>(acc, s_w) - acc;
    for (int j = 0; j < per; j++) {
        const unsigned long long k = base + (unsigned long long)threadIdx.x * per + j;
        run += v[j];
        if (k < n) cum[k] = run;
    }
}

// Camera segments of the cam-major sorted order.
__global__ void sel_segments_kernel(const uint32_t *vals, const uint16_t *rec_cam, uint2 *seg, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    if (ctr->error != 0) return; // a sort that gave up: its order is not a permutation
    const unsigned long long n = ctr->n_records;
    for (unsigned long long k = (unsigned long long)blockIdx.x * 256 + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * 256) {
        const int c = rec_cam[vals[k]];
        if (k == 0 || rec_cam[vals[k - 1]] != c) seg[c].x = (uint32_t)k;
        if (k == n - 1 || rec_cam[vals[k + 1]] != c) seg[c].y = (uint32_t)(k + 1);
    }
}

// The fixed-association FP64 prefix of w in sorted order with explicit
// buffers (no workspace): bsum [ceil(cap / 4096)] doubles, cum [cap] doubles;
// the item count is ctr->n_records.
cudaError_t launch_mass_scan(cudaStream_t st, const uint32_t *sorted, const float *w, double *bsum, double *cum,
                             const DevCounters *ctr, unsigned long long cap)
{
    const unsigned sblocks = (unsigned)((cap + kScanTile - 1) / kScanTile);
    if (sblocks == 0) return cudaSuccess;
    launch_pdl(sel_block_sum_kernel<double>, sblocks, 256, 0, st, sorted, w, bsum, ctr);
    note_launch();
    launch_pdl(sel_block_scan_kernel<double>, 1, kBScanThreads, 0, st, bsum, (int)sblocks);
    note_launch();
    launch_pdl(sel_scan_kernel<double>, sblocks, 256, 0, st, sorted, w, bsum, cum, ctr);
    note_launch();
    return cudaGetLastError();
}

// The same prefix in 64-bit fixed point (32 fractional bits), the arithmetic
// of gs_importance's selection: exact, so identical in any association.
cudaError_t launch_mass_scan_fixed(cudaStream_t st, const uint32_t *sorted, const float *w, unsigned long long *bsum,
                                   unsigned long long *cum, const DevCounters *ctr, unsigned long long cap)
{
    const unsigned sblocks = (unsigned)((cap + kScanTile - 1) / kScanTile);
    if (sblocks == 0) return cudaSuccess;
    launch_pdl(sel_block_sum_kernel<unsigned long long>, sblocks, 256, 0, st, sorted, w, bsum, ctr);
    note_launch();
    launch_pdl(sel_block_scan_kernel<unsigned long long>, 1, kBScanThreads, 0, st, bsum, (int)sblocks);
    note_launch();
    launch_pdl(sel_scan_kernel<unsigned long long>, sblocks, 256, 0, st, sorted, w, bsum, cum, ctr);
    note_launch();
    return cudaGetLastError();
}

struct SelApplyArgs {
    const uint32_t *vals;
    const uint32_t *rec_g;
    const uint16_t *rec_cam;
    const float *imp_w;
    const unsigned long long *cum; // fixed-point inclusive prefix of w (mass_of)
    const uint2 *seg;
    uint32_t *cull_out;
    uint32_t *cvis;
    long long words;
    float vis_mass;
    const DevCounters *ctr;
};

__global__ void sel_apply_kernel(SelApplyArgs a)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    if (a.ctr->error != 0) return; // a sort that gave up: every Gaussian stays culled
    const unsigned long long n = a.ctr->n_records;
    for (unsigned long long k = (unsigned long long)blockIdx.x * 256 + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * 256) {
        const uint32_t r = a.vals[k];
        const float w = a.imp_w[r];
        if (!(w > 0.f)) continue;
        const int c = a.rec_cam[r];
        const uint2 sg = a.seg[c];
        const unsigned long long before = sg.x > 0 ? a.cum[sg.x - 1] : 0ull;
        const unsigned long long total = a.cum[sg.y - 1] - before;
        const unsigned long long excl = (k > 0 ? a.cum[k - 1] : 0ull) - before;
        if ((double)excl < (double)a.vis_mass * (double)total) {
            const uint32_t g = a.rec_g[r];
            if (a.cull_out) atomicAnd(&a.cull_out[(long long)c * a.words + (g >> 5)], ~(1u << (g & 31)));
            if (a.cvis) atomicAdd(&a.cvis[g], 1u);
        }
    }
}

// Cull words start at "culled" for every valid bit.
__global__ void cull_init_kernel(uint32_t *cull, long long words, long long n, int n_cams)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long total = words * n_cams;
    for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < total; k += (long long)gridDim.x * 256) {
        const long long wi = k % words;
        const long long bits = n - wi * 32;
        cull[k] = bits >= 32 ? 0xffffffffu : ((1u << bits) - 1u);
    }
}

// w and a of every record from the importance slots of the current binning
cudaError_t launch_importance_reduce(gs_workspace *ws, cudaStream_t st)
{
    const unsigned long long rcap = (unsigned long long)ws->cap.max_records;
    const unsigned blocks = (unsigned)std::max<unsigned long long>(
        1, std::min<unsigned long long>((rcap + 8 * kImpRecs - 1) / (8 * kImpRecs), 16ull * ws->sm_count));
    launch_pdl(imp_reduce_kernel, blocks, 256, 0, st, ws->inst_off, ws->tt,
                                              ws->imp_slots, ws->imp_w, ws->imp_a,
                                              ws->ctr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_importance(gs_workspace *ws, cudaStream_t st, float *w, uint32_t *a, float *s_accum,
                              uint32_t *crad, uint32_t *cvis, uint32_t *cull_out)
{
    cudaError_t e;
    const long long n = ws->g.n;
    const int ncam = ws->cams.n;
    const unsigned long long rcap = (unsigned long long)ws->cap.max_records;
    const unsigned rblocks = (unsigned)((rcap + 255) / 256);
    // w and a per record: from the raster here, unless gs_render_fwd_importance took them already
    if (!ws->imp_ready) {
        if ((e = launch_importance_raster(ws, st)) != cudaSuccess) return e;
        if ((e = launch_importance_reduce(ws, st)) != cudaSuccess) return e;
    }
    if (w && (e = cudaMemsetAsync(w, 0, (size_t)ncam * n * sizeof(float), st)) != cudaSuccess) return e;
    if (a && (e = cudaMemsetAsync(a, 0, (size_t)ncam * n * sizeof(uint32_t), st)) != cudaSuccess) return e;
    if (n > 0) {
        ImpGaussArgs ga{ws->rec_g, ws->rec_cam, ws->imp_w, ws->imp_a, w, a, s_accum, crad, n, ws->rc.eps_score,
                        ws->ctr};
        launch_pdl(imp_gauss_kernel, rblocks, 256, 0, st, ga);
        note_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!cull_out && !cvis) return cudaSuccess;
    const long long words = (n + 31) / 32;
    if (cull_out && words > 0) {
        launch_pdl(cull_init_kernel, 1216, 256, 0, st, cull_out, words, n, ncam);
        note_launch();
    }
    // sort records by w descending (stable), then by camera (stable); own
    // buffers, so the depth order stays valid for a later backward
    uint32_t *sk[2] = {ws->selk[0], ws->selk[1]};
    uint32_t *sv[2] = {ws->selv[0], ws->selv[1]};
    launch_pdl(sel_keys_kernel, rblocks, 256, 0, st, ws->imp_w, sk[0], ws->ctr);
    note_launch();
    int ob = 0;
    const unsigned long long *cnt = &ws->ctr->n_records;
    if ((e = launch_radix_sort(ws, st, sk, sv, cnt, rcap, 32, true, ob, ws->sel_spin_limit)) != cudaSuccess)
        return e;
    uint32_t *sorted = sv[ob];
    if (ncam > 1) {
        uint32_t *k2[2] = {sk[ob ^ 1], sk[ob]};
        uint32_t *v2[2] = {sv[ob], sv[ob ^ 1]};
        launch_pdl(sel_camkeys_kernel, rblocks, 256, 0, st, v2[0], ws->rec_cam, k2[0], ws->ctr);
        note_launch();
        int ob2 = 0;
        if ((e = launch_radix_sort(ws, st, k2, v2, cnt, rcap, 8, false, ob2, ws->sel_spin_limit)) !=
            cudaSuccess)
            return e;
        sorted = v2[ob2];
    }
    const unsigned sblocks = (unsigned)((rcap + kScanTile - 1) / kScanTile);
    // fixed-point masses: exact sums in any association
    unsigned long long *bsum = ws->sel_bsum;
    unsigned long long *cum = reinterpret_cast<unsigned long long *>(ws->sel_cum);
    launch_pdl(sel_block_sum_kernel<unsigned long long>, sblocks, 256, 0, st, sorted, ws->imp_w, bsum, ws->ctr);
    note_launch();
    launch_pdl(sel_block_scan_kernel<unsigned long long>, 1, kBScanThreads, 0, st, bsum, (int)sblocks);
    note_launch();
    launch_pdl(sel_scan_kernel<unsigned long long>, sblocks, 256, 0, st, sorted, ws->imp_w, bsum, cum, ws->ctr);
    note_launch();
    uint2 *seg = reinterpret_cast<uint2 *>(ws->rx_hist); // 64 uint2 fit in the histogram scratch
    if ((e = cudaMemsetAsync(seg, 0, GS_MAX_CAMERAS * sizeof(uint2), st)) != cudaSuccess) return e;
    launch_pdl(sel_segments_kernel, 1216, 256, 0, st, sorted, ws->rec_cam, seg, ws->ctr);
    note_launch();
    SelApplyArgs sa{sorted, ws->rec_g, ws->rec_cam, ws->imp_w, cum, seg, cull_out, cvis, words,
                    ws->rc.vis_mass, ws->ctr};
    launch_pdl(sel_apply_kernel, 1216, 256, 0, st, sa);
    note_launch();
    return cudaGetLastError();
}

} // namespace gs
