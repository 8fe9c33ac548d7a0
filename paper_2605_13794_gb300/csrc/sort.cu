// sort.cu -- device LSD radix sort of (32-bit key, value) pairs, stable, for
// the importance selection (records by w, then by camera) and the
// model-level selections (Gaussians by score).
// The passes are single-pass ("onesweep"): each block ranks its 1024, 2048
// or 4096 keys (a tuning of the workspace) in shared memory, publishes
// per-digit counts and finds its global offsets by a per-digit decoupled
// look-back, so every pass reads and writes each key once.  Item counts stay
// on the device, so nothing here needs a host synchronisation.
#include "gs_internal.cuh"

namespace gs {

constexpr uint32_t kRxAgg = 1u << 30;
constexpr uint32_t kRxInc = 2u << 30;
constexpr uint32_t kRxVal = (1u << 30) - 1;

__device__ __forceinline__ unsigned long long clamp_count(const unsigned long long *count, unsigned long long cap)
{
    unsigned long long c = *count;
    return c < cap ? c : cap;
}

// Histograms of all passes in one read of the keys.
__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t *keys, const unsigned long long *count,
                                                         unsigned long long cap, int passes, uint32_t *hist)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ uint32_t h[4][256];
    for (int k = threadIdx.x; k < 4 * 256; k += 256) (&h[0][0])[k] = 0;
    __syncthreads();
    const unsigned long long n = clamp_count(count, cap);
    for (unsigned long long i = (unsigned long long)blockIdx.x * 256 + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * 256) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; p++) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < passes * 256; k += 256) {
        const uint32_t v = (&h[0][0])[k];
        if (v) atomicAdd(&hist[k], v);
    }
}

// One stable LSD pass over digit (key >> shift) & 255; each block ranks
// 256 * ITEMS keys.  The global offset of each digit is the exclusive scan of
// the pass's histogram, which every block computes for itself (256 values).
template <int ITEMS, bool VALS_IDENTITY, bool WRITE_KEYS>
__global__ void __launch_bounds__(kSortThreads) radix_pass_kernel(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const unsigned long long *count, unsigned long long cap, int shift,
    const uint32_t *__restrict__ hist, uint32_t *status /* ticket at [0], then [blocks][256] */,
    DevCounters *ctr, unsigned long long spin_limit)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const uint32_t hd = hist[threadIdx.x]; // this thread's digit: count over all keys
    constexpr int kTileKeys = kSortThreads * ITEMS;
    __shared__ uint32_t s_keys[kTileKeys];
    __shared__ uint32_t s_vals[kTileKeys];
    __shared__ uint32_t s_wcnt[8][256];
    __shared__ uint32_t s_blk[256];
    __shared__ uint32_t s_glob[256];
    __shared__ uint32_t s_warp[8];
    __shared__ unsigned s_bid;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bid = atomicAdd(&status[0], 1u);
    for (int k = tid; k < 8 * 256; k += kSortThreads) (&s_wcnt[0][0])[k] = 0;
    __syncthreads();
    const unsigned bid = s_bid;
    const unsigned long long n = clamp_count(count, cap);
    const unsigned long long base = (unsigned long long)bid * kTileKeys;
    if (base >= n) return;
    uint32_t *st = status + 1;

    // load in warp-striped order: item j of lane l is base + warp*512 + j*32 + l
    uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const unsigned long long idx = base + (unsigned long long)warp * (32 * ITEMS) + j * 32 + lane;
        const bool valid = idx < n;
        key[j] = valid ? keys_in[idx] : 0u;
        val[j] = valid ? (VALS_IDENTITY ? (uint32_t)idx : vals_in[idx]) : 0u;
        const uint32_t d = (key[j] >> shift) & 255u;
        // peers with the same digit (and valid) via 8 ballots
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const unsigned bits = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bits : ~bits;
        }
        const uint32_t before = s_wcnt[warp][d];
        __syncwarp();
        rank[j] = before + __popc(peers & lt_mask);
        if (valid && (peers & lt_mask) == 0) s_wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        if (!valid) key[j] = 0xffffffffu, rank[j] = 0xffffffffu; // marks invalid
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, block total
    const int d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = run;
        run += c;
    }
    const uint32_t dtotal = run;
    // block-local exclusive scan over digits, and the global start of each digit
    uint32_t tot;
    const uint32_t dexcl = block_exclusive_scan_256<uint32_t>(dtotal, s_warp, tot);
    s_blk[d] = dexcl;
    const uint32_t boff = block_exclusive_scan_256<uint32_t>(hd, s_warp, tot);
    // publish aggregate, then per-digit look-back (one thread per digit)
    volatile uint32_t *vst = st;
    if (bid == 0) {
        vst[d] = kRxInc | dtotal;
        s_glob[d] = boff;
    } else {
        vst[(unsigned long long)bid * 256 + d] = kRxAgg | dtotal;
        // walk back 8 predecessors at a time (independent loads in flight):
        // add aggregates until an inclusive prefix; wait where one is missing
        constexpr int kWin = 8;
        uint32_t excl = 0;
        long long pred = (long long)bid - 1;
        unsigned long long spins = 0;
        while (pred >= 0) {
            uint32_t sv[kWin];
#pragma unroll
            for (int q = 0; q < kWin; q++)
                sv[q] = pred - q >= 0 ? (uint32_t)vst[(unsigned long long)(pred - q) * 256 + d] : (uint32_t)kRxInc; // block -1: prefix 0
            int q = 0;
            bool done = false;
            for (; q < kWin; q++) {
                const uint32_t sq = sv[q];
                if ((sq >> 30) == 0) break; // not published yet
                excl += sq & kRxVal;
                if ((sq >> 30) == 2) { done = true; break; }
            }
            if (done) break;
            pred -= q;
            if (q == kWin) continue;
            if (++spins > spin_limit) {
                set_error(ctr, GS_ERR_TIMEOUT, kSiteRadix);
                break;
            }
            __nanosleep(40);
        }
        vst[(unsigned long long)bid * 256 + d] = kRxInc | (excl + dtotal);
        s_glob[d] = boff + excl;
    }
    __syncthreads();
    // scatter into shared memory in block-sorted order
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        if (rank[j] == 0xffffffffu) continue;
        const uint32_t dd = (key[j] >> shift) & 255u;
        const uint32_t pos = s_blk[dd] + s_wcnt[warp][dd] + rank[j];
        s_keys[pos] = key[j];
        s_vals[pos] = val[j];
    }
    __syncthreads();
    const unsigned long long rem = n - base;
    const int nvalid = rem < (unsigned long long)kTileKeys ? (int)rem : kTileKeys;
    for (int i = tid; i < nvalid; i += kSortThreads) {
        const uint32_t k = s_keys[i];
        const uint32_t dd = (k >> shift) & 255u;
        const unsigned long long out = (unsigned long long)s_glob[dd] + (uint32_t)(i - (int)s_blk[dd]);
        // always below n for a complete look-back; after one gave up (or a pass that
        // follows it) the offsets are wrong but never beyond the output
        if (out >= n) continue;
        if (WRITE_KEYS) keys_out[out] = k;
        vals_out[out] = s_vals[i];
    }
}

// The passes of one sort.  status: with `region` > 0, pass p's look-back
// state is status + p * region, all of it zeroed by the caller; with region 0
// every pass zeroes and uses status itself.
template <int ITEMS>
static cudaError_t radix_passes(cudaStream_t st, uint32_t *keys[2], uint32_t *vals[2], const unsigned long long *count,
                                unsigned long long cap, int passes, bool vals_identity, uint32_t *status,
                                size_t region, const uint32_t *hist, DevCounters *ctr, int &out_buf,
                                unsigned long long spin_limit)
{
    const unsigned long long blocks = (cap + kSortThreads * ITEMS - 1) / (kSortThreads * ITEMS);
    cudaError_t e;
    int src = 0;
    for (int p = 0; p < passes; p++) {
        const int dst = src ^ 1;
        uint32_t *stp = status + (size_t)p * region;
        if (region == 0 && (e = cudaMemsetAsync(stp, 0, (blocks * 256 + 1) * sizeof(uint32_t), st)) != cudaSuccess)
            return e;
        if (vals_identity && p == 0)
            launch_pdl(radix_pass_kernel<ITEMS, true, true>, (unsigned)blocks, kSortThreads, 0, st,
                keys[src], vals[src], keys[dst], vals[dst], count, cap, 8 * p, hist + 256 * p, stp, ctr, spin_limit);
        else
            launch_pdl(radix_pass_kernel<ITEMS, false, true>, (unsigned)blocks, kSortThreads, 0, st,
                keys[src], vals[src], keys[dst], vals[dst], count, cap, 8 * p, hist + 256 * p, stp, ctr, spin_limit);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        src = dst;
    }
    out_buf = src;
    return cudaSuccess;
}

// LSD radix sort of (key, value) pairs, `bits` significant key bits, count on
// the device (clamped to cap).  keys[0]/vals[0] hold the input; the sorted
// result lands in keys[out_buf]/vals[out_buf].  With vals_identity the input
// values are the item indices and vals[0] is not read.  Blocks rank
// ws->sort_items * 256 keys (the workspace's tuning: 1024, 2048 or 4096, or
// chosen by the size of the sort).  One memset clears the histograms and the
// look-back state of every pass (ws->rx_status: [4][256] histogram words,
// then one region per pass), so the sort's kernels follow one another with
// programmatic dependent launch.
// Keys per block of a sort of up to cap keys: the workspace's tuning, or by
// size (0): small sorts take small blocks so that enough SMs work on them,
// large ones large blocks, whose look-back chains are shorter (measured on the
// city view: 94k depth keys 34.5 us in 1024-key blocks against 56.6 us in
// 4096-key blocks; 1.2M tile keys 77 us in 2048-key blocks against 70 us in
// 4096-key blocks, emission included).
static int radix_items(const gs_workspace *ws, unsigned long long cap)
{
    int items = ws->sort_items;
    if (items == 0) items = cap <= (1ull << 18) ? 4 : (cap <= (1ull << 20) ? 8 : 16);
    if (items != 4 && items != 8) items = kSortItems;
    return items;
}

// Words of ws->rx_status a sort of up to cap keys of `bits` bits uses: the
// histograms, then one look-back region per pass.
static size_t radix_words(const gs_workspace *ws, unsigned long long cap, int bits, size_t &region)
{
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    const int items = radix_items(ws, cap);
    const unsigned long long blocks = (cap + kSortThreads * items - 1) / (kSortThreads * items);
    region = (size_t)blocks * 256 + 1;
    return kRxHistWords + passes * region;
}

cudaError_t launch_radix_sort(gs_workspace *ws, cudaStream_t st, uint32_t *keys[2], uint32_t *vals[2],
                              const unsigned long long *count, unsigned long long cap, int bits, bool vals_identity,
                              int &out_buf, unsigned long long spin_limit)
{
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    cudaError_t e;
    out_buf = 0;
    if (cap == 0) return cudaSuccess;
    const int items = radix_items(ws, cap);
    size_t region;
    const size_t words = radix_words(ws, cap, bits, region);
    uint32_t *hist = ws->rx_status, *status = ws->rx_status + kRxHistWords;
    if (words > ws->rx_words) return cudaErrorInvalidValue; // sized for this cap
    if ((e = cudaMemsetAsync(hist, 0, words * sizeof(uint32_t), st)) != cudaSuccess) return e;
    unsigned hblocks = (unsigned)((cap + 255) / 256);
    if (hblocks > 1216) hblocks = 1216;
    launch_pdl(radix_hist_kernel, hblocks, 256, 0, st, keys[0], count, cap, passes, hist);
    note_launch();
    if (items == 4)
        return radix_passes<4>(st, keys, vals, count, cap, passes, vals_identity, status, region, hist, ws->ctr,
                               out_buf, spin_limit);
    if (items == 8)
        return radix_passes<8>(st, keys, vals, count, cap, passes, vals_identity, status, region, hist, ws->ctr,
                               out_buf, spin_limit);
    return radix_passes<kSortItems>(st, keys, vals, count, cap, passes, vals_identity, status, region, hist, ws->ctr,
                                    out_buf, spin_limit);
}

// The same LSD sort with every scratch buffer passed in (no workspace) and
// 4096-key blocks: status [ceil(cap / 4096) * 256 + 1] uint32 (zeroed before
// each pass), hist [4 * 256] uint32, ctr receives a timeout error.  Used by
// the entry point without allocation.
cudaError_t launch_radix_sort_scratch(cudaStream_t st, uint32_t *keys[2], uint32_t *vals[2],
                                      const unsigned long long *count, unsigned long long cap, int bits,
                                      bool vals_identity, uint32_t *status, uint32_t *hist, DevCounters *ctr,
                                      int &out_buf)
{
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    cudaError_t e;
    out_buf = 0;
    if (cap == 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(hist, 0, 4 * 256 * sizeof(uint32_t), st)) != cudaSuccess) return e;
    unsigned hblocks = (unsigned)((cap + 255) / 256);
    if (hblocks > 1216) hblocks = 1216;
    launch_pdl(radix_hist_kernel, hblocks, 256, 0, st, keys[0], count, cap, passes, hist);
    note_launch();
    return radix_passes<kSortItems>(st, keys, vals, count, cap, passes, vals_identity, status, 0, hist, ctr, out_buf,
                                    kSpinLimit);
}

} // namespace gs
