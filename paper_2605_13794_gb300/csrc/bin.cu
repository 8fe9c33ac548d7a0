// bin.cu -- the tile lists of a binning (App. A: tile-based rasterisation of
// depth-ordered projected Gaussians), built by tile first and sorted by depth
// inside each tile.
//
// Order of the work:
//   1. count: records in record order ((Gaussian, camera) order), blocks of
//      kBinThreads; a block scans its records' tile counts and finds its
//      global offset by a decoupled look-back, so each record's first
//      instance (inst_off, the base of its gradient slots) follows record
//      order; every instance adds one to its tile's count;
//   2. tile scan: exclusive scan of the tile counts (decoupled look-back over
//      blocks of tiles) gives each tile's range and a fill cursor;
//   3. scatter: every instance takes the next position of its tile (an
//      atomic on the cursor) and writes its record and depth key there;
//   4. per-tile sort: one warp per tile sorts the tile's (depth bits,
//      record) pairs -- unique keys, so the order is the same in any
//      scatter order -- in registers (a bitonic network over shuffles, up
//      to kTileSortMax entries) or, for a longer list, in chunks merged
//      through a scratch copy in global memory.
// The final order of a tile's list is (depth bits, record): depth ties go to
// the lower record, i.e. the lower Gaussian index.  Counts stay on the
// device; nothing here synchronises with the host.
#include "gs_internal.cuh"

namespace gs {

constexpr int kBinThreads = 128;       // threads (and records) per block of the count pass
constexpr int kScatterRecs = 32;       // records per block of the scatter pass (kBinThreads threads)
constexpr int kTileScanItems = 4;      // tiles per thread of the tile scan (1024 per block)
constexpr int kTileSortMax = 512;      // entries a warp sorts in registers (16 per lane)
constexpr int kTileSortWarps = 4;      // tiles per block of the per-tile sort

struct BinArgs {
    const uint32_t *tt;
    const uint2 *rect;
    const uint16_t *rec_cam;
    const uint32_t *dkey;          // FP32 bits of each record's camera depth
    uint32_t *inst_off;            // first instance of each record (record order)
    uint32_t *tile_cnt;            // [tiles] instances per tile (zeroed before the count)
    uint32_t *tile_cur;            // [tiles] fill cursor of each tile
    uint32_t *tile_last;           // [tiles] the forward's largest n_contrib per tile: zeroed here
    uint2 *ranges;                 // [tiles] [start, end) of each tile's list
    uint32_t *skey, *sval;         // [instances] scattered depth keys and records; sval ends sorted
    uint32_t *xkey, *xval;         // [instances] scratch of the merges of long lists
    unsigned long long *lb_count;  // look-back of the count pass (ticket at word 0)
    unsigned long long *lb_tiles;  // look-back of the tile scan (ticket at word 0)
    DevCounters *ctr;
    unsigned long long max_instances;
    int total_tiles;
};

// The records of one block of the count or scatter pass in shared memory:
// inclusive prefix of their tile counts, rectangle and camera tile layout.
struct BinBlock {
    unsigned long long incl[kBinThreads];
    uint32_t rec[kBinThreads];
    uint2 rect[kBinThreads];
    int tile_base[kBinThreads], tiles_x[kBinThreads];
    unsigned long long warp[kBinThreads / 32];
};

// Instance j (block-local, below the block's total) of the block: its record
// slot in the block and its global tile id.
__device__ __forceinline__ uint32_t bin_instance(const BinBlock &s, unsigned long long j, int &slot)
{
    int lo = 0, hi = kBinThreads - 1; // first record whose inclusive prefix exceeds j
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s.incl[mid] > j) hi = mid; else lo = mid + 1;
    }
    slot = lo;
    const unsigned long long first = lo ? s.incl[lo - 1] : 0ull;
    const uint32_t local = (uint32_t)(j - first);
    int x0, y0, x1, y1;
    unpack_rect(s.rect[lo], x0, y0, x1, y1);
    const uint32_t w = (uint32_t)(x1 - x0);
    const int tx = x0 + (int)(local % w), ty = y0 + (int)(local / w);
    return (uint32_t)(s.tile_base[lo] + ty * s.tiles_x[lo] + tx);
}

// Loads the block's records k0 .. k0 + recs - 1 (those below nrec; recs <=
// kBinThreads, one per thread) and scans their tile counts; returns this
// thread's exclusive prefix and the block's total.
__device__ __forceinline__ unsigned long long bin_load(const BinArgs &a, const CamTable &ct, BinBlock &s,
                                                       unsigned long long k0, unsigned long long nrec, int recs,
                                                       unsigned long long &c, unsigned long long &total)
{
    const unsigned long long k = k0 + threadIdx.x;
    c = 0;
    if ((int)threadIdx.x < recs && k < nrec) {
        const uint32_t r = (uint32_t)k;
        c = a.tt[r];
        const int cam = a.rec_cam[r];
        s.rect[threadIdx.x] = a.rect[r];
        s.tile_base[threadIdx.x] = ct.c[cam].tile_base;
        s.tiles_x[threadIdx.x] = ct.c[cam].tiles_x;
    }
    s.rec[threadIdx.x] = (uint32_t)k;
    const unsigned long long excl = block_exclusive_scan<kBinThreads / 32, unsigned long long>(c, s.warp, total);
    s.incl[threadIdx.x] = excl + c;
    __syncthreads();
    return excl;
}

// 1. Count: each record's first instance (record order) and every tile's count.
__global__ void __launch_bounds__(kBinThreads) bin_count_kernel(BinArgs a, const CamTable *__restrict__ ctp)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ BinBlock s;
    __shared__ unsigned s_bid;
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) s_bid = atomicAdd((unsigned *)a.lb_count, 1u); // blocks in ticket order
    __syncthreads();
    const unsigned bid = s_bid;
    const unsigned long long nrec = a.ctr->n_records;
    const unsigned long long k0 = (unsigned long long)bid * kBinThreads;
    if (k0 >= nrec) return;
    unsigned long long c, total;
    const unsigned long long excl = bin_load(a, *ctp, s, k0, nrec, kBinThreads, c, total);
    if (threadIdx.x < 32) {
        const unsigned long long b = lookback_exclusive(a.lb_count + 1, bid, total, a.ctr, kSiteEmit);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    const unsigned long long base = s_base;
    const unsigned long long k = k0 + threadIdx.x;
    if (k < nrec) a.inst_off[k] = (uint32_t)(base + excl);
    if (k == nrec - 1) {
        const unsigned long long end = base + excl + c;
        a.ctr->instances_needed = end;
        a.ctr->n_instances = end < a.max_instances ? end : a.max_instances;
        if (end > a.max_instances) set_error(a.ctr, GS_ERR_CAPACITY, kSiteEmit);
    }
    for (unsigned long long j = threadIdx.x; j < total; j += kBinThreads) {
        int slot;
        const uint32_t t = bin_instance(s, j, slot);
        atomicAdd(&a.tile_cnt[t], 1u);
    }
}

// 2. Tile scan: exclusive scan of the tile counts; ranges clamped to the
// instance capacity (an overflow is already an error), cursors at the start,
// the forward's per-tile maxima of n_contrib cleared.
__global__ void __launch_bounds__(256) tile_scan_kernel(BinArgs a)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ unsigned long long s_warp[8];
    __shared__ unsigned s_bid;
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) s_bid = atomicAdd((unsigned *)a.lb_tiles, 1u);
    __syncthreads();
    const unsigned bid = s_bid;
    const long long t0 = ((long long)bid * 256 + threadIdx.x) * kTileScanItems;
    if ((long long)bid * 256 * kTileScanItems >= a.total_tiles) return;
    uint32_t cnt[kTileScanItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < kTileScanItems; q++) {
        cnt[q] = t0 + q < a.total_tiles ? a.tile_cnt[t0 + q] : 0u;
        sum += cnt[q];
    }
    unsigned long long total;
    const unsigned long long excl = block_exclusive_scan_256<unsigned long long>(sum, s_warp, total);
    if (threadIdx.x < 32) {
        const unsigned long long b = lookback_exclusive(a.lb_tiles + 1, bid, total, a.ctr, kSiteEmit);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    unsigned long long off = s_base + excl;
#pragma unroll
    for (int q = 0; q < kTileScanItems; q++) {
        if (t0 + q >= a.total_tiles) break;
        const unsigned long long e = off + cnt[q];
        a.ranges[t0 + q] = make_uint2((uint32_t)min(off, a.max_instances), (uint32_t)min(e, a.max_instances));
        a.tile_cur[t0 + q] = (uint32_t)min(off, a.max_instances);
        a.tile_last[t0 + q] = 0u;
        off = e;
    }
}

// 3. Scatter: every instance to the next position of its tile.  A block of
// kBinThreads threads takes kScatterRecs records, so that twice as many
// cursor atomics are in flight per SM as records per thread would allow.
__global__ void __launch_bounds__(kBinThreads) bin_scatter_kernel(BinArgs a, const CamTable *__restrict__ ctp)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ BinBlock s;
    const unsigned long long nrec = a.ctr->n_records;
    const unsigned long long k0 = (unsigned long long)blockIdx.x * kScatterRecs;
    if (k0 >= nrec) return;
    unsigned long long c, total;
    bin_load(a, *ctp, s, k0, nrec, kScatterRecs, c, total);
    // four instances per round: their cursor atomics are in flight together
    constexpr int kRound = 4;
    for (unsigned long long j0 = threadIdx.x; j0 < total; j0 += kRound * kBinThreads) {
        uint32_t pos[kRound], r[kRound], end[kRound], dk[kRound];
#pragma unroll
        for (int q = 0; q < kRound; q++) { // every load and atomic of the round issued first
            const unsigned long long j = j0 + (unsigned long long)q * kBinThreads;
            if (j >= total) break;
            int slot;
            const uint32_t t = bin_instance(s, j, slot);
            r[q] = s.rec[slot];
            pos[q] = atomicAdd(&a.tile_cur[t], 1u);
            end[q] = a.ranges[t].y;
            dk[q] = a.dkey[r[q]];
        }
#pragma unroll
        for (int q = 0; q < kRound; q++) {
            const unsigned long long j = j0 + (unsigned long long)q * kBinThreads;
            if (j >= total) break;
            if (pos[q] < end[q]) { // within the capacity-clamped range
                a.skey[pos[q]] = dk[q];
                a.sval[pos[q]] = r[q];
            }
        }
    }
}

// Ascending bitonic sort of the warp's 32 * E keys held in registers: key
// x[e] of lane l is element g = E l + e.  A stage of stride s < E pairs
// registers of one lane (e, e ^ s); a stage of stride s >= E pairs lanes
// (l, l ^ s / E) by a shuffle.  The network is fixed, so the result is the
// sorted order of the keys (all distinct) whatever order they came in.
template <int E> __device__ __forceinline__ void warp_sort_regs(unsigned long long (&x)[E])
{
    // the loops over sizes and lane strides stay loops (a short kernel body
    // for the instruction cache); the registers' indices are unrolled
    const int lane = threadIdx.x & 31;
    for (int size = 2; size <= 32 * E; size <<= 1) {
        for (int stride = size >> 1; stride >= E; stride >>= 1) {
            const int ls = stride / E;
            const bool lower = (lane & ls) == 0;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const unsigned long long u = x[e];
                const unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)u, ls);
                const unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 32), ls);
                const unsigned long long v = ((unsigned long long)hi << 32) | lo;
                const bool up = ((lane * E + e) & size) == 0;
                x[e] = (u < v) == (lower == up) ? u : v;
            }
        }
#pragma unroll
        for (int stride = E / 2; stride > 0; stride >>= 1) {
            if (stride >= size) continue;
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & stride) continue; // the lower element of each pair
                const bool up = ((lane * E + e) & size) == 0;
                const unsigned long long u = x[e], v = x[e ^ stride];
                const bool swap = (u > v) == up;
                x[e] = swap ? v : u;
                x[e ^ stride] = swap ? u : v;
            }
        }
    }
}

__device__ __forceinline__ unsigned long long key_at(const uint32_t *kk, const uint32_t *vv, uint32_t i)
{
    return ((unsigned long long)kk[i] << 32) | vv[i];
}

// Number of the first d outputs of the merge of X (nx) and Y (ny) that come
// from X (merge path; keys unique).
__device__ __forceinline__ uint32_t merge_split(const uint32_t *xk, const uint32_t *xv, uint32_t nx,
                                                const uint32_t *yk, const uint32_t *yv, uint32_t ny, uint32_t d)
{
    uint32_t lo = d > ny ? d - ny : 0u, hi = d < nx ? d : nx;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (key_at(xk, xv, mid) < key_at(yk, yv, d - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Sorts the n <= 32 * E keys (depth bits, record) at position `at` of (kk,
// vv) -- padded with the largest key -- and writes the records (rv) or the
// keys (rk, rv) back in order.
template <int E>
__device__ __forceinline__ void sort_run(const uint32_t *kk, const uint32_t *vv, uint32_t n, uint32_t *rk, uint32_t *rv)
{
    const int lane = threadIdx.x & 31;
    unsigned long long x[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t g = (uint32_t)(lane * E + e);
        x[e] = g < n ? key_at(kk, vv, g) : ~0ull;
    }
    warp_sort_regs<E>(x);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t g = (uint32_t)(lane * E + e);
        if (g < n) {
            if (rk) rk[g] = (uint32_t)(x[e] >> 32);
            rv[g] = (uint32_t)x[e];
        }
    }
}

__device__ __forceinline__ void sort_short(const uint32_t *kk, const uint32_t *vv, uint32_t n, uint32_t *rk, uint32_t *rv)
{
    if (n <= 32) sort_run<1>(kk, vv, n, rk, rv);
    else if (n <= 64) sort_run<2>(kk, vv, n, rk, rv);
    else if (n <= 128) sort_run<4>(kk, vv, n, rk, rv);
    else if (n <= 256) sort_run<8>(kk, vv, n, rk, rv);
    else sort_run<16>(kk, vv, n, rk, rv);
}

// 4. Per-tile sort of the scattered (depth bits, record) pairs; the sorted
// records end in sval.  One warp per tile, keys in registers.
__global__ void __launch_bounds__(32 * kTileSortWarps, 8) tile_sort_kernel(BinArgs a)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long t = (long long)blockIdx.x * kTileSortWarps + warp;
    if (t >= a.total_tiles) return;
    const uint2 rg = a.ranges[t];
    const uint32_t start = rg.x, n = rg.y - rg.x;
    if (n <= 1) return; // a single record is in place
    if (n <= (uint32_t)kTileSortMax) {
        sort_short(a.skey + start, a.sval + start, n, nullptr, a.sval + start);
        return;
    }
    // a long list: sorted chunks of kTileSortMax into the scratch, then
    // pairwise merges of runs, the warp's lanes on equal shares of each merge
    for (uint32_t c0 = 0; c0 < n; c0 += kTileSortMax)
        sort_short(a.skey + start + c0, a.sval + start + c0, min((uint32_t)kTileSortMax, n - c0), a.xkey + start + c0,
                   a.xval + start + c0);
    const uint32_t *srck = a.xkey + start, *srcv = a.xval + start;
    uint32_t *dstk = a.skey + start, *dstv = a.sval + start;
    for (uint32_t width = kTileSortMax; width < n; width <<= 1) {
        __syncwarp(); // the previous level's writes, before this level reads them
        for (uint32_t p = 0; p < n; p += 2 * width) {
            const uint32_t nx = min(width, n - p), ny = p + width < n ? min(width, n - p - width) : 0u;
            const uint32_t *xk = srck + p, *xv = srcv + p, *yk = srck + p + nx, *yv = srcv + p + nx;
            const uint32_t L = nx + ny, d0 = (uint32_t)(((unsigned long long)L * lane) / 32),
                           d1 = (uint32_t)(((unsigned long long)L * (lane + 1)) / 32);
            uint32_t i = merge_split(xk, xv, nx, yk, yv, ny, d0), j = d0 - i;
            for (uint32_t d = d0; d < d1; d++) {
                const bool take_x = j >= ny || (i < nx && key_at(xk, xv, i) < key_at(yk, yv, j));
                const unsigned long long v = take_x ? key_at(xk, xv, i) : key_at(yk, yv, j);
                if (take_x) i++;
                else j++;
                dstk[p + d] = (uint32_t)(v >> 32);
                dstv[p + d] = (uint32_t)v;
            }
        }
        const uint32_t *tk = srck, *tv = srcv;
        srck = dstk; srcv = dstv;
        dstk = const_cast<uint32_t *>(tk); dstv = const_cast<uint32_t *>(tv);
    }
    __syncwarp();
    if (srcv != a.sval + start) // the last level wrote the scratch: the records back into sval
        for (uint32_t i = lane; i < n; i += 32) a.sval[start + i] = srcv[i];
}

// The tile lists of the records of the last preprocess: ranges and
// ws->tval[0] (records sorted by (tile, depth bits, record)), inst_off, the
// instance counters.  Scratch: tile_cnt, tile_cur, the two look-back regions
// of lb_status, tkey[0..1], tval[1].
cudaError_t launch_bin(gs_workspace *ws, cudaStream_t st)
{
    const unsigned long long rcap = (unsigned long long)ws->cap.max_records;
    const int tiles = ws->cams.total_tiles;
    const unsigned cblocks = (unsigned)((rcap + kBinThreads - 1) / kBinThreads);
    const unsigned sblocks = (unsigned)((tiles + 256 * kTileScanItems - 1) / (256 * kTileScanItems));
    const size_t lb_need = (size_t)cblocks + 1 + sblocks + 1;
    if (lb_need > ws->lb_words) return cudaErrorInvalidValue; // sized at creation
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws->lb_status, 0, lb_need * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws->tile_cnt, 0, (size_t)tiles * sizeof(uint32_t), st)) != cudaSuccess) return e;
    BinArgs a;
    a.tt = ws->tt; a.rect = ws->rect; a.rec_cam = ws->rec_cam; a.dkey = ws->dkey;
    a.inst_off = ws->inst_off; a.tile_cnt = ws->tile_cnt; a.tile_cur = ws->tile_cur; a.ranges = ws->ranges;
    a.tile_last = ws->tile_last;
    a.skey = ws->tkey[0]; a.sval = ws->tval[0]; a.xkey = ws->tkey[1]; a.xval = ws->tval[1];
    a.lb_count = ws->lb_status; a.lb_tiles = ws->lb_status + cblocks + 1;
    a.ctr = ws->ctr; a.max_instances = (unsigned long long)ws->cap.max_instances; a.total_tiles = tiles;
    kt_begin(ws, GS_KT_BIN_COUNT, st);
    launch_pdl(bin_count_kernel, cblocks, kBinThreads, 0, st, a, ws->d_cams);
    kt_end(ws, GS_KT_BIN_COUNT, st);
    note_launch();
    kt_begin(ws, GS_KT_BIN_SORT, st);
    if (tiles > 0) {
        launch_pdl(tile_scan_kernel, sblocks, 256, 0, st, a);
        note_launch();
    }
    launch_pdl(bin_scatter_kernel, (unsigned)((rcap + kScatterRecs - 1) / kScatterRecs), kBinThreads, 0, st, a,
               ws->d_cams);
    note_launch();
    if (tiles > 0) {
        launch_pdl(tile_sort_kernel, (unsigned)((tiles + kTileSortWarps - 1) / kTileSortWarps), 32 * kTileSortWarps,
                   0, st, a);
        note_launch();
    }
    kt_end(ws, GS_KT_BIN_SORT, st);
    return cudaGetLastError();
}

} // namespace gs
