// gs_internal.cuh -- device-side building blocks shared by the gsblitz kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsblitz.h"

namespace gs {

// Programmatic dependent launch.  Every kernel of this library is launched
// with launch_pdl, which lets it be scheduled while the previous kernel on
// the stream drains, and begins with griddep_wait, which blocks until that
// kernel has completed and its writes are visible (a no-op when launched
// without the attribute).  Kernel-to-kernel gaps of a step shrink; inside a
// CUDA graph the launches become programmatic dependency edges.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the stream's priority, carried explicitly so that a kernel node captured
    // from the stream keeps it (graphs instantiated with per-node priorities)
    int prio = 0;
    if (cudaStreamGetPriority(st, &prio) == cudaSuccess && prio != 0) {
        attr[1].id = cudaLaunchAttributePriority;
        attr[1].val.priority = prio;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Single-instruction square root and reciprocal (PTX .approx forms).
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

constexpr size_t kRxHistWords = 4 * 256;  // radix histograms: 256 buckets for each of up to 4 passes
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;          // keys per thread in a radix pass (default)
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanTile = 4096;         // items per block of the selection's prefix sums
// per (record, tile) gradient slot, as the compositing adjoint writes it: the
// dG-weighted moments sum dG e, sum dG dy, sum dG dx^2, sum dG dx dy, sum dG dy^2
// (dG = dL/do of a pixel, (dx, dy) = pixel centre - mean, e = dx + k dy), then
// dL/do, dL/dr, dL/dg, dL/db; the per-record sum turns the moments into
// dL/du dL/dv dL/dA dL/dB dL/dC (slot_grads_from_moments)
constexpr int kSlotFloats = 9;
constexpr int kGradRow = 59;            // parameters per Gaussian: mean 3, log-scale 3, quat 4, opacity 1, SH 48
constexpr unsigned long long kSpinLimit = 1ull << 22;
constexpr int kMaxLod = 15;             // largest supported L_max

// The mean and conic gradients of a record from the sums of its slots' moments
// (see kSlotFloats).  With power = -1/2 (A dx^2 + C dy^2) - B dx dy
// = -1/2 (A e^2 + D dy^2) (k = B / A, D = C - B^2 / A) and dL/dpower = o dG at
// each pixel:  dL/du = o A sum dG e,  dL/dv = o (k A sum dG e + D sum dG dy),
// dL/dA = -o/2 sum dG dx^2,  dL/dB = -o sum dG dx dy,  dL/dC = -o/2 sum dG dy^2.
__device__ __forceinline__ void slot_grads_from_moments(float (&g)[kSlotFloats], float A, float k, float D, float o)
{
    const float oAe = o * A * g[0];
    const float gv = fmaf(k, oAe, o * D * g[1]);
    g[0] = oAe;
    g[1] = gv;
    g[2] = -0.5f * o * g[2];
    g[3] = -o * g[3];
    g[4] = -0.5f * o * g[4];
}

// Error sites recorded next to the error word (which kernel gave up).
enum ErrorSite {
    kSitePreprocess = 1, kSiteEmit = 2 /* binning */, kSiteRadix = 3, kSiteSelect = 4, kSiteScanF64 = 5, kSiteModel = 6,
    kSiteRender = 7,
};

// Device counters of one workspace.
struct DevCounters {
    unsigned long long n_records;
    unsigned long long n_instances;
    unsigned long long n_visible;
    unsigned long long records_needed;
    unsigned long long instances_needed;
    unsigned long long n_candidates;   // Gaussians passing the gate stage of preprocess
    unsigned long long n_catchup;      // candidates behind the current Adam step (deferred steps to replay)
    int error;
    int error_site;
    unsigned long long sel_count[GS_MAX_CAMERAS]; // w > 0 entries per camera (importance)
    unsigned long long fragments;      // sum over pixels of the entries up to the last composited one
    unsigned long long composited;     // ... of which composited (alpha >= alpha_min)
};

// Per-camera constants (the device camera table).
struct CamInfo {
    float R[9], t[3];
    float fx, fy, cx, cy;
    float campos[3];
    int width, height;
    int tiles_x, tiles_y;
    int tile_base;        // first global tile id of this camera
    long long pix_base;   // first pixel of this camera in the concatenated outputs
    float jbound;         // >= fx^2 (1 + limx^2) + fy^2 (1 + limy^2): bounds |J|_F^2 tz^2
};

// The cameras of one call and their tiling.  Kernels read it from device
// memory (the workspace's copy), so a captured CUDA graph replays with
// whatever cameras were uploaded last.
struct CamTable {
    int n;
    int total_tiles;
    int tile_w, tile_h;   // pixels per tile: 16 x 16, 32 x 8, 8 x 32 or 32 x 16
    CamInfo c[GS_MAX_CAMERAS];
};

// Index of a supported tile shape, -1 if unsupported.
__host__ __device__ inline int tile_shape_id(int tw, int th)
{
    return tw == 16 && th == 16 ? 0 : tw == 32 && th == 8 ? 1 : tw == 8 && th == 32 ? 2 : tw == 32 && th == 16 ? 3
         : tw == 16 && th == 8 ? 4 : tw == 8 && th == 16 ? 5 : -1;
}

// Render-time constants (FP32, as the kernels compare them).
struct RenderConsts {
    float bg[3];
    float alpha_min, alpha_max, T_min;
    float dilation, znear, fov_clamp;
    float lod_d0, lod_f;
    int lod_enable, lod_Lmax, cull_enable;
    float eps_score, vis_mass;
    // LOD gate in squared-distance form: a level-l Gaussian (1 <= l <= Lmax)
    // passes Eq. 1-2 iff d^2 <= lod_thr2[l] = (d0 f^(0.5 - l))^2
    float lod_thr2[kMaxLod + 1];
};

__device__ __forceinline__ void set_error(DevCounters *ctr, int code, int site)
{
    if (atomicCAS(&ctr->error, 0, code) == 0) ctr->error_site = site;
}

// Whether the error word was set before this block started, read by one thread
// so that the whole block takes the same branch (the kernels calling it use
// block barriers).
__device__ __forceinline__ bool block_error(const DevCounters *ctr)
{
    __shared__ int s_err;
    if (threadIdx.x == 0) s_err = *(volatile const int *)&ctr->error;
    __syncthreads();
    return s_err != 0;
}

// Camera of a global tile id (binary search over tile bases).
__device__ __forceinline__ int camera_of_tile(const CamTable &ct, int tile)
{
    int lo = 0, hi = ct.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ct.c[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Rectangle of a record, packed as (x0 | y0 << 16, x1 | y1 << 16) in tiles.
__device__ __forceinline__ void unpack_rect(uint2 r, int &x0, int &y0, int &x1, int &y1)
{
    x0 = (int)(r.x & 0xffffu); y0 = (int)(r.x >> 16);
    x1 = (int)(r.y & 0xffffu); y1 = (int)(r.y >> 16);
}

// ---- decoupled look-back (Merrill & Garland single-pass scan) -------------
// Status words: bits 63..62 = 0 empty, 1 block aggregate, 2 inclusive prefix.
constexpr unsigned long long kLbAgg = 1ull << 62;
constexpr unsigned long long kLbInc = 2ull << 62;
constexpr unsigned long long kLbVal = (1ull << 62) - 1;

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v)
{
    *(volatile unsigned long long *)p = v;
}

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p)
{
    return *(volatile const unsigned long long *)p;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Called by one full warp of block `bid`.  Publishes the block aggregate,
// walks back over predecessors 32 at a time and returns the exclusive prefix
// of this block (to every lane), then publishes the inclusive prefix.  Every
// wait is bounded: on timeout the error word is set and the walk stops.
__device__ __forceinline__ unsigned long long lookback_exclusive(unsigned long long *status, unsigned bid,
                                                                 unsigned long long aggregate, DevCounters *ctr,
                                                                 int site)
{
    const int lane = threadIdx.x & 31;
    if (bid == 0) {
        if (lane == 0) lb_store(&status[0], kLbInc | aggregate);
        return 0ull;
    }
    if (lane == 0) lb_store(&status[bid], kLbAgg | aggregate);
    unsigned long long excl = 0;
    long long pred = (long long)bid - 1;
    while (true) {
        long long idx = pred - lane;
        unsigned long long s = kLbInc; // before block 0: inclusive prefix 0
        if (idx >= 0) {
            unsigned long long spins = 0;
            while (true) {
                s = lb_load(&status[idx]);
                if ((s >> 62) != 0) break;
                if (++spins > kSpinLimit) {
                    set_error(ctr, GS_ERR_TIMEOUT, site);
                    s = kLbInc;
                    break;
                }
                __nanosleep(40);
            }
        }
        unsigned incl = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        unsigned long long v = s & kLbVal;
        if (incl) {
            int first = __ffs(incl) - 1;
            if (lane > first) v = 0;
            excl += warp_sum_u64(v);
            break;
        }
        excl += warp_sum_u64(v);
        pred -= 32;
    }
    if (lane == 0) lb_store(&status[bid], kLbInc | (excl + aggregate));
    return excl;
}

// Block-wide exclusive scan of one value per thread, NW warps per block.
template <int NW, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *smem_warp /*[NW]*/, T &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    T wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        T s = smem_warp[w];
        if (w < warp) wpre += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + x - v;
}

// The same for blockDim.x == 256.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan_256(T v, T *smem_warp /*[8]*/, T &total)
{
    return block_exclusive_scan<8, T>(v, smem_warp, total);
}

// ---- bulk copies (cp.async.bulk) and shared-memory barriers ----------------
// One thread arms a barrier with the bytes it expects and issues bulk copies
// from global to shared memory that complete on it; the threads that read the
// data wait on the barrier's phase.  Addresses and sizes of a bulk copy are
// multiples of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes initialised barriers visible to the bulk-copy engine
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Waits for the phase of the given parity to complete, at most `limit` tries;
// false when it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned long long limit)
{
    for (unsigned long long i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

} // namespace gs

// ---- workspace (host struct, device buffers) -------------------------------
struct gs_workspace {
    gs_capacity cap;
    unsigned long long sel_spin_limit; // bound on the look-back waits of gs_importance's selection sorts
    int device;
    int sm_count;        // multiprocessors of the device (persistent grids)
    void *base;          // one device allocation, carved into the buffers below
    size_t bytes;
    // per Gaussian (candidates of the gate stage, in index order)
    uint32_t *cand_g;              // [N]
    unsigned long long *cand_mask; // [N] bit per camera
    uint32_t *gate_g;              // [N] block-strided candidates of the gate's first pass
    unsigned long long *gate_mask; // [N]
    uint32_t *rec_first;           // [N] first record of each Gaussian, ~0 when none
    float *cgrad;                  // [R][59] compact gradient rows (fused backward + Adam)
    // per record
    uint32_t *rec_g;
    uint16_t *rec_cam;
    float4 *rd0;         // u, v (nearest floats to the mean), conic A, k
    float4 *rd1;         // conic D, opacity, r, g
    float4 *rd2;         // b, u_lo, v_lo (mean = u + u_lo), 0
    uint2 *rect;
    uint32_t *tt;
    uint32_t *inst_off;
    uint8_t *clampm;
    float *rgrad;        // [R][9] per-record summed gradients of u v A B C o r g b
    uint32_t *dkey;      // [R] FP32 bits of each record's camera depth
    uint32_t *tile_cnt, *tile_cur; // [T] the binning's tile counts and fill cursors
    uint32_t *tile_last;           // [T] largest n_contrib of each tile's pixels (zeroed by the binning, set by the forward)
    // per instance
    uint32_t *tkey[2], *tval[2];
    float *slots;        // [I][9] adjoint slots (training workspaces only)
    float2 *imp_slots;   // [I] importance slots (alpha-weight, composited pixels as uint32 bits); a buffer
                         // of their own, so the importance sweep shares no scratch with the training pass
    // per tile
    uint2 *ranges;       // [T]
    // per pixel
    uint32_t *n_contrib;
    float *T_final;
    // importance
    float *imp_w;        // [R] per-record alpha-weight
    uint32_t *imp_a;     // [R]
    double *sel_cum;     // [R] scratch for the mass scans (FP64, or fixed point for the selection)
    unsigned long long *sel_bsum; // [R / 4096 + 2] block masses of the selection scan
    uint32_t *selk[2], *selv[2]; // [R] selection sort pairs
    // loss scratch: 3 maps of [P][3]
    float *loss_maps;
    float *loss_partial; // [2 * blocks]
    size_t loss_partial_words;
    // scan / sort scratch
    unsigned long long *lb_status; // [max(blocks)+1] single-value look-back + ticket
    size_t lb_words;
    uint32_t *rx_status; // radix: [4][256] histograms, then per pass [blocks * 256 + 1] look-back + ticket
    size_t rx_words;
    uint32_t *rx_hist;   // [4][256]: the first kRxHistWords words of rx_status (also a scratch of 1024 words)
    float *red_partial;  // [blocks] reduction partials of the adjoint (scale regulariser)
    size_t red_words;
    gs::DevCounters *ctr;
    gs::CamTable *d_cams;  // device copy of the uploaded cameras, read by every kernel
    int sort_items;        // keys per thread of a radix pass: 16 (4096-key blocks) or 8 (2048)
    // model-level scratch (GS_CAP_MODEL_OPS): sorts and scans over all Gaussians
    uint32_t *mkey[2], *mval[2]; // [N]
    double *mcum;                // [N]
    double *mbsum;               // [N / 4096 + 2]
    uint32_t *mrx_status;        // radix look-back, [(N / 2048 + 1) * 256 + 1]
    unsigned long long *mlb;     // single-value look-back, [N / 256 + 3]
    uint32_t *mhist;             // [4][256]
    gs::DevCounters *mctr;       // item count (n_records) and errors of the model-level calls
    int *d_adam_step;      // device Adam step counter (graph-replayable optimizer step)
    // deferred zero-gradient Adam steps (gs_adam_lazy_enable): a Gaussian's p, m,
    // v are brought to the current step only when it is next used
    struct {
        int enabled;
        int max_steps;
        float *hist;       // device [max_steps + 1][10]: lr_c of the 5 groups, then 1/sqrt(1 - beta2^t)
        gs_gaussian_grads m, v;
        int32_t *last;     // [N] step at which a Gaussian's p, m, v are current
        float *drift;      // [N][2] bounds on the mean's and the largest log-scale's further drift
        float b1, b2, eps, drift_factor;
    } lazy;
    float *d_adam_coef;    // [2][GS_MAX_ADAM_GROUPS] bias-corrected lr and 1/sqrt(1 - beta2^t)
    // host staging of camera uploads: a ring of pinned tables, each reused only
    // after the copy that read it has completed
    static constexpr int kStageSlots = 8;
    gs::CamTable *h_stage; // [kStageSlots], pinned
    cudaEvent_t stage_ev[kStageSlots];
    bool stage_pending[kStageSlots];
    int stage_next;
    // last upload: the host copy of the table (launch sizes) and the parameters it depends on
    gs::CamTable cams;
    int have_upload;
    float up_fov_clamp;
    // state of the last preprocess
    gs::RenderConsts rc;
    gs_gaussians g;
    int have_preprocess;
    int have_binning;
    int have_compact;    // compact gradient rows of the current binning exist
    int imp_ready;       // the importance w, a of the current binning exist (gs_render_fwd_importance)
    int tile_buf;        // buffer holding sorted instances (0)
    // kernel timing (gs_kernel_timing): event pairs around the rasterisers' launches
    static constexpr int kTimedPairs = 64;
    struct {
        int on;
        unsigned mask; // (1 << GS_KT_*) bits of the kernels timed while on
        cudaEvent_t ev[GS_KT_COUNT][kTimedPairs][2];
        int used[GS_KT_COUNT];
        long long launches[GS_KT_COUNT]; // launches while on, recorded or not
    } kt;
};

namespace gs {
// Counts one kernel launch of this library (process-wide, see gs_kernel_launches).
void note_launch();
// Kernel timing: kt_begin/kt_end bracket one launch of kernel id on stream st
// while timing is on (nothing under stream capture, nothing past kTimedPairs).
void kt_begin(gs_workspace *ws, int id, cudaStream_t st);
void kt_end(gs_workspace *ws, int id, cudaStream_t st);
// Records msg as the calling thread's gs_last_error() and returns code.
int report_error(int code, const char *msg);
// Kernel launchers (defined in the .cu files).
cudaError_t launch_preprocess(gs_workspace *ws, cudaStream_t st, const uint32_t *cull);
cudaError_t launch_render_fwd_importance(gs_workspace *ws, cudaStream_t st, float *rgb, float *T_out);
cudaError_t launch_importance_reduce(gs_workspace *ws, cudaStream_t st);
cudaError_t launch_radix_sort(gs_workspace *ws, cudaStream_t st, uint32_t *keys[2], uint32_t *vals[2],
                              const unsigned long long *count, unsigned long long cap, int bits, bool vals_identity,
                              int &out_buf, unsigned long long spin_limit = kSpinLimit);
cudaError_t launch_bin(gs_workspace *ws, cudaStream_t st);
cudaError_t launch_render_fwd(gs_workspace *ws, cudaStream_t st, float *rgb, float *T_out);
cudaError_t launch_render_bwd(gs_workspace *ws, cudaStream_t st, const float *dL_drgb);
cudaError_t launch_reduce_slots(gs_workspace *ws, cudaStream_t st);
cudaError_t launch_preprocess_bwd(gs_workspace *ws, cudaStream_t st, const gs_gaussians &g,
                                  const gs_gaussian_grads &gr, int accumulate, float *absgrad, float beta,
                                  float *scale_reg_value, float *cgrad);
// Adam over the five parameter arrays with gradients taken from the compact
// rows (zero for Gaussians without a record).
cudaError_t launch_adam_sparse(gs_workspace *ws, cudaStream_t st, const gs_gaussian_grads &param,
                               const gs_gaussian_grads &m, const gs_gaussian_grads &v, long long n,
                               const float lr[5], float beta1, float beta2, float eps, int step);
cudaError_t launch_importance(gs_workspace *ws, cudaStream_t st, float *w, uint32_t *a, float *s_accum,
                              uint32_t *crad, uint32_t *cvis, uint32_t *cull_out);
cudaError_t launch_loss(gs_workspace *ws, cudaStream_t st, const float *img, const float *tgt, int B, int H, int W,
                        float lambda, float *loss_out, float *dL);
cudaError_t launch_adam(const gs_adam_group *groups, int n_groups, int step, cudaStream_t st);
cudaError_t launch_prune_sample(gs_workspace *ws, cudaStream_t st, const float *s, const float *expo, long long n,
                                long long k, uint32_t *keep);
cudaError_t launch_prune_mass(gs_workspace *ws, cudaStream_t st, const float *s, long long n, float mass,
                              uint32_t *keep);
cudaError_t launch_count_views(gs_workspace *ws, cudaStream_t st, uint32_t *counts);
cudaError_t launch_lazy_catchup(gs_workspace *ws, cudaStream_t st, const gs_gaussians &g);
cudaError_t launch_lazy_flush(gs_workspace *ws, cudaStream_t st, const gs_gaussians &g);
cudaError_t launch_compact(gs_workspace *ws, cudaStream_t st, const gs_model &src, const uint32_t *keep,
                           const gs_model &dst, long long dst_cap, long long *n_out);
cudaError_t launch_densify(gs_workspace *ws, cudaStream_t st, const gs_model &src, const float *absgrad,
                           const uint32_t *denom, const uint32_t *cvis, const uint32_t *crad, const float *noise,
                           const gs_densify_params &p, const gs_model &dst, long long dst_cap, long long *n_out);
} // namespace gs
