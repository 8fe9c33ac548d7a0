// noalloc.cu -- the per-view visible-set selection without any allocation.
//
// Some callers may not allocate device memory at all: code that runs where a
// cudaMalloc is forbidden or would stall other work (it can synchronise the
// device), such as a latency-critical serving thread, a host callback, or a
// plugin whose memory belongs to another allocator -- and that holds no
// gs_workspace.  For them gs_visible_set_static computes the same Cull column
// as gs_importance's selection step from a view's per-Gaussian alpha-weights,
// with its scratch in one fixed device array of this file instead of a
// workspace.
//
// The array (kVisScratchBytes, about 24.6 MB, for at most kVisMaxGaussians =
// 2^20 Gaussians per call) is a file-scope __device__ variable: every GPU on
// which the library's module is loaded keeps it until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device asks the runtime for it (cudaGetSymbolAddress, with that
// device current) and caches it; that first call should therefore come before
// any stream capture.  All calls share the array: calls whose work overlaps on
// the GPU (other streams, other threads) race and must be serialised by the
// caller.  Every value the selection reads is written earlier in the same call.
// The selection is gs_importance's, operation for operation: the same stable
// sort of w descending (ties toward the lower index) and the same exact 64-bit
// fixed-point prefix sums, so the two give the same Cull column bit for bit.
// A device-side failure (a bounded wait of the sort that gave up) leaves every
// Gaussian culled and is reported through the caller's error word.
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "gs_internal.cuh"

namespace gs {

cudaError_t launch_radix_sort_scratch(cudaStream_t st, uint32_t *keys[2], uint32_t *vals[2],
                                      const unsigned long long *count, unsigned long long cap, int bits,
                                      bool vals_identity, uint32_t *status, uint32_t *hist, DevCounters *ctr,
                                      int &out_buf);
cudaError_t launch_mass_scan_fixed(cudaStream_t st, const uint32_t *sorted, const float *w, unsigned long long *bsum,
                                   unsigned long long *cum, const DevCounters *ctr, unsigned long long cap);

constexpr long long kVisMaxGaussians = 1ll << 20;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// the sort's look-back status words are sized by its key blocks, the scan's block
// sums by its item blocks: each from its own constant
constexpr size_t kVisSortBlocks = (size_t)(kVisMaxGaussians + kSortTile - 1) / kSortTile;
constexpr size_t kVisScanBlocks = (size_t)(kVisMaxGaussians + kScanTile - 1) / kScanTile;
// layout of the scratch array
constexpr size_t kOffCtr = 0;
constexpr size_t kOffKey0 = align256(kOffCtr + sizeof(DevCounters));
constexpr size_t kOffKey1 = align256(kOffKey0 + 4 * (size_t)kVisMaxGaussians);
constexpr size_t kOffVal0 = align256(kOffKey1 + 4 * (size_t)kVisMaxGaussians);
constexpr size_t kOffVal1 = align256(kOffVal0 + 4 * (size_t)kVisMaxGaussians);
constexpr size_t kOffCum = align256(kOffVal1 + 4 * (size_t)kVisMaxGaussians);
constexpr size_t kOffBsum = align256(kOffCum + 8 * (size_t)kVisMaxGaussians);
constexpr size_t kOffStatus = align256(kOffBsum + 8 * (kVisScanBlocks + 1));
constexpr size_t kOffHist = align256(kOffStatus + 4 * (kVisSortBlocks * 256 + 1));
constexpr size_t kVisScratchBytes = align256(kOffHist + 4 * 1024);

static __device__ __align__(256) unsigned char g_vis_scratch[kVisScratchBytes];

__global__ void vis_init_kernel(const float *w, long long n, unsigned char *scratch)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    DevCounters *ctr = reinterpret_cast<DevCounters *>(scratch + kOffCtr);
    uint32_t *keys = reinterpret_cast<uint32_t *>(scratch + kOffKey0);
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i == 0) {
        memset(ctr, 0, sizeof(DevCounters));
        ctr->n_records = (unsigned long long)n; // the item count the sort and scan kernels read
    }
    // ascending keys = descending w; w = 0 sorts last
    if (i < n) keys[i] = ~__float_as_uint(w[i]);
}

__global__ void vis_cull_init_kernel(uint32_t *cull, long long words, long long n)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long k = (long long)blockIdx.x * 256 + threadIdx.x;
    if (k >= words) return;
    const long long bits = n - k * 32;
    cull[k] = bits >= 32 ? 0xffffffffu : ((1u << bits) - 1u);
}

__global__ void vis_apply_kernel(const float *w, long long n, const uint32_t *sorted, const unsigned long long *cum,
                                 float vis_mass, uint32_t *cull, uint32_t *cvis, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long k = (long long)blockIdx.x * 256 + threadIdx.x;
    if (k >= n || ctr->error != 0) return; // a failed sort: every Gaussian stays culled
    const uint32_t g = sorted[k];
    if (!(w[g] > 0.f)) return;
    const unsigned long long total = cum[n - 1];
    const unsigned long long excl = k > 0 ? cum[k - 1] : 0ull;
    if ((double)excl < (double)vis_mass * (double)total) {
        atomicAnd(&cull[g >> 5], ~(1u << (g & 31)));
        if (cvis) atomicAdd(&cvis[g], 1u);
    }
}

// The call's device error word (0: none) for the caller.
__global__ void vis_status_kernel(const DevCounters *ctr, uint32_t *error_out)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    if (threadIdx.x == 0) *error_out = (uint32_t)ctr->error;
}

namespace {
std::mutex g_vis_mutex;
void *g_vis_addr[256]; // per device ordinal

int vis_fail(int code, const char *fmt, long long a = 0, long long b = 0)
{
    char msg[256];
    snprintf(msg, sizeof(msg), fmt, a, b, b);
    return report_error(code, msg);
}
} // namespace

} // namespace gs

extern "C" {

int gs_visible_set_static(const float *w, int64_t n, float vis_mass, uint32_t *cull_out, uint32_t *cvis_accum,
                          uint32_t *error_out, gs_stream stream)
{
    using namespace gs;
    if (!w || !cull_out) return vis_fail(GS_ERR_INVALID_ARG, "gs_visible_set_static: NULL w or cull_out");
    if (n < 0 || n > kVisMaxGaussians)
        return vis_fail(GS_ERR_CAPACITY,
                        "gs_visible_set_static: n = %lld outside [0, %lld]: the fixed scratch holds at most %lld "
                        "Gaussians per call",
                        (long long)n, kVisMaxGaussians);
    if (!(vis_mass > 0.f) || vis_mass > 1.f)
        return vis_fail(GS_ERR_INVALID_ARG, "gs_visible_set_static: vis_mass must be in (0, 1]");
    if (n == 0) {
        if (error_out && cudaMemsetAsync(error_out, 0, sizeof(uint32_t), (cudaStream_t)stream) != cudaSuccess)
            return vis_fail(GS_ERR_CUDA, "gs_visible_set_static: clearing error_out failed");
        return GS_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256)
        return vis_fail(GS_ERR_CUDA, "gs_visible_set_static: cudaGetDevice failed");
    unsigned char *scratch;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_vis_mutex);
        if (!g_vis_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_vis_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return vis_fail(GS_ERR_CUDA, "gs_visible_set_static: cudaGetSymbolAddress of the scratch failed");
            }
            g_vis_addr[dev] = ptr;
        }
        scratch = static_cast<unsigned char *>(g_vis_addr[dev]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    DevCounters *ctr = reinterpret_cast<DevCounters *>(scratch + kOffCtr);
    uint32_t *keys[2] = {reinterpret_cast<uint32_t *>(scratch + kOffKey0),
                         reinterpret_cast<uint32_t *>(scratch + kOffKey1)};
    uint32_t *vals[2] = {reinterpret_cast<uint32_t *>(scratch + kOffVal0),
                         reinterpret_cast<uint32_t *>(scratch + kOffVal1)};
    unsigned long long *cum = reinterpret_cast<unsigned long long *>(scratch + kOffCum);
    unsigned long long *bsum = reinterpret_cast<unsigned long long *>(scratch + kOffBsum);
    uint32_t *status = reinterpret_cast<uint32_t *>(scratch + kOffStatus);
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + kOffHist);
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const long long words = (n + 31) / 32;
    launch_pdl(vis_init_kernel, blocks, 256, 0, st, w, n, scratch);
    note_launch();
    launch_pdl(vis_cull_init_kernel, (unsigned)((words + 255) / 256), 256, 0, st, cull_out, words, n);
    note_launch();
    int ob = 0;
    if ((e = launch_radix_sort_scratch(st, keys, vals, &ctr->n_records, (unsigned long long)n, 32, true, status, hist,
                                       ctr, ob)) != cudaSuccess ||
        (e = launch_mass_scan_fixed(st, vals[ob], w, bsum, cum, ctr, (unsigned long long)n)) != cudaSuccess)
        return vis_fail(GS_ERR_CUDA, "gs_visible_set_static: a kernel launch failed");
    launch_pdl(vis_apply_kernel, blocks, 256, 0, st, w, n, vals[ob], cum, vis_mass, cull_out, cvis_accum,
               (const DevCounters *)ctr);
    note_launch();
    if (error_out) {
        launch_pdl(vis_status_kernel, 1, 32, 0, st, (const DevCounters *)ctr, error_out);
        note_launch();
    }
    if ((e = cudaGetLastError()) != cudaSuccess)
        return vis_fail(GS_ERR_CUDA, "gs_visible_set_static: a kernel launch failed");
    return GS_OK;
}

} // extern "C"
