// render.cu -- per-tile compositing (App. A, Eq. for C(p) and T_i), its
// adjoint, and the instrumented colourless sweep of the importance pass
// (Sec. 3.2, Fig. 2).
//
// One block per tile; each warp owns an 8 x 8 pixel square of it (lane l the
// horizontal pixel pair (2 (l % 4), l / 4), packed FP32x2) and walks the
// tile's depth-ordered list on its own, staging each batch of 32 entries
// itself and visiting only the entries that can reach alpha_min in its square.
// Per-Gaussian quantities are warp reductions (recursive halving for the
// adjoint's nine values), then the warps' partials summed in warp order,
// rather than per-pixel global atomics.  The backward and the importance
// sweep write one gradient/score slot per (record, tile) -- slot index = the
// record's first instance + the tile's position inside the record's rectangle
// -- and a later per-record pass sums a record's slots in a fixed order, so
// results are bit-reproducible run to run.
#include "gs_internal.cuh"

namespace gs {

// Compositing works in tile-local pixel coordinates: pixel centres are exact
// small floats, and each staged entry's mean is moved to the tile's origin
// once, from its double-length form u + u_lo, so px - u keeps its full
// precision however far the tile lies from the image origin.

// ---- packed pair arithmetic (Blackwell FP32x2) ----------------------------------
// A lane's two pixels are one float2, so the exponent, alpha, transmittance
// and colour updates are packed FP32x2 operations.  The exponent is evaluated from the conic's form
// power = -1/2 (A (dx + k dy)^2 + D dy^2), with A and D pre-scaled at staging so
// it comes out in base 2: G = exp(power) = 2^(log2(e) power).  Every kernel
// that takes skip decisions (forward, backward, importance) stages and
// evaluates through these same functions.
constexpr float kNegHalfLog2e = -0.72134752044448170f; // -log2(e) / 2

// A staged entry: e0 = (u, v) tile-local, A and k; e1.x = D (A, D scaled to base 2)
__device__ __forceinline__ float4 stage_e0_at(float4 r0, float4 r2, float ox, float oy)
{
    return make_float4(__fadd_rn(__fsub_rn(r0.x, ox), r2.y), __fadd_rn(__fsub_rn(r0.y, oy), r2.z),
                       __fmul_rn(r0.z, kNegHalfLog2e), r0.w);
}
__device__ __forceinline__ float stage_D(float4 r1) { return __fmul_rn(r1.x, kNegHalfLog2e); }

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// alpha = min(alpha_max, o 2^p) of a pixel pair
__device__ __forceinline__ float2 pair_alpha(float2 p, float o, float amax, float2 &G)
{
    G = make_float2(ex2_approx(p.x), ex2_approx(p.y));
    const float2 og = __fmul2_rn(f2(o), G);
    return make_float2(fminf(amax, og.x), fminf(amax, og.y));
}

// Whether an entry can composite anywhere in a warp's square, the box
// [bx0, bx1] x [by0, by1] of its pixel centres (tile-local; (u, v) the entry's
// tile-local mean).  alpha >= alpha_min needs o G >= alpha_min, i.e.
// q = A (dx + k dy)^2 + D dy^2 <= tau, tau = 2 ln(o / alpha_min).  Two
// conservative tests, both of which must pass:
//  - the bounding box of that ellipse, half-widths sqrt(tau Sx), sqrt(tau Sy)
//    with (Sx, Sy) the diagonal of the inverse of the conic (Sx = 1/A +
//    k^2/D, Sy = 1/D), meets the square;
//  - a lower bound of q over the square is at most tau: D times the squared
//    distance of the dy range from 0 plus A times the squared gap between the
//    dx range and the range of -k dy (each term minimised on its own, so their
//    sum is below q at every point of the square).  It drops the squares that
//    only the corners of an elongated, tilted ellipse's box reach.
// Widened (tau by 0.2 % + 2e-3, the half-widths by 0.1 % + 1/32 px, the gaps
// narrowed by 1/32 px) far beyond the FP32 error of the exponent the kernels
// evaluate and of the approximate logarithm, reciprocals and square roots
// here (a few units in the last place), so no pixel of a square that fails
// either test can reach alpha_min in them; false when o is below alpha_min.
// A warp skips an entry that fails: it composites nowhere in the warp, so
// skipping it changes nothing.
__device__ __forceinline__ bool square_visit(float A, float k, float D, float o, float alpha_min, float u, float v,
                                             float bx0, float bx1, float by0, float by1)
{
    float tau = 2.f * __logf(__fdividef(o, alpha_min));
    tau = fmaf(tau, 1.002f, 2e-3f);
    if (!(tau > 0.f)) return false;
    const float iD = rcp_approx(D);
    const float hx = fmaf(sqrt_approx(tau * fmaf(k * k, iD, rcp_approx(A))), 1.001f, 0.03125f);
    const float hy = fmaf(sqrt_approx(tau * iD), 1.001f, 0.03125f);
    if (u + hx < bx0 || u - hx > bx1 || v + hy < by0 || v - hy > by1) return false;
    const float dx0 = bx0 - u, dx1 = bx1 - u, dy0 = by0 - v, dy1 = by1 - v;
    const float p0 = -k * dy0, p1 = -k * dy1;
    const float gy = fmaxf(fmaxf(dy0, -dy1) - 0.03125f, 0.f);
    const float gx = fmaxf(fmaxf(fminf(p0, p1) - dx1, dx0 - fmaxf(p0, p1)) - 0.03125f, 0.f);
    return fmaf(A * gx, gx, D * gy * gy) <= tau;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums the 9 slot values over the warp by recursive halving (a reduce-scatter):
// at each of the first four levels a lane keeps half of its values and trades
// the other half with its partner, so 5 + 3 + 2 + 1 + 1 = 12 shuffles replace
// the 45 of nine butterfly sums.  Lane l ends with the full sum of value
// red9_index(l), valid when red9_owner(l).
__device__ __forceinline__ float warp_reduce9(const float (&v)[kSlotFloats], int lane)
{
    static_assert(kSlotFloats == 9, "the halving schedule is laid out for 9 values");
    const bool h1 = lane & 16, h2 = lane & 8, h3 = lane & 4, h4 = lane & 2;
    float a[5], b[3], c[2];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float lo = v[i], hi = i + 5 < 9 ? v[i + 5] : 0.f;
        a[i] = (h1 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h1 ? lo : hi, 16);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float lo = a[i], hi = i + 3 < 5 ? a[i + 3] : 0.f;
        b[i] = (h2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h2 ? lo : hi, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float lo = b[i], hi = i + 2 < 3 ? b[i + 2] : 0.f;
        c[i] = (h3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h3 ? lo : hi, 4);
    }
    const float d = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 2);
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}
// value held by lane l after warp_reduce9: lane bit 4 picks 0-4 / 5-8, bits 3, 2
// and 1 pick within the halves (padding positions hold no value)
__device__ __forceinline__ int red9_index(int lane)
{
    return 5 * ((lane >> 4) & 1) + 3 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
}
__device__ __forceinline__ bool red9_owner(int lane)
{
    const int h1 = (lane >> 4) & 1, h2 = (lane >> 3) & 1, h3 = (lane >> 2) & 1, h4 = (lane >> 1) & 1;
    const int ai = 3 * h2 + 2 * h3 + h4;
    return (lane & 1) == 0 && (h2 ? h3 == 0 : 2 * h3 + h4 <= 2) && ai < (h1 ? 4 : 5);
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

// ---- warp squares ------------------------------------------------------------
//
// The forward and the adjoint give each warp an 8 x 8 pixel square of the
// tile: lane l holds the horizontal pixel pair (2 (l % 4), l / 4) of it, as
// FP32x2, and the warp walks the tile's list on its own.  The warp stages each
// batch of 32 entries itself (lane i the i-th), the staging lane tests its
// entry's alpha footprint against the square (square_visit), and one ballot gives the entries the
// warp visits; an entry whose box misses the square composites nowhere in it.

template <int TW, int TH> struct SquareShape {
    static_assert(TW % 8 == 0 && TH % 8 == 0, "the tile splits into 8 x 8 pixel squares");
    static constexpr int wx = TW / 8;
    static constexpr int warps = (TW / 8) * (TH / 8);
    static constexpr int threads = 32 * warps;
    // the adjoint's register budget: at least six resident blocks of 128 threads per
    // SM, which ptxas meets with 64 registers (so eight fit); on the 16 x 16 tile
    // 10-15 % faster than both its own choice (86 registers, five blocks) and tighter
    // budgets (56-57 registers)
    static constexpr int bwd_min_blocks = 768 / threads;
    // the importance walk's: eight blocks of 128 threads (64 registers; the fused walk
    // with the training image measured 8 % faster than with the compiler's 60)
    static constexpr int imp_min_blocks = 1024 / threads;
};

// Tile, camera and pixel geometry of one warp square.
struct SquareGeom {
    const CamInfo *ci;
    int tx, ty;            // tile coordinates in its camera
    float ox, oy;          // pixel origin of the tile
    int lx, ly;            // tile-local pixel of the lane's pair (left pixel)
    float2 pxc;            // its two pixel-centre x, tile-local
    float pyc;             // its pixel-centre y, tile-local
    float bx0, bx1, by0, by1; // the square's pixel-centre box, tile-local
};

template <int TW, int TH> __device__ __forceinline__ SquareGeom square_geom(const CamTable &ct, int tile, int warp,
                                                                            int lane)
{
    SquareGeom q;
    q.ci = &ct.c[camera_of_tile(ct, tile)];
    const int lt = tile - q.ci->tile_base;
    q.tx = lt % q.ci->tiles_x;
    q.ty = lt / q.ci->tiles_x;
    q.ox = (float)(q.tx * TW);
    q.oy = (float)(q.ty * TH);
    const int sx = 8 * (warp % SquareShape<TW, TH>::wx), sy = 8 * (warp / SquareShape<TW, TH>::wx);
    q.lx = sx + 2 * (lane & 3);
    q.ly = sy + (lane >> 2);
    q.pxc = make_float2((float)q.lx + 0.5f, (float)q.lx + 1.5f);
    q.pyc = (float)q.ly + 0.5f;
    q.bx0 = (float)sx + 0.5f; q.bx1 = (float)sx + 7.5f;
    q.by0 = (float)sy + 0.5f; q.by1 = (float)sy + 7.5f;
    return q;
}

// Base-2 exponent of a staged entry (e0 = (u, v, A, k), Ds = scaled D) at the
// lane's pixel pair; every kernel evaluates it through this function, so all
// take the same decisions.  e returns dx + k dy.
__device__ __forceinline__ float2 pair_power(float4 e0, float Ds, float2 pxc, float pyc, float2 &dx, float &dy,
                                             float2 &e)
{
    dx = __fadd2_rn(pxc, f2(-e0.x));
    dy = __fadd_rn(pyc, -e0.y);
    const float kdy = __fmul_rn(e0.w, dy);
    const float ddy = __fmul_rn(__fmul_rn(Ds, dy), dy);
    e = __fadd2_rn(dx, f2(kdy));
    return __ffma2_rn(f2(e0.z), __fmul2_rn(e, e), f2(ddy));
}

// ---- forward --------------------------------------------------------------
//
// Front to back over the visited entries of each batch; a warp stops once all
// of its pixels have (T would drop below T_min), with no block barrier.

template <int TW, int TH>
__global__ void __launch_bounds__(SquareShape<TW, TH>::threads)
    render_fwd_kernel(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
                      const float4 *__restrict__ rd0, const float4 *__restrict__ rd1, const float4 *__restrict__ rd2,
                      const CamTable *__restrict__ ctp, RenderConsts rc, float *__restrict__ rgb_out,
                      float *__restrict__ T_out, float *__restrict__ T_ws, uint32_t *__restrict__ n_contrib,
                      uint32_t *__restrict__ tile_last)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    constexpr int kWarps = SquareShape<TW, TH>::warps;
    __shared__ float4 s0[kWarps][32];
    __shared__ float4 s1[kWarps][32];
    __shared__ float s2[kWarps][32];
    const CamTable &ct = *ctp;
    if ((int)blockIdx.x >= ct.total_tiles) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SquareGeom q = square_geom<TW, TH>(ct, blockIdx.x, warp, lane);
    const CamInfo &cam = *q.ci;
    const uint2 rg = ranges[blockIdx.x];
    const int start = (int)rg.x, end = (int)rg.y;
    const int px = q.tx * TW + q.lx, py = q.ty * TH + q.ly;
    float2 T = f2(1.f), Cr = f2(0.f), Cg = f2(0.f), Cb = f2(0.f);
    uint32_t last0 = 0, last1 = 0;
    bool dn0 = px >= cam.width || py >= cam.height, dn1 = px + 1 >= cam.width || py >= cam.height;
    for (int b = start; b < end && !__all_sync(0xffffffffu, dn0 && dn1); b += 32) {
        const int cnt = min(32, end - b);
        bool visit = false;
        if (lane < cnt) {
            const uint32_t r = vals[b + lane];
            const float4 r0 = rd0[r], r1 = rd1[r], r2 = rd2[r];
            const float op = r2.w != 0.f ? 0.f : r1.y; // a record marked culled composites nowhere
            const float4 e0 = stage_e0_at(r0, r2, q.ox, q.oy);
            s0[warp][lane] = e0;
            s1[warp][lane] = make_float4(stage_D(r1), op, r1.z, r1.w);
            s2[warp][lane] = r2.x;
            visit = square_visit(r0.z, r0.w, r1.x, op, rc.alpha_min, e0.x, e0.y, q.bx0, q.bx1, q.by0, q.by1);
        }
        unsigned m = __ballot_sync(0xffffffffu, visit);
        __syncwarp();
        while (m != 0u) {
            const int jj = __ffs(m) - 1; // front to back
            m &= m - 1u;
            const float4 p0 = s0[warp][jj];
            const float4 p1 = s1[warp][jj];
            const uint32_t pos = (uint32_t)(b - start + jj + 1);
            float2 dx, e;
            float dy;
            const float2 pw = pair_power(p0, p1.x, q.pxc, q.pyc, dx, dy, e);
            float2 G;
            const float2 al = pair_alpha(pw, p1.y, rc.alpha_max, G);
            const float2 tT = __ffma2_rn(make_float2(-T.x, -T.y), al, T); // T (1 - alpha)
            const bool ok0 = !dn0 && al.x >= rc.alpha_min, ok1 = !dn1 && al.y >= rc.alpha_min;
            const bool st0 = ok0 && tT.x < rc.T_min, st1 = ok1 && tT.y < rc.T_min;
            const bool c0 = ok0 && !st0, c1 = ok1 && !st1;
            dn0 = dn0 || st0;
            dn1 = dn1 || st1;
            const float2 ae = make_float2(c0 ? al.x : 0.f, c1 ? al.y : 0.f); // skipped fragments add nothing
            const float2 w = __fmul2_rn(ae, T);
            Cr = __ffma2_rn(w, f2(p1.z), Cr);
            Cg = __ffma2_rn(w, f2(p1.w), Cg);
            Cb = __ffma2_rn(w, f2(s2[warp][jj]), Cb);
            T = __ffma2_rn(make_float2(-T.x, -T.y), ae, T);
            last0 = c0 ? pos : last0;
            last1 = c1 ? pos : last1;
            if (__all_sync(0xffffffffu, dn0 && dn1)) break;
        }
        __syncwarp();
    }
    const long long np = (long long)cam.width * cam.height;
    float *img = rgb_out + 3 * cam.pix_base;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (px + h >= cam.width || py >= cam.height) continue;
        const float Tk = h ? T.y : T.x;
        const long long pix = (long long)py * cam.width + px + h;
        img[pix] = (h ? Cr.y : Cr.x) + Tk * rc.bg[0];
        img[np + pix] = (h ? Cg.y : Cg.x) + Tk * rc.bg[1];
        img[2 * np + pix] = (h ? Cb.y : Cb.x) + Tk * rc.bg[2];
        const long long gp = cam.pix_base + pix;
        if (T_out) T_out[gp] = Tk;
        T_ws[gp] = Tk;
        n_contrib[gp] = h ? last1 : last0;
    }
    // the tile's largest n_contrib, where the adjoint's reverse walk starts
    const unsigned wl = __reduce_max_sync(0xffffffffu, max(last0, last1));
    if (lane == 0 && wl != 0u) atomicMax(&tile_last[blockIdx.x], wl);
}

template <int TW, int TH> static void fwd_launch(gs_workspace *ws, cudaStream_t st, float *rgb, float *T_out)
{
    launch_pdl(render_fwd_kernel<TW, TH>, ws->cams.total_tiles, SquareShape<TW, TH>::threads, 0, st,
        ws->ranges, ws->tval[ws->tile_buf], ws->rd0, ws->rd1, ws->rd2, ws->d_cams, ws->rc, rgb, T_out, ws->T_final,
        ws->n_contrib, ws->tile_last);
}

cudaError_t launch_render_fwd(gs_workspace *ws, cudaStream_t st, float *rgb, float *T_out)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    kt_begin(ws, GS_KT_RENDER_FWD, st);
    switch (tile_shape_id(ws->cams.tile_w, ws->cams.tile_h)) {
    case 0: fwd_launch<16, 16>(ws, st, rgb, T_out); break;
    case 1: fwd_launch<32, 8>(ws, st, rgb, T_out); break;
    case 2: fwd_launch<8, 32>(ws, st, rgb, T_out); break;
    case 3: fwd_launch<32, 16>(ws, st, rgb, T_out); break;
    case 4: fwd_launch<16, 8>(ws, st, rgb, T_out); break;
    case 5: fwd_launch<8, 16>(ws, st, rgb, T_out); break;
    default: return cudaErrorInvalidValue;
    }
    kt_end(ws, GS_KT_RENDER_FWD, st);
    note_launch();
    return cudaGetLastError();
}

// ---- backward ---------------------------------------------------------------
//
// Each warp owns an 8 x 8 pixel square of the tile -- lane l the horizontal
// pixel pair (2 (l % 4), l / 4) of it, packed as FP32x2 -- and walks the
// tile's list back to front on its own, in batches that start at the tile's
// last contribution (the forward's largest n_contrib of the tile), visiting
// only entries in front of its own pixels' last contribution and recovering T
// by T / (1 - alpha) from the final transmittance.  It stages each batch of 32
// entries itself (one per lane), so no block-wide barrier holds it while
// another warp of the tile has more to do; the staging lane also tests its
// entry's alpha footprint against the warp's square, and one ballot gives the
// batch's entries the warp must visit.  Per visited entry the warp's nine slot
// values are one warp reduction; the warps' partials of a batch are summed in
// warp order by the warp that finishes that batch last (shared-memory arrival
// counters) and written to the entries' slots.  A warp may run up to
// kBwdBufs - 1 batches ahead of the slowest warp of its tile; its wait for a
// partial buffer is bounded.

constexpr int kBwdBatch = 32; // entries staged per batch of the reverse walk (one per lane)
constexpr int kBwdBufs = 3;   // partial buffers: batches a warp may run ahead, plus one


struct BwdRenderArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float4 *rd0, *rd1, *rd2;
    const uint32_t *inst_off;
    const uint2 *rect;
    const float *T_final;
    const uint32_t *n_contrib;
    const uint32_t *tile_last; // largest n_contrib of each tile (the forward's)
    const float *dL_drgb;
    float *slots;
    DevCounters *ctr; // fragments += sum of the tile's n_contrib; composited += composited pairs
};

template <int TW, int TH>
__global__ void __launch_bounds__(SquareShape<TW, TH>::threads, SquareShape<TW, TH>::bwd_min_blocks)
    render_bwd_kernel(BwdRenderArgs a, const CamTable *__restrict__ ctp, RenderConsts rc)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    constexpr int kWarps = SquareShape<TW, TH>::warps, kRT = SquareShape<TW, TH>::threads;
    __shared__ float4 s0[kWarps][kBwdBatch];
    __shared__ float4 s1[kWarps][kBwdBatch];
    __shared__ float s2[kWarps][kBwdBatch];
    __shared__ unsigned long long s_slot[kWarps][kBwdBatch];
    __shared__ float s_part[kBwdBufs][kWarps][kBwdBatch][kSlotFloats];
    __shared__ unsigned s_mask[kBwdBufs][kWarps]; // entries of the batch each warp visited
    __shared__ int s_arrive[kBwdBufs], s_done[kBwdBufs];
    const CamTable &ct = *ctp;
    if ((int)blockIdx.x >= ct.total_tiles) return;
    const int tile = blockIdx.x;
    const CamInfo &ci = ct.c[camera_of_tile(ct, tile)];
    const int lt = tile - ci.tile_base;
    const int tx = lt % ci.tiles_x, ty = lt / ci.tiles_x;
    const float ox = (float)(tx * TW), oy = (float)(ty * TH);
    const uint2 rg = a.ranges[blockIdx.x];
    const int start = (int)rg.x, end = (int)rg.y;
    // the reverse walk starts after the tile's last contribution (the forward's
    // largest n_contrib); entries behind it carry zero gradient
    const int last = start + min((int)a.tile_last[blockIdx.x], end - start);
    if (threadIdx.x < kBwdBufs) { s_arrive[threadIdx.x] = 0; s_done[threadIdx.x] = 0; }
    __syncthreads(); // the only block barrier: the arrival counters are set
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool red_own = red9_owner(lane);
    const int red_q = red9_index(lane);
    // the warp's square and the lane's pixel pair (tile-local)
    const int sx = 8 * (warp % SquareShape<TW, TH>::wx), sy = 8 * (warp / SquareShape<TW, TH>::wx);
    const int lx = sx + 2 * (lane & 3), ly = sy + (lane >> 2);
    const float2 pxc = make_float2((float)lx + 0.5f, (float)lx + 1.5f);
    const float pyc = (float)ly + 0.5f;
    const float bx0 = (float)sx + 0.5f, bx1 = (float)sx + 7.5f, by0 = (float)sy + 0.5f, by1 = (float)sy + 7.5f;

    // per-pixel state of the pair: dL/dC (g), T (from T_final back to each
    // fragment's own), S = colour composited behind the current fragment plus
    // the background seen through T_final
    float2 T = f2(1.f), g0 = f2(0.f), g1 = f2(0.f), g2 = f2(0.f);
    int nc0 = 0, nc1 = 0;
    {
        const long long np = (long long)ci.width * ci.height;
        const float *gimg = a.dL_drgb + 3 * ci.pix_base;
        const int px = tx * TW + lx, py = ty * TH + ly;
        float t[2] = {1.f, 1.f}, c0[2] = {0.f, 0.f}, c1[2] = {0.f, 0.f}, c2[2] = {0.f, 0.f};
        int n[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (px + h < ci.width && py < ci.height) {
                const long long pix = (long long)py * ci.width + px + h;
                c0[h] = gimg[pix]; c1[h] = gimg[np + pix]; c2[h] = gimg[2 * np + pix];
                t[h] = a.T_final[ci.pix_base + pix];
                n[h] = (int)a.n_contrib[ci.pix_base + pix];
            }
        }
        T = make_float2(t[0], t[1]);
        g0 = make_float2(c0[0], c0[1]); g1 = make_float2(c1[0], c1[1]); g2 = make_float2(c2[0], c2[1]);
        nc0 = n[0]; nc1 = n[1];
    }
    float2 S0 = __fmul2_rn(T, f2(rc.bg[0])), S1 = __fmul2_rn(T, f2(rc.bg[1])), S2 = __fmul2_rn(T, f2(rc.bg[2]));
    const int wmax = __reduce_max_sync(0xffffffffu, max(nc0, nc1));
    {
        const unsigned f = __reduce_add_sync(0xffffffffu, (unsigned)(nc0 + nc1));
        if (lane == 0 && f) atomicAdd(&a.ctr->fragments, (unsigned long long)f);
    }
    int ncomp = 0;
    int b = 0;
    for (int hi = last; hi > start; hi -= kBwdBatch, b++) {
        const int lo = max(start, hi - kBwdBatch);
        const int cnt = hi - lo;
        const int buf = b % kBwdBufs;
        bool visit = false;
        if (lane < cnt) {
            const uint32_t r = a.vals[lo + lane];
            const float4 r0 = a.rd0[r], r1 = a.rd1[r], r2 = a.rd2[r];
            const float op = r2.w != 0.f ? 0.f : r1.y; // a record marked culled composites nowhere
            const float4 e0 = stage_e0_at(r0, r2, ox, oy);
            s0[warp][lane] = e0;
            s1[warp][lane] = make_float4(stage_D(r1), op, r1.z, r1.w);
            s2[warp][lane] = r2.x;
            s_slot[warp][lane] = slot_of(a.inst_off, a.rect, r, tx, ty);
            // visited: in front of the warp's last contribution, alpha footprint meeting the square
            visit = lo + lane - start < wmax &&
                    square_visit(r0.z, r0.w, r1.x, op, rc.alpha_min, e0.x, e0.y, bx0, bx1, by0, by1);
        }
        const unsigned vmask = __ballot_sync(0xffffffffu, visit);
        // the partial buffer of this batch is free once batch b - kBwdBufs has been summed
        if (b >= kBwdBufs) {
            const int want = b / kBwdBufs;
            unsigned long long spins = 0;
            bool gave_up = false;
            while (*(volatile int *)&s_done[buf] < want) {
                if (++spins > kSpinLimit) { gave_up = true; break; }
                __nanosleep(32);
            }
            if (__any_sync(0xffffffffu, gave_up)) {
                if (lane == 0) set_error(a.ctr, GS_ERR_TIMEOUT, kSiteRender);
                return;
            }
            __threadfence_block();
        }
        __syncwarp();
        float (*part)[kSlotFloats] = s_part[buf][warp];
        if (lane == 0) s_mask[buf][warp] = vmask;
        for (unsigned m = vmask; m != 0u;) {
            const int jj = 31 - __clz(m); // back to front
            m ^= 1u << jj;
            const int j = lo + jj - start; // position in the tile list
            const float4 p0 = s0[warp][jj];
            const float4 p1 = s1[warp][jj];
            // the forward's own exponent and alpha (the same operations, the same bits)
            float2 dx, e;
            float dy;
            const float2 pw = pair_power(p0, p1.x, pxc, pyc, dx, dy, e);
            float2 G;
            const float2 al = pair_alpha(pw, p1.y, rc.alpha_max, G);
            // composited pixels: in front of the pixel's last contribution, alpha >= alpha_min
            const bool m0 = j < nc0 && al.x >= rc.alpha_min;
            const bool m1 = j < nc1 && al.y >= rc.alpha_min;
            float r = 0.f;
            if (__any_sync(0xffffffffu, m0 || m1)) {
                // Every lane runs the adjoint (no divergent branch): a pixel that does not
                // composite here has aT = dG = 0, so it adds exact zeros and keeps its T and S
                // (all terms stay finite: alpha <= alpha_max < 1).
                ncomp += (int)m0 + (int)m1;
                const float cb = s2[warp][jj];
                const float2 inv = make_float2(rcp_approx(1.f - al.x), rcp_approx(1.f - al.y));
                const float2 Tj = __fmul2_rn(T, inv); // transmittance in front of this fragment
                const float2 aTf = __fmul2_rn(al, Tj);
                const float2 aT = make_float2(m0 ? aTf.x : 0.f, m1 ? aTf.y : 0.f);
                // dL/dalpha = Tj (g . c) - (g . S) / (1 - alpha)
                const float2 gc = __ffma2_rn(g2, f2(cb), __ffma2_rn(g1, f2(p1.w), __fmul2_rn(g0, f2(p1.z))));
                const float2 gS = __ffma2_rn(g2, S2, __ffma2_rn(g1, S1, __fmul2_rn(g0, S0)));
                const float2 dal = __ffma2_rn(make_float2(-inv.x, -inv.y), gS, __fmul2_rn(Tj, gc));
                S0 = __ffma2_rn(aT, f2(p1.z), S0);
                S1 = __ffma2_rn(aT, f2(p1.w), S1);
                S2 = __ffma2_rn(aT, f2(cb), S2);
                T = make_float2(m0 ? Tj.x : T.x, m1 ? Tj.y : T.y);
                // dL/do of the pixel = G dL/dalpha, zero where alpha is clamped at alpha_max;
                // dL/dpower = o times it
                const float2 dGf = __fmul2_rn(G, dal);
                const float2 dG = make_float2(m0 && al.x < rc.alpha_max ? dGf.x : 0.f,
                                              m1 && al.y < rc.alpha_max ? dGf.y : 0.f);
                // The slot takes dG-weighted moments of the pixel offsets: the record's
                // opacity and conic factors of the mean and conic gradients are applied
                // once per record, when its slots are summed (slot_grads_from_moments).
                float v[kSlotFloats];
                const float sG = dG.x + dG.y;
                const float2 gx = __fmul2_rn(dG, dx);
                v[0] = fmaf(dG.y, e.y, dG.x * e.x);   // sum dG e,  e = dx + k dy
                v[1] = sG * dy;                       // sum dG dy
                v[2] = fmaf(gx.y, dx.y, gx.x * dx.x); // sum dG dx^2
                v[3] = (gx.x + gx.y) * dy;            // sum dG dx dy
                v[4] = v[1] * dy;                     // sum dG dy^2
                v[5] = sG;                            // dL/do = sum dG
                v[6] = fmaf(aT.y, g0.y, aT.x * g0.x); // dL/dc = sum alpha T dL/dC
                v[7] = fmaf(aT.y, g1.y, aT.x * g1.x);
                v[8] = fmaf(aT.y, g2.y, aT.x * g2.x);
                r = warp_reduce9(v, lane);
            }
            if (red_own) part[jj][red_q] = r;
        }
        // arrive; the last warp of the tile to finish this batch sums it
        __syncwarp();
        int arrived = 0;
        if (lane == 0) {
            __threadfence_block();
            arrived = atomicAdd(&s_arrive[buf], 1);
        }
        arrived = __shfl_sync(0xffffffffu, arrived, 0);
        if (arrived == kWarps - 1) {
            __threadfence_block();
            // lane jj sums entry jj over the warps that visited it, in warp order
            if (lane < cnt) {
                float sum[kSlotFloats];
#pragma unroll
                for (int q = 0; q < kSlotFloats; q++) sum[q] = 0.f;
#pragma unroll
                for (int w = 0; w < kWarps; w++) {
                    if ((s_mask[buf][w] >> lane) & 1u) {
#pragma unroll
                        for (int q = 0; q < kSlotFloats; q++) sum[q] += s_part[buf][w][lane][q];
                    }
                }
                float *dst = a.slots + s_slot[warp][lane] * kSlotFloats;
#pragma unroll
                for (int q = 0; q < kSlotFloats; q++) dst[q] = sum[q];
            }
            __syncwarp();
            if (lane == 0) {
                s_arrive[buf] = 0;
                __threadfence_block();
                *(volatile int *)&s_done[buf] = b / kBwdBufs + 1;
            }
        }
    }
    // entries after the tile's last contribution carry zero gradient
    for (int s = last + threadIdx.x; s < end; s += kRT) {
        float *dst = a.slots + slot_of(a.inst_off, a.rect, a.vals[s], tx, ty) * kSlotFloats;
#pragma unroll
        for (int k = 0; k < kSlotFloats; k++) dst[k] = 0.f;
    }
    const unsigned f = __reduce_add_sync(0xffffffffu, (unsigned)ncomp);
    if (lane == 0 && f) atomicAdd(&a.ctr->composited, (unsigned long long)f);
}

cudaError_t launch_render_bwd(gs_workspace *ws, cudaStream_t st, const float *dL_drgb)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    BwdRenderArgs a;
    a.ranges = ws->ranges; a.vals = ws->tval[ws->tile_buf]; a.rd0 = ws->rd0; a.rd1 = ws->rd1; a.rd2 = ws->rd2;
    a.inst_off = ws->inst_off; a.rect = ws->rect; a.T_final = ws->T_final; a.n_contrib = ws->n_contrib;
    a.tile_last = ws->tile_last;
    a.dL_drgb = dL_drgb; a.slots = ws->slots; a.ctr = ws->ctr;
    const unsigned grid = (unsigned)ws->cams.total_tiles;
    kt_begin(ws, GS_KT_RENDER_BWD, st);
    switch (tile_shape_id(ws->cams.tile_w, ws->cams.tile_h)) {
    case 0: launch_pdl(render_bwd_kernel<16, 16>, grid, SquareShape<16, 16>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 1: launch_pdl(render_bwd_kernel<32, 8>, grid, SquareShape<32, 8>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 2: launch_pdl(render_bwd_kernel<8, 32>, grid, SquareShape<8, 32>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 3: launch_pdl(render_bwd_kernel<32, 16>, grid, SquareShape<32, 16>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 4: launch_pdl(render_bwd_kernel<16, 8>, grid, SquareShape<16, 8>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 5: launch_pdl(render_bwd_kernel<8, 16>, grid, SquareShape<8, 16>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    default: return cudaErrorInvalidValue;
    }
    kt_end(ws, GS_KT_RENDER_BWD, st);
    note_launch();
    return cudaGetLastError();
}

// ---- importance sweep (colourless forward), alone or fused with the forward ----
//
// The walk of render_fwd_kernel on warp squares with every record at its own
// opacity (the importance sweep never applies the Cull column it recomputes):
// per visited entry the warp sums alpha T and the count of composited pixels
// over its lanes, and, as in the adjoint, the warps' partials of a batch are
// summed in warp order by the warp that finishes the batch last and written to
// the entries' importance slots.  Every warp goes through every batch of the
// tile (staging only the slot ids once its pixels have stopped), so every
// slot is written.  With FWD the same walk also composites the training image
// (records marked culled composite nowhere in it): one evaluation of each
// entry's alpha serves both, the image, T and n_contrib equal
// render_fwd_kernel's and the slots this kernel's alone, bit for bit.

constexpr int kImpBufs = 3; // partial buffers: batches a warp may run ahead, plus one

struct ImpArgs {
    const uint2 *ranges;
    const uint32_t *vals;
    const float4 *rd0, *rd1, *rd2;
    const uint32_t *inst_off;
    const uint2 *rect;
    float2 *slots;         // [I]: alpha-weight (float), composited pixels (uint32 bits)
    DevCounters *ctr;
    // FWD only
    float *rgb_out, *T_out, *T_ws;
    uint32_t *n_contrib;
    uint32_t *tile_last;   // the tile's largest n_contrib (atomic max; zeroed by the binning)
};

template <int TW, int TH, bool FWD>
__global__ void __launch_bounds__(SquareShape<TW, TH>::threads, SquareShape<TW, TH>::imp_min_blocks)
    importance_raster_kernel(ImpArgs a, const CamTable *__restrict__ ctp, RenderConsts rc)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    constexpr int kWarps = SquareShape<TW, TH>::warps;
    __shared__ float4 s0[kWarps][32];
    __shared__ float4 s1[kWarps][32]; // (D scaled, own opacity, training opacity, blue)
    __shared__ float2 s3[FWD ? kWarps : 1][32]; // (red, green) of the training image
    __shared__ unsigned long long s_slot[kWarps][32];
    __shared__ float2 s_part[kImpBufs][kWarps][32];
    __shared__ unsigned s_mask[kImpBufs][kWarps];
    __shared__ int s_arrive[kImpBufs], s_done[kImpBufs];
    const CamTable &ct = *ctp;
    if ((int)blockIdx.x >= ct.total_tiles) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SquareGeom q = square_geom<TW, TH>(ct, blockIdx.x, warp, lane);
    const CamInfo &cam = *q.ci;
    const uint2 rg = a.ranges[blockIdx.x];
    const int start = (int)rg.x, end = (int)rg.y;
    const int px = q.tx * TW + q.lx, py = q.ty * TH + q.ly;
    const bool out0 = px >= cam.width || py >= cam.height, out1 = px + 1 >= cam.width || py >= cam.height;
    float2 Ti = f2(1.f);             // importance transmittance
    bool di0 = out0, di1 = out1;     // importance walk stopped
    float2 T = f2(1.f), Cr = f2(0.f), Cg = f2(0.f), Cb = f2(0.f); // training image (FWD)
    uint32_t last0 = 0, last1 = 0;
    bool dn0 = out0, dn1 = out1;
    if (threadIdx.x < kImpBufs) { s_arrive[threadIdx.x] = 0; s_done[threadIdx.x] = 0; }
    __syncthreads();
    int bi = 0;
    for (int b = start; b < end; b += 32, bi++) {
        const int cnt = min(32, end - b);
        const int buf = bi % kImpBufs;
        const bool wdone = __all_sync(0xffffffffu, di0 && di1 && (!FWD || (dn0 && dn1)));
        bool visit = false;
        if (lane < cnt) {
            const uint32_t r = a.vals[b + lane];
            s_slot[warp][lane] = slot_of(a.inst_off, a.rect, r, q.tx, q.ty);
            if (!wdone) {
                const float4 r0 = a.rd0[r], r1 = a.rd1[r], r2 = a.rd2[r];
                const float4 e0 = stage_e0_at(r0, r2, q.ox, q.oy);
                s0[warp][lane] = e0;
                s1[warp][lane] = make_float4(stage_D(r1), r1.y, r2.w != 0.f ? 0.f : r1.y, r2.x);
                if (FWD) s3[FWD ? warp : 0][lane] = make_float2(r1.z, r1.w);
                // the record's own opacity: the training opacity is the same or 0
                visit = square_visit(r0.z, r0.w, r1.x, r1.y, rc.alpha_min, e0.x, e0.y, q.bx0, q.bx1, q.by0, q.by1);
            }
        }
        const unsigned vmask = __ballot_sync(0xffffffffu, visit);
        // the partial buffer of this batch is free once batch bi - kImpBufs has been summed
        if (bi >= kImpBufs) {
            const int want = bi / kImpBufs;
            unsigned long long spins = 0;
            bool gave_up = false;
            while (*(volatile int *)&s_done[buf] < want) {
                if (++spins > kSpinLimit) { gave_up = true; break; }
                __nanosleep(32);
            }
            if (__any_sync(0xffffffffu, gave_up)) {
                if (lane == 0) set_error(a.ctr, GS_ERR_TIMEOUT, kSiteRender);
                return;
            }
            __threadfence_block();
        }
        __syncwarp();
        if (lane == 0) s_mask[buf][warp] = vmask;
        for (unsigned m = vmask; m != 0u;) {
            const int jj = __ffs(m) - 1; // front to back
            m &= m - 1u;
            const float4 p0 = s0[warp][jj];
            const float4 p1 = s1[warp][jj];
            float2 dx, e;
            float dy;
            const float2 pw = pair_power(p0, p1.x, q.pxc, q.pyc, dx, dy, e);
            float2 G;
            const float2 al = pair_alpha(pw, p1.y, rc.alpha_max, G);
            if (FWD && p1.z != 0.f) { // the training image: render_fwd_kernel's update
                const uint32_t pos = (uint32_t)(b - start + jj + 1);
                const float2 tT = __ffma2_rn(make_float2(-T.x, -T.y), al, T);
                const bool ok0 = !dn0 && al.x >= rc.alpha_min, ok1 = !dn1 && al.y >= rc.alpha_min;
                const bool st0 = ok0 && tT.x < rc.T_min, st1 = ok1 && tT.y < rc.T_min;
                const bool c0 = ok0 && !st0, c1 = ok1 && !st1;
                dn0 = dn0 || st0;
                dn1 = dn1 || st1;
                const float2 ae = make_float2(c0 ? al.x : 0.f, c1 ? al.y : 0.f);
                const float2 w = __fmul2_rn(ae, T);
                const float2 rgc = s3[FWD ? warp : 0][jj];
                Cr = __ffma2_rn(w, f2(rgc.x), Cr);
                Cg = __ffma2_rn(w, f2(rgc.y), Cg);
                Cb = __ffma2_rn(w, f2(p1.w), Cb);
                T = __ffma2_rn(make_float2(-T.x, -T.y), ae, T);
                last0 = c0 ? pos : last0;
                last1 = c1 ? pos : last1;
            }
            // the importance sweep
            const float2 tT = __ffma2_rn(make_float2(-Ti.x, -Ti.y), al, Ti);
            const bool ok0 = !di0 && al.x >= rc.alpha_min, ok1 = !di1 && al.y >= rc.alpha_min;
            const bool st0 = ok0 && tT.x < rc.T_min, st1 = ok1 && tT.y < rc.T_min;
            const bool c0 = ok0 && !st0, c1 = ok1 && !st1;
            di0 = di0 || st0;
            di1 = di1 || st1;
            const float2 ae = make_float2(c0 ? al.x : 0.f, c1 ? al.y : 0.f);
            const float2 w = __fmul2_rn(ae, Ti);
            float wv = w.x + w.y;
            uint32_t av = (uint32_t)c0 + (uint32_t)c1;
            Ti = __ffma2_rn(make_float2(-Ti.x, -Ti.y), ae, Ti);
            if (__any_sync(0xffffffffu, av != 0)) {
                wv = warp_sum_f(wv);
                av = __reduce_add_sync(0xffffffffu, av);
            }
            if (lane == 0) s_part[buf][warp][jj] = make_float2(wv, __uint_as_float(av));
        }
        // arrive; the last warp of the tile to finish this batch sums it
        __syncwarp();
        int arrived = 0;
        if (lane == 0) {
            __threadfence_block();
            arrived = atomicAdd(&s_arrive[buf], 1);
        }
        arrived = __shfl_sync(0xffffffffu, arrived, 0);
        if (arrived == kWarps - 1) {
            __threadfence_block();
            if (lane < cnt) {
                float ws = 0.f;
                uint32_t as = 0;
#pragma unroll
                for (int w = 0; w < kWarps; w++)
                    if ((s_mask[buf][w] >> lane) & 1u) {
                        const float2 pv = s_part[buf][w][lane];
                        ws += pv.x;
                        as += __float_as_uint(pv.y);
                    }
                a.slots[s_slot[warp][lane]] = make_float2(ws, __uint_as_float(as));
            }
            __syncwarp();
            if (lane == 0) {
                s_arrive[buf] = 0;
                __threadfence_block();
                *(volatile int *)&s_done[buf] = bi / kImpBufs + 1;
            }
        }
    }
    if (FWD) {
        const long long np = (long long)cam.width * cam.height;
        float *img = a.rgb_out + 3 * cam.pix_base;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (px + h >= cam.width || py >= cam.height) continue;
            const float Tk = h ? T.y : T.x;
            const long long pix = (long long)py * cam.width + px + h;
            img[pix] = (h ? Cr.y : Cr.x) + Tk * rc.bg[0];
            img[np + pix] = (h ? Cg.y : Cg.x) + Tk * rc.bg[1];
            img[2 * np + pix] = (h ? Cb.y : Cb.x) + Tk * rc.bg[2];
            const long long gp = cam.pix_base + pix;
            if (a.T_out) a.T_out[gp] = Tk;
            a.T_ws[gp] = Tk;
            a.n_contrib[gp] = h ? last1 : last0;
        }
        const unsigned wl = __reduce_max_sync(0xffffffffu, max(last0, last1));
        if (lane == 0 && wl != 0u) atomicMax(&a.tile_last[blockIdx.x], wl);
    }
}

template <bool FWD> static cudaError_t importance_launch(gs_workspace *ws, cudaStream_t st, const ImpArgs &a)
{
    const unsigned grid = (unsigned)ws->cams.total_tiles;
    switch (tile_shape_id(ws->cams.tile_w, ws->cams.tile_h)) {
    case 0: launch_pdl(importance_raster_kernel<16, 16, FWD>, grid, SquareShape<16, 16>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 1: launch_pdl(importance_raster_kernel<32, 8, FWD>, grid, SquareShape<32, 8>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 2: launch_pdl(importance_raster_kernel<8, 32, FWD>, grid, SquareShape<8, 32>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 3: launch_pdl(importance_raster_kernel<32, 16, FWD>, grid, SquareShape<32, 16>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 4: launch_pdl(importance_raster_kernel<16, 8, FWD>, grid, SquareShape<16, 8>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    case 5: launch_pdl(importance_raster_kernel<8, 16, FWD>, grid, SquareShape<8, 16>::threads, 0, st, a, ws->d_cams, ws->rc); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

static ImpArgs importance_args(gs_workspace *ws)
{
    ImpArgs a{};
    a.ranges = ws->ranges; a.vals = ws->tval[ws->tile_buf]; a.rd0 = ws->rd0; a.rd1 = ws->rd1; a.rd2 = ws->rd2;
    a.inst_off = ws->inst_off; a.rect = ws->rect; a.slots = ws->imp_slots; a.ctr = ws->ctr;
    return a;
}

cudaError_t launch_importance_raster(gs_workspace *ws, cudaStream_t st)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    kt_begin(ws, GS_KT_IMPORTANCE, st);
    cudaError_t e = importance_launch<false>(ws, st, importance_args(ws));
    if (e != cudaSuccess) return e;
    kt_end(ws, GS_KT_IMPORTANCE, st);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_render_fwd_importance(gs_workspace *ws, cudaStream_t st, float *rgb, float *T_out)
{
    if (ws->cams.total_tiles == 0) return cudaSuccess;
    ImpArgs a = importance_args(ws);
    a.rgb_out = rgb; a.T_out = T_out; a.T_ws = ws->T_final; a.n_contrib = ws->n_contrib; a.tile_last = ws->tile_last;
    kt_begin(ws, GS_KT_RENDER_FWD, st);
    cudaError_t e = importance_launch<true>(ws, st, a);
    if (e != cudaSuccess) return e;
    kt_end(ws, GS_KT_RENDER_FWD, st);
    note_launch();
    return cudaGetLastError();
}

} // namespace gs
