// preprocess.cu -- view gate, EWA projection, SH colour (forward) and the
// adjoint of the projection and colour (backward).
//
// Forward, one thread per Gaussian, all cameras of the call:
//   LOD gate (Sec. 3.3, Eq. 1-2) and Cull column (Eq. 3), near cull,
//   Sigma = R(q) S S^T R(q)^T, Sigma' = J W Sigma W^T J^T + dilation I,
//   conic, radius ceil(3 sqrt(lambda_max)), tile rectangle (App. A),
//   degree-3 SH colour, sigmoid opacity.
// Active (Gaussian, camera) pairs become records, compacted in (Gaussian,
// camera) order by a single-pass decoupled look-back scan, so later stages
// only touch active work.  The integer decisions (gate, near cull, det sign,
// radius, rectangle) are computed with explicitly rounded FP32 operations
// (no contraction) so they are reproducible on any FP32 IEEE implementation.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

#define FMUL __fmul_rn
#define FADD __fadd_rn
#define FSUB __fsub_rn
#define FDIV __fdiv_rn
#define FSQRT __fsqrt_rn

struct GaussPtrs {
    const float *mean, *log_scale, *quat, *opacity_logit, *sh;
    const uint8_t *lod;
    long long n;
};

// One projected (Gaussian, camera) pair.  The mean is kept to about 48 bits
// as u + u_lo (u = the float nearest the double-float mean): pixel
// coordinates near 2000 carry only 1e-4 px in one float, and at the edge of a
// small footprint that is a relative 1e-3 of alpha.  The conic is held as
// A (x + k y)^2 + D y^2, whose terms stay accurate for long thin footprints at
// any orientation (the A, B, C form loses them to cancellation).
struct Proj {
    float u, v, u_lo, v_lo; // projected mean
    float A, k, D;          // conic: A = c / det, k = -b / c, D = 1 / c
    float depth;
    int radius;
    int x0, y0, x1, y1;
};

// SH basis, degree 3, real form with the Condon-Shortley phase, m = -l..l,
// evaluated as homogeneous polynomials of the unit direction (x, y, z).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16])
{
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = C0;
    Y[1] = -C1 * y;
    Y[2] = C1 * z;
    Y[3] = -C1 * x;
    Y[4] = C2a * x * y;
    Y[5] = -C2a * y * z;
    Y[6] = C2b * (2.f * zz - xx - yy);
    Y[7] = -C2a * x * z;
    Y[8] = C2c * (xx - yy);
    Y[9] = -C3a * y * (3.f * xx - yy);
    Y[10] = C3b * x * y * z;
    Y[11] = -C3c * y * (4.f * zz - xx - yy);
    Y[12] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -C3c * x * (4.f * zz - xx - yy);
    Y[14] = C3e * z * (xx - yy);
    Y[15] = -C3a * x * (xx - 3.f * yy);
}

// Gradient of each basis polynomial with respect to (x, y, z).
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float dY[16][3])
{
    const float C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[0][0] = 0.f; dY[0][1] = 0.f; dY[0][2] = 0.f;
    dY[1][0] = 0.f; dY[1][1] = -C1; dY[1][2] = 0.f;
    dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = C1;
    dY[3][0] = -C1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    dY[4][0] = C2a * y; dY[4][1] = C2a * x; dY[4][2] = 0.f;
    dY[5][0] = 0.f; dY[5][1] = -C2a * z; dY[5][2] = -C2a * y;
    dY[6][0] = -2.f * C2b * x; dY[6][1] = -2.f * C2b * y; dY[6][2] = 4.f * C2b * z;
    dY[7][0] = -C2a * z; dY[7][1] = 0.f; dY[7][2] = -C2a * x;
    dY[8][0] = 2.f * C2c * x; dY[8][1] = -2.f * C2c * y; dY[8][2] = 0.f;
    dY[9][0] = -C3a * 6.f * x * y; dY[9][1] = -C3a * (3.f * xx - 3.f * yy); dY[9][2] = 0.f;
    dY[10][0] = C3b * y * z; dY[10][1] = C3b * x * z; dY[10][2] = C3b * x * y;
    dY[11][0] = C3c * 2.f * x * y; dY[11][1] = -C3c * (4.f * zz - xx - 3.f * yy); dY[11][2] = -C3c * 8.f * y * z;
    dY[12][0] = -C3d * 6.f * x * z; dY[12][1] = -C3d * 6.f * y * z; dY[12][2] = C3d * (6.f * zz - 3.f * xx - 3.f * yy);
    dY[13][0] = -C3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = C3c * 2.f * x * y; dY[13][2] = -C3c * 8.f * x * z;
    dY[14][0] = C3e * 2.f * x * z; dY[14][1] = -C3e * 2.f * y * z; dY[14][2] = C3e * (xx - yy);
    dY[15][0] = -C3a * (3.f * xx - 3.f * yy); dY[15][1] = C3a * 6.f * x * y; dY[15][2] = 0.f;
}

// g = sum_k c_k grad Y_k(x, y, z): the gradients of sh_basis_grad weighted
// and summed, without materialising the 16 x 3 table.
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, const float c[16], float g[3])
{
    float dY[16][3];
    sh_basis_grad(x, y, z, dY);
    g[0] = g[1] = g[2] = 0.f;
#pragma unroll
    for (int k = 1; k < 16; k++) {
        g[0] = fmaf(c[k], dY[k][0], g[0]);
        g[1] = fmaf(c[k], dY[k][1], g[1]);
        g[2] = fmaf(c[k], dY[k][2], g[2]);
    }
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) { return x < lo ? lo : (x > hi ? hi : x); }

// Distance LOD gate (Sec. 3.3, Eq. 1-2) in its squared-distance form:
// keep level l iff l == 0, or l <= Lmax and |mu - c|^2 <= (d0 f^(0.5 - l))^2,
// which is l <= clamp(round(log_f(d0 / d)), 0, Lmax) with half-away rounding.
// thr2: the squared-distance thresholds of RenderConsts::lod_thr2 (a copy in
// shared memory, so the level indexes it without a local-memory copy).
__device__ __forceinline__ bool lod_pass(const float m[3], int lod, const CamInfo &cam, const RenderConsts &rc,
                                         const float *thr2)
{
    if (!rc.lod_enable || lod == 0) return true;
    if (lod > rc.lod_Lmax) return false;
    const float dx = FSUB(m[0], cam.campos[0]), dy = FSUB(m[1], cam.campos[1]), dz = FSUB(m[2], cam.campos[2]);
    const float d2 = FADD(FADD(FMUL(dx, dx), FMUL(dy, dy)), FMUL(dz, dz));
    return d2 <= thr2[lod];
}

// lod_pass for a mean that may still move by up to D (deferred Adam steps):
// passes whenever some point within D of m passes.  D = 0 is lod_pass.
__device__ __forceinline__ bool lod_pass_margin(const float m[3], int lod, const CamInfo &cam, const RenderConsts &rc,
                                                const float *thr2, const float *thr, float D)
{
    if (D == 0.f) return lod_pass(m, lod, cam, rc, thr2);
    if (!rc.lod_enable || lod == 0) return true;
    if (lod > rc.lod_Lmax) return false;
    const float dx = m[0] - cam.campos[0], dy = m[1] - cam.campos[1], dz = m[2] - cam.campos[2];
    const float lim = 1.0001f * (thr[lod] + D);
    return dx * dx + dy * dy + dz * dz <= lim * lim;
}

// Depth row of camera_point alone (the near-plane test).
__device__ __forceinline__ void camera_z(const float m[3], const CamInfo &cam, float &tz, float &ez)
{
    const float *R = cam.R;
    tz = FADD(FADD(FADD(FMUL(R[6], m[0]), FMUL(R[7], m[1])), FMUL(R[8], m[2])), cam.t[2]);
    const float mag = fabsf(R[6] * m[0]) + fabsf(R[7] * m[1]) + fabsf(R[8] * m[2]) + fabsf(cam.t[2]);
    ez = 8.f * 5.9604645e-8f * mag + 1e-30f;
}

// Camera-space mean in float, for the gate only, with a bound on its distance
// from the double-float value the projection uses: three additions and
// the final rounding each err by at most 2^-24 of a partial sum bounded by
// sum_k |R_jk m_k| + |t_j|.
__device__ __forceinline__ void camera_point(const float m[3], const CamInfo &cam, float t[3], float err[3])
{
    const float *R = cam.R;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        t[j] = FADD(FADD(FADD(FMUL(R[3 * j], m[0]), FMUL(R[3 * j + 1], m[1])), FMUL(R[3 * j + 2], m[2])), cam.t[j]);
        const float mag = fabsf(R[3 * j] * m[0]) + fabsf(R[3 * j + 1] * m[1]) + fabsf(R[3 * j + 2] * m[2]) +
                          fabsf(cam.t[j]);
        err[j] = 8.f * 5.9604645e-8f * mag + 1e-30f;
    }
}

// Double-float arithmetic: a value carried as hi + lo, two floats (~48
// significant bits).  A product of floats splits exactly with an FMA
// (Dekker's product), a sum exactly with Knuth's two-sum; every operation is
// an explicitly rounded IEEE one, never contracted.  On GB300 the FP32 pipes
// run these many times faster than the FP64 unit runs doubles.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_prod(float a, float b)
{
    const float p = FMUL(a, b);
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = FADD(a, b), bb = FSUB(s, a);
    return {s, FADD(FSUB(a, FSUB(s, bb)), FSUB(b, bb))};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    const float s = FADD(a, b);
    return {s, FSUB(b, FSUB(s, a))};
}

// Camera-space mean x_cam = R x + t in double-float: the three products
// exactly, the three sums by two-sum, their error terms gathered in float
// and folded in once (relative error ~2^-46 of the largest term).
__device__ __forceinline__ void camera_point_df(const float m[3], const CamInfo &cam, DF t[3])
{
    const float *R = cam.R;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const DF p0 = two_prod(R[3 * j], m[0]), p1 = two_prod(R[3 * j + 1], m[1]), p2 = two_prod(R[3 * j + 2], m[2]);
        const DF s1 = two_sum(p0.hi, p1.hi);
        const DF s2 = two_sum(s1.hi, p2.hi);
        const DF s3 = two_sum(s2.hi, cam.t[j]);
        const float lo = FADD(FADD(FADD(FADD(FADD(p0.lo, p1.lo), s1.lo), p2.lo), s2.lo), s3.lo);
        t[j] = fast_two_sum(s3.hi, lo);
    }
}

// f * x / z + c in double-float (x, z double-float, f, c float): the quotient
// x.hi / z.hi corrected by the exactly formed remainder, then the product and
// the sum split exactly; returns the normalised pair (hi = the float nearest).
__device__ __forceinline__ DF df_project(float f, DF x, DF z, float c)
{
    const float iz = 1.f / z.hi;
    const float q = FMUL(x.hi, iz);
    const DF qz = two_prod(q, z.hi);
    const float r = FSUB(FADD(FSUB(FSUB(x.hi, qz.hi), qz.lo), x.lo), FMUL(q, z.lo)); // x - q z
    const float ql = FMUL(r, iz);
    const DF a = two_prod(f, q);
    const DF b = two_sum(a.hi, c);
    return fast_two_sum(b.hi, FADD(FADD(a.lo, FMUL(f, ql)), b.lo));
}

// Conservative screen test run before the exact covariance: false only when
// the exact tile rectangle is certainly empty.  lambda_max(Sigma') <=
// |J|_F^2 max_j s_j^2 + dilation, |J|_F^2 <= jbound / tz^2 (clamped Jacobian),
// plus sqrt(0.1) for the clamp of the discriminant, with margins for the
// rounding of this float evaluation (t, e from camera_point).
__device__ __forceinline__ bool maybe_on_screen(const float t[3], const float e[3], float smax, const CamInfo &cam,
                                                int tw, int th, const RenderConsts &rc)
{
    // approximate reciprocals and square root (a few ulp): the margins below
    // (1 % on lambda, 2 px on the radius, 1e-5 |u|) dwarf them
    const float tzl = t[2] - e[2]; // lower bound of the exact depth
    const float itz = __fdividef(1.f, t[2]), itzl = __fdividef(1.f, tzl);
    const float u = cam.fx * t[0] * itz + cam.cx, v = cam.fy * t[1] * itz + cam.cy;
    const float lam = 1.01f * (cam.jbound * itzl * itzl * smax * smax + rc.dilation) + 0.33f;
    const float R = 3.003f * (lam * rsqrtf(lam)) + 2.f;
    // |d(tx / tz)| <= (e_x + |tx / tz| e_z) / tz_low
    const float du = 1.01f * cam.fx * (e[0] + fabsf(t[0] * itz) * e[2]) * itzl;
    const float dv = 1.01f * cam.fy * (e[1] + fabsf(t[1] * itz) * e[2]) * itzl;
    const float ru = R + du + 1e-5f * fabsf(u), rv = R + dv + 1e-5f * fabsf(v);
    const bool off = u + ru < 0.f || u - ru >= (float)(cam.tiles_x * tw) || v + rv < 0.f ||
                     v - rv >= (float)(cam.tiles_y * th);
    return !(tzl > 1e-6f) || !off;
}

// Exact projection of one Gaussian into one camera, from the double-float
// camera-space mean td (the near plane already passed).  Every float
// operation is one explicitly rounded IEEE operation in a fixed order, so the
// integer results (radius, rectangle, depth key) are reproducible bit for bit.
// Sigma' = V V^T + dilation I with V = T M (T = J W, M = R(q) diag(s)); its
// determinant comes from the Cauchy-Binet identity (sum of the squared 2x2
// minors of V, plus the dilation terms), which is free of the cancellation of
// a c - b^2.  Returns false when the tile rectangle is empty.
__device__ __forceinline__ bool project_gaussian(const float ls[3], const float qin[4], const DF td[3],
                                                 const CamInfo &cam, int tile_w, int tile_h, const RenderConsts &rc,
                                                 Proj &o)
{
    const float *R = cam.R;
    const float tx = td[0].hi, ty = td[1].hi, tz = td[2].hi;
    float qw = qin[0], qx = qin[1], qy = qin[2], qz = qin[3];
    float qn = FSQRT(FADD(FADD(FADD(FMUL(qw, qw), FMUL(qx, qx)), FMUL(qy, qy)), FMUL(qz, qz)));
    qw = FDIV(qw, qn); qx = FDIV(qx, qn); qy = FDIV(qy, qn); qz = FDIV(qz, qn);
    float Q[3][3];
    Q[0][0] = FSUB(1.f, FMUL(2.f, FADD(FMUL(qy, qy), FMUL(qz, qz))));
    Q[0][1] = FMUL(2.f, FSUB(FMUL(qx, qy), FMUL(qw, qz)));
    Q[0][2] = FMUL(2.f, FADD(FMUL(qx, qz), FMUL(qw, qy)));
    Q[1][0] = FMUL(2.f, FADD(FMUL(qx, qy), FMUL(qw, qz)));
    Q[1][1] = FSUB(1.f, FMUL(2.f, FADD(FMUL(qx, qx), FMUL(qz, qz))));
    Q[1][2] = FMUL(2.f, FSUB(FMUL(qy, qz), FMUL(qw, qx)));
    Q[2][0] = FMUL(2.f, FSUB(FMUL(qx, qz), FMUL(qw, qy)));
    Q[2][1] = FMUL(2.f, FADD(FMUL(qy, qz), FMUL(qw, qx)));
    Q[2][2] = FSUB(1.f, FMUL(2.f, FADD(FMUL(qx, qx), FMUL(qy, qy))));
    float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M[i][j] = FMUL(Q[i][j], s[j]);

    const float fx = cam.fx, fy = cam.fy;
    float limx = FMUL(rc.fov_clamp, FDIV((float)cam.width, FMUL(2.f, fx)));
    float limy = FMUL(rc.fov_clamp, FDIV((float)cam.height, FMUL(2.f, fy)));
    float xr = FDIV(tx, tz), yr = FDIV(ty, tz);
    float txc = FMUL(clampf(xr, -limx, limx), tz);
    float tyc = FMUL(clampf(yr, -limy, limy), tz);
    float tz2 = FMUL(tz, tz);
    float j00 = FDIV(fx, tz), j02 = FDIV(-FMUL(fx, txc), tz2);
    float j11 = FDIV(fy, tz), j12 = FDIV(-FMUL(fy, tyc), tz2);
    float T[2][3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T[0][k] = FADD(FMUL(j00, R[k]), FMUL(j02, R[6 + k]));
        T[1][k] = FADD(FMUL(j11, R[3 + k]), FMUL(j12, R[6 + k]));
    }
    float V[2][3];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            V[r][k] = FADD(FADD(FMUL(T[r][0], M[0][k]), FMUL(T[r][1], M[1][k])), FMUL(T[r][2], M[2][k]));
    const float dil = rc.dilation;
    float s00 = FADD(FADD(FMUL(V[0][0], V[0][0]), FMUL(V[0][1], V[0][1])), FMUL(V[0][2], V[0][2]));
    float s01 = FADD(FADD(FMUL(V[0][0], V[1][0]), FMUL(V[0][1], V[1][1])), FMUL(V[0][2], V[1][2]));
    float s11 = FADD(FADD(FMUL(V[1][0], V[1][0]), FMUL(V[1][1], V[1][1])), FMUL(V[1][2], V[1][2]));
    float a = FADD(s00, dil), b = s01, c = FADD(s11, dil);
    float m01 = FSUB(FMUL(V[0][0], V[1][1]), FMUL(V[0][1], V[1][0]));
    float m02 = FSUB(FMUL(V[0][0], V[1][2]), FMUL(V[0][2], V[1][0]));
    float m12 = FSUB(FMUL(V[0][1], V[1][2]), FMUL(V[0][2], V[1][1]));
    float det = FADD(FADD(FADD(FADD(FMUL(m01, m01), FMUL(m02, m02)), FMUL(m12, m12)), FMUL(dil, FADD(s00, s11))),
                     FMUL(dil, dil));
    if (!(det > 0.f)) return false;
    float mid = FMUL(0.5f, FADD(a, c));
    float disc = FSUB(FMUL(mid, mid), det);
    if (disc < 0.1f) disc = 0.1f;
    float lam = FADD(mid, FSQRT(disc));
    float ext = FMUL(3.f, FSQRT(lam));
    int radius = (int)ceilf(ext);
    const DF ud = df_project(fx, td[0], td[2], cam.cx), vd = df_project(fy, td[1], td[2], cam.cy);
    float u = ud.hi, v = vd.hi;
    float rr = (float)radius, tw = (float)tile_w, th = (float)tile_h;
    int x0 = (int)floorf(FDIV(FSUB(u, rr), tw)), y0 = (int)floorf(FDIV(FSUB(v, rr), th));
    int x1 = (int)floorf(FDIV(FADD(u, rr), tw)) + 1, y1 = (int)floorf(FDIV(FADD(v, rr), th)) + 1;
    x0 = min(max(x0, 0), cam.tiles_x); x1 = min(max(x1, 0), cam.tiles_x);
    y0 = min(max(y0, 0), cam.tiles_y); y1 = min(max(y1, 0), cam.tiles_y);
    if (x1 <= x0 || y1 <= y0) return false;
    o.u = u; o.v = v;
    o.u_lo = ud.lo;
    o.v_lo = vd.lo;
    o.A = FDIV(c, det); o.k = FDIV(-b, c); o.D = FDIV(1.f, c);
    o.depth = tz;
    o.radius = radius;
    o.x0 = x0; o.y0 = y0; o.x1 = x1; o.y1 = y1;
    return true;
}

struct PreOut {
    uint32_t *rec_g, *tt, *dkey;
    uint16_t *rec_cam;
    float4 *rd0, *rd1, *rd2;
    uint2 *rect;
    uint8_t *clampm;
    uint32_t *cand_g;
    unsigned long long *cand_mask;
    uint32_t *gate_g;              // [N] block-strided candidates of the gate's first pass
    unsigned long long *gate_mask; // [N]
    const float *drift;            // [2][N] drift bounds (mean, log-scale) of deferred Adam steps, or NULL
    uint32_t *rec_first;           // first record of each Gaussian, ~0 when it has none
    unsigned long long *lb_status; // word 0: ticket
    DevCounters *ctr;
    long long max_records;
    const uint32_t *cull;
    long long cull_words;
};

struct GaussLoad {
    float m[3], ls[3], q[4];
    float smax;
    bool have_shape;
};

__device__ __forceinline__ void load_shape(const GaussPtrs &g, long long i, GaussLoad &L)
{
    if (L.have_shape) return;
    L.ls[0] = g.log_scale[3 * i]; L.ls[1] = g.log_scale[3 * i + 1]; L.ls[2] = g.log_scale[3 * i + 2];
    const float4 q = *reinterpret_cast<const float4 *>(g.quat + 4 * i); // 16-byte aligned rows
    L.q[0] = q.x; L.q[1] = q.y; L.q[2] = q.z; L.q[3] = q.w;
    L.smax = expf(fmaxf(L.ls[0], fmaxf(L.ls[1], L.ls[2])));
    L.have_shape = true;
}

constexpr int kGateItems = 4; // Gaussians per thread of the gate kernel: 1024 per block
static_assert((kGateItems * 8) % 32 == 0, "the gate ranks its (item, warp) counts with one warp");

__device__ __forceinline__ bool cull_bit(const PreOut &o, int c, long long i)
{
    return o.cull ? ((o.cull[c * o.cull_words + (i >> 5)] >> (i & 31)) & 1u) : false;
}

// The cameras of the call, copied from the device table into shared memory
// once per block (every Gaussian reads them).
__device__ __forceinline__ void stage_cameras(const CamTable &ct, CamInfo *s_cams)
{
    const int words = ct.n * (int)(sizeof(CamInfo) / sizeof(int));
    const int *src = reinterpret_cast<const int *>(ct.c);
    int *dst = reinterpret_cast<int *>(s_cams);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    __syncthreads();
}

// Stage 1, streaming over all Gaussians: the view gate (LOD, Cull), the near
// plane and the conservative screen test -- everything that is cheap and
// rejects most of a city scene -- producing an order-preserving list of
// candidate Gaussians with a bit per camera that may still be active.
// The Gaussians come in chunks of kGateChunk; thread t of the block that takes
// chunk c owns Gaussians c*kGateChunk + k*256 + t.  What every test needs
// (mean, level, mean drift) streams in: either as bulk copies of the chunk into
// shared memory, double-buffered so that the next chunk is in flight while this
// one is tested (persistent blocks), or, where the arrays are not 16-byte
// aligned, as plain loads issued up front.  The log-scales (and their drift)
// are read only for the few Gaussians past the LOD and near tests.
constexpr int kGateChunk = 256 * kGateItems;

struct GateShared {
    CamInfo cams[GS_MAX_CAMERAS];
    float thr2[kMaxLod + 1];
    float thr[kMaxLod + 1];  // sqrt of thr2, for the drift margin
    unsigned cnt[kGateItems][8];
    unsigned total;
    uint16_t surv[8][kGateChunk / 8]; // one camera: each warp's items past the LOD and near tests
    unsigned hit[8][kGateItems];      // one camera: (warp, item) bits by lane of the candidates
};

// One chunk as the bulk copies leave it in shared memory.
struct GateStage {
    float mean[3 * kGateChunk];
    float drift[kGateChunk];     // drift bound of the mean (deferred Adam steps)
    uint8_t lod[kGateChunk];
};

struct GateItems {
    float mx[kGateItems], my[kGateItems], mz[kGateItems];
    int lod[kGateItems];
    uint32_t cw[kGateItems]; // the Cull word of camera 0 (GS_CULL_DROP)
    float dm[kGateItems];    // drift bound of the mean, 0 when up to date
};

__device__ __forceinline__ void gate_load_plain(const GaussPtrs &g, const PreOut &o, const RenderConsts &rc,
                                                long long block0, GateItems &it)
{
    const long long n = g.n;
#pragma unroll
    for (int k = 0; k < kGateItems; k++) {
        const long long i = block0 + k * 256 + threadIdx.x;
        const bool ok = i < n;
        it.mx[k] = ok ? g.mean[3 * i] : 0.f;
        it.my[k] = ok ? g.mean[3 * i + 1] : 0.f;
        it.mz[k] = ok ? g.mean[3 * i + 2] : 0.f;
        it.lod[k] = (ok && rc.lod_enable && g.lod) ? (int)g.lod[i] : 0;
        it.cw[k] = (ok && rc.cull_enable == GS_CULL_DROP && o.cull) ? o.cull[i >> 5] : 0u;
        it.dm[k] = (ok && o.drift) ? o.drift[i] : 0.f;
    }
}

// A whole chunk (every item below n) from its staged copy.
__device__ __forceinline__ void gate_load_staged(const GateStage &sg, const GaussPtrs &g, const PreOut &o,
                                                 const RenderConsts &rc, long long block0, GateItems &it)
{
#pragma unroll
    for (int k = 0; k < kGateItems; k++) {
        const int j = k * 256 + threadIdx.x;
        const long long i = block0 + j;
        it.mx[k] = sg.mean[3 * j];
        it.my[k] = sg.mean[3 * j + 1];
        it.mz[k] = sg.mean[3 * j + 2];
        it.lod[k] = (rc.lod_enable && g.lod) ? (int)sg.lod[j] : 0;
        it.cw[k] = (rc.cull_enable == GS_CULL_DROP && o.cull) ? o.cull[i >> 5] : 0u;
        it.dm[k] = o.drift ? sg.drift[j] : 0.f;
    }
}

// Issues the bulk copies of chunk c (a whole chunk) into sg, completing on bar.
__device__ __forceinline__ void gate_issue(GateStage &sg, unsigned long long *bar, const GaussPtrs &g,
                                           const PreOut &o, const RenderConsts &rc, long long c)
{
    const bool lod = rc.lod_enable && g.lod, drift = o.drift != nullptr;
    const unsigned bytes = 12u * kGateChunk + (lod ? kGateChunk : 0u) + (drift ? 4u * kGateChunk : 0u);
    mbar_expect_tx(bar, bytes);
    bulk_copy_g2s(sg.mean, g.mean + 3 * kGateChunk * c, 12u * kGateChunk, bar);
    if (lod) bulk_copy_g2s(sg.lod, g.lod + kGateChunk * c, kGateChunk, bar);
    if (drift) bulk_copy_g2s(sg.drift, o.drift + kGateChunk * c, 4u * kGateChunk, bar);
}

// sg: the chunk's staged copy (bulk copies), or nullptr (plain loads)
template <bool kOneCam>
__device__ __forceinline__ void gate_masks(const GaussPtrs &g, const PreOut &o, const CamTable &ct,
                                           const RenderConsts &rc, GateShared &sh, long long block0,
                                           const GateItems &it, const GateStage *sg,
                                           unsigned long long mask[kGateItems])
{
    const int ncam = ct.n, tw = ct.tile_w, th = ct.tile_h;
    const long long n = g.n;
    if (kOneCam) {
        // one camera: the LOD, Cull and near tests of every item; the few items
        // still in (a twentieth of a city scene) are compacted per warp, in
        // item order, and the warp's lanes take them together through their
        // shape (log-scales, their drift) and the screen test
        const CamInfo &cam = sh.cams[0];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned lt = (1u << lane) - 1u;
        unsigned nsurv = 0;
#pragma unroll
        for (int k = 0; k < kGateItems; k++) {
            const long long i = block0 + k * 256 + threadIdx.x;
            const float m[3] = {it.mx[k], it.my[k], it.mz[k]};
            const bool lod_ok = lod_pass_margin(m, it.lod[k], cam, rc, sh.thr2, sh.thr, it.dm[k]);
            const bool culled = rc.cull_enable == GS_CULL_DROP && ((it.cw[k] >> (i & 31)) & 1u);
            float tz, ez;
            camera_z(m, cam, tz, ez);
            const bool near_ok = tz + ez + it.dm[k] > rc.znear; // the exact near test is the projection's
            const bool in = i < n && lod_ok && !culled && near_ok;
            const unsigned b = __ballot_sync(0xffffffffu, in);
            if (in) sh.surv[warp][nsurv + __popc(b & lt)] = (uint16_t)(k * 256 + threadIdx.x);
            nsurv += __popc(b);
        }
        if (lane < kGateItems) sh.hit[warp][lane] = 0u;
        __syncwarp();
        for (unsigned q = lane; q < nsurv; q += 32) {
            const int j = sh.surv[warp][q]; // chunk-local item: k * 256 + warp * 32 + its lane
            const long long i = block0 + j;
            float m[3], dm;
            if (sg) {
                m[0] = sg->mean[3 * j]; m[1] = sg->mean[3 * j + 1]; m[2] = sg->mean[3 * j + 2];
                dm = o.drift ? sg->drift[j] : 0.f;
            } else {
                m[0] = g.mean[3 * i]; m[1] = g.mean[3 * i + 1]; m[2] = g.mean[3 * i + 2];
                dm = o.drift ? o.drift[i] : 0.f;
            }
            const float dl = o.drift ? o.drift[n + i] : 0.f;
            const float lsmax = fmaxf(g.log_scale[3 * i], fmaxf(g.log_scale[3 * i + 1], g.log_scale[3 * i + 2])) + dl;
            float t[3], te[3];
            camera_point(m, cam, t, te);
            te[0] += dm; te[1] += dm; te[2] += dm;
            const float smax = 1.0001f * __expf(lsmax);
            if (maybe_on_screen(t, te, smax, cam, tw, th, rc)) atomicOr(&sh.hit[warp][j >> 8], 1u << (j & 31));
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kGateItems; k++) mask[k] = (sh.hit[warp][k] >> lane) & 1u;
    } else {
#pragma unroll
        for (int k = 0; k < kGateItems; k++) {
            mask[k] = 0;
            const long long i = block0 + k * 256 + threadIdx.x;
            if (i >= n) continue;
            const float m[3] = {it.mx[k], it.my[k], it.mz[k]};
            const float dm = it.dm[k];
            float smax = -1.f;
            for (int c = 0; c < ncam; c++) {
                const CamInfo &cam = sh.cams[c];
                if (!lod_pass_margin(m, it.lod[k], cam, rc, sh.thr2, sh.thr, dm)) continue;
                if (rc.cull_enable == GS_CULL_DROP && (c == 0 ? ((it.cw[k] >> (i & 31)) & 1u) : cull_bit(o, c, i)))
                    continue;
                float t[3], te[3];
                camera_point(m, cam, t, te);
                te[0] += dm; te[1] += dm; te[2] += dm;
                if (!(t[2] + te[2] > rc.znear)) continue; // the exact near test is the projection's
                if (smax < 0.f) {
                    const float dl = o.drift ? o.drift[n + i] : 0.f;
                    smax = 1.0001f * __expf(fmaxf(g.log_scale[3 * i], fmaxf(g.log_scale[3 * i + 1],
                                                                            g.log_scale[3 * i + 2])) + dl);
                }
                if (maybe_on_screen(t, te, smax, cam, tw, th, rc)) mask[k] |= 1ull << c;
            }
        }
    }
}

// Block-local order of the candidates: item (k, thread) precedes (k', thread')
// iff k < k', or k == k' and thread < thread'.  Returns the block's count.
__device__ __forceinline__ unsigned gate_ranks(const unsigned long long mask[kGateItems], unsigned bal[kGateItems],
                                               GateShared &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kGateItems; k++) {
        bal[k] = __ballot_sync(0xffffffffu, mask[k] != 0);
        if (lane == 0) sh.cnt[k][warp] = __popc(bal[k]);
    }
    __syncthreads();
    if (threadIdx.x < 32) { // warp 0: exclusive scan of the (item, warp) counts in (k, warp) order
        constexpr int kPer = kGateItems * 8 / 32; // consecutive counts per lane
        unsigned c[kPer], sum = 0;
#pragma unroll
        for (int p = 0; p < kPer; p++) {
            const int e = lane * kPer + p;
            c[p] = sh.cnt[e >> 3][e & 7];
            sum += c[p];
        }
        unsigned x = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        unsigned run = x - sum;
#pragma unroll
        for (int p = 0; p < kPer; p++) {
            const int e = lane * kPer + p;
            sh.cnt[e >> 3][e & 7] = run;
            run += c[p];
        }
        if (lane == 31) sh.total = x;
    }
    __syncthreads();
    return sh.total;
}

// The gate runs as count, scan, gather: no block waits on another (an
// in-order look-back chain makes the blocks of a wave, which all finish their
// counts together, wait for one another); each chunk's candidates go first to
// the chunk's own range, and the gather moves only candidates.
// kBulk: persistent blocks, chunk c, c + gridDim.x, ...; the chunks copied
// whole (all but a partial last one) arrive by bulk copies one chunk ahead.  A
// copy that does not complete within spin_limit waits sets GS_ERR_TIMEOUT; the
// block then waits (again bounded) for its copies in flight, records empty
// counts for its remaining chunks and returns.
template <bool kOneCam, bool kBulk>
__global__ void __launch_bounds__(256, kOneCam ? 4 : 3) gate_count_kernel(GaussPtrs g, PreOut o,
                                                                         const CamTable *__restrict__ ctp,
                                                                         RenderConsts rc, unsigned long long *counts,
                                                                         unsigned long long spin_limit)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ GateShared sh;
    __shared__ __align__(16) GateStage stage[kBulk ? 2 : 1];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_fail;
    const long long nchunks = (g.n + kGateChunk - 1) / kGateChunk;
    const long long nwhole = kBulk ? g.n / kGateChunk : 0; // chunks that come by bulk copy
    if (threadIdx.x == 0) {
#pragma unroll
        for (int l = 0; l <= kMaxLod; l++) {
            sh.thr2[l] = rc.lod_thr2[l];
            sh.thr[l] = sqrtf(rc.lod_thr2[l]);
        }
        s_fail = 0;
        if (kBulk) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_init_fence();
            if ((long long)blockIdx.x < nwhole) gate_issue(stage[0], &bar[0], g, o, rc, blockIdx.x);
        }
    }
    stage_cameras(*ctp, sh.cams); // ends with a block barrier
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int k = 0;
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x, k++) {
        const long long block0 = c * kGateChunk;
        GateItems it;
        if (kBulk && c < nwhole) {
            const long long cn = c + gridDim.x;
            // the next chunk's copy, into the buffer the previous chunk used
            if (threadIdx.x == 0 && cn < nwhole) gate_issue(stage[(k + 1) & 1], &bar[(k + 1) & 1], g, o, rc, cn);
            if (!mbar_wait(&bar[k & 1], (unsigned)(k >> 1) & 1u, spin_limit)) {
                set_error(o.ctr, GS_ERR_TIMEOUT, kSitePreprocess);
                s_fail = 1;
            }
            __syncthreads();
            if (s_fail) {
                if (threadIdx.x == 0) { // the copies still in flight land before the block's memory is released
                    mbar_wait(&bar[k & 1], (unsigned)(k >> 1) & 1u, spin_limit);
                    if (cn < nwhole) mbar_wait(&bar[(k + 1) & 1], (unsigned)((k + 1) >> 1) & 1u, spin_limit);
                }
                for (long long r = c + threadIdx.x * (long long)gridDim.x; r < nchunks; r += 256ll * gridDim.x)
                    counts[r] = 0;
                return;
            }
            gate_load_staged(stage[k & 1], g, o, rc, block0, it);
        } else {
            gate_load_plain(g, o, rc, block0, it);
        }
        unsigned long long mask[kGateItems];
        unsigned bal[kGateItems];
        gate_masks<kOneCam>(g, o, *ctp, rc, sh, block0, it, (kBulk && c < nwhole) ? &stage[k & 1] : nullptr, mask);
        const unsigned total = gate_ranks(mask, bal, sh);
        if (threadIdx.x == 0) counts[c] = total;
        // the chunk's candidates, in order, at the start of its own range
#pragma unroll
        for (int q = 0; q < kGateItems; q++) {
            if (mask[q]) {
                const long long pos = block0 + sh.cnt[q][warp] + __popc(bal[q] & lt);
                o.gate_g[pos] = (uint32_t)(block0 + q * 256 + threadIdx.x);
                o.gate_mask[pos] = mask[q];
            }
        }
        __syncthreads(); // the staged chunk and the ranks are free for the next chunk
    }
}

// Exclusive scan of the block counts in place (one block); the total is the
// candidate count.
__global__ void __launch_bounds__(1024) gate_scan_kernel(unsigned long long *counts, long long nblocks,
                                                         DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ unsigned long long s[1024];
    const long long per = (nblocks + 1023) / 1024;
    const long long b0 = (long long)threadIdx.x * per;
    unsigned long long acc = 0;
    for (long long b = b0; b < b0 + per && b < nblocks; b++) acc += counts[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned long long v = threadIdx.x >= off ? s[threadIdx.x - off] : 0ull;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = s[threadIdx.x] - acc; // exclusive prefix of this chunk
    for (long long b = b0; b < b0 + per && b < nblocks; b++) {
        const unsigned long long c = counts[b];
        counts[b] = run;
        run += c;
    }
    if (threadIdx.x == 1023) ctr->n_candidates = s[1023];
}

// Moves each block's candidates from its own range to their place in the
// ordered list (offsets from gate_scan_kernel).
__global__ void __launch_bounds__(256) gate_gather_kernel(PreOut o, const unsigned long long *offsets,
                                                          long long nblocks, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const long long b = blockIdx.x;
    const unsigned long long off = offsets[b];
    const unsigned long long end = b + 1 < nblocks ? offsets[b + 1] : ctr->n_candidates;
    const long long src = b * 256 * kGateItems;
    for (unsigned long long t = threadIdx.x; off + t < end; t += 256) {
        o.cand_g[off + t] = o.gate_g[src + t];
        o.cand_mask[off + t] = o.gate_mask[src + t];
    }
}

// Stage 2, one thread per candidate (converged warps): the exact FP32
// projection decides which cameras are active; the records are compacted in
// (Gaussian, camera) order with a look-back scan and written with their
// conic, colour, opacity, rectangle and depth key.
struct RecOut {
    float4 rd0, rd1, rd2;
    uint2 rect;
    uint32_t tt, dkey;
    uint8_t clm;
};

// The record of Gaussian i (loaded as L, opacity op) in camera cam from its
// (passing) projection p: the colour from the SH coefficients, the rectangle
// and the depth key.
__device__ __forceinline__ RecOut make_record(const GaussPtrs &g, long long i, const GaussLoad &L, float op,
                                              const CamInfo &cam, const Proj &p, const RenderConsts &rc, bool marked)
{
    const float dx = L.m[0] - cam.campos[0], dy = L.m[1] - cam.campos[1], dz = L.m[2] - cam.campos[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    float Y[16];
    sh_basis(dx * inv, dy * inv, dz * inv, Y);
    float col[3] = {0.f, 0.f, 0.f};
    uint8_t clm = 0;
    const float4 *shv = reinterpret_cast<const float4 *>(g.sh + 48 * i); // [16][3], 16-byte aligned
#pragma unroll
    for (int v4 = 0; v4 < 12; v4++) {
        const float4 c4 = shv[v4];
        const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int flat = 4 * v4 + e; // coefficient flat / 3, channel flat % 3
            col[flat % 3] = fmaf(cc[e], Y[flat / 3], col[flat % 3]);
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float acc = col[ch] + 0.5f;
        if (acc < 0.f) { acc = 0.f; clm |= (uint8_t)(1u << ch); }
        col[ch] = acc;
    }
    RecOut o;
    o.rd0 = make_float4(p.u, p.v, p.A, p.k);
    o.rd1 = make_float4(p.D, op, col[0], col[1]);
    o.rd2 = make_float4(col[2], p.u_lo, p.v_lo, marked ? 1.f : 0.f);
    o.rect = make_uint2((uint32_t)p.x0 | ((uint32_t)p.y0 << 16), (uint32_t)p.x1 | ((uint32_t)p.y1 << 16));
    o.tt = (uint32_t)((p.x1 - p.x0) * (p.y1 - p.y0));
    o.dkey = __float_as_uint(p.depth);
    o.clm = clm;
    return o;
}

__device__ __forceinline__ void store_record(const PreOut &o, unsigned long long r, long long i, int c,
                                             const RecOut &q)
{
    o.rec_g[r] = (uint32_t)i;
    o.rec_cam[r] = (uint16_t)c;
    o.rd0[r] = q.rd0;
    o.rd1[r] = q.rd1;
    o.rd2[r] = q.rd2;
    o.rect[r] = q.rect;
    o.tt[r] = q.tt;
    o.dkey[r] = q.dkey;
    o.clampm[r] = q.clm;
}

// kOneCam: a candidate has at most one record, which is computed (colour
// included, from the projection that decided it) before the block's scan and
// look-back, so the look-back of one warp does not leave the others idle in
// front of the colour's loads.  Blocks of kProjThreads take chunks of as many
// candidates.
constexpr int kProjThreads = 128;
template <bool kOneCam>
__global__ void __launch_bounds__(kProjThreads) project_kernel(GaussPtrs g, PreOut o, const CamTable *__restrict__ ctp,
                                                               RenderConsts rc)
{
    constexpr int kNW = kProjThreads / 32;
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    const CamTable &ct = *ctp;
    __shared__ CamInfo s_cams[GS_MAX_CAMERAS];
    __shared__ float s_thr2[kMaxLod + 1];
    __shared__ unsigned s_bid;
    __shared__ unsigned long long s_warp[kNW];
    __shared__ unsigned long long s_base;
    const unsigned long long ncand = o.ctr->n_candidates;
    const int tw = ct.tile_w, th = ct.tile_h;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int l = 0; l <= kMaxLod; l++) s_thr2[l] = rc.lod_thr2[l];
    }
    stage_cameras(ct, s_cams);
    // persistent blocks: each takes the next chunk of candidates (tickets in
    // order, so every look-back waits only on chunks already being processed)
    for (;;) {
    if (threadIdx.x == 0) s_bid = atomicAdd((unsigned *)o.lb_status, 1u);
    __syncthreads();
    const unsigned bid = s_bid;
    if ((unsigned long long)bid * kProjThreads >= ncand) return;
    const unsigned long long j = (unsigned long long)bid * kProjThreads + threadIdx.x;
    GaussLoad L;
    L.have_shape = false;
    long long i = 0;
    unsigned long long act = 0;
    float op = 0.f;
    Proj p_one; // one camera: the projection of the active record
    if (j < ncand) {
        i = o.cand_g[j];
        const unsigned long long cm = o.cand_mask[j];
        L.m[0] = g.mean[3 * i]; L.m[1] = g.mean[3 * i + 1]; L.m[2] = g.mean[3 * i + 2];
        load_shape(g, i, L);
        const float ol = g.opacity_logit[i];
        const int lod = (rc.lod_enable && g.lod) ? (int)g.lod[i] : 0;
        for (unsigned long long mm = cm; mm; mm &= mm - 1) {
            const int c = __ffsll((long long)mm) - 1;
            // the exact LOD decision (the gate's is widened for Gaussians with deferred steps)
            if (!lod_pass(L.m, lod, s_cams[c], rc, s_thr2)) continue;
            DF td[3];
            camera_point_df(L.m, s_cams[c], td);
            if (!(td[2].hi > rc.znear)) continue;
            Proj p;
            if (project_gaussian(L.ls, L.q, td, s_cams[c], tw, th, rc, p)) {
                act |= 1ull << c;
                if (kOneCam) p_one = p;
            }
        }
        op = 1.f / (1.f + expf(-ol));
    }
    const unsigned long long cnt = __popcll(act);
    // GS_CULL_MARK: records of the cameras whose Cull bit is set are kept and marked
    unsigned long long marked = 0;
    if (rc.cull_enable == GS_CULL_MARK)
        for (unsigned long long mm = act; mm; mm &= mm - 1) {
            const int c = __ffsll((long long)mm) - 1;
            if (cull_bit(o, c, i)) marked |= 1ull << c;
        }
    RecOut one;
    if (kOneCam && act) one = make_record(g, i, L, op, s_cams[0], p_one, rc, marked & 1ull);
    unsigned long long total, tvis;
    const unsigned long long excl = block_exclusive_scan<kNW, unsigned long long>(cnt, s_warp, total);
    block_exclusive_scan<kNW, unsigned long long>((unsigned long long)((act & ~marked) != 0), s_warp, tvis);
    if (threadIdx.x < 32) {
        const unsigned long long b = lookback_exclusive(o.lb_status + 1, bid, total, o.ctr, kSitePreprocess);
        if (threadIdx.x == 0) {
            s_base = b;
            if (tvis) atomicAdd(&o.ctr->n_visible, tvis); // the visible set of Eq. 5
        }
    }
    __syncthreads();
    const unsigned long long base = s_base + excl;
    if (j == ncand - 1) {
        const unsigned long long end = base + cnt;
        o.ctr->records_needed = end;
        o.ctr->n_records = end < (unsigned long long)o.max_records ? end : o.max_records;
    }
    if (act) {
        if (base < (unsigned long long)o.max_records) o.rec_first[i] = (uint32_t)base;
        if (kOneCam) {
            if (base >= (unsigned long long)o.max_records) set_error(o.ctr, GS_ERR_CAPACITY, kSitePreprocess);
            else store_record(o, base, i, 0, one);
        } else {
            unsigned long long r = base;
            for (unsigned long long mm = act; mm; mm &= mm - 1, r++) {
                const int c = __ffsll((long long)mm) - 1;
                if (r >= (unsigned long long)o.max_records) {
                    set_error(o.ctr, GS_ERR_CAPACITY, kSitePreprocess);
                    break;
                }
                const CamInfo &cam = s_cams[c];
                DF td[3];
                camera_point_df(L.m, cam, td);
                Proj p;
                project_gaussian(L.ls, L.q, td, cam, tw, th, rc, p); // same inputs: same (passing) result
                store_record(o, r, i, c, make_record(g, i, L, op, cam, p, rc, (marked >> c) & 1ull));
            }
        }
    }
    __syncthreads(); // every thread is done with this chunk's shared values
    } // chunks
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t launch_preprocess(gs_workspace *ws, cudaStream_t st, const uint32_t *cull)
{
    const long long n = ws->g.n;
    const unsigned gblocks = (unsigned)((n + kGateChunk - 1) / kGateChunk); // chunks
    const unsigned pchunks = (unsigned)((n + kProjThreads - 1) / kProjThreads); // projection chunks (at most)
    cudaError_t e;
    // counters, then the look-back state of each stage (ticket in word 0)
    if ((e = cudaMemsetAsync(ws->ctr, 0, sizeof(DevCounters), st)) != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    GaussPtrs gp{ws->g.mean, ws->g.log_scale, ws->g.quat, ws->g.opacity_logit, ws->g.sh, ws->g.lod, n};
    PreOut o;
    o.rec_g = ws->rec_g; o.tt = ws->tt; o.dkey = ws->dkey;
    o.rec_cam = ws->rec_cam; o.rd0 = ws->rd0; o.rd1 = ws->rd1; o.rd2 = ws->rd2; o.rect = ws->rect;
    o.clampm = ws->clampm; o.cand_g = ws->cand_g; o.cand_mask = ws->cand_mask; o.rec_first = ws->rec_first;
    o.gate_g = ws->gate_g; o.gate_mask = ws->gate_mask;
    o.drift = ws->lazy.enabled ? ws->lazy.drift : nullptr;
    o.lb_status = ws->lb_status;
    o.ctr = ws->ctr; o.max_records = ws->cap.max_records;
    o.cull = ws->rc.cull_enable ? cull : nullptr;
    o.cull_words = (n + 31) / 32;
    if ((e = cudaMemsetAsync(ws->rec_first, 0xff, (size_t)n * sizeof(uint32_t), st)) != cudaSuccess) return e;
    // gate: per-block counts (in lb_status) and candidates (block-strided), the
    // scan of the counts, the gather into one ordered list
    kt_begin(ws, GS_KT_GATE, st);
    // the camera count of the upload (a captured graph replays uploads of the
    // same count); bulk copies where every streamed array is 16-byte aligned
    const bool one = ws->cams.n == 1;
    const bool bulk = n >= kGateChunk && aligned16(gp.mean) && (!gp.lod || aligned16(gp.lod)) &&
                      (!o.drift || aligned16(o.drift));
    const unsigned per_sm = one ? 4u : 3u;
    const unsigned ggrid = bulk ? std::min<unsigned>(gblocks, per_sm * (unsigned)ws->sm_count) : gblocks;
    const unsigned long long spins = kSpinLimit;
    if (one && bulk)
        launch_pdl(gate_count_kernel<true, true>, ggrid, 256, 0, st, gp, o, ws->d_cams, ws->rc, ws->lb_status, spins);
    else if (one)
        launch_pdl(gate_count_kernel<true, false>, ggrid, 256, 0, st, gp, o, ws->d_cams, ws->rc, ws->lb_status, spins);
    else if (bulk)
        launch_pdl(gate_count_kernel<false, true>, ggrid, 256, 0, st, gp, o, ws->d_cams, ws->rc, ws->lb_status, spins);
    else
        launch_pdl(gate_count_kernel<false, false>, ggrid, 256, 0, st, gp, o, ws->d_cams, ws->rc, ws->lb_status, spins);
    kt_end(ws, GS_KT_GATE, st);
    note_launch();
    launch_pdl(gate_scan_kernel, 1, 1024, 0, st, ws->lb_status, (long long)gblocks, ws->ctr);
    note_launch();
    launch_pdl(gate_gather_kernel, gblocks, 256, 0, st, o, ws->lb_status, (long long)gblocks, ws->ctr);
    note_launch();
    if ((e = cudaMemsetAsync(ws->lb_status, 0, (pchunks + 1) * sizeof(unsigned long long), st)) != cudaSuccess)
        return e;
    // deferred Adam steps: bring the candidates up to date before projecting them
    if (ws->lazy.enabled && (e = launch_lazy_catchup(ws, st, ws->g)) != cudaSuccess) return e;
    // projection: persistent blocks, about as many as stay resident (five per
    // SM at their registers), taking the candidates' chunks by ticket
    const unsigned pgrid = std::min<unsigned>(pchunks, 5u * (unsigned)ws->sm_count);
    kt_begin(ws, GS_KT_PROJECT, st);
    if (ws->cams.n == 1)
        launch_pdl(project_kernel<true>, pgrid, kProjThreads, 0, st, gp, o, ws->d_cams, ws->rc);
    else
        launch_pdl(project_kernel<false>, pgrid, kProjThreads, 0, st, gp, o, ws->d_cams, ws->rc);
    kt_end(ws, GS_KT_PROJECT, st);
    note_launch();
    return cudaGetLastError();
}

// ---- backward ---------------------------------------------------------------

// Sum of the per-(record, tile) gradient slots of each record, turned into the
// record's mean and conic gradients by its opacity and conic
// (slot_grads_from_moments).  A warp takes kReduceRecs consecutive records
// (whose slots are contiguous: a record's first instance follows record
// order); each of its first lanes loads one record's indices.  Records of
// at most kReduceBig tiles are added up by groups of kReduceLanes lanes, 32 /
// kReduceLanes records at a time (a group's lanes read the record's slots
// strided by kReduceLanes, then a fixed shuffle tree adds the lanes), so the
// loads of a round are in flight together; larger records then take the whole
// warp each (lanes strided by 32, a fixed tree over 32 lanes).  Which way a
// record is summed depends only on its tile count, so the sum is the same on
// every run.  Records marked culled are skipped: the projection adjoint never
// reads them.
constexpr int kReduceLanes = 8;
constexpr int kReduceRecs = 2 * (32 / kReduceLanes); // records per warp: two rounds of the groups
constexpr uint32_t kReduceBig = 4 * kReduceLanes;    // tiles above which a record takes the whole warp
static_assert(kReduceLanes < kSlotFloats && kSlotFloats <= 2 * kReduceLanes, "a slot is written by one group");
__global__ void __launch_bounds__(256) reduce_slots_kernel(const uint32_t *inst_off, const uint32_t *tt,
                                                           const float4 *rd0, const float4 *rd1, const float4 *rd2,
                                                           const float *slots, float *rgrad, const DevCounters *ctr)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    constexpr int kGroups = 32 / kReduceLanes;
    constexpr uint32_t kSkip = 0xffffffffu;
    const unsigned long long nrec = ctr->n_records, ninst = ctr->n_instances;
    const int lane = threadIdx.x & 31, sub = lane & (kReduceLanes - 1), grp = lane / kReduceLanes;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * 8;
    for (unsigned long long k0 = ((unsigned long long)blockIdx.x * 8 + (threadIdx.x >> 5)) * kReduceRecs; k0 < nrec;
         k0 += nwarps * kReduceRecs) {
        // lane l < kReduceRecs: record k0 + l
        uint32_t r = 0, cnt = kSkip;
        unsigned long long off = 0;
        if (lane < kReduceRecs && k0 + lane < nrec) {
            r = (uint32_t)(k0 + lane);
            off = inst_off[r];
            cnt = tt[r];
            // capacity error already recorded, or marked: nothing to sum
            if (off + cnt > ninst || rd2[r].w != 0.f) cnt = kSkip;
        }
        const unsigned big = __ballot_sync(0xffffffffu, cnt != kSkip && cnt > kReduceBig);
#pragma unroll
        for (int round = 0; round < kReduceRecs / kGroups; round++) {
            const int src = round * kGroups + grp; // the record of this group in this round
            const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
            const uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
            const unsigned long long o = __shfl_sync(0xffffffffu, off, src);
            const bool live = c <= kReduceBig;
            float acc[kSlotFloats];
#pragma unroll
            for (int j = 0; j < kSlotFloats; j++) acc[j] = 0.f;
            if (live) {
                #pragma unroll 4 // the loads of four iterations in flight (the adds keep their order)
                for (uint32_t t = sub; t < c; t += kReduceLanes) {
                    const float *sl = slots + (o + t) * kSlotFloats;
#pragma unroll
                    for (int j = 0; j < kSlotFloats; j++) acc[j] += sl[j];
                }
            }
#pragma unroll
            for (int j = 0; j < kSlotFloats; j++)
#pragma unroll
                for (int x = kReduceLanes / 2; x > 0; x >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], x);
            if (live) {
                const float4 q0 = rd0[rr], q1 = rd1[rr];
                slot_grads_from_moments(acc, q0.z, q0.w, q1.x, q1.y);
                // lane sub writes component sub, and component sub + kReduceLanes where there is one
                float v = acc[0];
#pragma unroll
                for (int j = 1; j < kReduceLanes; j++) v = sub == j ? acc[j] : v;
                float w = acc[kReduceLanes];
#pragma unroll
                for (int j = kReduceLanes + 1; j < kSlotFloats; j++) w = sub + kReduceLanes == j ? acc[j] : w;
                float *dst = rgrad + (unsigned long long)rr * kSlotFloats;
                dst[sub] = v;
                if (sub + kReduceLanes < kSlotFloats) dst[sub + kReduceLanes] = w;
            }
        }
        for (unsigned rest = big; rest; rest &= rest - 1) {
            const int src = __ffs(rest) - 1;
            const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
            const uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
            const unsigned long long o = __shfl_sync(0xffffffffu, off, src);
            float acc[kSlotFloats];
#pragma unroll
            for (int j = 0; j < kSlotFloats; j++) acc[j] = 0.f;
            #pragma unroll 4 // the loads of four iterations in flight (the adds keep their order)
            for (uint32_t t = lane; t < c; t += 32) {
                const float *sl = slots + (o + t) * kSlotFloats;
#pragma unroll
                for (int j = 0; j < kSlotFloats; j++) acc[j] += sl[j];
            }
#pragma unroll
            for (int j = 0; j < kSlotFloats; j++)
#pragma unroll
                for (int x = 16; x > 0; x >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], x);
            if (lane < kSlotFloats) {
                const float4 q0 = rd0[rr], q1 = rd1[rr];
                slot_grads_from_moments(acc, q0.z, q0.w, q1.x, q1.y);
                float v = acc[0];
#pragma unroll
                for (int j = 1; j < kSlotFloats; j++) v = lane == j ? acc[j] : v;
                rgrad[(unsigned long long)rr * kSlotFloats + lane] = v;
            }
        }
    }
}

cudaError_t launch_reduce_slots(gs_workspace *ws, cudaStream_t st)
{
    const long long cap = ws->cap.max_records;
    long long blocks = (cap + 8 * kReduceRecs - 1) / (8 * kReduceRecs); // kReduceRecs records per warp
    if (blocks > 16ll * ws->sm_count) blocks = 16ll * ws->sm_count;
    if (blocks < 1) blocks = 1;
    kt_begin(ws, GS_KT_REDUCE_SLOTS, st);
    launch_pdl(reduce_slots_kernel, (unsigned)blocks, 256, 0, st, ws->inst_off, ws->tt, (const float4 *)ws->rd0,
               (const float4 *)ws->rd1, (const float4 *)ws->rd2, (const float *)ws->slots, ws->rgrad,
               (const DevCounters *)ws->ctr);
    kt_end(ws, GS_KT_REDUCE_SLOTS, st);
    note_launch();
    return cudaGetLastError();
}

struct BwdArgs {
    GaussPtrs g;
    float *gmean, *gls, *gquat, *gop, *gsh;
    const uint32_t *rec_g;
    const uint16_t *rec_cam;
    const uint8_t *clampm;
    const float4 *rd2;  // .w != 0: record marked culled (GS_CULL_MARK), no gradient
    const float *rgrad;
    float *cgrad;      // non-NULL: write each Gaussian's gradient row here (at its first record) instead
    float *absgrad;
    int accumulate;
    float beta;
    float *red_partial;
    const DevCounters *ctr;
};

// Chain rule from the gradients of (u, v, conic A B C, opacity, rgb) of each
// record to the parameters of its Gaussian, summed over the Gaussian's records.
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(BwdArgs a, const CamTable *__restrict__ ctp,
                                                             RenderConsts rc)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ CamInfo s_cams[GS_MAX_CAMERAS];
    __shared__ float s_red[4];
    // each thread's gradient row: the SH part accumulates here over the records,
    // and with a.cgrad the warp copies its 32 consecutive rows out together
    __shared__ float s_row[4][32 * kGradRow];
    stage_cameras(*ctp, s_cams);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *myrow = &s_row[warp][lane * kGradRow];
    // one thread per Gaussian that has records: the thread of its first record
    const unsigned long long rh = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long nrec = a.ctr->n_records;
    float smin_val = 0.f;
    const bool head = rh < nrec && (rh == 0 || a.rec_g[rh - 1] != a.rec_g[rh]);
    if (head) {
        const long long i = a.rec_g[rh];
        unsigned long long r0 = rh, r1 = rh + 1; // a Gaussian's records are contiguous
        while (r1 < nrec && a.rec_g[r1] == (uint32_t)i) r1++;
        float gm[3] = {0, 0, 0}, gls[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gop = 0.f;
        bool vis = false; // an unmarked record (the visible set of Eq. 5)
        float *gsh = myrow + 11; // the 48 SH gradients, summed over the records
#pragma unroll
        for (int k = 0; k < 48; k++) gsh[k] = 0.f;
        const float m[3] = {a.g.mean[3 * i], a.g.mean[3 * i + 1], a.g.mean[3 * i + 2]};
        const float ls[3] = {a.g.log_scale[3 * i], a.g.log_scale[3 * i + 1], a.g.log_scale[3 * i + 2]};
        {
            const float qr[4] = {a.g.quat[4 * i], a.g.quat[4 * i + 1], a.g.quat[4 * i + 2], a.g.quat[4 * i + 3]};
            const float qn = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
            const float q[4] = {qr[0] / qn, qr[1] / qn, qr[2] / qn, qr[3] / qn};
            const float w = q[0], x = q[1], y = q[2], z = q[3];
            float Q[3][3];
            Q[0][0] = 1.f - 2.f * (y * y + z * z); Q[0][1] = 2.f * (x * y - w * z); Q[0][2] = 2.f * (x * z + w * y);
            Q[1][0] = 2.f * (x * y + w * z); Q[1][1] = 1.f - 2.f * (x * x + z * z); Q[1][2] = 2.f * (y * z - w * x);
            Q[2][0] = 2.f * (x * z - w * y); Q[2][1] = 2.f * (y * z + w * x); Q[2][2] = 1.f - 2.f * (x * x + y * y);
            const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
            float M[3][3];
            for (int p = 0; p < 3; p++)
                for (int c = 0; c < 3; c++) M[p][c] = Q[p][c] * s[c];
            const float o = 1.f / (1.f + expf(-a.g.opacity_logit[i]));
            // H[a][b] = w_a^T G w_b summed over the records, w_k = C v_k: the scale and
            // rotation gradients below are these bilinear forms (see after the loop)
            float H00 = 0.f, H11 = 0.f, H22 = 0.f, H01 = 0.f, H02 = 0.f, H12 = 0.f;
            float absacc = 0.f;
            for (unsigned long long r = r0; r < r1; r++) {
                if (a.rd2[r].w != 0.f) continue; // marked culled: composited nowhere
                vis = true;
                const CamInfo &cam = s_cams[a.rec_cam[r]];
                const float *rg = a.rgrad + r * kSlotFloats;
                const float gu = rg[0], gv = rg[1], gA = rg[2], gB = rg[3], gC = rg[4], go = rg[5];
                const float grgb[3] = {rg[6], rg[7], rg[8]};
                absacc += sqrtf(gu * gu + gv * gv);
                const float *W = cam.R;
                DF td[3];
                camera_point_df(m, cam, td); // the camera-space mean the forward projected
                const float t[3] = {td[0].hi, td[1].hi, td[2].hi};
                const float fx = cam.fx, fy = cam.fy;
                const float limx = rc.fov_clamp * ((float)cam.width / (2.f * fx));
                const float limy = rc.fov_clamp * ((float)cam.height / (2.f * fy));
                const float xr = t[0] / t[2], yr = t[1] / t[2];
                const bool clx = xr < -limx || xr > limx, cly = yr < -limy || yr > limy;
                const float xc = clampf(xr, -limx, limx), yc = clampf(yr, -limy, limy);
                const float tz = t[2], itz = 1.f / tz, itz2 = itz * itz;
                float J[2][3] = {{fx * itz, 0.f, -fx * xc * itz}, {0.f, fy * itz, -fy * yc * itz}};
                float T[2][3];
                for (int r2 = 0; r2 < 2; r2++)
                    for (int k = 0; k < 3; k++) T[r2][k] = J[r2][0] * W[k] + J[r2][1] * W[3 + k] + J[r2][2] * W[6 + k];
                // Sigma' = V V^T + dilation I, V = T M; determinant by Cauchy-Binet
                float V[2][3];
                for (int r2 = 0; r2 < 2; r2++)
                    for (int k = 0; k < 3; k++) V[r2][k] = T[r2][0] * M[0][k] + T[r2][1] * M[1][k] + T[r2][2] * M[2][k];
                const float s00 = V[0][0] * V[0][0] + V[0][1] * V[0][1] + V[0][2] * V[0][2];
                const float s11 = V[1][0] * V[1][0] + V[1][1] * V[1][1] + V[1][2] * V[1][2];
                const float m01 = V[0][0] * V[1][1] - V[0][1] * V[1][0];
                const float m02 = V[0][0] * V[1][2] - V[0][2] * V[1][0];
                const float m12 = V[0][1] * V[1][2] - V[0][2] * V[1][1];
                const float det = m01 * m01 + m02 * m02 + m12 * m12 + rc.dilation * (s00 + s11 + rc.dilation);
                const float idet = 1.f / det;
                // conic C = (V V^T + d I)^-1 and dL/dV = -2 C G C V, G = dL/dC (symmetric).  C is applied
                // through its adjugate, adj(V V^T + d I) = (P V)(P V)^T + d I with P the quarter turn
                // (P v = (-v_y, v_x)), so (P V)^T v_k holds the 2x2 minors cross(v_i, v_k) of V: every
                // product keeps its accuracy along both axes of a long thin footprint, where the
                // entries of C and of dL/dSigma' in image axes would cancel.
                const float mn[3][3] = {{0.f, m01, m02}, {-m01, 0.f, m12}, {-m02, -m12, 0.f}};
                const float PV[2][3] = {{-V[1][0], -V[1][1], -V[1][2]}, {V[0][0], V[0][1], V[0][2]}};
                const float G[2][2] = {{gA, 0.5f * gB}, {0.5f * gB, gC}};
                float Wk[2][3]; // w_k = C v_k
                float GW[2][3]; // G C v_k
                for (int k = 0; k < 3; k++) {
                    float w[2];
                    for (int r2 = 0; r2 < 2; r2++)
                        w[r2] = (PV[r2][0] * mn[0][k] + PV[r2][1] * mn[1][k] + PV[r2][2] * mn[2][k] +
                                 rc.dilation * V[r2][k]) * idet;
                    Wk[0][k] = w[0]; Wk[1][k] = w[1];
                    for (int r2 = 0; r2 < 2; r2++) GW[r2][k] = G[r2][0] * w[0] + G[r2][1] * w[1];
                }
                H00 += Wk[0][0] * GW[0][0] + Wk[1][0] * GW[1][0];
                H11 += Wk[0][1] * GW[0][1] + Wk[1][1] * GW[1][1];
                H22 += Wk[0][2] * GW[0][2] + Wk[1][2] * GW[1][2];
                H01 += Wk[0][0] * GW[0][1] + Wk[1][0] * GW[1][1];
                H02 += Wk[0][0] * GW[0][2] + Wk[1][0] * GW[1][2];
                H12 += Wk[0][1] * GW[0][2] + Wk[1][1] * GW[1][2];
                float gV[2][3];
                for (int k = 0; k < 3; k++) {
                    float pv[3];
                    for (int i2 = 0; i2 < 3; i2++) pv[i2] = PV[0][i2] * GW[0][k] + PV[1][i2] * GW[1][k];
                    for (int r2 = 0; r2 < 2; r2++)
                        gV[r2][k] = -2.f * idet *
                                    (PV[r2][0] * pv[0] + PV[r2][1] * pv[1] + PV[r2][2] * pv[2] + rc.dilation * GW[r2][k]);
                }
                // V = T M: dL/dT = dL/dV M^T (dL/dM enters through H)
                float gT[2][3];
                for (int r2 = 0; r2 < 2; r2++)
                    for (int k = 0; k < 3; k++)
                        gT[r2][k] = gV[r2][0] * M[k][0] + gV[r2][1] * M[k][1] + gV[r2][2] * M[k][2];
                float gJ[2][3];
                for (int r2 = 0; r2 < 2; r2++)
                    for (int k = 0; k < 3; k++) gJ[r2][k] = gT[r2][0] * W[3 * k] + gT[r2][1] * W[3 * k + 1] + gT[r2][2] * W[3 * k + 2];
                float gt[3] = {0.f, 0.f, 0.f};
                gt[2] += gJ[0][0] * (-fx * itz2) + gJ[1][1] * (-fy * itz2);
                if (!clx) { gt[0] += gJ[0][2] * (-fx * itz2); gt[2] += gJ[0][2] * (2.f * fx * t[0] * itz2 * itz); }
                else      { gt[2] += gJ[0][2] * (fx * xc * itz2); }
                if (!cly) { gt[1] += gJ[1][2] * (-fy * itz2); gt[2] += gJ[1][2] * (2.f * fy * t[1] * itz2 * itz); }
                else      { gt[2] += gJ[1][2] * (fy * yc * itz2); }
                gt[0] += gu * fx * itz;
                gt[1] += gv * fy * itz;
                gt[2] += -(gu * fx * t[0] + gv * fy * t[1]) * itz2;
                for (int k = 0; k < 3; k++) gm[k] += W[k] * gt[0] + W[3 + k] * gt[1] + W[6 + k] * gt[2];
                gop += go * o * (1.f - o);
                // colour: rgb = max(sum_k sh_k Y_k(d) + 0.5, 0), d = (mu - campos) / |mu - campos|
                const float dv[3] = {m[0] - cam.campos[0], m[1] - cam.campos[1], m[2] - cam.campos[2]};
                const float dn = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                const float idn = 1.f / dn;
                const float d[3] = {dv[0] * idn, dv[1] * idn, dv[2] * idn};
                float Y[16];
                sh_basis(d[0], d[1], d[2], Y);
                const uint8_t cm = a.clampm[r];
                // dL/dd = sum_k c_k grad Y_k(d) with c_k = sum over unclamped channels of
                // dL/drgb_ch * sh_k,ch: the 16 weights first, then one gradient sum
                float ck[16];
#pragma unroll
                for (int k = 0; k < 16; k++) ck[k] = 0.f;
                const float4 *shv = reinterpret_cast<const float4 *>(a.g.sh + 48 * i); // [16][3]
#pragma unroll
                for (int v4 = 0; v4 < 12; v4++) {
                    const float4 c4 = shv[v4];
                    const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                    for (int e2 = 0; e2 < 4; e2++) {
                        const int flat = 4 * v4 + e2, k = flat / 3, ch = flat % 3;
                        if (cm & (1u << ch)) continue;
                        gsh[flat] += grgb[ch] * Y[k];
                        ck[k] += grgb[ch] * cc[e2];
                    }
                }
                float gd[3];
                sh_grad_dot(d[0], d[1], d[2], ck, gd);
                const float ddot = d[0] * gd[0] + d[1] * gd[1] + d[2] * gd[2];
                for (int e = 0; e < 3; e++) gm[e] += (gd[e] - d[e] * ddot) * idn;
            }
            // Scale and rotation.  With V = T R diag(s) and dL/dV = -2 C G C V (C the
            // conic, G = dL/dC), Omega = R^T dL/dR = diag(1/s) V^T dL/dV diag(s) has
            // entries -2 (s_b / s_a) H[a][b], H[a][b] = w_a^T G w_b.  The log-scale
            // gradient is its diagonal, -2 H[k][k]; the rotation gradient is its
            // antisymmetric part, dL/dtheta = (O21 - O12, O02 - O20, O10 - O01) for
            // R(q) R(I + [theta]x).  Forming them from H instead of through T^T dL/dV
            // and R's columns avoids the cancellation of a long thin footprint, whose
            // short axis projects to a short V column although T and R are large.
            gls[0] = -2.f * H00; gls[1] = -2.f * H11; gls[2] = -2.f * H22;
            const float th0 = -2.f * H12 * (s[1] / s[2] - s[2] / s[1]);
            const float th1 = -2.f * H02 * (s[2] / s[0] - s[0] / s[2]);
            const float th2 = -2.f * H01 * (s[0] / s[1] - s[1] / s[0]);
            // unit quaternion: dL/dq = 2 q (x) (0, dL/dtheta), tangent to the sphere;
            // the stored one is q |q_raw|, so dL/dq_raw = dL/dq / |q_raw|
            const float iq = 2.f / qn;
            gq[0] = iq * (-(x * th0 + y * th1 + z * th2));
            gq[1] = iq * (w * th0 + (y * th2 - z * th1));
            gq[2] = iq * (w * th1 + (z * th0 - x * th2));
            gq[3] = iq * (w * th2 + (x * th1 - y * th0));
            if (a.absgrad) a.absgrad[i] += absacc;
            // scale regulariser (Eq. 5): beta / |V| * min_j s_j on the first smallest axis
            if (a.beta > 0.f && vis) {
                int jm = 0;
                if (s[1] < s[jm]) jm = 1;
                if (s[2] < s[jm]) jm = 2;
                const float nv = (float)a.ctr->n_visible;
                gls[jm] += a.beta * s[jm] / nv;
                smin_val = s[jm];
            }
        }
        if (a.cgrad) {
            // compact row of 59 gradients (mean, log-scale, quat, opacity, SH) at the first
            // record: the SH part is in place, the rest goes beside it
            for (int k = 0; k < 3; k++) { myrow[k] = gm[k]; myrow[3 + k] = gls[k]; }
            for (int k = 0; k < 4; k++) myrow[6 + k] = gq[k];
            myrow[10] = gop;
        } else {
            // the grads of Gaussians without records were zeroed (overwrite mode) or are left as they are
            for (int k = 0; k < 3; k++) {
                a.gmean[3 * i + k] += gm[k];
                a.gls[3 * i + k] += gls[k];
            }
            for (int k = 0; k < 4; k++) a.gquat[4 * i + k] += gq[k];
            a.gop[i] += gop;
            for (int k = 0; k < 48; k++) a.gsh[48 * i + k] += gsh[k];
        }
    }
    if (a.cgrad) {
        // rows of records that are not a Gaussian's first are never read: zeros
        if (!head)
            for (int k = 0; k < kGradRow; k++) myrow[k] = 0.f;
        __syncwarp();
        const unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + warp * 32;
        if (base < nrec) {
            const unsigned rows = (unsigned)min(32ull, nrec - base);
            float *dst = a.cgrad + base * kGradRow;
            for (unsigned e = lane; e < rows * kGradRow; e += 32) dst[e] = s_row[warp][e];
        }
    }
    if (a.red_partial) {
        float v = smin_val;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) a.red_partial[blockIdx.x] = s_red[0] + s_red[1] + s_red[2] + s_red[3];
    }
}

__global__ void scale_reg_finalize_kernel(const float *partial, int nblocks, float beta, const DevCounters *ctr,
                                          float *out)
{
    griddep_wait(); // programmatic dependent launch: the previous kernel is complete
    __shared__ double s[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) acc += (double)partial[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nv = (double)ctr->n_visible;
        *out = nv > 0 ? (float)(beta * s[0] / nv) : 0.f;
    }
}

cudaError_t launch_preprocess_bwd(gs_workspace *ws, cudaStream_t st, const gs_gaussians &g,
                                  const gs_gaussian_grads &gr, int accumulate, float *absgrad, float beta,
                                  float *scale_reg_value, float *cgrad)
{
    const long long n = g.n;
    if (n == 0) return cudaSuccess;
    cudaError_t e;
    if (!accumulate && !cgrad) {
        // overwrite mode: Gaussians without a record get zero gradients
        float *arr[5] = {gr.mean, gr.log_scale, gr.quat, gr.opacity_logit, gr.sh};
        const int rows[5] = {3, 3, 4, 1, 48};
        for (int k = 0; k < 5; k++)
            if ((e = cudaMemsetAsync(arr[k], 0, (size_t)rows[k] * n * sizeof(float), st)) != cudaSuccess) return e;
    }
    const unsigned blocks = (unsigned)((ws->cap.max_records + 127) / 128);
    BwdArgs a;
    a.g = GaussPtrs{g.mean, g.log_scale, g.quat, g.opacity_logit, g.sh, g.lod, n};
    a.gmean = gr.mean; a.gls = gr.log_scale; a.gquat = gr.quat; a.gop = gr.opacity_logit; a.gsh = gr.sh;
    a.rec_g = ws->rec_g; a.rec_cam = ws->rec_cam; a.clampm = ws->clampm; a.rd2 = ws->rd2;
    a.rgrad = ws->rgrad;
    a.cgrad = cgrad;
    a.absgrad = absgrad; a.accumulate = accumulate; a.beta = beta;
    const bool reduce = beta > 0.f && scale_reg_value && blocks <= ws->red_words;
    a.red_partial = reduce ? ws->red_partial : nullptr;
    a.ctr = ws->ctr;
    kt_begin(ws, GS_KT_PREPROCESS_BWD, st);
    launch_pdl(preprocess_bwd_kernel, blocks, 128, 0, st, a, ws->d_cams, ws->rc);
    kt_end(ws, GS_KT_PREPROCESS_BWD, st);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (reduce) {
        launch_pdl(scale_reg_finalize_kernel, 1, 256, 0, st, ws->red_partial, (int)blocks, beta, ws->ctr, scale_reg_value);
        note_launch();
        e = cudaGetLastError();
    }
    return e;
}

} // namespace gs
