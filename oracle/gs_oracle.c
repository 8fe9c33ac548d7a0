/* gs_oracle.c -- plain, slow FP64 CPU oracle for the 3DGS render hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no source with the CUDA library.
 *
 * What it computes, following the paper (BlitzGS, arXiv 2605.13794):
 *   - App. A: Gaussian G_i (Eq. for G_i), tile-based front-to-back alpha
 *     compositing (Eq. for C(p) and T_i), projection to screen-space ellipses;
 *     the projection details the paper leaves to "standard 3DGS" follow the
 *     EWA splatting of 3DGS (Jacobian clamp, 0.3 dilation, 3-sigma radius).
 *   - Sec. 3.3, Eq. 1-3: distance-based LOD gate and the per-view cull mask.
 *   - Sec. 3.2 and Fig. 2: per-(Gaussian, view) alpha-weight w = sum_p alpha T
 *     and qualifying-pixel count a, accumulated during compositing.
 *   - The exact adjoint (reverse-mode derivative) of all of the above.
 * Everything is computed in FP64 from the FP32 inputs, decisions included.
 * A renderer that computes in FP32 can take a decision the other way only
 * where the FP64 value lies within its rounding error of the boundary: each
 * such decision is flagged (tie bits per Gaussian, flag bits per pixel) from
 * a stated FP32 error bound, so callers can exclude exactly those cases from
 * exact comparisons.  The bounds are:
 *   - projection decisions (LOD level, near plane, radius): a running
 *     forward-error bound of an FP32 evaluation of the same formulas
 *     (Wilkinson's running error analysis; Higham, "Accuracy and Stability
 *     of Numerical Algorithms", ch. 3), valid in any association order;
 *   - tile rectangle: the FP32 projected mean (the float nearest a mean held
 *     to at least 2^-38 relative), the rectangle's arithmetic being exact;
 *   - compositing thresholds: a renderer whose per-Gaussian exponent form
 *     A (x + k y)^2 + D y^2 carries at most prec_conic relative error in A, D
 *     and prec_conic (|k| + sqrt(D / A)) in k, and whose mean carries at most
 *     prec_mean pixels, evaluating the exponent in FP32.
 *
 * The SH basis is built from its definition: associated Legendre functions
 * from Rodrigues' formula, normalisation sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
 * Condon-Shortley phase, real form with m = -l..l (the 3DGS ordering).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ACTIVE 0
#define OR_GATED_LOD 1
#define OR_GATED_CULL 2
#define OR_NEAR 3
#define OR_DEGENERATE 4
#define OR_EMPTY 5

#define OR_TIE_LOD 1u
#define OR_TIE_NEAR 2u
#define OR_TIE_DET 4u
#define OR_TIE_RADIUS 8u
#define OR_TIE_RECT 16u
#define OR_TIE_CLAMP 32u
#define OR_TIE_DEPTH 64u

/* pixel flags */
#define OR_PIX_ALPHA_MIN 1u  /* some fragment's alpha within band of alpha_min */
#define OR_PIX_T_MIN 2u      /* some fragment's T(1-alpha) within band of T_min */
#define OR_PIX_ALPHA_MAX 4u  /* some fragment's o*G within band of alpha_max */
#define OR_PIX_POWER 8u      /* some fragment's exponent within band of 0 */

typedef struct {
    double R[9], t[3];
    double fx, fy, cx, cy;
    double campos[3];
    int32_t width, height;
} or_camera;

typedef struct {
    int32_t tile_w, tile_h; /* tile size in pixels (16 x 16 in 3DGS) */
    int32_t lod_enable, lod_Lmax, cull_enable;
    double bg[3];
    double alpha_min, alpha_max, T_min;
    double dilation, znear, fov_clamp;
    double lod_d0, lod_f;
    double prec_mean;      /* renderer's projected-mean error bound, pixels */
    double prec_conic;     /* renderer's exponent-form coefficient error bound (relative) */
    double comp_band;      /* extra log-space band for compositing thresholds */
} or_params;

/* ---- FP32 forward-error bounds -------------------------------------------
 * Each quantity v of a formula is carried with a bound e such that an FP32
 * evaluation of the same formula, whatever the association order of its sums,
 * is within e of v: every FP32 operation adds one rounding of at most
 * U32 = 2^-24 of its result, and errors of the operands propagate to first
 * order plus the product of the two errors.  Sums of n terms take
 * gamma_{n-1} = (n - 1) U32 of the sum of their magnitudes (Higham, Eq. 3.5);
 * library exp is taken as at most 2 ulp, sqrt and division as correctly
 * rounded. */
#define U32 5.9604644775390625e-08

typedef struct { double v, e; } eb_t;

static eb_t eb(double v, double e) { eb_t r; r.v = v; r.e = e; return r; }
static eb_t eb_round(double v, double e) { return eb(v, e + U32 * (fabs(v) + e)); }
static eb_t eb_add(eb_t a, eb_t b) { return eb_round(a.v + b.v, a.e + b.e); }
static eb_t eb_sub(eb_t a, eb_t b) { return eb_round(a.v - b.v, a.e + b.e); }
static eb_t eb_neg(eb_t a) { return eb(-a.v, a.e); }
static eb_t eb_scale(eb_t a, double k) { return eb(k * a.v, fabs(k) * a.e); } /* k a power of two: exact */
static eb_t eb_mul(eb_t a, eb_t b)
{
    return eb_round(a.v * b.v, fabs(a.v) * b.e + fabs(b.v) * a.e + a.e * b.e);
}
static eb_t eb_div(eb_t a, eb_t b)
{
    const double v = a.v / b.v, den = fabs(b.v) - b.e;
    return eb_round(v, den > 0.0 ? (a.e + fabs(v) * b.e) / den : INFINITY);
}
static eb_t eb_sqrt(eb_t a)
{
    const double v = sqrt(a.v > 0.0 ? a.v : 0.0);
    const double hi = sqrt(a.v + a.e), lo = sqrt(a.v - a.e > 0.0 ? a.v - a.e : 0.0);
    return eb_round(v, fmax(hi - v, v - lo));
}
static eb_t eb_exp(eb_t a)
{
    const double v = exp(a.v), e = v * expm1(a.e);
    return eb(v, e + 4.0 * U32 * (v + e));
}
/* sum of n terms in any order */
static eb_t eb_sum(const eb_t *t, int n)
{
    double v = 0.0, mag = 0.0, e = 0.0;
    for (int i = 0; i < n; i++) { v += t[i].v; mag += fabs(t[i].v) + t[i].e; e += t[i].e; }
    return eb(v, e + (double)n * U32 * mag); /* gamma_{n-1} of the terms plus the final rounding */
}
/* clamp to [-lim, lim]: 1-Lipschitz in x and in lim */
static eb_t eb_clamp(eb_t x, eb_t lim)
{
    const double v = x.v < -lim.v ? -lim.v : (x.v > lim.v ? lim.v : x.v);
    return eb(v, fmax(x.e, lim.e));
}
static eb_t eb_in(double v) { return eb(v, 0.0); } /* an FP32 input, exact */

/* ---- projection (App. A; view gate Eq. 1-3) -------------------------------
 * Steps, all in FP64:
 *   1. LOD gate L = clamp(round(log_f(d0 / d)), 0, Lmax), keep lod <= L (Eq. 1, 2)
 *   2. cull mask column (Eq. 3)
 *   3. camera transform, near-plane cull
 *   4. Sigma = R(q) diag(exp(2 log s)) R(q)^T
 *   5. Sigma' = J W Sigma W^T J^T + dilation I     (EWA splatting, 3DGS)
 *   6. conic = inverse of Sigma' (det = a c - b^2), radius = ceil(3 sqrt(lambda_max)),
 *      tile rectangle covering [u - r, u + r] x [v - r, v + r].
 * Tie bits mark the decisions an FP32 renderer may take the other way. */
typedef struct {
    int status;            /* OR_ACTIVE or the first failed test */
    unsigned tie;          /* OR_TIE_* bits */
    double tx, ty, tz;     /* camera-space mean */
    double u, v;           /* projected mean, pixels */
    double a, b, c, det;   /* Sigma' (with dilation) and its determinant */
    double conA, conB, conC;
    double extent, extent_err; /* 3 sqrt(lambda_max) and its FP32 error bound */
    int radius;
    int rect[4];           /* x0, y0, x1, y1 in tiles, half-open */
} proj_t;

static double ulp32(double x)
{
    const double ax = fabs(x);
    if (ax < 1.1754943508222875e-38) return 1.401298464324817e-45;
    int ex;
    frexp(ax, &ex); /* ax = m 2^ex, 0.5 <= m < 1 */
    return ldexp(1.0, ex - 24);
}

/* frac distance of x to the nearest integer */
static double dist_int(double x) { return fabs(x - floor(x + 0.5)); }

/* The rotation of a quaternion (w, x, y, z), normalised, with its FP32 error bounds. */
static void quat_rot_eb(const double q4[4], eb_t Q[3][3])
{
    eb_t sq[4];
    for (int k = 0; k < 4; k++) sq[k] = eb_mul(eb_in(q4[k]), eb_in(q4[k]));
    const eb_t qn = eb_sqrt(eb_sum(sq, 4));
    const eb_t w = eb_div(eb_in(q4[0]), qn), x = eb_div(eb_in(q4[1]), qn);
    const eb_t y = eb_div(eb_in(q4[2]), qn), z = eb_div(eb_in(q4[3]), qn);
    const eb_t one = eb_in(1.0);
    Q[0][0] = eb_sub(one, eb_scale(eb_add(eb_mul(y, y), eb_mul(z, z)), 2.0));
    Q[0][1] = eb_scale(eb_sub(eb_mul(x, y), eb_mul(w, z)), 2.0);
    Q[0][2] = eb_scale(eb_add(eb_mul(x, z), eb_mul(w, y)), 2.0);
    Q[1][0] = eb_scale(eb_add(eb_mul(x, y), eb_mul(w, z)), 2.0);
    Q[1][1] = eb_sub(one, eb_scale(eb_add(eb_mul(x, x), eb_mul(z, z)), 2.0));
    Q[1][2] = eb_scale(eb_sub(eb_mul(y, z), eb_mul(w, x)), 2.0);
    Q[2][0] = eb_scale(eb_sub(eb_mul(x, z), eb_mul(w, y)), 2.0);
    Q[2][1] = eb_scale(eb_add(eb_mul(y, z), eb_mul(w, x)), 2.0);
    Q[2][2] = eb_sub(one, eb_scale(eb_add(eb_mul(x, x), eb_mul(y, y)), 2.0));
}

/* lambda_max of Sigma' = [[a, b], [b, c]]: mid + sqrt(max(0.1, mid^2 - det)) */
static eb_t lambda_max_eb(eb_t a, eb_t c, eb_t det)
{
    const eb_t mid = eb_scale(eb_add(a, c), 0.5);
    eb_t disc = eb_sub(eb_mul(mid, mid), det);
    if (disc.v < 0.1) disc.v = 0.1; /* max(0.1, .) is 1-Lipschitz: the bound stays */
    return eb_add(mid, eb_sqrt(disc));
}

static void project_one(const double *mean3, const double *ls3, const double *q4, int lod, int culled,
                        const or_camera *cam, const or_params *P, proj_t *o)
{
    memset(o, 0, sizeof(*o));
    o->status = OR_ACTIVE;
    const double mx = mean3[0], my = mean3[1], mz = mean3[2];

    /* 1. distance-based LOD gate (Eq. 1 and Eq. 2).  An FP32 renderer forms
     * d^2 from the float coordinates with relative error <= 7 U32; the level
     * log_f(d0 / d) then moves by <= 3.5 U32 / ln f, and a threshold rounded
     * to float adds U32 / ln f: flagged within twice that of a half-integer. */
    if (P->lod_enable) {
        const double dx = mx - cam->campos[0], dy = my - cam->campos[1], dz = mz - cam->campos[2];
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        int L;
        if (d > 0.0) {
            const double x = log(P->lod_d0 / d) / log(P->lod_f);
            const double r = x >= 0.0 ? floor(x + 0.5) : -floor(-x + 0.5); /* half away from zero */
            L = (int)r;
            if (dist_int(x + 0.5) <= 2.0 * 4.5 * U32 / log(P->lod_f)) o->tie |= OR_TIE_LOD;
        } else {
            L = P->lod_Lmax;
        }
        if (L < 0) L = 0;
        if (L > P->lod_Lmax) L = P->lod_Lmax;
        if (lod > L) {
            o->status = OR_GATED_LOD;
            if (!(o->tie & OR_TIE_LOD)) return; /* a tied gate: the values below are still wanted */
        }
    }
    /* 2. importance-based per-view cull (Eq. 3) */
    if (P->cull_enable && culled) { o->status = OR_GATED_CULL; return; }

    /* 3. camera transform, t = W mu + t0 (W row-major) */
    const double *W = cam->R;
    const double tx = W[0] * mx + W[1] * my + W[2] * mz + cam->t[0];
    const double ty = W[3] * mx + W[4] * my + W[5] * mz + cam->t[1];
    const double tz = W[6] * mx + W[7] * my + W[8] * mz + cam->t[2];
    o->tx = tx; o->ty = ty; o->tz = tz;
    /* the renderer compares its float depth (nearest to a mean held to 2^-38) with znear */
    const double zmag = fabs(W[6] * mx) + fabs(W[7] * my) + fabs(W[8] * mz) + fabs(cam->t[2]);
    if (fabs(tz - P->znear) <= ulp32(P->znear) + 0x1p-38 * zmag) o->tie |= OR_TIE_NEAR;
    if (!(tz > P->znear) && o->status == OR_ACTIVE) {
        o->status = OR_NEAR;
        if (!(o->tie & OR_TIE_NEAR)) return;
    }
    if (!(tz > 0.0)) { if (o->status == OR_ACTIVE) o->status = OR_NEAR; return; }
    /* the depth key is the float nearest the depth: flagged where a depth held
     * to 2^-38 could round to the neighbouring float */
    {
        const double d32 = (double)(float)tz, half = 0.5 * ulp32(d32);
        if (fabs(half - fabs(tz - d32)) <= 0x1p-38 * zmag) o->tie |= OR_TIE_DEPTH;
    }

    /* 4. 3D covariance from the normalised quaternion and the scales */
    double qn = sqrt(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
    const double w = q4[0] / qn, x = q4[1] / qn, y = q4[2] / qn, z = q4[3] / qn;
    const double Q[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    const double sc[3] = {exp(ls3[0]), exp(ls3[1]), exp(ls3[2])};
    double Sg[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += Q[i][k] * sc[k] * sc[k] * Q[j][k];
            Sg[i][j] = acc;
        }

    /* 5. EWA: Jacobian of the perspective map at the (clamped) mean */
    const double fx = cam->fx, fy = cam->fy;
    const double limx = P->fov_clamp * (cam->width / (2.0 * fx));
    const double limy = P->fov_clamp * (cam->height / (2.0 * fy));
    const double xr = tx / tz, yr = ty / tz;
    const double xc = xr < -limx ? -limx : (xr > limx ? limx : xr);
    const double yc = yr < -limy ? -limy : (yr > limy ? limy : yr);
    const double J[2][3] = {{fx / tz, 0.0, -fx * xc / tz}, {0.0, fy / tz, -fy * yc / tz}};
    double T[2][3];
    for (int r = 0; r < 2; r++)
        for (int k = 0; k < 3; k++) T[r][k] = J[r][0] * W[k] + J[r][1] * W[3 + k] + J[r][2] * W[6 + k];
    double S2[2][2];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double acc = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) acc += T[r][i] * Sg[i][j] * T[c][j];
            S2[r][c] = acc;
        }
    const double a = S2[0][0] + P->dilation, b = S2[0][1], c = S2[1][1] + P->dilation;
    o->a = a; o->b = b; o->c = c;

    /* 6. conic, extent, footprint */
    const double det = a * c - b * b;
    o->det = det;

    /* FP32 error bounds of det and of the extent, for the two standard ways of
     * forming Sigma': as V V^T with V = J W R diag(s) (det by the Cauchy-Binet
     * identity), and as J W Sigma W^T J^T with Sigma formed first (det as
     * a c - b^2).  The larger bound of the two is taken. */
    double det_err, ext_err;
    {
        eb_t Qe[3][3];
        quat_rot_eb(q4, Qe);
        eb_t se[3];
        for (int k = 0; k < 3; k++) se[k] = eb_exp(eb_in(ls3[k]));
        eb_t M[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) M[i][j] = eb_mul(Qe[i][j], se[j]);
        /* the renderer's float camera-space mean: nearest float to a value held to 2^-38 */
        const double tmag[3] = {fabs(W[0] * mx) + fabs(W[1] * my) + fabs(W[2] * mz) + fabs(cam->t[0]),
                                fabs(W[3] * mx) + fabs(W[4] * my) + fabs(W[5] * mz) + fabs(cam->t[1]), zmag};
        const eb_t te[3] = {eb(tx, 0.5 * ulp32(tx) + 0x1p-38 * tmag[0]), eb(ty, 0.5 * ulp32(ty) + 0x1p-38 * tmag[1]),
                            eb(tz, 0.5 * ulp32(tz) + 0x1p-38 * tmag[2])};
        const eb_t fxe = eb_in(fx), fye = eb_in(fy), fc = eb_in(P->fov_clamp);
        const eb_t lx = eb_mul(fc, eb_div(eb_in(cam->width), eb_scale(fxe, 2.0)));
        const eb_t ly = eb_mul(fc, eb_div(eb_in(cam->height), eb_scale(fye, 2.0)));
        const eb_t xce = eb_clamp(eb_div(te[0], te[2]), lx), yce = eb_clamp(eb_div(te[1], te[2]), ly);
        const eb_t tz2 = eb_mul(te[2], te[2]);
        const eb_t j00 = eb_div(fxe, te[2]), j02 = eb_neg(eb_div(eb_mul(fxe, eb_mul(xce, te[2])), tz2));
        const eb_t j11 = eb_div(fye, te[2]), j12 = eb_neg(eb_div(eb_mul(fye, eb_mul(yce, te[2])), tz2));
        eb_t Te[2][3];
        for (int k = 0; k < 3; k++) {
            Te[0][k] = eb_add(eb_mul(j00, eb_in(W[k])), eb_mul(j02, eb_in(W[6 + k])));
            Te[1][k] = eb_add(eb_mul(j11, eb_in(W[3 + k])), eb_mul(j12, eb_in(W[6 + k])));
        }
        const eb_t dil = eb_in(P->dilation);
        /* (i) V = T M, Sigma' = V V^T + dil I, det by Cauchy-Binet */
        eb_t V[2][3];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                eb_t t3[3] = {eb_mul(Te[r][0], M[0][k]), eb_mul(Te[r][1], M[1][k]), eb_mul(Te[r][2], M[2][k])};
                V[r][k] = eb_sum(t3, 3);
            }
        eb_t t00[3], t11[3];
        for (int k = 0; k < 3; k++) { t00[k] = eb_mul(V[0][k], V[0][k]); t11[k] = eb_mul(V[1][k], V[1][k]); }
        const eb_t s00 = eb_sum(t00, 3), s11 = eb_sum(t11, 3);
        const eb_t av = eb_add(s00, dil), cv = eb_add(s11, dil);
        const eb_t m01 = eb_sub(eb_mul(V[0][0], V[1][1]), eb_mul(V[0][1], V[1][0]));
        const eb_t m02 = eb_sub(eb_mul(V[0][0], V[1][2]), eb_mul(V[0][2], V[1][0]));
        const eb_t m12 = eb_sub(eb_mul(V[0][1], V[1][2]), eb_mul(V[0][2], V[1][1]));
        const eb_t dterms[5] = {eb_mul(m01, m01), eb_mul(m02, m02), eb_mul(m12, m12),
                                eb_mul(dil, eb_add(s00, s11)), eb_mul(dil, dil)};
        const eb_t detv = eb_sum(dterms, 5);
        const eb_t lamv = lambda_max_eb(av, cv, detv);
        /* (ii) Sigma = M M^T, Sigma' = T Sigma T^T + dil I, det = a c - b^2 */
        eb_t Se[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                eb_t t3[3] = {eb_mul(M[i][0], M[j][0]), eb_mul(M[i][1], M[j][1]), eb_mul(M[i][2], M[j][2])};
                Se[i][j] = eb_sum(t3, 3);
            }
        eb_t S2e[2][2];
        for (int r = 0; r < 2; r++)
            for (int cc = 0; cc < 2; cc++) {
                eb_t t9[9];
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) t9[3 * i + j] = eb_mul(eb_mul(Te[r][i], Se[i][j]), Te[cc][j]);
                S2e[r][cc] = eb_sum(t9, 9);
            }
        const eb_t as = eb_add(S2e[0][0], dil), bs = S2e[0][1], cs = eb_add(S2e[1][1], dil);
        const eb_t dets = eb_sub(eb_mul(as, cs), eb_mul(bs, bs));
        const eb_t lams = lambda_max_eb(as, cs, dets);
        /* ext = 3 sqrt(lambda): its bound from each lambda bound */
        const eb_t e1 = eb_mul(eb_in(3.0), eb_sqrt(lamv)), e2 = eb_mul(eb_in(3.0), eb_sqrt(lams));
        det_err = fmax(detv.e, dets.e);
        ext_err = fmax(e1.e, e2.e);
    }
    if (fabs(det) <= 2.0 * det_err) o->tie |= OR_TIE_DET;
    if (!(det > 0.0)) { if (o->status == OR_ACTIVE) o->status = OR_DEGENERATE; return; }
    o->conA = c / det; o->conB = -b / det; o->conC = a / det;
    const double mid = 0.5 * (a + c);
    double disc = mid * mid - det;
    if (disc < 0.1) disc = 0.1;
    const double lam = mid + sqrt(disc);
    const double ext = 3.0 * sqrt(lam);
    o->extent = ext;
    o->extent_err = ext_err;
    /* ceil(ext) changes where ext crosses an integer */
    if (dist_int(ext) <= 2.0 * ext_err) o->tie |= OR_TIE_RADIUS;
    o->radius = (int)ceil(ext);
    const double u = fx * tx / tz + cam->cx;
    const double v = fy * ty / tz + cam->cy;
    o->u = u; o->v = v;
    const int r = o->radius, tw = P->tile_w, th = P->tile_h;
    const int tiles_x = (cam->width + tw - 1) / tw;
    const int tiles_y = (cam->height + th - 1) / th;
    /* the rectangle from the renderer's float mean (within 1/2 ulp + 2^-38 of
     * the exact one) and the integer radius is exact arithmetic: an edge can
     * move only where (u +- r) lies within that of a tile boundary */
    const double bu = 0.5 * ulp32(u) + 0x1p-38 * fabs(u) + 1e-300, bv = 0.5 * ulp32(v) + 0x1p-38 * fabs(v) + 1e-300;
    const double e[4] = {(u - r) / tw, (v - r) / th, (u + r) / tw, (v + r) / th};
    const double be[4] = {2.0 * bu / tw, 2.0 * bv / th, 2.0 * bu / tw, 2.0 * bv / th};
    for (int k = 0; k < 4; k++)
        if (dist_int(e[k]) <= be[k]) o->tie |= OR_TIE_RECT;
    int x0 = (int)floor(e[0]), y0 = (int)floor(e[1]);
    int x1 = (int)floor(e[2]) + 1, y1 = (int)floor(e[3]) + 1;
    x0 = x0 < 0 ? 0 : (x0 > tiles_x ? tiles_x : x0);
    x1 = x1 < 0 ? 0 : (x1 > tiles_x ? tiles_x : x1);
    y0 = y0 < 0 ? 0 : (y0 > tiles_y ? tiles_y : y0);
    y1 = y1 < 0 ? 0 : (y1 > tiles_y ? tiles_y : y1);
    o->rect[0] = x0; o->rect[1] = y0; o->rect[2] = x1; o->rect[3] = y1;
    if ((x1 <= x0 || y1 <= y0) && o->status == OR_ACTIVE) o->status = OR_EMPTY;
}

/* ---- spherical harmonics from the definition ---------------------------- */
static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
}

/* coefficients (ascending powers of z) of d^m/dz^m P_l(z), P_l by Rodrigues:
 * P_l(z) = 1/(2^l l!) d^l/dz^l (z^2 - 1)^l */
static void legendre_deriv_coeffs(int l, int m, double *c /* [2l+1] */)
{
    double p[16] = {0};
    /* (z^2 - 1)^l = sum_k C(l,k) z^{2k} (-1)^{l-k} */
    for (int k = 0; k <= l; k++) {
        double binom = factorial(l) / (factorial(k) * factorial(l - k));
        p[2 * k] = binom * (((l - k) & 1) ? -1.0 : 1.0);
    }
    int deg = 2 * l;
    for (int d = 0; d < l + m && deg >= 0; d++) { /* differentiate l + m times */
        for (int i = 0; i < deg; i++) p[i] = p[i + 1] * (i + 1);
        p[deg] = 0.0;
        deg--;
    }
    double norm = 1.0 / (pow(2.0, l) * factorial(l));
    for (int i = 0; i <= 2 * l; i++) c[i] = (i <= deg && deg >= 0) ? p[i] * norm : 0.0;
}

static double poly_eval(const double *c, int n, double z)
{
    double r = 0.0;
    for (int i = n - 1; i >= 0; i--) r = r * z + c[i];
    return r;
}

/* Real SH Y_k, k = l^2 + l + m, at the unit vector (x, y, z), and optionally the
 * gradient of each Y_k (as a polynomial on R^3) with respect to (x, y, z).
 * P_l^m(cos t) = (-1)^m sin^m t Q_lm(cos t), Q_lm = d^m P_l / dz^m, and
 * sin^m t e^{i m phi} = (x + i y)^m. */
void or_sh_basis(const double *dirs, int64_t count, double *Y, double *dY)
{
    for (int64_t n = 0; n < count; n++) {
        double x = dirs[3 * n], y = dirs[3 * n + 1], z = dirs[3 * n + 2];
        /* powers of (x + i y) */
        double re[5], im[5];
        re[0] = 1.0; im[0] = 0.0;
        for (int m = 1; m < 5; m++) {
            re[m] = re[m - 1] * x - im[m - 1] * y;
            im[m] = re[m - 1] * y + im[m - 1] * x;
        }
        for (int l = 0; l <= 3; l++) {
            for (int m = -l; m <= l; m++) {
                int am = m < 0 ? -m : m;
                double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
                double sgn = (am & 1) ? -1.0 : 1.0; /* Condon-Shortley phase */
                double q[8], q1[8];
                legendre_deriv_coeffs(l, am, q);
                legendre_deriv_coeffs(l, am + 1, q1);
                double Q = poly_eval(q, 2 * l + 1, z), dQ = poly_eval(q1, 2 * l + 1, z);
                double pref, trig, dtrig_dx, dtrig_dy;
                if (m == 0) {
                    pref = K; trig = 1.0; dtrig_dx = 0.0; dtrig_dy = 0.0;
                } else if (m > 0) {
                    pref = sqrt(2.0) * K * sgn;
                    trig = re[am];
                    dtrig_dx = am * re[am - 1];
                    dtrig_dy = -am * im[am - 1];
                } else {
                    pref = sqrt(2.0) * K * sgn;
                    trig = im[am];
                    dtrig_dx = am * im[am - 1];
                    dtrig_dy = am * re[am - 1];
                }
                int k = l * l + l + m;
                Y[16 * n + k] = pref * Q * trig;
                if (dY) {
                    dY[48 * n + 3 * k + 0] = pref * Q * dtrig_dx;
                    dY[48 * n + 3 * k + 1] = pref * Q * dtrig_dy;
                    dY[48 * n + 3 * k + 2] = pref * dQ * trig;
                }
            }
        }
    }
}

/* ---- forward: projection + colour ------------------------------------- */
typedef struct {
    int8_t *status;     /* n */
    uint8_t *tie;       /* n */
    double *uv;         /* 2n */
    double *depth;      /* n, FP64 camera z */
    float *depth32;     /* n, FP32 camera z (sort key) */
    double *conic;      /* 3n: A, B, C */
    double *opacity;    /* n */
    double *rgb;        /* 3n */
    uint8_t *clamp;     /* n: bit c set when colour channel c was clamped at 0 */
    int32_t *radius;    /* n */
    int32_t *rect;      /* 4n */
    int32_t *tiles;     /* n */
    double *extent;     /* 2n: 3 sqrt(lambda_max) and the FP32 error bound of it */
} or_proj_out;

static int cull_bit(const uint32_t *cull, int64_t i)
{
    return cull ? (int)((cull[i >> 5] >> (i & 31)) & 1u) : 0;
}

int or_project(int64_t n, const double *mean, const double *log_scale, const double *quat,
               const double *opacity_logit, const double *sh, const uint8_t *lod,
               const uint32_t *cull, const or_camera *cam, const or_params *P, or_proj_out *out)
{
    for (int64_t i = 0; i < n; i++) {
        double m3[3] = {mean[i], mean[n + i], mean[2 * n + i]};
        double s3[3] = {log_scale[i], log_scale[n + i], log_scale[2 * n + i]};
        double q4[4] = {quat[i], quat[n + i], quat[2 * n + i], quat[3 * n + i]};
        int l = lod ? lod[i] : 0;
        int cb = cull_bit(cull, i);
        proj_t pj;
        project_one(m3, s3, q4, l, cb, cam, P, &pj);
        out->status[i] = (int8_t)pj.status;
        out->tie[i] = (uint8_t)pj.tie;
        out->depth32[i] = (float)pj.tz; /* the depth key: the FP32 value of the exact depth */
        out->depth[i] = pj.tz;
        out->radius[i] = pj.radius;
        for (int k = 0; k < 4; k++) out->rect[4 * i + k] = pj.rect[k];
        out->tiles[i] = pj.status == OR_ACTIVE ? (pj.rect[2] - pj.rect[0]) * (pj.rect[3] - pj.rect[1]) : 0;
        out->uv[2 * i] = pj.u;
        out->uv[2 * i + 1] = pj.v;
        if (out->extent) { out->extent[2 * i] = pj.extent; out->extent[2 * i + 1] = pj.extent_err; }
        out->conic[3 * i] = pj.conA;
        out->conic[3 * i + 1] = pj.conB;
        out->conic[3 * i + 2] = pj.conC;
        out->opacity[i] = 1.0 / (1.0 + exp(-opacity_logit[i]));
        /* view-dependent colour, degree-3 SH, +0.5 offset, clamped at 0 */
        double d[3] = {m3[0] - cam->campos[0], m3[1] - cam->campos[1], m3[2] - cam->campos[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        d[0] /= dn; d[1] /= dn; d[2] /= dn;
        double Y[16];
        or_sh_basis(d, 1, Y, NULL);
        uint8_t cm = 0;
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
            for (int k = 0; k < 16; k++) acc += sh[(int64_t)(3 * k + c) * n + i] * Y[k];
            acc += 0.5;
            if (fabs(acc) <= 1e-6) out->tie[i] |= OR_TIE_CLAMP;
            if (acc < 0.0) { acc = 0.0; cm |= (uint8_t)(1u << c); }
            out->rgb[3 * i + c] = acc;
        }
        out->clamp[i] = cm;
    }
    return 0;
}

/* ---- binning: per-tile lists ordered by (depth bits, index) ------------ */
typedef struct { uint32_t key; int32_t idx; } kv_t;

static int kv_cmp(const void *pa, const void *pb)
{
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

static uint32_t f32_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Fills tile_start[0..ntiles] and list[]; returns the instance count or -1 if
 * it exceeds cap.  Tile t = ty * tiles_x + tx. */
int64_t or_bin(int64_t n, const int8_t *status, const int32_t *rect, const float *depth32,
               int32_t tiles_x, int32_t tiles_y, int64_t *tile_start, int32_t *list, int64_t cap)
{
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t *count = (int64_t *)calloc((size_t)ntiles, sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        if (status[i] != OR_ACTIVE) continue;
        for (int y = rect[4 * i + 1]; y < rect[4 * i + 3]; y++)
            for (int x = rect[4 * i]; x < rect[4 * i + 2]; x++) count[(int64_t)y * tiles_x + x]++;
    }
    tile_start[0] = 0;
    for (int64_t t = 0; t < ntiles; t++) tile_start[t + 1] = tile_start[t] + count[t];
    int64_t total = tile_start[ntiles];
    if (total > cap) { free(count); return -1; }
    memset(count, 0, (size_t)ntiles * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        if (status[i] != OR_ACTIVE) continue;
        for (int y = rect[4 * i + 1]; y < rect[4 * i + 3]; y++)
            for (int x = rect[4 * i]; x < rect[4 * i + 2]; x++) {
                int64_t t = (int64_t)y * tiles_x + x;
                list[tile_start[t] + count[t]++] = (int32_t)i;
            }
    }
    kv_t *buf = NULL;
    int64_t bufcap = 0;
    for (int64_t t = 0; t < ntiles; t++) {
        int64_t len = tile_start[t + 1] - tile_start[t];
        if (len > bufcap) { free(buf); bufcap = len; buf = (kv_t *)malloc((size_t)bufcap * sizeof(kv_t)); }
        for (int64_t j = 0; j < len; j++) {
            int32_t g = list[tile_start[t] + j];
            buf[j].key = f32_bits(depth32[g]);
            buf[j].idx = g;
        }
        qsort(buf, (size_t)len, sizeof(kv_t), kv_cmp);
        for (int64_t j = 0; j < len; j++) list[tile_start[t] + j] = buf[j].idx;
    }
    free(buf);
    free(count);
    return total;
}

/* ---- compositing of one pixel (App. A, Eq. for C(p)) -------------------- */
typedef struct {
    double C[3], T;
    int32_t n_contrib;
    uint8_t flags;
} pix_t;

/* x within a relative distance band of thr, measured in log space so that an
 * error bound on an exponent applies directly (band ~ |log(x / thr)|). */
static int near_log(double x, double thr, double band)
{
    return x > 0.0 && fabs(log(x / thr)) <= band;
}

/* How far an FP32 renderer's exponent for this fragment can be from the exact
 * one, for a renderer that holds each Gaussian's exponent as
 * A (x + k y)^2 + D y^2 (k = B / A, D = C - B^2 / A) with |dA| <= pc A,
 * |dD| <= pc D, |dk| <= pc (|k| + sqrt(D / A)) (pc = prec_conic) and its mean
 * within pm = prec_mean pixels, and evaluates the form, the exponential and
 * o G in FP32.  With e = dx + k dy:
 *   |de|  <= pm (1 + |k|) + |dy| pc (|k| + sqrt(D / A)) + 2 U32 (|dx| + 2 |k dy|)
 *   |dp|  <= pc |p| + A |e| |de| + A |de|^2 / 2 + D |dy| pm + 4 U32 |p|
 * plus 2^-21 for the exponential and 8 U32 for the opacity.  Returned
 * doubled: a fragment whose alpha lies within this (in log space) of a
 * threshold may be decided the other way by such a renderer. */
static double fp32_power_err(const or_params *P, const double *conic, int32_t g, double dx, double dy,
                             double power)
{
    const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
    const double k = B / A, D = C - B * k;
    const double pm = P->prec_mean, pc = P->prec_conic;
    const double e = dx + k * dy;
    const double de = pm * (1.0 + fabs(k)) + fabs(dy) * pc * (fabs(k) + sqrt(fabs(D / A)))
                    + 2.0 * U32 * (fabs(dx) + 2.0 * fabs(k * dy));
    const double dp = pc * fabs(power) + A * fabs(e) * de + 0.5 * A * de * de + fabs(D * dy) * pm
                    + 4.0 * U32 * fabs(power);
    return 2.0 * (dp + 0x1p-21 + 8.0 * U32);
}

/* Composites the ordered Gaussians ids[0..len) at pixel centre (px, py).
 * Optional w/a accumulate the importance alpha-weight and pixel count.
 * Flags: a fragment within comp_band plus its own FP32 error bound (log
 * space) of the alpha_min, alpha_max or T_min threshold, or at the
 * exponent's maximum 0.
 * When the pixel is flagged and gcount is given, every Gaussian the pixel
 * composited or nearly composited has its count of such pixels raised. */
static void composite_pixel(const or_params *P, double px, double py, const int32_t *ids, int64_t len,
                            const double *uv, const double *conic, const double *opacity,
                            const double *rgb, pix_t *o, double *w, double *a, int32_t *gcount)
{
    double T = 1.0, C[3] = {0, 0, 0};
    double T_relerr = 0.0; /* bound on the relative error of T in FP32 */
    int32_t nc = 0;
    uint8_t fl = 0;
    int64_t jstop = len;
    for (int64_t j = 0; j < len; j++) {
        int32_t g = ids[j];
        double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
        double A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
        double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        const double perr = fp32_power_err(P, conic, g, dx, dy, power);
        if (power > 0.0) { fl |= OR_PIX_POWER; continue; } /* only from rounding at the centre */
        double G = exp(power);
        double og = opacity[g] * G;
        if (near_log(og, P->alpha_max, P->comp_band + perr)) fl |= OR_PIX_ALPHA_MAX;
        const int clamped = og >= P->alpha_max;
        double alpha = clamped ? P->alpha_max : og;
        if (near_log(alpha, P->alpha_min, P->comp_band + perr)) fl |= OR_PIX_ALPHA_MIN;
        if (alpha < P->alpha_min) continue;
        double testT = T * (1.0 - alpha);
        const double trel = T_relerr + (clamped ? 0.0 : perr * alpha / (1.0 - alpha));
        if (near_log(testT, P->T_min, P->comp_band + trel)) fl |= OR_PIX_T_MIN;
        if (testT < P->T_min) { jstop = j; break; }
        for (int c = 0; c < 3; c++) C[c] += alpha * T * rgb[3 * g + c];
        if (w) w[g] += alpha * T;
        if (a) a[g] += 1.0;
        T = testT;
        T_relerr = trel + 2.0 * 5.9604644775390625e-08;
        nc = (int32_t)(j + 1);
    }
    for (int c = 0; c < 3; c++) o->C[c] = C[c] + T * P->bg[c];
    o->T = T;
    o->n_contrib = nc;
    o->flags = fl;
    if (fl && gcount) {
        for (int64_t j = 0; j <= jstop && j < len; j++) {
            int32_t g = ids[j];
            double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
            double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
            if (opacity[g] * exp(power) >= 0.5 * P->alpha_min) gcount[g] += 1;
        }
    }
}

/* Tiled render: image (3,H,W) planar, T_final (H,W), n_contrib (H,W), flags
 * (H,W); w, a (n) accumulate the importance signals when non-NULL; gcount (n)
 * counts, per Gaussian, the flagged pixels it takes part in, when non-NULL. */
int or_render(const or_camera *cam, const or_params *P, int64_t n, const double *uv, const double *conic,
              const double *opacity, const double *rgb, const int64_t *tile_start, const int32_t *list,
              double *image, double *T_final, int32_t *n_contrib, uint8_t *flags, double *w, double *a,
              int32_t *gcount)
{
    (void)n;
    const int W = cam->width, H = cam->height, tw = P->tile_w, th = P->tile_h;
    const int tiles_x = (W + tw - 1) / tw;
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int64_t t = (int64_t)(py / th) * tiles_x + px / tw;
            pix_t o;
            composite_pixel(P, px + 0.5, py + 0.5, list + tile_start[t], tile_start[t + 1] - tile_start[t],
                            uv, conic, opacity, rgb, &o, w, a, gcount);
            int64_t p = (int64_t)py * W + px;
            for (int c = 0; c < 3; c++) image[(int64_t)c * W * H + p] = o.C[c];
            T_final[p] = o.T;
            n_contrib[p] = o.n_contrib;
            flags[p] = o.flags;
        }
    return 0;
}

/* Untiled brute force: every pixel composites ALL active Gaussians in
 * (depth bits, index) order, with no tile lists and no rectangles. */
int or_render_brute(const or_camera *cam, const or_params *P, int64_t n, const int8_t *status,
                    const float *depth32, const double *uv, const double *conic, const double *opacity,
                    const double *rgb, double *image, double *T_final)
{
    kv_t *buf = (kv_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv_t));
    int32_t *ids = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (status[i] == OR_ACTIVE) { buf[m].key = f32_bits(depth32[i]); buf[m].idx = (int32_t)i; m++; }
    qsort(buf, (size_t)m, sizeof(kv_t), kv_cmp);
    for (int64_t j = 0; j < m; j++) ids[j] = buf[j].idx;
    const int W = cam->width, H = cam->height;
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            pix_t o;
            composite_pixel(P, px + 0.5, py + 0.5, ids, m, uv, conic, opacity, rgb, &o, NULL, NULL, NULL);
            int64_t p = (int64_t)py * W + px;
            for (int c = 0; c < 3; c++) image[(int64_t)c * W * H + p] = o.C[c];
            T_final[p] = o.T;
        }
    free(buf);
    free(ids);
    return 0;
}

/* Composites a list of pixels (px, py given as integer pixel indices) with
 * explicit per-pixel Gaussian lists: used for sampled checks at full size. */
int or_render_pixels(const or_params *P, int64_t npix, const int32_t *pxy, const int64_t *list_start,
                     const int32_t *lists, const double *uv, const double *conic, const double *opacity,
                     const double *rgb, double *C, double *T, int32_t *n_contrib, uint8_t *flags)
{
    for (int64_t k = 0; k < npix; k++) {
        pix_t o;
        composite_pixel(P, pxy[2 * k] + 0.5, pxy[2 * k + 1] + 0.5, lists + list_start[k],
                        list_start[k + 1] - list_start[k], uv, conic, opacity, rgb, &o, NULL, NULL, NULL);
        for (int c = 0; c < 3; c++) C[3 * k + c] = o.C[c];
        T[k] = o.T;
        n_contrib[k] = o.n_contrib;
        flags[k] = o.flags;
    }
    return 0;
}

/* ---- backward of the compositing --------------------------------------
 * For one pixel with composited fragments k = 1..K (alpha_k, T_k, c_k) and
 * upstream gradient g = dL/dC(p):
 *   dL/dc_k     = alpha_k T_k g
 *   dL/dalpha_k = g . (T_k c_k - S_k / (1 - alpha_k)) - T_K+1 (g . bg) / (1 - alpha_k)
 * with S_k = sum_{m > k} alpha_m T_m c_m (every later term carries the factor
 * (1 - alpha_k), and so does the final transmittance).  alpha = min(amax, o G):
 * when o G >= amax the derivative through alpha is zero. */
int or_render_bwd(const or_camera *cam, const or_params *P, int64_t n, const double *uv, const double *conic,
                  const double *opacity, const double *rgb, const int64_t *tile_start, const int32_t *list,
                  const double *dL_dimage, double *dL_duv, double *dL_dconic, double *dL_dopacity,
                  double *dL_drgb, double *dL_dconic_abs)
{
    (void)n;
    const int W = cam->width, H = cam->height, tw = P->tile_w, th = P->tile_h;
    const int tiles_x = (W + tw - 1) / tw;
    int64_t cap = 0;
    int32_t *frag = NULL;
    double *fa = NULL, *fT = NULL, *fG = NULL, *fog = NULL;
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int64_t t = (int64_t)(py / th) * tiles_x + px / tw;
            const int32_t *ids = list + tile_start[t];
            int64_t len = tile_start[t + 1] - tile_start[t];
            if (len > cap) {
                cap = len;
                frag = (int32_t *)realloc(frag, (size_t)cap * sizeof(int32_t));
                fa = (double *)realloc(fa, (size_t)cap * sizeof(double));
                fT = (double *)realloc(fT, (size_t)cap * sizeof(double));
                fG = (double *)realloc(fG, (size_t)cap * sizeof(double));
                fog = (double *)realloc(fog, (size_t)cap * sizeof(double));
            }
            const double pxc = px + 0.5, pyc = py + 0.5;
            /* forward pass recording the composited fragments */
            double T = 1.0;
            int64_t K = 0;
            for (int64_t j = 0; j < len; j++) {
                int32_t g = ids[j];
                double dx = pxc - uv[2 * g], dy = pyc - uv[2 * g + 1];
                double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
                if (power > 0.0) continue;
                double G = exp(power), og = opacity[g] * G;
                double alpha = og < P->alpha_max ? og : P->alpha_max;
                if (alpha < P->alpha_min) continue;
                double testT = T * (1.0 - alpha);
                if (testT < P->T_min) break;
                frag[K] = g; fa[K] = alpha; fT[K] = T; fG[K] = G; fog[K] = og;
                K++;
                T = testT;
            }
            const double Tfin = T;
            int64_t p = (int64_t)py * W + px;
            double gpix[3] = {dL_dimage[p], dL_dimage[(int64_t)W * H + p], dL_dimage[2 * (int64_t)W * H + p]};
            double gbg = gpix[0] * P->bg[0] + gpix[1] * P->bg[1] + gpix[2] * P->bg[2];
            double S[3] = {0, 0, 0}; /* sum over later fragments of alpha T c */
            for (int64_t k = K - 1; k >= 0; k--) {
                int32_t g = frag[k];
                const double *c = rgb + 3 * g;
                double dalpha = 0.0;
                for (int ch = 0; ch < 3; ch++) {
                    dL_drgb[3 * g + ch] += fa[k] * fT[k] * gpix[ch];
                    dalpha += gpix[ch] * (fT[k] * c[ch] - S[ch] / (1.0 - fa[k]));
                }
                dalpha -= Tfin * gbg / (1.0 - fa[k]);
                for (int ch = 0; ch < 3; ch++) S[ch] += fa[k] * fT[k] * c[ch];
                if (fog[k] >= P->alpha_max) continue; /* clamped: no derivative */
                dL_dopacity[g] += fG[k] * dalpha;
                double dG = opacity[g] * dalpha;
                double dpower = fG[k] * dG;
                double dx = pxc - uv[2 * g], dy = pyc - uv[2 * g + 1];
                double A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
                /* power = -A dx^2 / 2 - B dx dy - C dy^2 / 2, dx = px - u */
                dL_duv[2 * g] += dpower * (A * dx + B * dy);
                dL_duv[2 * g + 1] += dpower * (Cc * dy + B * dx);
                dL_dconic[3 * g] += dpower * (-0.5 * dx * dx);
                dL_dconic[3 * g + 1] += dpower * (-dx * dy);
                dL_dconic[3 * g + 2] += dpower * (-0.5 * dy * dy);
                if (dL_dconic_abs) { /* magnitudes of the pixel terms, for FP32 error bounds */
                    dL_dconic_abs[3 * g] += fabs(dpower * 0.5 * dx * dx);
                    dL_dconic_abs[3 * g + 1] += fabs(dpower * dx * dy);
                    dL_dconic_abs[3 * g + 2] += fabs(dpower * 0.5 * dy * dy);
                }
            }
        }
    free(frag); free(fa); free(fT); free(fG); free(fog);
    return 0;
}

/* ---- backward of the projection and colour (chain rule) ---------------- */
static void quat_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* dR/dq_k for the rotation matrix of a (unit) quaternion, as a polynomial in q */
static void quat_rot_grad(const double q[4], double dR[4][3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double Dw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
    double Dx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
    double Dy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
    double Dz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
    memcpy(dR[0], Dw, sizeof(Dw));
    memcpy(dR[1], Dx, sizeof(Dx));
    memcpy(dR[2], Dy, sizeof(Dy));
    memcpy(dR[3], Dz, sizeof(Dz));
}

/* Accumulates (+=) parameter gradients of every Gaussian with status ACTIVE
 * from the gradients of its projected quantities u, v, conic (A, B, C),
 * opacity and rgb, for one camera. */
int or_project_bwd(int64_t n, const double *mean, const double *log_scale, const double *quat,
                   const double *opacity_logit, const double *sh, const int8_t *status, const uint8_t *clamp,
                   const or_camera *cam, const or_params *P, const double *dL_duv, const double *dL_dconic,
                   const double *dL_dopacity, const double *dL_drgb, double *g_mean, double *g_log_scale,
                   double *g_quat, double *g_opacity_logit, double *g_sh)
{
    const double *Wc = cam->R;
    const double fx = cam->fx, fy = cam->fy;
    for (int64_t i = 0; i < n; i++) {
        if (status[i] != OR_ACTIVE) continue;
        double m3[3] = {mean[i], mean[n + i], mean[2 * n + i]};
        double t[3];
        for (int r = 0; r < 3; r++) t[r] = Wc[3 * r] * m3[0] + Wc[3 * r + 1] * m3[1] + Wc[3 * r + 2] * m3[2] + cam->t[r];
        double qraw[4] = {quat[i], quat[n + i], quat[2 * n + i], quat[3 * n + i]};
        double qn = sqrt(qraw[0] * qraw[0] + qraw[1] * qraw[1] + qraw[2] * qraw[2] + qraw[3] * qraw[3]);
        double q[4] = {qraw[0] / qn, qraw[1] / qn, qraw[2] / qn, qraw[3] / qn};
        double Q[3][3];
        quat_rot(q, Q);
        double s[3] = {exp(log_scale[i]), exp(log_scale[n + i]), exp(log_scale[2 * n + i])};
        double M[3][3], Sg[3][3];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) M[a][b] = Q[a][b] * s[b];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) Sg[a][b] = M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2];
        /* Jacobian with the field-of-view clamp */
        double limx = P->fov_clamp * (cam->width / (2.0 * fx));
        double limy = P->fov_clamp * (cam->height / (2.0 * fy));
        double xr = t[0] / t[2], yr = t[1] / t[2];
        int cx_cl = xr < -limx || xr > limx, cy_cl = yr < -limy || yr > limy;
        double xc = xr < -limx ? -limx : (xr > limx ? limx : xr); /* clamped tx/tz */
        double yc = yr < -limy ? -limy : (yr > limy ? limy : yr);
        double J[2][3] = {{fx / t[2], 0.0, -fx * xc / t[2]}, {0.0, fy / t[2], -fy * yc / t[2]}};
        double T[2][3];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) T[r][k] = J[r][0] * Wc[k] + J[r][1] * Wc[3 + k] + J[r][2] * Wc[6 + k];
        double S2[2][2];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) {
                double acc = 0.0;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) acc += T[r][a] * Sg[a][b] * T[c][b];
                S2[r][c] = acc;
            }
        double a = S2[0][0] + P->dilation, b = S2[0][1], c = S2[1][1] + P->dilation;
        double det = a * c - b * b, det2 = det * det;
        /* conic (A, B, C) = (c, -b, a) / det */
        double gA = dL_dconic[3 * i], gB = dL_dconic[3 * i + 1], gC = dL_dconic[3 * i + 2];
        double ga = gA * (-c * c / det2) + gB * (b * c / det2) + gC * (1.0 / det - a * c / det2);
        double gb = gA * (2.0 * b * c / det2) + gB * (-1.0 / det - 2.0 * b * b / det2) + gC * (2.0 * a * b / det2);
        double gc = gA * (1.0 / det - a * c / det2) + gB * (a * b / det2) + gC * (-a * a / det2);
        /* symmetric dL/dSigma' (b appears in both off-diagonal entries) */
        double G2[2][2] = {{ga, 0.5 * gb}, {0.5 * gb, gc}};
        /* Sigma' = T Sigma T^T: dL/dSigma = T^T G2 T, dL/dT = 2 G2 T Sigma */
        double gS[3][3], gT[2][3];
        for (int p = 0; p < 3; p++)
            for (int q2 = 0; q2 < 3; q2++) {
                double acc = 0.0;
                for (int r = 0; r < 2; r++)
                    for (int c2 = 0; c2 < 2; c2++) acc += T[r][p] * G2[r][c2] * T[c2][q2];
                gS[p][q2] = acc;
            }
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int c2 = 0; c2 < 2; c2++)
                    for (int m = 0; m < 3; m++) acc += 2.0 * G2[r][c2] * T[c2][m] * Sg[m][k];
                gT[r][k] = acc;
            }
        /* T = J W  ->  dL/dJ = dL/dT W^T */
        double gJ[2][3];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) gJ[r][k] = gT[r][0] * Wc[3 * k] + gT[r][1] * Wc[3 * k + 1] + gT[r][2] * Wc[3 * k + 2];
        /* J entries as functions of t (exact derivative of the clamp) */
        double tz = t[2], tz2 = tz * tz, tz3 = tz2 * tz;
        double gt[3] = {0, 0, 0};
        gt[2] += gJ[0][0] * (-fx / tz2) + gJ[1][1] * (-fy / tz2);
        if (!cx_cl) { gt[0] += gJ[0][2] * (-fx / tz2); gt[2] += gJ[0][2] * (2.0 * fx * t[0] / tz3); }
        else        { gt[2] += gJ[0][2] * (fx * xc / tz2); }
        if (!cy_cl) { gt[1] += gJ[1][2] * (-fy / tz2); gt[2] += gJ[1][2] * (2.0 * fy * t[1] / tz3); }
        else        { gt[2] += gJ[1][2] * (fy * yc / tz2); }
        /* u = fx tx / tz + cx, v = fy ty / tz + cy */
        double gu = dL_duv[2 * i], gv = dL_duv[2 * i + 1];
        gt[0] += gu * fx / tz;
        gt[1] += gv * fy / tz;
        gt[2] += gu * (-fx * t[0] / tz2) + gv * (-fy * t[1] / tz2);
        /* t = W mu + t0 */
        double gm[3];
        for (int k = 0; k < 3; k++) gm[k] = Wc[k] * gt[0] + Wc[3 + k] * gt[1] + Wc[6 + k] * gt[2];
        /* Sigma = M M^T, M = Q diag(s): dL/dM = 2 dL/dSigma M (dL/dSigma symmetric) */
        double gSs[3][3];
        for (int p = 0; p < 3; p++)
            for (int q2 = 0; q2 < 3; q2++) gSs[p][q2] = 0.5 * (gS[p][q2] + gS[q2][p]);
        double gM[3][3];
        for (int p = 0; p < 3; p++)
            for (int q2 = 0; q2 < 3; q2++) gM[p][q2] = 2.0 * (gSs[p][0] * M[0][q2] + gSs[p][1] * M[1][q2] + gSs[p][2] * M[2][q2]);
        double gs[3] = {0, 0, 0}, gQ[3][3];
        for (int p = 0; p < 3; p++)
            for (int q2 = 0; q2 < 3; q2++) { gs[q2] += gM[p][q2] * Q[p][q2]; gQ[p][q2] = gM[p][q2] * s[q2]; }
        for (int k = 0; k < 3; k++) g_log_scale[(int64_t)k * n + i] += gs[k] * s[k];
        double dR[4][3][3];
        quat_rot_grad(q, dR);
        double gq[4];
        for (int k = 0; k < 4; k++) {
            double acc = 0.0;
            for (int p = 0; p < 3; p++)
                for (int q2 = 0; q2 < 3; q2++) acc += gQ[p][q2] * dR[k][p][q2];
            gq[k] = acc;
        }
        /* q = qraw / |qraw| */
        double qdot = q[0] * gq[0] + q[1] * gq[1] + q[2] * gq[2] + q[3] * gq[3];
        for (int k = 0; k < 4; k++) g_quat[(int64_t)k * n + i] += (gq[k] - q[k] * qdot) / qn;
        /* opacity = sigmoid(logit) */
        double o = 1.0 / (1.0 + exp(-opacity_logit[i]));
        g_opacity_logit[i] += dL_dopacity[i] * o * (1.0 - o);
        /* colour: rgb_c = max(sum_k sh_kc Y_k(d) + 0.5, 0), d = (mu - campos)/|mu - campos| */
        double dv[3] = {m3[0] - cam->campos[0], m3[1] - cam->campos[1], m3[2] - cam->campos[2]};
        double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double d[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
        double Y[16], dY[48];
        or_sh_basis(d, 1, Y, dY);
        double gd[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ch++) {
            if (clamp[i] & (1u << ch)) continue;
            double gr = dL_drgb[3 * i + ch];
            for (int k = 0; k < 16; k++) {
                double coef = sh[(int64_t)(3 * k + ch) * n + i];
                g_sh[(int64_t)(3 * k + ch) * n + i] += gr * Y[k];
                for (int e = 0; e < 3; e++) gd[e] += gr * coef * dY[3 * k + e];
            }
        }
        double ddot = d[0] * gd[0] + d[1] * gd[1] + d[2] * gd[2];
        for (int e = 0; e < 3; e++) gm[e] += (gd[e] - d[e] * ddot) / dn;
        for (int k = 0; k < 3; k++) g_mean[(int64_t)k * n + i] += gm[k];
    }
    return 0;
}

/* ---- FP32 error bounds of the scale and rotation gradients ----------------
 * With V = J W R(q) diag(s) and C = (V V^T + dilation I)^-1, w_k = C v_k (v_k the
 * columns of V) and G = dL/dconic = [[gA, gB/2], [gB/2, gC]]:
 *   dL/dlog s_k = -2 w_k^T G w_k,
 *   the rotation gradient (body frame) theta_i = -2 w_a^T G w_b (s_a/s_b - s_b/s_a)
 *   for (i, a, b) = (0, 1, 2), (1, 2, 0), (2, 0, 1), and dL/dq = (2/|q|) q (x) (0, theta).
 * Each pixel adds dpow (w_a . d)(w_b . d) to w_a^T G w_b: a short axis of a long
 * thin footprint sees pixel terms of gA, gB, gC that nearly cancel.  An FP32
 * renderer holds the summed G to within eps_sum of the sums of the magnitudes of
 * its pixel terms (dL_dconic_abs) and w_k to within prec_conic; the bound below
 * propagates both through the bilinear forms (first order, magnitudes):
 *   |d(w_a^T G w_b)| <= (eps_sum + 2 prec_conic) S_ab,
 *   S_ab = |w_a0 w_b0| SA + (|w_a0 w_b1| + |w_a1 w_b0|) SB / 2 + |w_a1 w_b1| SC.
 * Accumulates (+=) into ls_err (3n) and q_err (4n) for every ACTIVE Gaussian. */
int or_grad_bounds(int64_t n, const double *mean, const double *log_scale, const double *quat, const int8_t *status,
                   const or_camera *cam, const or_params *P, const double *dL_dconic_abs, double eps_sum,
                   double *ls_err, double *q_err)
{
    const double *Wc = cam->R;
    for (int64_t i = 0; i < n; i++) {
        if (status[i] != OR_ACTIVE) continue;
        double m3[3] = {mean[i], mean[n + i], mean[2 * n + i]};
        double t[3];
        for (int r = 0; r < 3; r++) t[r] = Wc[3 * r] * m3[0] + Wc[3 * r + 1] * m3[1] + Wc[3 * r + 2] * m3[2] + cam->t[r];
        double qr[4] = {quat[i], quat[n + i], quat[2 * n + i], quat[3 * n + i]};
        const double qn = sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
        const double q[4] = {qr[0] / qn, qr[1] / qn, qr[2] / qn, qr[3] / qn};
        double Q[3][3];
        quat_rot(q, Q);
        const double s[3] = {exp(log_scale[i]), exp(log_scale[n + i]), exp(log_scale[2 * n + i])};
        const double limx = P->fov_clamp * (cam->width / (2.0 * cam->fx));
        const double limy = P->fov_clamp * (cam->height / (2.0 * cam->fy));
        const double xr = t[0] / t[2], yr = t[1] / t[2];
        const double xc = xr < -limx ? -limx : (xr > limx ? limx : xr);
        const double yc = yr < -limy ? -limy : (yr > limy ? limy : yr);
        const double J[2][3] = {{cam->fx / t[2], 0.0, -cam->fx * xc / t[2]}, {0.0, cam->fy / t[2], -cam->fy * yc / t[2]}};
        double V[2][3];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int a = 0; a < 3; a++) {
                    double ta = J[r][0] * Wc[a] + J[r][1] * Wc[3 + a] + J[r][2] * Wc[6 + a];
                    acc += ta * Q[a][k] * s[k];
                }
                V[r][k] = acc;
            }
        const double a = V[0][0] * V[0][0] + V[0][1] * V[0][1] + V[0][2] * V[0][2] + P->dilation;
        const double b = V[0][0] * V[1][0] + V[0][1] * V[1][1] + V[0][2] * V[1][2];
        const double c = V[1][0] * V[1][0] + V[1][1] * V[1][1] + V[1][2] * V[1][2] + P->dilation;
        const double det = a * c - b * b;
        const double C00 = c / det, C01 = -b / det, C11 = a / det;
        double w[3][2];
        for (int k = 0; k < 3; k++) {
            w[k][0] = C00 * V[0][k] + C01 * V[1][k];
            w[k][1] = C01 * V[0][k] + C11 * V[1][k];
        }
        const double SA = dL_dconic_abs[3 * i], SB = dL_dconic_abs[3 * i + 1], SC = dL_dconic_abs[3 * i + 2];
        const double f = eps_sum + 2.0 * P->prec_conic;
#define S_AB(x, y) (fabs(w[x][0] * w[y][0]) * SA + 0.5 * (fabs(w[x][0] * w[y][1]) + fabs(w[x][1] * w[y][0])) * SB + \
                    fabs(w[x][1] * w[y][1]) * SC)
        for (int k = 0; k < 3; k++) ls_err[(int64_t)k * n + i] += 2.0 * f * S_AB(k, k);
        const double th[3] = {2.0 * f * S_AB(1, 2) * fabs(s[1] / s[2] - s[2] / s[1]),
                              2.0 * f * S_AB(2, 0) * fabs(s[2] / s[0] - s[0] / s[2]),
                              2.0 * f * S_AB(0, 1) * fabs(s[0] / s[1] - s[1] / s[0])};
#undef S_AB
        const double aw = fabs(q[0]), ax = fabs(q[1]), ay = fabs(q[2]), az = fabs(q[3]);
        const double iq = 2.0 / qn;
        q_err[i] += iq * (ax * th[0] + ay * th[1] + az * th[2]);
        q_err[n + i] += iq * (aw * th[0] + ay * th[2] + az * th[1]);
        q_err[2 * n + i] += iq * (aw * th[1] + az * th[0] + ax * th[2]);
        q_err[3 * n + i] += iq * (aw * th[2] + ax * th[1] + ay * th[0]);
    }
    return 0;
}
