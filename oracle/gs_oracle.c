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
 * Continuous values are FP64; integer decisions of the projection are taken in
 * FP32 (project.inc compiled with REAL = float); compositing thresholds are
 * compared in FP64 and pixels where a fragment lies within tie_band of a
 * threshold are flagged, so callers can exclude them from exact comparisons.
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
    double tie_band;       /* relative band for projection decisions */
    double comp_band;      /* relative band for compositing thresholds */
} or_params;

/* ---- projection, two precisions ---------------------------------------- */
#define REAL double
#define PFN(x) x##_f64
#define SQRT sqrt
#define EXP exp
#define LOG2 log2
#define FLOOR floor
#define CEIL ceil
#include "project.inc"
#undef REAL
#undef PFN
#undef SQRT
#undef EXP
#undef LOG2
#undef FLOOR
#undef CEIL
#define REAL float
#define PFN(x) x##_f32
#define SQRT sqrtf
#define EXP expf
#define LOG2 log2f
#define FLOOR floorf
#define CEIL ceilf
#include "project.inc"
#undef REAL
#undef PFN

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
    double *ldl32;      /* 3n: (A, k, D) of the FP32 instance's conic, NULL if not wanted */
    double *uv32;       /* 2n: projected mean in double, before the FP32 instance rounds it */
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
        proj_t_f32 d32;
        proj_t_f64 d64;
        project_one_f32(m3, s3, q4, l, cb, cam, P, &d32);
        project_one_f64(m3, s3, q4, l, cb, cam, P, &d64);
        out->status[i] = (int8_t)d32.status;
        out->tie[i] = (uint8_t)(d32.tie | d64.tie);
        out->depth32[i] = d32.tz;
        out->depth[i] = d64.tz;
        out->radius[i] = d32.radius;
        for (int k = 0; k < 4; k++) out->rect[4 * i + k] = d32.rect[k];
        out->tiles[i] = d32.status == OR_ACTIVE ? (d32.rect[2] - d32.rect[0]) * (d32.rect[3] - d32.rect[1]) : 0;
        out->uv[2 * i] = d64.u;
        out->uv[2 * i + 1] = d64.v;
        if (out->ldl32) {
            out->ldl32[3 * i] = d32.ldlA;
            out->ldl32[3 * i + 1] = d32.ldlK;
            out->ldl32[3 * i + 2] = d32.ldlD;
            out->uv32[2 * i] = d32.ud;
            out->uv32[2 * i + 1] = d32.vd;
        }
        out->conic[3 * i] = d64.conA;
        out->conic[3 * i + 1] = d64.conB;
        out->conic[3 * i + 2] = d64.conC;
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
 * one.  An FP32 renderer composites with the FP32 instance's conic, held as
 * A (x + k y)^2 + D y^2 (ldl32), and a mean kept to double precision (uv32).
 * The exponent these give, evaluated exactly, differs from the exact exponent
 * by the projection's own rounding; evaluating that form in FP32 adds, per
 * operation, a relative 2^-24 of the terms it combines, and 2^x in FP32 a few
 * more units.  A fragment whose alpha lies within this of a threshold may be
 * decided the other way by a correct FP32 renderer. */
static double fp32_power_err(const double *ldl32, const double *uv32, int32_t g, double px, double py,
                             double power)
{
    const double eps32 = 5.9604644775390625e-08; /* 2^-24 */
    if (!ldl32) return 16.0 * eps32 * (fabs(power) + 1.0);
    const double A = ldl32[3 * g], k = ldl32[3 * g + 1], D = ldl32[3 * g + 2];
    const double dx = px - uv32[2 * g], dy = py - uv32[2 * g + 1];
    const double e = dx + k * dy;
    const double p32 = -0.5 * (A * e * e + D * dy * dy);
    const double de = 2.0 * eps32 * (fabs(dx) + 2.0 * fabs(k * dy));
    const double eval = 0.5 * A * (2.0 * fabs(e) * de + de * de) + 4.0 * eps32 * (fabs(p32) + 1.0);
    return 2.0 * (fabs(p32 - power) + eval);
}

/* Composites the ordered Gaussians ids[0..len) at pixel centre (px, py).
 * Optional w/a accumulate the importance alpha-weight and pixel count.
 * Flags: a fragment within tie band (comp_band, widened by its own FP32 error
 * bound) of the alpha_min or T_min threshold, or at the exponent's maximum 0.
 * When the pixel is flagged and gcount is given, every Gaussian the pixel
 * composited or nearly composited has its count of such pixels raised. */
static void composite_pixel(const or_params *P, double px, double py, const int32_t *ids, int64_t len,
                            const double *uv, const double *conic, const double *opacity,
                            const double *rgb, pix_t *o, double *w, double *a, int32_t *gcount,
                            const double *ldl32, const double *uv32)
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
        const double perr = fp32_power_err(ldl32, uv32, g, px, py, power);
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
 * counts, per Gaussian, the flagged pixels it takes part in, when non-NULL.
 * ldl32 (3n) and uv32 (2n), from the projection's FP32 instance, widen the
 * flag bands by how far an FP32 renderer's exponents can be from the exact
 * ones; NULL leaves only the fixed bands. */
int or_render(const or_camera *cam, const or_params *P, int64_t n, const double *uv, const double *conic,
              const double *opacity, const double *rgb, const int64_t *tile_start, const int32_t *list,
              double *image, double *T_final, int32_t *n_contrib, uint8_t *flags, double *w, double *a,
              int32_t *gcount, const double *ldl32, const double *uv32)
{
    (void)n;
    const int W = cam->width, H = cam->height, tw = P->tile_w, th = P->tile_h;
    const int tiles_x = (W + tw - 1) / tw;
    for (int py = 0; py < H; py++)
        for (int px = 0; px < W; px++) {
            int64_t t = (int64_t)(py / th) * tiles_x + px / tw;
            pix_t o;
            composite_pixel(P, px + 0.5, py + 0.5, list + tile_start[t], tile_start[t + 1] - tile_start[t],
                            uv, conic, opacity, rgb, &o, w, a, gcount, ldl32, uv32);
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
            composite_pixel(P, px + 0.5, py + 0.5, ids, m, uv, conic, opacity, rgb, &o, NULL, NULL, NULL, NULL, NULL);
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
                        list_start[k + 1] - list_start[k], uv, conic, opacity, rgb, &o, NULL, NULL, NULL, NULL,
                        NULL);
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
                  double *dL_drgb)
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
