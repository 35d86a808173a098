/*
 * FP64 CPU oracle for the two-stage adaptive AD-census stereo matcher of
 * "Mixed Reality Depth Contour Occlusion Using Binocular Similarity Matching
 * and Three-dimensional Contour Optimisation" (arXiv 2203.02300), Sect. 4.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * Plain and slow on purpose: every aggregated cost is an explicit double
 * sum over the support region, every cost term calls libm exp() in double.
 * No prefix sums, no lookup tables, no blocking.  OpenMP (if enabled) only
 * splits independent rows; each value is summed in the same order either way.
 *
 * Readings of points the paper leaves open (fixed here and in the tests):
 *   - grey level  Y = (77 R + 150 G + 29 B + 128) >> 8  (integer)
 *   - census (Sect. 4.2.1): cw x ch window (9x7) on Y, centre excluded,
 *     clamp-to-edge, bit k = [Y(n) < Y(p)] with k running over window rows
 *     top to bottom, columns left to right.
 *   - C_AD = mean of the three absolute channel differences (grey levels),
 *     C_census = Hamming distance of the census strings.
 *   - arms (Sect. 4.1, colour + distance double threshold): arm length in
 *     direction e is the largest k <= L1 such that for every 1 <= j <= k,
 *     p + j e lies in the image, Dc(p_j, p) < tau1, Dc(p_j, p_{j-1}) < tau1,
 *     and Dc(p_j, p) < tau2 whenever j > L2; Dc = max channel difference.
 *   - L_min = the shortest of the four arms of p (Eq. 1).
 *   - smooth cross-support window (Sect. 4.1, "morphological processing";
 *     the figure is missing), when enabled: a grey-level opening of each of
 *     the four arm-length maps (3x3 minimum, then 3x3 maximum, windows cut to
 *     the image); L_min and the regions use the opened arms.
 *   - support region (Eq. 2): union over q on the vertical arm of p of q's
 *     horizontal segment; N = its pixel count.  Reference-view arms only.
 *     The other order (union over q on p's horizontal arm of q's vertical
 *     segment) is available as a variant.
 *   - d in [d_min, d_min + D - 1] (Eq. 3's [d_min, d_max], D values; d_min = 0
 *     by default); a match outside the image costs 1 (upper bound of Eq. 1).
 *   - WTA (Eq. 3) takes the smallest d among equal minima.
 *   - the decision in the kernel's precision (optional outputs qdisp_*):
 *     the paper fixes no precision, so where floating point decides the
 *     argmin the oracle can also take it as the GPU does: lambda_AD,
 *     lambda_census, gamma_L and eps rounded to FP32; the tables
 *     T_AD[k] = 1 - exp(-(k/3)/lambda_AD) (k = channel sum 0..765),
 *     T_cen[h] = 1 - exp(-h/lambda_census) (h = 0..64) and
 *     alphaS[l] = alpha(l) * S evaluated in FP64 and rounded to FP32 once;
 *     the cost of Eq. 1 in FP32 as fma(alphaS, T_AD[k], (S - alphaS) *
 *     T_cen[h]) (one rounding per operation), rounded to the nearest
 *     integer (ties to even) at the fixed-point scale
 *     S = floor((2^32 - 1) / (2 L1 + 1)^2) - 1, a match outside the image
 *     costing S; the region sums of these integers are exact and the
 *     smallest sum wins, the smallest d among equal sums.
 *   - outlier removal: left-right consistency, valid iff x - dL >= 0 and
 *     |dL(x) - dR(x - dL)| <= tol, otherwise -1.
 *   - parallax optimisation (Sect. 4.3, Eq. 4), applied to the checked map:
 *     every valid pixel p takes the disparity that occurs most often among
 *     the valid pixels of its support region N_p (the same region as Eq. 2,
 *     left-view arms), the smallest such d on equal counts; invalid pixels
 *     (any value outside [0, D-1], -1 after the check) cast no vote and are
 *     written as -1.  k iterations each read the whole map
 *     of the previous one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ---------------------------------------------------------------- grey */
static int grey_of(const uint8_t *px)
{
    return (77 * (int)px[0] + 150 * (int)px[1] + 29 * (int)px[2] + 128) >> 8;
}

int orc_grey(const uint8_t *rgb, int W, int H, int32_t *out)
{
    if (!rgb || !out || W < 1 || H < 1) return ORC_EINVAL;
    for (long i = 0; i < (long)W * H; i++) out[i] = grey_of(rgb + 3 * i);
    return ORC_OK;
}

/* -------------------------------------------------------------- census */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int orc_census(const uint8_t *rgb, int W, int H, int cw, int ch, uint64_t *out)
{
    if (!rgb || !out || W < 1 || H < 1) return ORC_EINVAL;
    if (cw < 1 || ch < 1 || !(cw & 1) || !(ch & 1) || cw * ch - 1 > 64) return ORC_EINVAL;
    int32_t *Y = (int32_t *)malloc(sizeof(int32_t) * (size_t)W * H);
    if (!Y) return ORC_ENOMEM;
    orc_grey(rgb, W, H, Y);
    int rx = cw / 2, ry = ch / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int yc = Y[(long)y * W + x];
            uint64_t bits = 0;
            int k = 0;
            for (int dy = -ry; dy <= ry; dy++) {
                for (int dx = -rx; dx <= rx; dx++) {
                    if (dx == 0 && dy == 0) continue;
                    int nx = clampi(x + dx, 0, W - 1), ny = clampi(y + dy, 0, H - 1);
                    if (Y[(long)ny * W + nx] < yc) bits |= (uint64_t)1 << k;
                    k++;
                }
            }
            out[(long)y * W + x] = bits;
        }
    }
    free(Y);
    return ORC_OK;
}

int orc_hamming(uint64_t a, uint64_t b)
{
    uint64_t v = a ^ b;
    int n = 0;
    while (v) { n += (int)(v & 1u); v >>= 1; }
    return n;
}

/* ---------------------------------------------------------------- arms */
static int dc_max(const uint8_t *a, const uint8_t *b)
{
    int m = 0;
    for (int c = 0; c < 3; c++) {
        int v = abs((int)a[c] - (int)b[c]);
        if (v > m) m = v;
    }
    return m;
}

/* arms: 4 bytes per pixel, order {left, right, up, down} */
int orc_arms(const uint8_t *rgb, int W, int H, int L1, int L2, int tau1, int tau2,
             uint8_t *arms)
{
    if (!rgb || !arms || W < 1 || H < 1 || L1 < 0 || L1 > 255 || L2 < 0) return ORC_EINVAL;
    static const int ex[4] = {-1, 1, 0, 0}, ey[4] = {0, 0, -1, 1};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            const uint8_t *p = rgb + 3 * ((long)y * W + x);
            for (int e = 0; e < 4; e++) {
                int k = 0;
                for (int j = 1; j <= L1; j++) {
                    int qx = x + j * ex[e], qy = y + j * ey[e];
                    if (qx < 0 || qx >= W || qy < 0 || qy >= H) break;
                    const uint8_t *q = rgb + 3 * ((long)qy * W + qx);
                    const uint8_t *qprev = rgb + 3 * ((long)(qy - ey[e]) * W + (qx - ex[e]));
                    if (dc_max(q, p) >= tau1) break;
                    if (dc_max(q, qprev) >= tau1) break;
                    if (j > L2 && dc_max(q, p) >= tau2) break;
                    k = j;
                }
                arms[4 * ((long)y * W + x) + e] = (uint8_t)k;
            }
        }
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- cost */
typedef struct {
    double lambda_ad, lambda_census, gamma_l, eps;
} orc_cost_params;

/* Eq. 1: adaptive weight from the shortest arm */
/*
 * Morphological smoothing of the cross-support window (Sect. 4.1): opening
 * of every arm-length map, out(p) = max over q in W(p) of min over r in W(q)
 * of arms(r), W(p) the 3x3 window around p cut to the image.  An opening
 * never lengthens an arm, so the result stays inside the image and <= L1.
 */
int orc_arms_smooth(const uint8_t *arms, int W, int H, uint8_t *out)
{
    if (!arms || !out || W < 1 || H < 1) return ORC_EINVAL;
    long n = (long)W * H;
    uint8_t *er = (uint8_t *)malloc(4 * n);
    if (!er) return ORC_ENOMEM;
    for (int pass = 0; pass < 2; pass++) {
        const uint8_t *src = pass == 0 ? arms : er;
        uint8_t *dst = pass == 0 ? er : out;
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++)
                for (int k = 0; k < 4; k++) {
                    int v = pass == 0 ? 255 : 0;
                    for (int yy = y - 1; yy <= y + 1; yy++)
                        for (int xx = x - 1; xx <= x + 1; xx++) {
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            int a = src[4 * ((long)yy * W + xx) + k];
                            v = pass == 0 ? (a < v ? a : v) : (a > v ? a : v);
                        }
                    dst[4 * ((long)y * W + x) + k] = (uint8_t)v;
                }
    }
    free(er);
    return ORC_OK;
}

double orc_alpha(int lmin, double gamma_l, double eps)
{
    return 1.0 - exp(-gamma_l / ((double)lmin + eps));
}

/* Eq. 1: robust exponential combination of the AD and census measures.
 * ad_sum = |dR| + |dG| + |dB|, ham = Hamming distance. */
double orc_cost_terms(int ad_sum, int ham, int lmin, double lambda_ad, double lambda_census,
                      double gamma_l, double eps)
{
    double alpha = orc_alpha(lmin, gamma_l, eps);
    double c_ad = (double)ad_sum / 3.0;
    double c_census = (double)ham;
    return alpha * (1.0 - exp(-c_ad / lambda_ad)) +
           (1.0 - alpha) * (1.0 - exp(-c_census / lambda_census));
}

typedef struct {
    int W, H, D;
    int dmin;                           /* d in [dmin, dmin + D - 1] */
    const uint8_t *ref_rgb, *oth_rgb;   /* reference view and the other view */
    const uint64_t *ref_cen, *oth_cen;
    const uint8_t *ref_arms;
    int sign;                           /* -1: left reference (q = p - d); +1: right */
    orc_cost_params cp;
    int order;                          /* 0: region H then V (Eq. 2 reading); 1: V then H */
    /* the decision in the kernel's precision (see the header) */
    float q_ad[766], q_cen[65], q_as[64];
    float qS;
    uint32_t qSint;
} view_ctx;

/* fixed-point scale: the largest full region ((2 L1 + 1)^2 costs <= 1) fits
   in 32 bits, with one unit of margin */
static uint32_t fixed_scale(int L1)
{
    uint64_t n = (uint64_t)(2 * L1 + 1) * (uint64_t)(2 * L1 + 1);
    return (uint32_t)(0xffffffffull / n - 1);
}

/* the FP32 tables of Eq. 1 with the parameters rounded to FP32 */
static void quant_tables(view_ctx *v, int L1)
{
    double lad = (double)(float)v->cp.lambda_ad, lcen = (double)(float)v->cp.lambda_census;
    double gam = (double)(float)v->cp.gamma_l, eps = (double)(float)v->cp.eps;
    v->qSint = fixed_scale(L1);
    v->qS = (float)v->qSint;
    for (int k = 0; k <= 765; k++) v->q_ad[k] = (float)(1.0 - exp(-((double)k / 3.0) / lad));
    for (int h = 0; h <= 64; h++) v->q_cen[h] = (float)(1.0 - exp(-(double)h / lcen));
    for (int l = 0; l < 64; l++) v->q_as[l] = (float)((1.0 - exp(-gam / ((double)l + eps))) * (double)v->qSint);
}

static int lmin_of(const uint8_t *a)
{
    int m = a[0];
    for (int e = 1; e < 4; e++) if (a[e] < m) m = a[e];
    return m;
}

/* raw cost C(p, d) of Eq. 1 for the reference pixel (x, y) */
static double pixel_cost(const view_ctx *v, int x, int y, int d)
{
    int xo = x + v->sign * d;
    if (xo < 0 || xo >= v->W) return 1.0;
    long ip = (long)y * v->W + x, io = (long)y * v->W + xo;
    const uint8_t *a = v->ref_rgb + 3 * ip, *b = v->oth_rgb + 3 * io;
    int ad = abs((int)a[0] - (int)b[0]) + abs((int)a[1] - (int)b[1]) + abs((int)a[2] - (int)b[2]);
    int ham = orc_hamming(v->ref_cen[ip], v->oth_cen[io]);
    int lmin = lmin_of(v->ref_arms + 4 * ip);
    return orc_cost_terms(ad, ham, lmin, v->cp.lambda_ad, v->cp.lambda_census,
                          v->cp.gamma_l, v->cp.eps);
}

/* the same cost in the kernel's precision, as an integer at scale S */
static uint32_t pixel_qcost(const view_ctx *v, int x, int y, int d)
{
    int xo = x + v->sign * d;
    if (xo < 0 || xo >= v->W) return v->qSint;
    long ip = (long)y * v->W + x, io = (long)y * v->W + xo;
    const uint8_t *a = v->ref_rgb + 3 * ip, *b = v->oth_rgb + 3 * io;
    int ad = abs((int)a[0] - (int)b[0]) + abs((int)a[1] - (int)b[1]) + abs((int)a[2] - (int)b[2]);
    int ham = orc_hamming(v->ref_cen[ip], v->oth_cen[io]);
    float as = v->q_as[lmin_of(v->ref_arms + 4 * ip)];
    float rest = v->qS - as;               /* FP32 difference */
    float cen = rest * v->q_cen[ham];      /* FP32 product */
    float c = fmaf(as, v->q_ad[ad], cen);  /* one rounding */
    return (uint32_t)nearbyintf(c);        /* nearest integer, ties to even */
}

/* Eq. 2 support-region size N of pixel (x, y): order 0 sums, over q on p's
   vertical arm, q's horizontal segment; order 1 sums, over q on p's
   horizontal arm, q's vertical segment */
static long region_size(const view_ctx *v, int x, int y)
{
    const uint8_t *ap = v->ref_arms + 4 * ((long)y * v->W + x);
    long n = 0;
    if (v->order == 0) {
        for (int yy = y - ap[2]; yy <= y + ap[3]; yy++) {
            const uint8_t *aq = v->ref_arms + 4 * ((long)yy * v->W + x);
            n += (long)aq[0] + aq[1] + 1;
        }
    } else {
        for (int xx = x - ap[0]; xx <= x + ap[1]; xx++) {
            const uint8_t *aq = v->ref_arms + 4 * ((long)y * v->W + xx);
            n += (long)aq[2] + aq[3] + 1;
        }
    }
    return n;
}

/*
 * Aggregated cost (Eq. 2), WTA (Eq. 3) for one view, rows [y0, y1).
 * For each d the raw costs of rows [y0-L1, y1+L1) are evaluated, the
 * horizontal segment sums S_H formed by explicit summation, then the
 * vertical sums of S_H over the vertical arm, divided by N.
 * Outputs per pixel of the row range: disparity, best and second-best
 * aggregated cost; optionally the whole aggregated volume [d][y-y0][x].
 */
static int run_view(const view_ctx *v, int y0, int y1, int reach, int16_t *disp,
                    double *best, double *second, double *vol, int16_t *qdisp)
{
    int W = v->W, H = v->H;
    int ya = y0 - reach < 0 ? 0 : y0 - reach;
    int yb = y1 + reach > H ? H : y1 + reach;
    int nr = yb - ya, no = y1 - y0;
    double *C = (double *)malloc(sizeof(double) * (size_t)W * nr);
    double *SH = (double *)malloc(sizeof(double) * (size_t)W * nr);
    long *N = (long *)malloc(sizeof(long) * (size_t)W * no);
    /* kernel-precision decision: integer costs, their segment sums, the best sum */
    uint32_t *QC = qdisp ? (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W * nr) : NULL;
    uint64_t *QH = qdisp ? (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * nr) : NULL;
    uint64_t *qbest = qdisp ? (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * no) : NULL;
    if (!C || !SH || !N || (qdisp && (!QC || !QH || !qbest))) {
        free(C); free(SH); free(N); free(QC); free(QH); free(qbest);
        return ORC_ENOMEM;
    }
    for (int y = y0; y < y1; y++)
        for (int x = 0; x < W; x++) N[(long)(y - y0) * W + x] = region_size(v, x, y);
    for (long i = 0; i < (long)W * no; i++) { best[i] = INFINITY; second[i] = INFINITY; disp[i] = 0; }
    if (qdisp)
        for (long i = 0; i < (long)W * no; i++) { qbest[i] = UINT64_MAX; qdisp[i] = 0; }

    for (int d = v->dmin; d < v->dmin + v->D; d++) {
#pragma omp parallel for schedule(static)
        for (int y = ya; y < yb; y++)
            for (int x = 0; x < W; x++) C[(long)(y - ya) * W + x] = pixel_cost(v, x, y, d);
        if (qdisp) {
#pragma omp parallel for schedule(static)
            for (int y = ya; y < yb; y++)
                for (int x = 0; x < W; x++) QC[(long)(y - ya) * W + x] = pixel_qcost(v, x, y, d);
        }
        if (v->order == 0) {
            /* segment sums along each row (q's horizontal segment) */
#pragma omp parallel for schedule(static)
            for (int y = ya; y < yb; y++) {
                for (int x = 0; x < W; x++) {
                    const uint8_t *a = v->ref_arms + 4 * ((long)y * W + x);
                    double s = 0.0;
                    for (int xx = x - a[0]; xx <= x + a[1]; xx++) s += C[(long)(y - ya) * W + xx];
                    SH[(long)(y - ya) * W + x] = s;
                    if (qdisp) {
                        uint64_t qs = 0;
                        for (int xx = x - a[0]; xx <= x + a[1]; xx++) qs += QC[(long)(y - ya) * W + xx];
                        QH[(long)(y - ya) * W + x] = qs;
                    }
                }
            }
        } else {
            /* segment sums along each column (q's vertical segment), output rows only */
#pragma omp parallel for schedule(static)
            for (int y = y0; y < y1; y++) {
                for (int x = 0; x < W; x++) {
                    const uint8_t *a = v->ref_arms + 4 * ((long)y * W + x);
                    double s = 0.0;
                    for (int yy = y - a[2]; yy <= y + a[3]; yy++) s += C[(long)(yy - ya) * W + x];
                    SH[(long)(y - ya) * W + x] = s;
                    if (qdisp) {
                        uint64_t qs = 0;
                        for (int yy = y - a[2]; yy <= y + a[3]; yy++) qs += QC[(long)(yy - ya) * W + x];
                        QH[(long)(y - ya) * W + x] = qs;
                    }
                }
            }
        }
#pragma omp parallel for schedule(static)
        for (int y = y0; y < y1; y++) {
            for (int x = 0; x < W; x++) {
                const uint8_t *a = v->ref_arms + 4 * ((long)y * W + x);
                double s = 0.0;
                if (v->order == 0)
                    for (int yy = y - a[2]; yy <= y + a[3]; yy++) s += SH[(long)(yy - ya) * W + x];
                else
                    for (int xx = x - a[0]; xx <= x + a[1]; xx++) s += SH[(long)(y - ya) * W + xx];
                long i = (long)(y - y0) * W + x;
                double cbar = s / (double)N[i];
                if (vol) vol[(long)(d - v->dmin) * W * no + i] = cbar;
                if (cbar < best[i]) { second[i] = best[i]; best[i] = cbar; disp[i] = (int16_t)d; }
                else if (cbar < second[i]) { second[i] = cbar; }
                if (qdisp) {
                    /* exact integer region sum; N does not depend on d */
                    uint64_t qs = 0;
                    if (v->order == 0)
                        for (int yy = y - a[2]; yy <= y + a[3]; yy++) qs += QH[(long)(yy - ya) * W + x];
                    else
                        for (int xx = x - a[0]; xx <= x + a[1]; xx++) qs += QH[(long)(y - ya) * W + xx];
                    if (qs < qbest[i]) { qbest[i] = qs; qdisp[i] = (int16_t)d; }
                }
            }
        }
    }
    free(C); free(SH); free(N); free(QC); free(QH); free(qbest);
    return ORC_OK;
}

/* Left-right consistency check on rows of width W (outlier removal, Sect. 4.3). */
int orc_lr_check(const int16_t *dl, const int16_t *dr, int W, int rows, int tol, int16_t *out)
{
    if (!dl || !dr || !out || W < 1 || rows < 0) return ORC_EINVAL;
    for (int y = 0; y < rows; y++) {
        for (int x = 0; x < W; x++) {
            long i = (long)y * W + x;
            int d = dl[i];
            int16_t r = -1;
            if (tol < 0) r = (int16_t)d;
            else if (d >= 0 && x - d >= 0) {
                int d2 = dr[(long)y * W + (x - d)];
                if (d2 >= 0 && abs(d - d2) <= tol) r = (int16_t)d;
            }
            out[i] = r;
        }
    }
    return ORC_OK;
}

/*
 * Full matcher on rows [y0, y1) of a W x H pair with the D disparities
 * dmin .. dmin + D - 1.  Every output array holds (y1 - y0) x W values;
 * vol_l / vol_r (optional) hold D x (y1 - y0) x W aggregated costs, plane k
 * for disparity dmin + k.  Census and arms are computed on
 * the whole image (they are cheap next to the aggregation).  qdisp_l /
 * qdisp_r (optional, both or neither) receive the Eq. 3 decisions taken in
 * the kernel's precision (header); disp_* are the FP64 decisions.
 */
int orc_match(const uint8_t *left, const uint8_t *right, int W, int H, int D, int dmin,
              double lambda_ad, double lambda_census, double gamma_l, double eps,
              int cw, int ch, int L1, int L2, int tau1, int tau2, int lr_tol, int smooth, int order,
              int y0, int y1,
              int16_t *disp_l, int16_t *disp_r, int16_t *disp_final,
              double *best_l, double *second_l, double *best_r, double *second_r,
              double *vol_l, double *vol_r, int16_t *qdisp_l, int16_t *qdisp_r)
{
    if (!left || !right || W < 1 || H < 1 || D < 1 || dmin < 0 || y0 < 0 || y1 > H || y0 > y1)
        return ORC_EINVAL;
    if (!disp_l || !disp_r || !disp_final || !best_l || !second_l || !best_r || !second_r)
        return ORC_EINVAL;
    size_t npx = (size_t)W * H;
    uint64_t *cl = (uint64_t *)malloc(8 * npx), *cr = (uint64_t *)malloc(8 * npx);
    uint8_t *al = (uint8_t *)malloc(4 * npx), *ar = (uint8_t *)malloc(4 * npx);
    int rc = ORC_ENOMEM;
    if (!cl || !cr || !al || !ar) goto done;
    if ((rc = orc_census(left, W, H, cw, ch, cl)) != ORC_OK) goto done;
    if ((rc = orc_census(right, W, H, cw, ch, cr)) != ORC_OK) goto done;
    if ((rc = orc_arms(left, W, H, L1, L2, tau1, tau2, al)) != ORC_OK) goto done;
    if ((rc = orc_arms(right, W, H, L1, L2, tau1, tau2, ar)) != ORC_OK) goto done;
    if (smooth) {
        if ((rc = orc_arms_smooth(al, W, H, al)) != ORC_OK) goto done;
        if ((rc = orc_arms_smooth(ar, W, H, ar)) != ORC_OK) goto done;
    }
    {
        orc_cost_params cp = {lambda_ad, lambda_census, gamma_l, eps};
        view_ctx *vl = (view_ctx *)calloc(1, sizeof(view_ctx)), *vr = (view_ctx *)calloc(1, sizeof(view_ctx));
        if (!vl || !vr) { free(vl); free(vr); rc = ORC_ENOMEM; goto done; }
        *vl = (view_ctx){W, H, D, dmin, left, right, cl, cr, al, -1, cp, order};
        *vr = (view_ctx){W, H, D, dmin, right, left, cr, cl, ar, +1, cp, order};
        if (qdisp_l && qdisp_r) { quant_tables(vl, L1); quant_tables(vr, L1); }
        rc = run_view(vl, y0, y1, L1, disp_l, best_l, second_l, vol_l, qdisp_l && qdisp_r ? qdisp_l : NULL);
        if (rc == ORC_OK)
            rc = run_view(vr, y0, y1, L1, disp_r, best_r, second_r, vol_r, qdisp_l && qdisp_r ? qdisp_r : NULL);
        free(vl); free(vr);
        if (rc != ORC_OK) goto done;
        rc = orc_lr_check(disp_l, disp_r, W, y1 - y0, lr_tol, disp_final);
    }
done:
    free(cl); free(cr); free(al); free(ar);
    return rc;
}

/*
 * Parallax optimisation (Sect. 4.3, Eq. 4): `iters` rounds of
 *   d'(p) = argmax_d hist(d, N_p)
 * on a W x H map with disparities in [dmin, dmin + D - 1] (any other value,
 * -1 after the consistency check, is invalid and casts no vote), N_p being the
 * support region of Eq. 2 built from `arms` (4 bytes per pixel: l, r, u, d).
 * The histogram counts every pixel of the region explicitly (pixels of the
 * region are enumerated row by row; the region is a union of disjoint row
 * segments, so no pixel is counted twice).
 */
int orc_vote(const int16_t *disp, const uint8_t *arms, int W, int H, int D, int dmin, int iters, int16_t *out)
{
    if (!disp || !arms || !out || W < 1 || H < 1 || D < 1 || dmin < 0 || iters < 0) return ORC_EINVAL;
    long n = (long)W * H;
    int16_t *cur = (int16_t *)malloc(sizeof(int16_t) * n);
    int16_t *nxt = (int16_t *)malloc(sizeof(int16_t) * n);
    if (!cur || !nxt) { free(cur); free(nxt); return ORC_ENOMEM; }
    memcpy(cur, disp, sizeof(int16_t) * n);
    int rc = ORC_OK;
    for (int it = 0; it < iters && rc == ORC_OK; it++) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int y = 0; y < H; y++) {
            long *hist = (long *)malloc(sizeof(long) * D);
            if (!hist) { rc = ORC_ENOMEM; continue; }
            for (int x = 0; x < W; x++) {
                long i = (long)y * W + x;
                if (cur[i] < dmin || cur[i] >= dmin + D) { nxt[i] = -1; continue; }   /* invalid */
                for (int d = 0; d < D; d++) hist[d] = 0;
                const uint8_t *ap = arms + 4 * i;
                for (int yy = y - ap[2]; yy <= y + ap[3]; yy++) {
                    const uint8_t *aq = arms + 4 * ((long)yy * W + x);
                    for (int xx = x - aq[0]; xx <= x + aq[1]; xx++) {
                        int v = cur[(long)yy * W + xx];
                        if (v >= dmin && v < dmin + D) hist[v - dmin]++;
                    }
                }
                int best = 0;
                for (int d = 1; d < D; d++)
                    if (hist[d] > hist[best]) best = d;   /* strict: smallest d on ties */
                nxt[i] = (int16_t)(dmin + best);
            }
            free(hist);
        }
        int16_t *t = cur; cur = nxt; nxt = t;
    }
    if (rc == ORC_OK) memcpy(out, cur, sizeof(int16_t) * n);
    free(cur); free(nxt);
    return rc;
}

/*
 * Quarter-size input (Sect. 4, Sect. 4.4: the pair is matched at a quarter
 * of its size).  Reading: half of each axis, every output channel the
 * rounded mean of its 2x2 input block, (a + b + c + d + 2) >> 2; an odd last
 * row or column is dropped.  out: (W/2) x (H/2) x 3.
 */
int orc_downscale(const uint8_t *rgb, int W, int H, uint8_t *out)
{
    if (!rgb || !out || W < 2 || H < 2) return ORC_EINVAL;
    int Wh = W / 2, Hh = H / 2;
    for (int y = 0; y < Hh; y++)
        for (int x = 0; x < Wh; x++)
            for (int c = 0; c < 3; c++) {
                int s = rgb[((long)(2 * y) * W + 2 * x) * 3 + c] + rgb[((long)(2 * y) * W + 2 * x + 1) * 3 + c] +
                        rgb[((long)(2 * y + 1) * W + 2 * x) * 3 + c] +
                        rgb[((long)(2 * y + 1) * W + 2 * x + 1) * 3 + c];
                out[((long)y * Wh + x) * 3 + c] = (uint8_t)((s + 2) >> 2);
            }
    return ORC_OK;
}

/*
 * Sparse depth map (Sect. 4.4, Eq. 14 convention 0 = missing).  The
 * disparity d of the half-size map is doubled back to full size and
 * converted with the binocular parameters: Z = f * B / (2 d), f in pixels of
 * the full image, B the baseline; d <= 0 (invalid or at infinity) gives 0.
 * Reading of "discretised into the original size": every half-size pixel
 * covers its 2x2 block of the W x H output; an odd last row or column is 0.
 */
int orc_depth(const int16_t *disp_half, int W, int H, double f, double B, double *out)
{
    if (!disp_half || !out || W < 2 || H < 2) return ORC_EINVAL;
    int Wh = W / 2, Hh = H / 2;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int hx = x / 2, hy = y / 2;
            double z = 0.0;
            if (hx < Wh && hy < Hh) {
                int d = disp_half[(long)hy * Wh + hx];
                if (d > 0) z = f * B / (2.0 * d);
            }
            out[(long)y * W + x] = z;
        }
    return ORC_OK;
}
