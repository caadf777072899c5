/*
 * rick_oracle.c -- plain, slow FP64 reference implementation of the w-stacking
 * imager of arXiv 2504.00959 (RICK).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library
 * (paper_2504_00959_gb300/csrc); neither includes nor links the other.
 *
 * What it computes, step by step in the order of the paper's workflow (Sec. 2.1):
 *   1. place each measurement: nearest w-plane (Sec. 2.1, "mapped to the
 *      closest w-plane") and the first cell of its S x S kernel footprint;
 *   2. convolutional gridding, Eq. 3: every measurement V_m, times its weight,
 *      is spread onto the cells of its plane with a separable kernel (Gaussian
 *      or Kaiser-Bessel, Sec. 2.1) whose taps are normalised to sum 1 per axis;
 *   3. per-plane 2D inverse FFT (step 3 of the workflow) -- a textbook
 *      radix-2 Cooley-Tukey FFT written here (direct DFT for other lengths),
 *      with the fftshift done by explicit circular shifts;
 *   4. w-term correction and reduction of the planes (step 4 / Eq. 1):
 *      I(l,m) = sum_k P_k(l,m) exp(+2 pi i w_k (n-1)), n = sqrt(1-l^2-m^2),
 *      w_k the centre of plane k;
 *   5. normalisation by the sum of weights, optional division by the taper
 *      (Fourier transform of the gridding kernel) and optional factor n.
 *
 * Readings where the paper is silent (the same readings the GPU library
 * documents): Nw uniform w-bins over [w_min, w_max] with centres
 * w_min + (k+1/2) dw; footprint cells f..f+S-1 with f = floor(p - S/2) + 1;
 * Gaussian exp(-x^2 / 2 sigma^2), sigma default S/6; Kaiser-Bessel
 * I0(beta sqrt(1 - (2x/S)^2)), beta default 2.34 S; phase centre at pixel
 * (N/2, N/2); uv cell j <-> u = (j - N/2) du with du = 1/(N dl).
 *
 * Precision rule: every decision that turns a float into an integer (plane
 * index, first footprint cell, nearest cell for the density grid) is taken in
 * IEEE binary32 with the operation sequence spelled out in oracle_place(), the
 * precision of the kernels under test.  Every value (kernel taps, positions,
 * FFT, phases, sums) is FP64.
 *
 * Extra entry points used to pin this oracle: a brute-force direct DFT with
 * the exact w-term (Eq. 1 evaluated per measurement, no gridding, no
 * w-quantisation), a per-pixel evaluation of the discrete algorithm that needs
 * no FFT, the adjoint (degridding) operator, and the FFT / I0 / kernel /
 * taper building blocks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_GAUSS 0
#define OR_KB 1
#define OR_MAX_SUPPORT 64
#define OR_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* configuration                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n, nw, kernel, support;
    double pixel_rad, w_min, w_max, kparam; /* kparam: sigma (cells) or beta */
    double uvscale;                         /* cells per wavelength = n * pixel_rad */
    double dw;                              /* plane width in w */
    /* binary32 copies used only for the integer decisions */
    float uvscale_f, half_n_f, half_s_f, wmin_f, invdw_f;
    /* w-support (Eq. 3's kernel in w): sw planes per measurement with the
     * kernel family of u and v, support sw, parameter wkparam; 1 = the
     * nearest plane (Sec. 2.1).  half_sw_f: sw / 2 in binary32. */
    int sw;
    double wkparam;
    float half_sw_f;
    double wq[4097];  /* Simpson-weighted samples of h over [-sw/2, sw/2] (sw > 1) */
} or_cfg;

static int or_make_cfg(or_cfg* c, int n, int nw, double pixel_rad, double w_min,
                       double w_max, int kernel, int support, double kparam)
{
    if (n < 2 || (n & 1) || nw < 1 || support < 1 || support > OR_MAX_SUPPORT ||
        support > n || !(pixel_rad > 0.0) || (kernel != OR_GAUSS && kernel != OR_KB))
        return -1;
    if (nw > 1 && !(w_max > w_min)) return -1;
    c->n = n; c->nw = nw; c->kernel = kernel; c->support = support;
    c->pixel_rad = pixel_rad; c->w_min = w_min; c->w_max = w_max;
    if (kparam <= 0.0) kparam = (kernel == OR_GAUSS) ? support / 6.0 : 2.34 * support;
    c->kparam = kparam;
    c->uvscale = (double)n * pixel_rad;
    c->dw = (nw > 1) ? (w_max - w_min) / nw : (w_max - w_min);
    c->uvscale_f = (float)c->uvscale;
    c->half_n_f = (float)(n / 2);
    c->half_s_f = (float)(0.5 * support);
    c->wmin_f = (float)w_min;
    c->invdw_f = (nw > 1) ? (float)(1.0 / c->dw) : 0.0f;
    c->sw = 1;
    c->wkparam = 0.0;
    c->half_sw_f = 0.5f;
    return 0;
}

/* The w-support rides in bits 8..15 of the flags (0 or 1: nearest plane). */
#define OR_WSUPPORT(flags) ((int)(((flags) >> 8) & 0xffu))
#define OR_MAX_WSUPPORT 16

static int or_set_wsupport(or_cfg* c, unsigned flags)
{
    int sw = OR_WSUPPORT(flags);
    if (sw < 1) sw = 1;
    if (sw > OR_MAX_WSUPPORT || (sw > 1 && c->nw < sw)) return -1;
    c->sw = sw;
    c->wkparam = (c->kernel == OR_GAUSS) ? sw / 6.0 : 2.34 * sw;
    c->half_sw_f = (float)(0.5 * sw);
    return 0;
}

static double or_kernel_w(const or_cfg* c, double x);

/* Samples of the w correction's quadrature (after or_set_wsupport). */
static void or_prepare_wcorr(or_cfg* c)
{
    if (c->sw == 1) return;
    const int K = 4096;
    const double a = -0.5 * c->sw, h = (double)c->sw / K;
    for (int i = 0; i <= K; ++i) {
        double q = (i == 0 || i == K) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        c->wq[i] = q * or_kernel_w(c, a + i * h);
    }
}

/* ------------------------------------------------------------------------ */
/* kernels                                                                  */
/* ------------------------------------------------------------------------ */

/* Modified Bessel function I0 from its power series
 * I0(x) = sum_k (x^2/4)^k / (k!)^2  (Abramowitz & Stegun 9.6.10). */
double oracle_bessel_i0(double x)
{
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 1000; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* Un-normalised 1D gridding kernel at offset x (cells) from the measurement.
 * Gaussian or Kaiser-Bessel (Sec. 2.1, Jackson 1991 for KB). */
static double or_kernel(const or_cfg* c, double x)
{
    if (c->kernel == OR_GAUSS) {
        double s = c->kparam;
        return exp(-x * x / (2.0 * s * s));
    }
    double t = 2.0 * x / c->support;
    double a = 1.0 - t * t;
    if (a < 0.0) a = 0.0;
    return oracle_bessel_i0(c->kparam * sqrt(a));
}

/* The kernel in w: the same family with support sw, at x plane widths. */
static double or_kernel_w(const or_cfg* c, double x)
{
    if (c->kernel == OR_GAUSS) {
        double s = c->wkparam;
        return exp(-x * x / (2.0 * s * s));
    }
    double t = 2.0 * x / c->sw;
    double a = 1.0 - t * t;
    if (a < 0.0) a = 0.0;
    return oracle_bessel_i0(c->wkparam * sqrt(a));
}

double oracle_kernel(int kernel, int support, double kparam, double x)
{
    or_cfg c;
    if (or_make_cfg(&c, 2 * OR_MAX_SUPPORT, 1, 1.0, 0.0, 0.0, kernel, support, kparam)) return NAN;
    return or_kernel(&c, x);
}

/* ------------------------------------------------------------------------ */
/* placement of one measurement                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int k;          /* w-plane (sw = 1), first plane of the w-footprint (sw > 1) */
    int fu, fv;     /* first footprint cell */
    int cu, cv;     /* nearest cell (density grid) */
    double pu, pv;  /* continuous cell coordinates, FP64 */
    double pw;      /* continuous plane coordinate (plane k's centre at k), FP64 */
} or_place;

/* Returns 1 when the measurement is gridded, 0 when it is dropped (a
 * non-finite coordinate or a footprint that leaves the grid). */
static int oracle_place(const or_cfg* c, float u, float v, float w, or_place* pl)
{
    if (!isfinite(u) || !isfinite(v) || !isfinite(w)) return 0;
    /* binary32 decisions */
    float pu32 = fmaf(u, c->uvscale_f, c->half_n_f);
    float pv32 = fmaf(v, c->uvscale_f, c->half_n_f);
    float au = floorf(pu32 - c->half_s_f);
    float av = floorf(pv32 - c->half_s_f);
    float lim = (float)(c->n - c->support - 1);
    if (!(au >= -1.0f && au <= lim && av >= -1.0f && av <= lim)) return 0;
    pl->fu = (int)au + 1;
    pl->fv = (int)av + 1;
    pl->cu = (int)floorf(pu32 + 0.5f);
    pl->cv = (int)floorf(pv32 + 0.5f);
    if (pl->cu > c->n - 1) pl->cu = c->n - 1;
    if (pl->cv > c->n - 1) pl->cv = c->n - 1;
    if (c->nw == 1) {
        pl->k = 0;
    } else if (c->sw == 1) {
        float t = (w - c->wmin_f) * c->invdw_f;
        float fk = floorf(t);
        if (fk < 0.0f) pl->k = 0;
        else if (fk > (float)(c->nw - 1)) pl->k = c->nw - 1;
        else pl->k = (int)fk;
    } else {
        /* planes fk .. fk + sw - 1, fk = floor(pw - sw/2) + 1, like a uv footprint */
        float pw32 = (w - c->wmin_f) * c->invdw_f - 0.5f;
        pl->k = (int)floorf(pw32 - c->half_sw_f) + 1;
    }
    pl->pw = ((double)w - c->w_min) / c->dw - 0.5;
    /* FP64 continuous positions */
    pl->pu = (double)u * c->uvscale + 0.5 * c->n;
    pl->pv = (double)v * c->uvscale + 0.5 * c->n;
    return 1;
}

/* Normalised taps g_t = g(f + t - p) / sum_t' g(f + t' - p). */
static void or_taps(const or_cfg* c, int f, double p, double* g)
{
    double s = 0.0;
    for (int t = 0; t < c->support; ++t) {
        g[t] = or_kernel(c, (double)(f + t) - p);
        s += g[t];
    }
    for (int t = 0; t < c->support; ++t) g[t] /= s;
}

/* Weight of plane k for a placed measurement: 1 for its nearest plane
 * (sw = 1), else the normalised w-tap h(k - pw) / sum_t h(fk + t - pw) when
 * k lies in fk .. fk + sw - 1 (planes outside 0 .. nw-1 are dropped with
 * their taps); 0 otherwise. */
static double or_plane_weight(const or_cfg* c, const or_place* pl, int k)
{
    if (c->sw == 1) return k == pl->k ? 1.0 : 0.0;
    int t = k - pl->k;
    if (t < 0 || t >= c->sw) return 0.0;
    double s = 0.0;
    for (int q = 0; q < c->sw; ++q) s += or_kernel_w(c, (double)(pl->k + q) - pl->pw);
    return or_kernel_w(c, (double)k - pl->pw) / s;
}

/* Grid correction in w (sw > 1): hw(xi) = int h(x) cos(2 pi x xi) dx / int h
 * over [-sw/2, sw/2] (Simpson, 4096 intervals), the factor the stacked image
 * is divided by at xi = dw (n - 1). */
static double or_wcorr(const or_cfg* c, double xi)
{
    const int K = 4096;
    const double a = -0.5 * c->sw, h = (double)c->sw / K;
    double num = 0.0, den = 0.0;
    for (int i = 0; i <= K; ++i) {
        num += c->wq[i] * cos(OR_TWO_PI * (a + i * h) * xi);
        den += c->wq[i];
    }
    return num / den;
}

static double or_plane_w(const or_cfg* c, int k)
{
    return c->w_min + (k + 0.5) * c->dw;
}

/* n - 1 without cancellation; returns 0 and sets *ok = 0 outside the sky. */
static double or_nm1(double l, double m, int* ok)
{
    double r2 = l * l + m * m;
    if (r2 >= 1.0) { *ok = 0; return 0.0; }
    *ok = 1;
    return -r2 / (1.0 + sqrt(1.0 - r2));
}

/* Exported helper: placement decisions of a batch (for tests). */
int oracle_place_batch(int n, int nw, double pixel_rad, double w_min, double w_max,
                       int kernel, int support, double kparam, int64_t m,
                       const float* u, const float* v, const float* w,
                       int32_t* k_out, int32_t* fu_out, int32_t* fv_out)
{
    or_cfg c;
    if (or_make_cfg(&c, n, nw, pixel_rad, w_min, w_max, kernel, support, kparam)) return -1;
    for (int64_t i = 0; i < m; ++i) {
        or_place pl;
        if (oracle_place(&c, u[i], v[i], w[i], &pl)) {
            k_out[i] = pl.k; fu_out[i] = pl.fu; fv_out[i] = pl.fv;
        } else {
            k_out[i] = -1; fu_out[i] = -1; fv_out[i] = -1;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* weights                                                                  */
/* ------------------------------------------------------------------------ */

/* Effective weight of every measurement: its weight, divided by the number of
 * gridded measurements whose nearest cell it shares when uniform weighting is
 * on; 0 for dropped measurements.  Returns the number dropped. */
static int64_t or_weights(const or_cfg* c, int uniform, int64_t m, const float* u,
                          const float* v, const float* w, const float* wt,
                          const float* vis, double* weff)
{
    int64_t dropped = 0;
    uint32_t* count = NULL;
    if (uniform) {
        count = (uint32_t*)calloc((size_t)c->n * c->n, sizeof(uint32_t));
        if (!count) return -1;
    }
    for (int64_t i = 0; i < m; ++i) {
        or_place pl;
        float wi = wt ? wt[i] : 1.0f;
        int ok = oracle_place(c, u[i], v[i], w[i], &pl) && isfinite(wi) &&
                 isfinite(vis[2 * i]) && isfinite(vis[2 * i + 1]);
        if (!ok) { weff[i] = 0.0; ++dropped; continue; }
        weff[i] = wi;
        if (uniform) count[(size_t)pl.cv * c->n + pl.cu] += 1;
    }
    if (uniform) {
        for (int64_t i = 0; i < m; ++i) {
            if (weff[i] == 0.0) continue;
            or_place pl;
            oracle_place(c, u[i], v[i], w[i], &pl);
            weff[i] /= (double)count[(size_t)pl.cv * c->n + pl.cu];
        }
        free(count);
    }
    return dropped;
}

/* ------------------------------------------------------------------------ */
/* gridding (Eq. 3)                                                         */
/* ------------------------------------------------------------------------ */

/* planes: complex double [k1-k0][n][n] (row = v cell, column = u cell),
 * accumulated into (caller zeroes).  Only planes k0 .. k1-1 are gridded,
 * each measurement with its weight on that plane (or_plane_weight). */
static void or_grid(const or_cfg* c, int64_t m, const float* u, const float* v,
                    const float* w, const float* vis, const double* weff, int k0,
                    int k1, double complex* planes)
{
    const size_t nn = (size_t)c->n * c->n;
    double gu[OR_MAX_SUPPORT], gv[OR_MAX_SUPPORT];
    for (int64_t i = 0; i < m; ++i) {
        if (weff[i] == 0.0) continue;
        or_place pl;
        if (!oracle_place(c, u[i], v[i], w[i], &pl)) continue;
        /* taps only for a measurement with a plane in [k0, k1) */
        int on_range = 0;
        for (int k = k0; k < k1 && !on_range; ++k) on_range = or_plane_weight(c, &pl, k) != 0.0;
        if (!on_range) continue;
        or_taps(c, pl.fu, pl.pu, gu);
        or_taps(c, pl.fv, pl.pv, gv);
        for (int k = k0; k < k1; ++k) {
            const double hk = or_plane_weight(c, &pl, k);
            if (hk == 0.0) continue;
            double complex a = hk * weff[i] * ((double)vis[2 * i] + I * (double)vis[2 * i + 1]);
            double complex* P = planes + (size_t)(k - k0) * nn;
            for (int r = 0; r < c->support; ++r)
                for (int q = 0; q < c->support; ++q)
                    P[(size_t)(pl.fv + r) * c->n + (pl.fu + q)] += a * gv[r] * gu[q];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FFT                                                                      */
/* ------------------------------------------------------------------------ */

static int or_is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* In-place 1D DFT  X[q] = sum_p x[p] exp(sign * 2 pi i p q / n), unnormalised.
 * Radix-2 decimation-in-time Cooley-Tukey for powers of two (bit reversal,
 * then log2 n butterfly stages with twiddles evaluated directly), the direct
 * O(n^2) sum otherwise.  `scratch` holds n elements. */
static void or_fft1d(int n, double complex* x, int sign, double complex* scratch)
{
    if (n <= 1) return;
    if (!or_is_pow2(n)) {
        for (int q = 0; q < n; ++q) {
            double complex s = 0.0;
            for (int p = 0; p < n; ++p) {
                long long pq = ((long long)p * q) % n;
                double ang = sign * OR_TWO_PI * (double)pq / n;
                s += x[p] * (cos(ang) + I * sin(ang));
            }
            scratch[q] = s;
        }
        memcpy(x, scratch, sizeof(double complex) * (size_t)n);
        return;
    }
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { double complex t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int j = 0; j < half; ++j) {
            double ang = sign * OR_TWO_PI * (double)j / len;
            double complex tw = cos(ang) + I * sin(ang);
            for (int s = 0; s < n; s += len) {
                double complex a = x[s + j], b = x[s + j + half] * tw;
                x[s + j] = a + b;
                x[s + j + half] = a - b;
            }
        }
    }
}

void oracle_fft(int n, double* data, int sign)
{
    double complex* sc = (double complex*)malloc(sizeof(double complex) * (size_t)n);
    or_fft1d(n, (double complex*)data, sign, sc);
    free(sc);
}

/* Unnormalised 2D transform with exponent sign, rows then columns. */
static void or_fft2d(int n, double complex* a, int sign)
{
#pragma omp parallel
    {
        double complex* sc = (double complex*)malloc(sizeof(double complex) * (size_t)n);
        double complex* col = (double complex*)malloc(sizeof(double complex) * (size_t)n);
#pragma omp for schedule(static)
        for (int r = 0; r < n; ++r) or_fft1d(n, a + (size_t)r * n, sign, sc);
#pragma omp for schedule(static)
        for (int q = 0; q < n; ++q) {
            for (int r = 0; r < n; ++r) col[r] = a[(size_t)r * n + q];
            or_fft1d(n, col, sign, sc);
            for (int r = 0; r < n; ++r) a[(size_t)r * n + q] = col[r];
        }
        free(sc);
        free(col);
    }
}

/* Circular shift by n/2 in both axes (fftshift == ifftshift for even n). */
static void or_shift_half(int n, double complex* a)
{
    int h = n / 2;
    for (int r = 0; r < h; ++r)
        for (int q = 0; q < n; ++q) {
            int q2 = (q + h) % n;
            double complex t = a[(size_t)r * n + q];
            a[(size_t)r * n + q] = a[(size_t)(r + h) * n + q2];
            a[(size_t)(r + h) * n + q2] = t;
        }
}

/* Plane image P[y][x] = sum_{jv,ju} G[jv][ju] exp(+2 pi i ((ju - n/2)(x - n/2) +
 * (jv - n/2)(y - n/2)) / n): ifftshift, unnormalised inverse DFT, fftshift.
 * With sign = -1 this is its adjoint (forward DFT between the same shifts). */
static void or_plane_transform(int n, double complex* a, int sign)
{
    or_shift_half(n, a);
    or_fft2d(n, a, sign);
    or_shift_half(n, a);
}

void oracle_plane_image(int n, double* grid_inout, int sign)
{
    or_plane_transform(n, (double complex*)grid_inout, sign);
}

/* ------------------------------------------------------------------------ */
/* taper (grid correction)                                                  */
/* ------------------------------------------------------------------------ */

/* c(x) = int g(t) cos(2 pi t (x - n/2) / n) dt / int g(t) dt over
 * t in [-S/2, S/2], composite Simpson with 2*nq intervals. */
static void or_taper(const or_cfg* c, double* taper)
{
    const int nq = 4096;
    const int npt = 2 * nq + 1;
    const double a = -0.5 * c->support, h = (double)c->support / (2 * nq);
    double* gw = (double*)malloc(sizeof(double) * npt);
    double* tt = (double*)malloc(sizeof(double) * npt);
    double norm = 0.0;
    for (int i = 0; i < npt; ++i) {
        double wgt = (i == 0 || i == npt - 1) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        tt[i] = a + i * h;
        gw[i] = wgt * or_kernel(c, tt[i]);
        norm += gw[i];
    }
#pragma omp parallel for schedule(static)
    for (int x = 0; x < c->n; ++x) {
        double xi = (double)(x - c->n / 2) / c->n;
        double s = 0.0;
        for (int i = 0; i < npt; ++i) s += gw[i] * cos(OR_TWO_PI * tt[i] * xi);
        taper[x] = s / norm;
    }
    free(gw);
    free(tt);
}

int oracle_taper(int n, int kernel, int support, double kparam, double* taper)
{
    or_cfg c;
    if (or_make_cfg(&c, n, 1, 1.0, 0.0, 0.0, kernel, support, kparam)) return -1;
    or_taper(&c, taper);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* the imager                                                               */
/* ------------------------------------------------------------------------ */

#define OR_FLAG_CORRECT 1u
#define OR_FLAG_APPLY_N 4u
#define OR_FLAG_UNIFORM 8u
#define OR_FLAG_FOLD 32u

/* Hermitian fold (real images): the visibility of a real sky satisfies
 * V(-u, -v, -w) = conj V(u, v, w), and a measurement imaged as its mirror
 * (-u, -v, -w, conj V) adds the complex conjugate of its own image term
 * (Eq. 1 and Eq. 3 with the mirrored cells: the plane transform of a mirrored,
 * conjugated grid is the conjugate of the plane image, and the screen
 * exp(2 pi i (-w)(n-1)) is the conjugate screen), so the real part of the
 * image is unchanged.  With the flag, every measurement with w < 0 is
 * replaced by its mirror before anything else; binary32 negation is exact.
 * The copies are released with or_unfold. */
typedef struct {
    float *u, *v, *w, *vis;
} or_fold_buf;

static void or_fold(unsigned flags, int64_t m, const float** u, const float** v, const float** w,
                    const float** vis, or_fold_buf* b)
{
    b->u = b->v = b->w = b->vis = NULL;
    if (!(flags & OR_FLAG_FOLD) || m <= 0) return;
    b->u = (float*)malloc(sizeof(float) * (size_t)m);
    b->v = (float*)malloc(sizeof(float) * (size_t)m);
    b->w = (float*)malloc(sizeof(float) * (size_t)m);
    b->vis = (float*)malloc(sizeof(float) * 2 * (size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        const int mirror = (*w)[i] < 0.0f;
        b->u[i] = mirror ? -(*u)[i] : (*u)[i];
        b->v[i] = mirror ? -(*v)[i] : (*v)[i];
        b->w[i] = mirror ? -(*w)[i] : (*w)[i];
        b->vis[2 * i] = (*vis)[2 * i];
        b->vis[2 * i + 1] = mirror ? -(*vis)[2 * i + 1] : (*vis)[2 * i + 1];
    }
    *u = b->u;
    *v = b->v;
    *w = b->w;
    *vis = b->vis;
}

static void or_unfold(or_fold_buf* b)
{
    free(b->u);
    free(b->v);
    free(b->w);
    free(b->vis);
}

/* Finalise pixel (x, y) of the stacked sum s: divide by the weight sum, by the
 * taper, multiply by n -- each as the flags ask. */
static double complex or_finalize_pixel(const or_cfg* c, unsigned flags, const double* taper,
                                        double sum_w, int x, int y, double complex s)
{
    double l = (x - c->n / 2) * c->pixel_rad, mm = (y - c->n / 2) * c->pixel_rad;
    int ok;
    double nm1 = or_nm1(l, mm, &ok);
    if (!ok) return 0.0;
    double complex d = (sum_w != 0.0) ? s / sum_w : 0.0;
    if (flags & OR_FLAG_CORRECT) d /= taper[x] * taper[y];
    if (flags & OR_FLAG_APPLY_N) d *= 1.0 + nm1;
    if (c->sw > 1) d /= or_wcorr(c, c->dw * nm1);
    return d;
}

/* Gridded planes only: planes_out complex double [k1-k0][n][n].  Returns the
 * number of dropped measurements (or -1 on bad arguments). */
int64_t oracle_grid(int n, int nw, double pixel_rad, double w_min, double w_max,
                    int kernel, int support, double kparam, unsigned flags,
                    int64_t m, const float* u, const float* v, const float* w,
                    const float* wt, const float* vis, int k0, int k1,
                    double* planes_out, double* sum_w_out)
{
    or_cfg c;
    if (or_make_cfg(&c, n, nw, pixel_rad, w_min, w_max, kernel, support, kparam)) return -1;
    if (or_set_wsupport(&c, flags)) return -1;
    or_prepare_wcorr(&c);
    if (k0 < 0 || k1 > nw || k0 > k1) return -1;
    or_fold_buf fold_buf;
    or_fold(flags, m, &u, &v, &w, &vis, &fold_buf);
    double* weff = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int64_t dropped = or_weights(&c, (flags & OR_FLAG_UNIFORM) != 0, m, u, v, w, wt, vis, weff);
    double sw = 0.0;
    for (int64_t i = 0; i < m; ++i) sw += weff[i];
    memset(planes_out, 0, sizeof(double complex) * (size_t)(k1 - k0) * n * n);
    or_grid(&c, m, u, v, w, vis, weff, k0, k1, (double complex*)planes_out);
    free(weff);
    if (sum_w_out) *sum_w_out = sw;
    or_unfold(&fold_buf);
    return dropped;
}

/* The full pipeline: grid planes [k0, k1), inverse FFT each, apply the w-term
 * phase screen, stack, finalise.  image_out: complex double [n][n].  With
 * k0 = 0, k1 = nw this is the dirty image; a sub-range gives the contribution
 * of those planes (normalised by the full weight sum). */
int64_t oracle_dirty_image(int n, int nw, double pixel_rad, double w_min, double w_max,
                           int kernel, int support, double kparam, unsigned flags,
                           int64_t m, const float* u, const float* v, const float* w,
                           const float* wt, const float* vis, int k0, int k1,
                           double* image_out, double* sum_w_out)
{
    or_cfg c;
    if (or_make_cfg(&c, n, nw, pixel_rad, w_min, w_max, kernel, support, kparam)) return -1;
    if (or_set_wsupport(&c, flags)) return -1;
    or_prepare_wcorr(&c);
    if (k0 < 0 || k1 > nw || k0 > k1) return -1;
    or_fold_buf fold_buf;
    or_fold(flags, m, &u, &v, &w, &vis, &fold_buf);
    const size_t nn = (size_t)n * n;
    double* weff = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int64_t dropped = or_weights(&c, (flags & OR_FLAG_UNIFORM) != 0, m, u, v, w, wt, vis, weff);
    double sw = 0.0;
    for (int64_t i = 0; i < m; ++i) sw += weff[i];
    double complex* acc = (double complex*)calloc(nn, sizeof(double complex));
    double complex* plane = (double complex*)malloc(sizeof(double complex) * nn);
    for (int k = k0; k < k1; ++k) {
        memset(plane, 0, sizeof(double complex) * nn);
        or_grid(&c, m, u, v, w, vis, weff, k, k + 1, plane);
        or_plane_transform(n, plane, +1);
        double wk = or_plane_w(&c, k);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                int ok;
                double nm1 = or_nm1((x - n / 2) * pixel_rad, (y - n / 2) * pixel_rad, &ok);
                if (!ok) continue;
                double ph = OR_TWO_PI * wk * nm1;
                acc[(size_t)y * n + x] += plane[(size_t)y * n + x] * (cos(ph) + I * sin(ph));
            }
    }
    double* taper = (double*)malloc(sizeof(double) * n);
    or_taper(&c, taper);
    double complex* out = (double complex*)image_out;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            out[(size_t)y * n + x] = or_finalize_pixel(&c, flags, taper, sw, x, y, acc[(size_t)y * n + x]);
    free(taper);
    free(plane);
    free(acc);
    free(weff);
    if (sum_w_out) *sum_w_out = sw;
    or_unfold(&fold_buf);
    return dropped;
}

/* The same discrete algorithm evaluated at chosen pixels without any FFT:
 * because the gridding kernel is separable, each measurement's contribution to
 * pixel (x, y) of its plane image is
 *   a_m * [sum_t gu_t e^{2 pi i (fu+t-n/2)(x-n/2)/n}] [sum_t gv_t e^{2 pi i (fv+t-n/2)(y-n/2)/n}],
 * multiplied by the plane's phase screen.  Used for sampled checks at sizes
 * where the full FFT oracle is too slow.  pix: int32 pairs (x, y).
 *
 * The u-axis sum depends on the pixel's x only and the v-axis sum on its y
 * only, so each is formed once per distinct column x and row y among the
 * pixels; the phase factors e^{2 pi i ((j-n/2)(x-n/2) mod n)/n} of every cell
 * j and the screens e^{2 pi i w_k (n-1)} of every plane are tabulated once
 * (the same expressions evaluated once instead of per measurement). */
int64_t oracle_image_at(int n, int nw, double pixel_rad, double w_min, double w_max,
                        int kernel, int support, double kparam, unsigned flags,
                        int64_t m, const float* u, const float* v, const float* w,
                        const float* wt, const float* vis, int npix, const int32_t* pix,
                        double* values_out, double* sum_w_out)
{
    or_cfg c;
    if (or_make_cfg(&c, n, nw, pixel_rad, w_min, w_max, kernel, support, kparam)) return -1;
    if (or_set_wsupport(&c, flags)) return -1;
    for (int q = 0; q < npix; ++q)
        if (pix[2 * q] < 0 || pix[2 * q] >= n || pix[2 * q + 1] < 0 || pix[2 * q + 1] >= n) return -1;
    or_prepare_wcorr(&c);
    or_fold_buf fold_buf;
    or_fold(flags, m, &u, &v, &w, &vis, &fold_buf);
    double* weff = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int64_t dropped = or_weights(&c, (flags & OR_FLAG_UNIFORM) != 0, m, u, v, w, wt, vis, weff);
    double sw = 0.0;
    for (int64_t i = 0; i < m; ++i) sw += weff[i];
    double* taper = (double*)malloc(sizeof(double) * n);
    or_taper(&c, taper);
    double complex* out = (double complex*)values_out;
    const int np1 = npix > 0 ? npix : 1;
    /* per pixel: its n - 1 (or outside the sky), its column and row index */
    double* nm1 = (double*)malloc(sizeof(double) * (size_t)np1);
    int* sky = (int*)malloc(sizeof(int) * (size_t)np1);
    int* xi = (int*)malloc(sizeof(int) * (size_t)np1);
    int* yi = (int*)malloc(sizeof(int) * (size_t)np1);
    int* xmap = (int*)malloc(sizeof(int) * (size_t)n);
    int* ymap = (int*)malloc(sizeof(int) * (size_t)n);
    int* xs = (int*)malloc(sizeof(int) * (size_t)np1);
    int* ys = (int*)malloc(sizeof(int) * (size_t)np1);
    int nx = 0, ny = 0;
    for (int j = 0; j < n; ++j) xmap[j] = ymap[j] = -1;
    for (int q = 0; q < npix; ++q) {
        const int x = pix[2 * q], y = pix[2 * q + 1];
        nm1[q] = or_nm1((x - n / 2) * pixel_rad, (y - n / 2) * pixel_rad, &sky[q]);
        if (xmap[x] < 0) { xmap[x] = nx; xs[nx++] = x; }
        if (ymap[y] < 0) { ymap[y] = ny; ys[ny++] = y; }
        xi[q] = xmap[x];
        yi[q] = ymap[y];
    }
    /* phase factor tables: eu[a * n + j] for column xs[a] and cell j (ev: rows) */
    double complex* eu = (double complex*)malloc(sizeof(double complex) * (size_t)(nx > 0 ? nx : 1) * n);
    double complex* ev = (double complex*)malloc(sizeof(double complex) * (size_t)(ny > 0 ? ny : 1) * n);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < nx; ++a)
        for (int j = 0; j < n; ++j) {
            double au = OR_TWO_PI * (double)((long long)(j - n / 2) * (xs[a] - n / 2) % n) / n;
            eu[(size_t)a * n + j] = cos(au) + I * sin(au);
        }
#pragma omp parallel for schedule(static)
    for (int b = 0; b < ny; ++b)
        for (int j = 0; j < n; ++j) {
            double av = OR_TWO_PI * (double)((long long)(j - n / 2) * (ys[b] - n / 2) % n) / n;
            ev[(size_t)b * n + j] = cos(av) + I * sin(av);
        }
    /* screen table: scr[q * nw + k] = e^{2 pi i w_k (n-1)} at pixel q */
    double complex* scr = (double complex*)malloc(sizeof(double complex) * (size_t)np1 * nw);
    for (int q = 0; q < npix; ++q)
        for (int k = 0; k < nw; ++k) {
            double ph = OR_TWO_PI * or_plane_w(&c, k) * nm1[q];
            scr[(size_t)q * nw + k] = cos(ph) + I * sin(ph);
        }
    double complex* sum = (double complex*)calloc((size_t)np1, sizeof(double complex));
    /* measurement-outer: taps and axis sums once per measurement, then every pixel */
#pragma omp parallel
    {
        double complex* part = (double complex*)calloc((size_t)np1, sizeof(double complex));
        double complex* su = (double complex*)malloc(sizeof(double complex) * (size_t)(nx > 0 ? nx : 1));
        double complex* sv = (double complex*)malloc(sizeof(double complex) * (size_t)(ny > 0 ? ny : 1));
        int kl[OR_MAX_SUPPORT];
        double hl[OR_MAX_SUPPORT];
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            if (weff[i] == 0.0) continue;
            or_place pl;
            if (!oracle_place(&c, u[i], v[i], w[i], &pl)) continue;
            double gu[OR_MAX_SUPPORT], gv[OR_MAX_SUPPORT];
            or_taps(&c, pl.fu, pl.pu, gu);
            or_taps(&c, pl.fv, pl.pv, gv);
            double complex a = weff[i] * ((double)vis[2 * i] + I * (double)vis[2 * i + 1]);
            for (int b = 0; b < nx; ++b) {
                const double complex* e = eu + (size_t)b * n + pl.fu;
                double complex s = 0.0;
                for (int t = 0; t < c.support; ++t) s += gu[t] * e[t];
                su[b] = s;
            }
            for (int b = 0; b < ny; ++b) {
                const double complex* e = ev + (size_t)b * n + pl.fv;
                double complex s = 0.0;
                for (int t = 0; t < c.support; ++t) s += gv[t] * e[t];
                sv[b] = s;
            }
            /* the planes the measurement is gridded onto and their weights */
            int nl = 0;
            const int ka = c.sw == 1 ? pl.k : (pl.k > 0 ? pl.k : 0);
            const int kb = c.sw == 1 ? pl.k + 1 : (pl.k + c.sw < nw ? pl.k + c.sw : nw);
            for (int k = ka; k < kb; ++k) {
                const double hk = or_plane_weight(&c, &pl, k);
                if (hk == 0.0) continue;
                kl[nl] = k;
                hl[nl++] = hk;
            }
            for (int q = 0; q < npix; ++q) {
                if (!sky[q]) continue;
                double complex sw_sum = 0.0;
                for (int r = 0; r < nl; ++r) sw_sum += hl[r] * scr[(size_t)q * nw + kl[r]];
                part[q] += a * su[xi[q]] * sv[yi[q]] * sw_sum;
            }
        }
#pragma omp critical
        for (int q = 0; q < npix; ++q) sum[q] += part[q];
        free(sv);
        free(su);
        free(part);
    }
    for (int q = 0; q < npix; ++q)
        out[q] = or_finalize_pixel(&c, flags, taper, sw, pix[2 * q], pix[2 * q + 1], sky[q] ? sum[q] : 0.0);
    free(sum);
    free(scr);
    free(ev);
    free(eu);
    free(ys);
    free(xs);
    free(ymap);
    free(xmap);
    free(yi);
    free(xi);
    free(sky);
    free(nm1);
    free(taper);
    free(weff);
    if (sum_w_out) *sum_w_out = sw;
    or_unfold(&fold_buf);
    return dropped;
}

/* Brute-force direct DFT with the exact w-term (Eq. 1 with the plane sum
 * replaced by the exact phase of every measurement, Eq. 2's kernel):
 *   D(l,m) = sum_k wt_k V_k exp(2 pi i (u_k l + v_k m + w_k (n-1))) / sum wt_k,
 * over the measurements the imager grids (same weights, same drops).  No
 * gridding, no FFT, no w-quantisation, no taper.  pix: int32 pairs (x, y). */
int64_t oracle_dft(int n, int nw, double pixel_rad, double w_min, double w_max,
                   int kernel, int support, double kparam, unsigned flags,
                   int64_t m, const float* u, const float* v, const float* w,
                   const float* wt, const float* vis, int npix, const int32_t* pix,
                   double* values_out)
{
    or_cfg c;
    if (or_make_cfg(&c, n, nw, pixel_rad, w_min, w_max, kernel, support, kparam)) return -1;
    if (or_set_wsupport(&c, flags)) return -1;
    or_prepare_wcorr(&c);
    or_fold_buf fold_buf;
    or_fold(flags, m, &u, &v, &w, &vis, &fold_buf);
    double* weff = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int64_t dropped = or_weights(&c, (flags & OR_FLAG_UNIFORM) != 0, m, u, v, w, wt, vis, weff);
    double sw = 0.0;
    for (int64_t i = 0; i < m; ++i) sw += weff[i];
    double complex* out = (double complex*)values_out;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < npix; ++q) {
        int x = pix[2 * q], y = pix[2 * q + 1];
        double l = (x - n / 2) * pixel_rad, mm = (y - n / 2) * pixel_rad;
        int ok;
        double nm1 = or_nm1(l, mm, &ok);
        double complex s = 0.0;
        if (ok)
            for (int64_t i = 0; i < m; ++i) {
                if (weff[i] == 0.0) continue;
                double ph = OR_TWO_PI * ((double)u[i] * l + (double)v[i] * mm + (double)w[i] * nm1);
                s += weff[i] * ((double)vis[2 * i] + I * (double)vis[2 * i + 1]) * (cos(ph) + I * sin(ph));
            }
        double complex d = (ok && sw != 0.0) ? s / sw : 0.0;
        if (ok && (flags & OR_FLAG_APPLY_N)) d *= 1.0 + nm1;
        out[q] = d;
    }
    free(weff);
    or_unfold(&fold_buf);
    return dropped;
}

/* Adjoint of the complex dirty-image operator V -> D (flags as in
 * oracle_dirty_image), applied to a complex image r: for every plane k,
 * Q = r / sum_w / taper * n * exp(-2 pi i w_k (n-1)), F_k = forward DFT of Q
 * between the same shifts, then each measurement gathers its footprint of
 * F_k with the same normalised taps, times its effective weight.
 * grad_out: complex double [m]. */
static int64_t or_degrid(int n, int nw, double pixel_rad, double w_min, double w_max,
                         int kernel, int support, double kparam, unsigned flags,
                         int64_t m, const float* u, const float* v, const float* w,
                         const float* wt, const float* vis, const double* r_in,
                         double* grad_out, int predict)
{
    or_cfg c;
    if (or_make_cfg(&c, n, nw, pixel_rad, w_min, w_max, kernel, support, kparam)) return -1;
    if (or_set_wsupport(&c, flags)) return -1;
    or_prepare_wcorr(&c);
    const float* w_given = w;  /* signs before the fold: mirrored gradients are conjugated */
    or_fold_buf fold_buf;
    or_fold(flags, m, &u, &v, &w, &vis, &fold_buf);
    const size_t nn = (size_t)n * n;
    double* weff = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int64_t dropped = or_weights(&c, (flags & OR_FLAG_UNIFORM) != 0, m, u, v, w, wt, vis, weff);
    double sw = 0.0;
    for (int64_t i = 0; i < m; ++i) sw += weff[i];
    if (predict) sw = 1.0;  /* prediction: no normalisation by the weight sum */
    double* taper = (double*)malloc(sizeof(double) * n);
    or_taper(&c, taper);
    const double complex* r = (const double complex*)r_in;
    double complex* R = (double complex*)malloc(sizeof(double complex) * nn);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            /* the finaliser is real-linear per pixel: apply the same factors */
            R[(size_t)y * n + x] = or_finalize_pixel(&c, flags, taper, sw, x, y, r[(size_t)y * n + x]);
    double complex* F = (double complex*)malloc(sizeof(double complex) * nn);
    double complex* g = (double complex*)grad_out;
    for (int64_t i = 0; i < m; ++i) g[i] = 0.0;
    for (int k = 0; k < nw; ++k) {
        double wk = or_plane_w(&c, k);
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                int ok;
                double nm1 = or_nm1((x - n / 2) * pixel_rad, (y - n / 2) * pixel_rad, &ok);
                double ph = -OR_TWO_PI * wk * nm1;
                F[(size_t)y * n + x] = ok ? R[(size_t)y * n + x] * (cos(ph) + I * sin(ph)) : 0.0;
            }
        or_plane_transform(n, F, -1);
        for (int64_t i = 0; i < m; ++i) {
            if (weff[i] == 0.0) continue;
            or_place pl;
            if (!oracle_place(&c, u[i], v[i], w[i], &pl)) continue;
            const double hk = or_plane_weight(&c, &pl, k);
            if (hk == 0.0) continue;
            double gu[OR_MAX_SUPPORT], gv[OR_MAX_SUPPORT];
            or_taps(&c, pl.fu, pl.pu, gu);
            or_taps(&c, pl.fv, pl.pv, gv);
            double complex s = 0.0;
            for (int rr = 0; rr < c.support; ++rr)
                for (int q = 0; q < c.support; ++q)
                    s += gv[rr] * gu[q] * F[(size_t)(pl.fv + rr) * n + (pl.fu + q)];
            g[i] += hk * weff[i] * s;
        }
    }
    free(F);
    free(R);
    free(taper);
    free(weff);
    if (flags & OR_FLAG_FOLD)
        for (int64_t i = 0; i < m; ++i)
            if (w_given[i] < 0.0f) g[i] = conj(g[i]);
    or_unfold(&fold_buf);
    return dropped;
}

int64_t oracle_degrid(int n, int nw, double pixel_rad, double w_min, double w_max,
                      int kernel, int support, double kparam, unsigned flags,
                      int64_t m, const float* u, const float* v, const float* w,
                      const float* wt, const float* vis, const double* r_in,
                      double* grad_out)
{
    return or_degrid(n, nw, pixel_rad, w_min, w_max, kernel, support, kparam, flags, m, u, v, w, wt, vis, r_in,
                     grad_out, 0);
}

/* Model visibilities of the image `model` (complex double [n][n]): the same
 * chain as the adjoint with unit weights and no division by their sum, i.e.
 * the w-stacking evaluation of the measurement equation (Eq. 2 with the
 * image in place of I/n): model / taper * n (per flags) * exp(-2 pi i w_k
 * (n-1)), forward DFT, gather with the normalised taps.  Measurements that
 * cannot be placed get 0.  vis_out: complex double [m]. */
int64_t oracle_predict(int n, int nw, double pixel_rad, double w_min, double w_max,
                       int kernel, int support, double kparam, unsigned flags,
                       int64_t m, const float* u, const float* v, const float* w,
                       const double* model, double* vis_out)
{
    float* one = (float*)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
    float* zero = (float*)calloc(2 * (size_t)(m > 0 ? m : 1), sizeof(float));
    for (int64_t i = 0; i < m; ++i) one[i] = 1.0f;
    const int64_t d = or_degrid(n, nw, pixel_rad, w_min, w_max, kernel, support, kparam, flags & ~OR_FLAG_UNIFORM,
                                m, u, v, w, one, zero, model, vis_out, 1);
    free(one);
    free(zero);
    return d;
}

/* Number of OpenMP threads the oracle runs on. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
