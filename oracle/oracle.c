/*
 * oracle.c -- CPU oracle for table-free Gaussian-mixture rANS coding.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library. The product path
 * (the CUDA library) shares no code, header, table or constant generator
 * with it, and never calls it.
 *
 * What it computes, in the paper's terms:
 *   - the GMM of Sec. II-A, Eq. 2: p(y) = sum_k w_k N(y; mu_k, sigma_k);
 *   - symbol s owns the mixture-CDF interval [F(s-1/2), F(s+1/2)), the
 *     per-symbol mass of the CDF table of Sec. II-C, Eqs. 4-5;
 *   - Phi is approximated by Abramowitz & Stegun 26.2.17 (Sec. III-B, Eq. 8)
 *     evaluated in FP32, or (selected by or_set_phi) by the logistic or the
 *     Polya approximation (Sec. III-B), for the comparison of Sec. V,
 *     Table II;
 *   - the CDF is quantised to 16-bit rANS frequencies on the fly for the one
 *     symbol being coded (Sec. III-A), coded with rANS (Sec. II-B, Eq. 3),
 *     and decoded by binary search over the same quantised CDF (Sec. III-A);
 *   - an FP64 rate audit against the exact mixture (Sec. V "no
 *     approximation" row, std::erfc).
 * The paper leaves every bit-level choice open; the readings taken here
 * (window, escape, rANS word size, interleaving, the 2^-22 grid on z) are
 * stated where they are used.
 *
 * Plain and slow on purpose: one symbol at a time, no blocking, no fusion.
 * Compile with -ffp-contract=off and without -ffast-math: every FP32
 * operation below is one IEEE round-to-nearest operation, fmaf is one fused
 * rounding, '/' is correctly rounded.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PREC_BITS 16
#define OR_M (1u << OR_PREC_BITS)  /* total frequency, 2^16 */
#define OR_L (1u << 16)            /* rANS lower bound and initial state */
#define OR_YMAX 255                /* window clamp: alphabet [-255, 255] */
#define OR_ZC 12.0f                /* |z| clamp of the Phi approximation */
#define OR_MAXK 4

/* status codes (same meaning as the library's, defined independently) */
#define OR_OK 0
#define OR_INVALID 1
#define OR_BAD_PARAMS 2
#define OR_CAPACITY 3
#define OR_CORRUPT 4

#define OR_PHI_AS 0
#define OR_PHI_LOGISTIC 1
#define OR_PHI_POLYA 2

/* ---------------------------------------------------------------------
 * exp(a) for a in [-72, 21] in FP32, written from the Cody-Waite method:
 * a = k ln2 + r with k = rint(a / ln2), ln2 split in a high part with a
 * short mantissa and a low part, |r| <= ln2/2; exp(r) by its Taylor series
 * to degree 7 (truncation < 2^-27 relative); scale by 2^k through the
 * exponent field (the result stays normal for -72 <= a <= 21).
 * ------------------------------------------------------------------- */
float or_exp(float a)
{
    const float log2e = 0x1.715476p+0f;      /* float(1/ln 2) */
    const float ln2_hi = 0x1.62e4p-1f;       /* ln 2 with the low 8 bits of float(ln 2) cleared */
    const float ln2_lo = 0x1.7f7d1cp-20f;    /* float(ln 2 - ln2_hi) */
    float k = rintf(a * log2e);
    float r = fmaf(-k, ln2_hi, a);
    r = fmaf(-k, ln2_lo, r);
    /* Taylor coefficients 1/i!, i = 7 .. 0, Horner in fmaf */
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    uint32_t u;
    memcpy(&u, &p, 4);
    u += (uint32_t)(int32_t)k << 23;
    memcpy(&p, &u, 4);
    return p;
}

/* ---------------------------------------------------------------------
 * Phi-hat(z): A&S 26.2.17 (Sec. III-B, Eq. 8),
 *   Phi(x) ~ 1 - Z(x) (b1 t + b2 t^2 + b3 t^3 + b4 t^4 + b5 t^5),
 *   t = 1/(1 + p x), Z the standard normal density, for x >= 0, and
 *   Phi(-x) = 1 - Phi(x).
 * Constants from the handbook: p = 0.2316419, b1..b5 = 0.319381530,
 * -0.356563782, 1.781477937, -1.821255978, 1.330274429. The factor
 * 1/sqrt(2 pi) of Z is folded into the b_i (c_i = float(b_i / sqrt(2 pi))).
 * z is clamped to [-12, 12] and rounded (half to even) to the grid 2^-22,
 * on which the FP32 evaluation is monotone non-decreasing (checked by an
 * exhaustive sweep of the grid in the test suite).
 * ------------------------------------------------------------------- */
float or_phi(float z)
{
    const float p = 0x1.da6712p-3f;          /* float(0.2316419) */
    const float c1 = 0x1.04f20cp-3f;
    const float c2 = -0x1.23531cp-3f;
    const float c3 = 0x1.6be1c6p-1f;
    const float c4 = -0x1.7401c6p-1f;
    const float c5 = 0x1.0fb844p-1f;
    float zc = fminf(fmaxf(z, -OR_ZC), OR_ZC);
    float zs = rintf(zc * 0x1p22f) * 0x1p-22f;
    float x = fabsf(zs);
    float d = fmaf(p, x, 1.0f);
    float t = 1.0f / d;
    float h = fmaf(c5, t, c4);
    h = fmaf(h, t, c3);
    h = fmaf(h, t, c2);
    h = fmaf(h, t, c1);
    float g = h * t;
    float a = -0.5f * (x * x);
    float e = or_exp(a);
    float q = e * g;
    return zs >= 0.0f ? 1.0f - q : q;
}

/* ---------------------------------------------------------------------
 * The other two approximations of Sec. III-B, on the same clamp and grid:
 * each returns the lower tail q = Phi-hat(-x) for x = |z| >= 0, and
 * Phi-hat(z) = z >= 0 ? 1 - q : q.
 *
 * Logistic (Sec. III-B): Phi(x) ~ 1 / (1 + exp(-1.702 x)), so
 *   q = 1 / (1 + exp(1.702 x)),
 * one correctly rounded reciprocal of a non-decreasing quantity.
 *
 * Polya (Sec. III-B): Phi(x) ~ (1 + sqrt(1 - exp(-2 x^2 / pi))) / 2 for
 * x >= 0. The paper prints exp(-x^2) inside the root; Polya's (1949) form
 * has the factor 2/pi, which the approximation needs to stay within 0.003
 * of Phi; that form is the reading taken here. The tail is evaluated
 * without cancellation as
 *   q = (1 - sqrt(1 - e)) / 2 = (e / 2) * (1 / (1 + sqrt(1 - e))),
 *   e = exp(max(-(2/pi) x^2, -72)),
 * a product of a non-increasing and a non-increasing factor.
 * Both are monotone on the grid when exp is (checked exhaustively).
 * ------------------------------------------------------------------- */
static float logistic_tail(float x)
{
    float E = or_exp(1.702f * x);
    return 1.0f / (1.0f + E);
}

static float polya_tail(float x)
{
    const float two_over_pi = 0x1.45f306p-1f;   /* float(2/pi) */
    float a = fmaxf(-(two_over_pi * (x * x)), -72.0f);
    float e = or_exp(a);
    float s = sqrtf(1.0f - e);
    return (0.5f * e) * (1.0f / (1.0f + s));
}

float or_phi_v(float z, int v)
{
    if (v == OR_PHI_AS) return or_phi(z);
    float zc = fminf(fmaxf(z, -OR_ZC), OR_ZC);
    float zs = rintf(zc * 0x1p22f) * 0x1p-22f;
    float x = fabsf(zs);
    float q = v == OR_PHI_LOGISTIC ? logistic_tail(x) : polya_tail(x);
    return zs >= 0.0f ? 1.0f - q : q;
}

/* The approximation used by the coding functions below (A&S by default). */
static int g_phi = OR_PHI_AS;

int or_set_phi(int v)
{
    if (v < OR_PHI_AS || v > OR_PHI_POLYA) return OR_INVALID;
    g_phi = v;
    return OR_OK;
}

/* ---------------------------------------------------------------------
 * One symbol's mixture parameters, read from the planar layout
 * params[(c*K + k)*N + n], c = 0 (w), 1 (mu), 2 (sigma).
 * ------------------------------------------------------------------- */
typedef struct {
    int K;
    float w[OR_MAXK], mu[OR_MAXK], sig[OR_MAXK];
} or_mix;

static void load_mix(const float *params, int K, int64_t N, int64_t n, or_mix *m)
{
    m->K = K;
    for (int k = 0; k < K; ++k) {
        m->w[k] = params[(int64_t)(0 * K + k) * N + n];
        m->mu[k] = params[(int64_t)(1 * K + k) * N + n];
        m->sig[k] = params[(int64_t)(2 * K + k) * N + n];
    }
}

/* Valid parameters: weights finite and >= 0, means finite, scales finite
 * and > 0 (Eq. 2 requires w_k >= 0 and sigma_k > 0). */
static int mix_ok(const or_mix *m)
{
    for (int k = 0; k < m->K; ++k) {
        if (!isfinite(m->w[k]) || m->w[k] < 0.0f) return 0;
        if (!isfinite(m->mu[k])) return 0;
        if (!isfinite(m->sig[k]) || !(m->sig[k] > 0.0f)) return 0;
    }
    return 1;
}

/* Scale floor 0.11, the lowest level of the scale table described in
 * Sec. II-B (the paper does not floor scales itself). */
static float sig_floor(float s) { return fmaxf(s, 0.11f); }

/* F-hat(b) = sum_k w_k Phi-hat((b - mu_k)/sigma'_k), k ascending, with the
 * component argument z = (b - mu_k) * (1/sigma'_k): two roundings, monotone
 * in b, and no cancellation when |mu_k| >> sigma'_k. */
float or_mixcdf_one(const or_mix *m, float b)
{
    float acc = 0.0f;
    for (int k = 0; k < m->K; ++k) {
        float sp = sig_floor(m->sig[k]);
        float inv = 1.0f / sp;
        float z = (b - m->mu[k]) * inv;
        acc = fmaf(m->w[k], or_phi_v(z, g_phi), acc);
    }
    return acc;
}

/* Window [lo, hi]: mu_k -/+ R sigma'_k with R = 8 over all components,
 * floored/ceiled and clamped to [-255, 255]. Symbols outside it are coded
 * through the escape slot (the paper fixes no tail rule; this is the
 * reading taken here). */
static void window_of(const or_mix *m, int *lo, int *hi)
{
    float a = INFINITY, b = -INFINITY;
    for (int k = 0; k < m->K; ++k) {
        float sp = sig_floor(m->sig[k]);
        a = fminf(a, fmaf(-8.0f, sp, m->mu[k]));
        b = fmaxf(b, fmaf(8.0f, sp, m->mu[k]));
    }
    a = fminf(fmaxf(floorf(a), -(float)OR_YMAX), (float)OR_YMAX);
    b = fminf(fmaxf(ceilf(b), -(float)OR_YMAX), (float)OR_YMAX);
    int l = (int)a, h = (int)b;
    if (l > h) { int t = l; l = h; h = t; }
    *lo = l;
    *hi = h;
}

/* Quantised CDF Q(j), lo <= j <= hi+1:
 *   Q(lo) = 0, Q(j) = (j - lo) + floor(T' * min(F-hat(j - 1/2), 1)),
 *   T' = 2^16 - W - 1, W = hi - lo + 1.
 * Every in-window symbol then gets frequency >= 1, and the escape slot
 * [Q(hi+1), 2^16) gets at least 1. */
static uint32_t Qof(const or_mix *m, int lo, int hi, int j)
{
    if (j == lo) return 0;
    int W = hi - lo + 1;
    float Tp = (float)(int)(OR_M - (uint32_t)W - 1u);
    float v = fminf(or_mixcdf_one(m, (float)j - 0.5f), 1.0f);
    return (uint32_t)(j - lo) + (uint32_t)floorf(Tp * v);
}

/* The rANS interval (start, freq) of symbol s; returns 1 for an escape. */
static int interval_of(const or_mix *m, int32_t s, uint32_t *start, uint32_t *freq)
{
    int lo, hi;
    window_of(m, &lo, &hi);
    if (s >= lo && s <= hi) {
        uint32_t a = Qof(m, lo, hi, s);
        uint32_t b = Qof(m, lo, hi, s + 1);
        *start = a;
        *freq = b - a;
        return 0;
    }
    uint32_t e = Qof(m, lo, hi, hi + 1);
    *start = e;
    *freq = OR_M - e;
    return 1;
}

/* ---- exported helpers for tests --------------------------------------- */

void or_phi_many(const float *z, float *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_phi(z[i]);
}

void or_exp_many(const float *a, float *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_exp(a[i]);
}

/* Exhaustive sweep of Phi-hat over the grid points i * 2^-22 for
 * i in [i0, i1]: counts decreases between consecutive points, and the
 * largest |Phi-hat - Phi| with Phi = erfc(-z/sqrt 2)/2 in FP64 (evaluated on
 * every `err_stride`-th point). out[0] = violations, out[1] = max error,
 * out[2] = z of max error. */
void or_phi_grid_sweep(int64_t i0, int64_t i1, int64_t err_stride, double *out)
{
    double viol = 0.0, maxerr = 0.0, zmax = 0.0;
    float prev = or_phi((float)i0 * 0x1p-22f);
    for (int64_t i = i0; i <= i1; ++i) {
        float z = (float)i * 0x1p-22f;
        float v = or_phi(z);
        if (v < prev) viol += 1.0;
        prev = v;
        if (err_stride > 0 && (i - i0) % err_stride == 0) {
            double ex = 0.5 * erfc(-(double)z / sqrt(2.0));
            double e = fabs((double)v - ex);
            if (e > maxerr) { maxerr = e; zmax = z; }
        }
    }
    out[0] = viol;
    out[1] = maxerr;
    out[2] = zmax;
}

/* The sweep of or_phi_grid_sweep for approximation v, against v's own
 * formula in FP64 (out[1], out[2]) and against Phi (out[3], out[4]):
 * out[0] = decreases between consecutive grid points in [i0, i1]. */
void or_phi_v_grid_sweep(int64_t i0, int64_t i1, int64_t err_stride, int v, double *out)
{
    double viol = 0.0, maxf = 0.0, zf = 0.0, maxg = 0.0, zg = 0.0;
    float prev = or_phi_v((float)i0 * 0x1p-22f, v);
    for (int64_t i = i0; i <= i1; ++i) {
        float z = (float)i * 0x1p-22f;
        float val = or_phi_v(z, v);
        if (val < prev) viol += 1.0;
        prev = val;
        if (err_stride > 0 && (i - i0) % err_stride == 0) {
            double x = (double)z, f;
            if (v == OR_PHI_LOGISTIC) f = 1.0 / (1.0 + exp(-1.702 * x));
            else if (v == OR_PHI_POLYA) {
                double r = sqrt(1.0 - exp(-2.0 * x * x / 3.14159265358979323846));
                f = x >= 0.0 ? 0.5 * (1.0 + r) : 0.5 * (1.0 - r);
            } else f = 0.5 * erfc(-x / sqrt(2.0));
            double ef = fabs((double)val - f), eg = fabs((double)val - 0.5 * erfc(-x / sqrt(2.0)));
            if (ef > maxf) { maxf = ef; zf = x; }
            if (eg > maxg) { maxg = eg; zg = x; }
        }
    }
    out[0] = viol;
    out[1] = maxf;
    out[2] = zf;
    out[3] = maxg;
    out[4] = zg;
}

void or_phi_v_many(const float *z, float *out, int64_t n, int v)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_phi_v(z[i], v);
}

/* Grid sweep that returns the values themselves (for CPU/GPU bit checks). */
void or_phi_grid(int64_t i0, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = or_phi((float)(i0 + i) * 0x1p-22f);
}

/* F-hat(b) for symbol n at boundary b (tests). */
float or_mixcdf(const float *params, int K, int64_t N, int64_t n, float b)
{
    or_mix m;
    load_mix(params, K, N, n, &m);
    return or_mixcdf_one(&m, b);
}

void or_window(const float *params, int K, int64_t N, int32_t *lo, int32_t *hi)
{
    for (int64_t n = 0; n < N; ++n) {
        or_mix m;
        load_mix(params, K, N, n, &m);
        int a, b;
        window_of(&m, &a, &b);
        lo[n] = a;
        hi[n] = b;
    }
}

/* Per-symbol intervals. sf[n] = start | freq << 16; escape iff
 * start + freq == 2^16. Returns OR_BAD_PARAMS if any parameter is invalid
 * (nothing written then). */
int or_freqs(const float *params, int K, int64_t N, const int32_t *sym, uint32_t *sf)
{
    if (K < 1 || K > OR_MAXK || N < 0) return OR_INVALID;
    for (int64_t n = 0; n < N; ++n) {
        or_mix m;
        load_mix(params, K, N, n, &m);
        if (!mix_ok(&m)) return OR_BAD_PARAMS;
    }
    for (int64_t n = 0; n < N; ++n) {
        or_mix m;
        load_mix(params, K, N, n, &m);
        uint32_t st, fr;
        interval_of(&m, sym[n], &st, &fr);
        sf[n] = st | (fr << 16);
    }
    return OR_OK;
}

/* Full table over the alphabet j in [-255, 256] by direct evaluation of Q
 * at every point (the table of Sec. II-C, Eqs. 4-5, quantised as above):
 * tab[n*512 + (j+255)] = Q(clamp(j, lo, hi+1)). */
int or_table(const float *params, int K, int64_t N, uint16_t *tab)
{
    if (K < 1 || K > OR_MAXK || N < 0) return OR_INVALID;
    for (int64_t n = 0; n < N; ++n) {
        or_mix m;
        load_mix(params, K, N, n, &m);
        if (!mix_ok(&m)) return OR_BAD_PARAMS;
        int lo, hi;
        window_of(&m, &lo, &hi);
        for (int j = -OR_YMAX; j <= OR_YMAX + 1; ++j) {
            int jj = j < lo ? lo : (j > hi + 1 ? hi + 1 : j);
            tab[n * 512 + (j + OR_YMAX)] = (uint16_t)Qof(&m, lo, hi, jj);
        }
    }
    return OR_OK;
}

/* ---------------------------------------------------------------------
 * rANS (Sec. II-B, Eq. 3): C(s, x) = M floor(x / l_s) + b_s + (x mod l_s),
 * M = 2^16, state x in [2^16, 2^32), 16-bit renormalisation words, initial
 * state 2^16. Before coding (start, freq): if x >= freq * 2^16, emit the low
 * 16 bits and shift (at most once).
 * ------------------------------------------------------------------- */
static void rans_put(uint32_t *x, uint32_t start, uint32_t freq, uint16_t *buf, int64_t *len)
{
    if (*x >= (freq << 16)) {
        buf[(*len)++] = (uint16_t)(*x & 0xFFFFu);
        *x >>= 16;
    }
    *x = ((*x / freq) << 16) + (*x % freq) + start;
}

/* Interleaving (the format of this coder; the paper codes one stream):
 * S streams (S a positive multiple of 32), symbol n -> stream n mod S at
 * step n div S; streams are grouped 32 to a segment (segment g holds streams
 * 32g .. 32g+31, lane = stream mod 32). Per segment the encoder runs the
 * steps t = T-1 .. 0 (T = ceil(N/S)); each step has three sub-phases:
 * low 16-bit chunk of escaped values (freq 1), high chunk (freq 1), then the
 * main symbol of every active lane. Within a sub-phase the renormalisation
 * words are appended in ascending lane order. Afterwards each lane appends
 * its final state as (x & 0xFFFF, x >> 16), lanes 0..31. Segments are
 * concatenated in order; offsets[g] is the exclusive prefix sum of segment
 * lengths, offsets[nseg] the total.
 *
 * encode_segment codes segment g into buf (room for 3 * 32 * T + 64 words)
 * and returns its length in words; or_encode returns the total number of
 * words, or a negative status. */
static int64_t encode_segment(const float *params, int K, int64_t N, const int32_t *sym, int32_t S, int64_t T,
                              int64_t g, uint16_t *buf)
{
    int64_t len = 0;
    uint32_t x[32];
    for (int l = 0; l < 32; ++l) x[l] = OR_L;
    for (int64_t t = T - 1; t >= 0; --t) {
        uint32_t st[32], fr[32];
        int esc[32], act[32];
        for (int l = 0; l < 32; ++l) {
            int64_t n = t * S + g * 32 + l;
            act[l] = n < N;
            esc[l] = 0;
            if (act[l]) {
                or_mix m;
                load_mix(params, K, N, n, &m);
                esc[l] = interval_of(&m, sym[n], &st[l], &fr[l]);
            }
        }
        for (int l = 0; l < 32; ++l)       /* low chunk of escapes */
            if (act[l] && esc[l])
                rans_put(&x[l], (uint32_t)sym[t * S + g * 32 + l] & 0xFFFFu, 1u, buf, &len);
        for (int l = 0; l < 32; ++l)       /* high chunk of escapes */
            if (act[l] && esc[l])
                rans_put(&x[l], (uint32_t)sym[t * S + g * 32 + l] >> 16, 1u, buf, &len);
        for (int l = 0; l < 32; ++l)       /* main symbol */
            if (act[l]) rans_put(&x[l], st[l], fr[l], buf, &len);
    }
    for (int l = 0; l < 32; ++l) {
        buf[len++] = (uint16_t)(x[l] & 0xFFFFu);
        buf[len++] = (uint16_t)(x[l] >> 16);
    }
    return len;
}

static int params_ok(const float *params, int K, int64_t N)
{
    for (int64_t n = 0; n < N; ++n) {
        or_mix m;
        load_mix(params, K, N, n, &m);
        if (!mix_ok(&m)) return 0;
    }
    return 1;
}

int64_t or_encode(const float *params, int K, int64_t N, const int32_t *sym, int32_t S,
                  uint16_t *words, int64_t cap, int64_t *offsets)
{
    if (K < 1 || K > OR_MAXK || N < 0 || S <= 0 || S % 32 != 0) return -OR_INVALID;
    if (!params_ok(params, K, N)) return -OR_BAD_PARAMS;
    int64_t nseg = S / 32;
    int64_t T = (N + S - 1) / S;
    uint16_t *buf = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(3 * 32 * T + 64));
    if (!buf) return -OR_INVALID;
    int64_t total = 0;
    for (int64_t g = 0; g < nseg; ++g) {
        int64_t len = encode_segment(params, K, N, sym, S, T, g, buf);
        offsets[g] = total;
        if (total + len > cap) { free(buf); return -OR_CAPACITY; }
        memcpy(words + total, buf, sizeof(uint16_t) * (size_t)len);
        total += len;
    }
    offsets[nseg] = total;
    free(buf);
    return total;
}

/* Binary search over the on-the-fly quantised CDF (Sec. III-A): the symbol
 * s in [lo, hi] with Q(s) <= slot < Q(s+1), or the escape slot when
 * slot >= Q(hi+1). Returns 1 for escape. */
static int search_slot(const or_mix *m, uint32_t slot, int32_t *s, uint32_t *start, uint32_t *freq)
{
    int lo, hi;
    window_of(m, &lo, &hi);
    uint32_t qe = Qof(m, lo, hi, hi + 1);
    if (slot >= qe) {
        *start = qe;
        *freq = OR_M - qe;
        return 1;
    }
    int a = lo, b = hi + 1;
    uint32_t qa = 0, qb = qe;
    while (b - a > 1) {
        int mid = a + ((b - a) >> 1);
        uint32_t qm = Qof(m, lo, hi, mid);
        if (qm <= slot) { a = mid; qa = qm; }
        else { b = mid; qb = qm; }
    }
    *s = a;
    *start = qa;
    *freq = qb - qa;
    return 0;
}

/* Decoder: the exact inverse of or_encode. Within a sub-phase the lanes
 * that fall below 2^16 refill from the end of the unread words; the lane of
 * rank r among c such lanes takes word [ptr - c + r]. At the end every
 * state must be 2^16 and the read pointer at the segment start, else
 * OR_CORRUPT. */
static int decode_segment(const float *params, int K, int64_t N, const uint16_t *words, const int64_t *offsets,
                          int32_t S, int64_t T, int64_t g, int32_t *out)
{
    int64_t beg = offsets[g], end = offsets[g + 1];
    if (end - beg < 64) return OR_CORRUPT;
    uint32_t x[32];
    for (int l = 0; l < 32; ++l)
        x[l] = (uint32_t)words[end - 64 + 2 * l] | ((uint32_t)words[end - 64 + 2 * l + 1] << 16);
    int64_t ptr = end - 64;
    int bad = 0;
    for (int64_t t = 0; t < T && !bad; ++t) {
        int act[32], esc[32];
        uint32_t hi16[32];
        /* main symbol */
        for (int l = 0; l < 32; ++l) {
            int64_t n = t * S + g * 32 + l;
            act[l] = n < N;
            esc[l] = 0;
            if (!act[l]) continue;
            or_mix m;
            load_mix(params, K, N, n, &m);
            uint32_t slot = x[l] & 0xFFFFu, st, fr;
            int32_t s = 0;
            esc[l] = search_slot(&m, slot, &s, &st, &fr);
            x[l] = fr * (x[l] >> 16) + slot - st;
            out[n] = s;
        }
        for (int l = 31; l >= 0; --l)
            if (act[l] && x[l] < OR_L) {
                if (ptr <= beg) { bad = 1; break; }
                x[l] = (x[l] << 16) | words[--ptr];
            }
        if (bad) break;
        /* high chunk of escapes */
        for (int l = 0; l < 32; ++l)
            if (act[l] && esc[l]) { hi16[l] = x[l] & 0xFFFFu; x[l] >>= 16; }
        for (int l = 31; l >= 0; --l)
            if (act[l] && esc[l] && x[l] < OR_L) {
                if (ptr <= beg) { bad = 1; break; }
                x[l] = (x[l] << 16) | words[--ptr];
            }
        if (bad) break;
        /* low chunk of escapes */
        for (int l = 0; l < 32; ++l)
            if (act[l] && esc[l]) {
                uint32_t lo16 = x[l] & 0xFFFFu;
                x[l] >>= 16;
                out[t * S + g * 32 + l] = (int32_t)((hi16[l] << 16) | lo16);
            }
        for (int l = 31; l >= 0; --l)
            if (act[l] && esc[l] && x[l] < OR_L) {
                if (ptr <= beg) { bad = 1; break; }
                x[l] = (x[l] << 16) | words[--ptr];
            }
    }
    if (bad || ptr != beg) return OR_CORRUPT;
    for (int l = 0; l < 32; ++l)
        if (x[l] != OR_L) return OR_CORRUPT;
    return OR_OK;
}

int or_decode(const float *params, int K, int64_t N, const uint16_t *words, const int64_t *offsets,
              int32_t S, int32_t *out)
{
    if (K < 1 || K > OR_MAXK || N < 0 || S <= 0 || S % 32 != 0) return OR_INVALID;
    if (!params_ok(params, K, N)) return OR_BAD_PARAMS;
    int64_t nseg = S / 32;
    int64_t T = (N + S - 1) / S;
    int status = OR_OK;
    for (int64_t g = 0; g < nseg; ++g)
        if (decode_segment(params, K, N, words, offsets, S, T, g, out) != OR_OK) status = OR_CORRUPT;
    return status;
}

/* ---------------------------------------------------------------------
 * The same coding with the segments spread over nthreads POSIX threads
 * (segments are independent by construction of the interleaving); used to
 * time the oracle on all host cores. The per-segment arithmetic is the
 * single-thread code above, so the output is identical.
 * ------------------------------------------------------------------- */
typedef struct {
    const float *params;
    int K;
    int64_t N;
    const int32_t *sym;
    const uint16_t *words;
    const int64_t *offsets;
    int32_t S;
    int64_t T, nseg;
    uint16_t *bufs;      /* encode: nseg buffers of seg_cap words */
    int64_t seg_cap;
    int64_t *lens;       /* encode: segment lengths */
    int32_t *out;        /* decode: symbols */
    int *status;         /* decode: per-segment status */
    int64_t next;        /* next segment to take (shared counter) */
    pthread_mutex_t mu;
} mt_job;

static int64_t mt_take(mt_job *j)
{
    pthread_mutex_lock(&j->mu);
    int64_t g = j->next++;
    pthread_mutex_unlock(&j->mu);
    return g;
}

static void *mt_encode_worker(void *arg)
{
    mt_job *j = (mt_job *)arg;
    for (int64_t g = mt_take(j); g < j->nseg; g = mt_take(j))
        j->lens[g] = encode_segment(j->params, j->K, j->N, j->sym, j->S, j->T, g, j->bufs + g * j->seg_cap);
    return NULL;
}

static void *mt_decode_worker(void *arg)
{
    mt_job *j = (mt_job *)arg;
    for (int64_t g = mt_take(j); g < j->nseg; g = mt_take(j))
        j->status[g] = decode_segment(j->params, j->K, j->N, j->words, j->offsets, j->S, j->T, g, j->out);
    return NULL;
}

static void mt_run(mt_job *j, int nthreads, void *(*fn)(void *))
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[started], NULL, fn, j) == 0) ++started;
    fn(j);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
}

int64_t or_encode_mt(const float *params, int K, int64_t N, const int32_t *sym, int32_t S, uint16_t *words,
                     int64_t cap, int64_t *offsets, int nthreads)
{
    if (K < 1 || K > OR_MAXK || N < 0 || S <= 0 || S % 32 != 0) return -OR_INVALID;
    if (!params_ok(params, K, N)) return -OR_BAD_PARAMS;
    mt_job j;
    memset(&j, 0, sizeof j);
    j.params = params; j.K = K; j.N = N; j.sym = sym; j.S = S;
    j.nseg = S / 32;
    j.T = (N + S - 1) / S;
    j.seg_cap = 3 * 32 * j.T + 64;
    j.bufs = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(j.seg_cap * j.nseg));
    j.lens = (int64_t *)malloc(sizeof(int64_t) * (size_t)j.nseg);
    if (!j.bufs || !j.lens) { free(j.bufs); free(j.lens); return -OR_INVALID; }
    pthread_mutex_init(&j.mu, NULL);
    mt_run(&j, nthreads, mt_encode_worker);
    pthread_mutex_destroy(&j.mu);
    int64_t total = 0;
    for (int64_t g = 0; g < j.nseg; ++g) {
        offsets[g] = total;
        if (total + j.lens[g] > cap) { free(j.bufs); free(j.lens); return -OR_CAPACITY; }
        memcpy(words + total, j.bufs + g * j.seg_cap, sizeof(uint16_t) * (size_t)j.lens[g]);
        total += j.lens[g];
    }
    offsets[j.nseg] = total;
    free(j.bufs);
    free(j.lens);
    return total;
}

int or_decode_mt(const float *params, int K, int64_t N, const uint16_t *words, const int64_t *offsets, int32_t S,
                 int32_t *out, int nthreads)
{
    if (K < 1 || K > OR_MAXK || N < 0 || S <= 0 || S % 32 != 0) return OR_INVALID;
    if (!params_ok(params, K, N)) return OR_BAD_PARAMS;
    mt_job j;
    memset(&j, 0, sizeof j);
    j.params = params; j.K = K; j.N = N; j.words = words; j.offsets = offsets; j.S = S;
    j.nseg = S / 32;
    j.T = (N + S - 1) / S;
    j.out = out;
    j.status = (int *)malloc(sizeof(int) * (size_t)(j.nseg > 0 ? j.nseg : 1));
    if (!j.status) return OR_INVALID;
    pthread_mutex_init(&j.mu, NULL);
    mt_run(&j, nthreads, mt_decode_worker);
    pthread_mutex_destroy(&j.mu);
    int status = OR_OK;
    for (int64_t g = 0; g < j.nseg; ++g)
        if (j.status[g] != OR_OK) status = OR_CORRUPT;
    free(j.status);
    return status;
}

/* ---------------------------------------------------------------------
 * FP64 rate audit (the "no approximation" reference of Sec. V, with
 * std::erfc): p64(s) = sum_k w_k [Phi(z_k(s+1/2)) - Phi(z_k(s-1/2))], the
 * per-symbol mass of Eq. 5, with the difference taken on the tail side of
 * each component so that it does not cancel. The coded cost of a symbol is
 * -log2(freq / 2^16), plus 32 bits of raw payload for an escape.
 * out[0] = sum -log2 p64 (ideal bits), out[1] = coded bits,
 * out[2] = max |F-hat(b) - F64(b)| over the boundaries the encoder
 * evaluates, out[3] = number of escapes.
 * ------------------------------------------------------------------- */
static double ncdf64(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

static double nmass64(double a, double b)   /* Phi(b) - Phi(a), a <= b */
{
    const double r2 = sqrt(2.0);
    if (a >= 0.0) return 0.5 * (erfc(a / r2) - erfc(b / r2));
    if (b <= 0.0) return 0.5 * (erfc(-b / r2) - erfc(-a / r2));
    return 1.0 - 0.5 * erfc(b / r2) - 0.5 * erfc(-a / r2);
}

double or_p64(const float *params, int K, int64_t N, int64_t n, int32_t s)
{
    or_mix m;
    load_mix(params, K, N, n, &m);
    double p = 0.0;
    for (int k = 0; k < K; ++k) {
        double sp = (double)sig_floor(m.sig[k]);
        double a = ((double)s - 0.5 - (double)m.mu[k]) / sp;
        double b = ((double)s + 0.5 - (double)m.mu[k]) / sp;
        p += (double)m.w[k] * nmass64(a, b);
    }
    return p;
}

static double F64(const or_mix *m, double b)
{
    double acc = 0.0;
    for (int k = 0; k < m->K; ++k)
        acc += (double)m->w[k] * ncdf64((b - (double)m->mu[k]) / (double)sig_floor(m->sig[k]));
    return acc;
}

int or_rate_audit(const float *params, int K, int64_t N, const int32_t *sym, double *out)
{
    if (K < 1 || K > OR_MAXK || N < 0) return OR_INVALID;
    double ideal = 0.0, coded = 0.0, maxerr = 0.0, nesc = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        or_mix m;
        load_mix(params, K, N, n, &m);
        if (!mix_ok(&m)) return OR_BAD_PARAMS;
        uint32_t st, fr;
        int esc = interval_of(&m, sym[n], &st, &fr);
        double p = or_p64(params, K, N, n, sym[n]);
        if (p < 2.2250738585072014e-308) p = 2.2250738585072014e-308;
        ideal += -log2(p);
        coded += 16.0 - log2((double)fr) + (esc ? 32.0 : 0.0);
        nesc += esc;
        int lo, hi;
        window_of(&m, &lo, &hi);
        /* boundaries evaluated by the encoder: s-1/2 (if s > lo) and s+1/2,
         * or hi+1/2 for an escape */
        float bs[2];
        int nb = 0;
        if (esc) bs[nb++] = (float)hi + 0.5f;
        else {
            if (sym[n] > lo) bs[nb++] = (float)sym[n] - 0.5f;
            bs[nb++] = (float)sym[n] + 0.5f;
        }
        for (int i = 0; i < nb; ++i) {
            double e = fabs((double)or_mixcdf_one(&m, bs[i]) - F64(&m, (double)bs[i]));
            if (e > maxerr) maxerr = e;
        }
    }
    out[0] = ideal;
    out[1] = coded;
    out[2] = maxerr;
    out[3] = nesc;
    return OR_OK;
}

/* ---------------------------------------------------------------------
 * Gaussian single model with pre-built tables (the scheme of Sec. II-C
 * that the paper attributes to CompressAI, its GSM anchor). The quantiser
 * shifts the latent by its mean, so the coder receives the integer
 * residual q and only the scale sigma: q is coded with N(0, sigma). The
 * scale is quantised to one of a fixed set of levels (by default 64 spaced
 * evenly in log between 0.11 and 256), so only one CDF table per level
 * exists and all can be built ahead of time.
 * Readings: the level of sigma is the smallest level >= sigma among the
 * first L - 1, else the last; default level i = float(exp(ln 0.11 +
 * i (ln 256 - ln 0.11) / 63)) in FP64; each level's table is this coder's
 * quantised CDF of N(0, level) (the same window, escape and 0.11 scale
 * floor). The GSM coder is then exactly this file's K = 1 coder on w = 1,
 * mu = 0, sigma = level: or_gsm_params produces those parameters.
 * ------------------------------------------------------------------- */
void or_gsm_levels(float *lv)
{
    const double a = log(0.11), b = log(256.0);
    for (int i = 0; i < 64; ++i) lv[i] = (float)exp(a + (b - a) * (double)i / 63.0);
}

/* Scales sigma[N] and levels lv[L] -> K = 1 parameters [3][1][N] =
 * (1, 0, level) and level indices (level_idx may be NULL). Returns
 * OR_BAD_PARAMS for a scale that is not finite and > 0. */
int or_gsm_params(const float *lv, int L, const float *sigma, int64_t N, float *params_out, int32_t *level_idx)
{
    for (int64_t n = 0; n < N; ++n) {
        const float sg = sigma[n];
        if (!isfinite(sg) || !(sg > 0.0f)) return OR_BAD_PARAMS;
        int i = L - 1;
        for (int j = 0; j < L - 1; ++j)
            if (sg <= lv[j]) { i = j; break; }
        params_out[0 * N + n] = 1.0f;
        params_out[1 * N + n] = 0.0f;
        params_out[2 * N + n] = lv[i];
        if (level_idx) level_idx[n] = i;
    }
    return OR_OK;
}

/* ---------------------------------------------------------------------
 * Checkerboard two-pass coding (the context model of the paper's codecs,
 * Sec. IV-A): in every channel of a C x H x W latent the positions with
 * h + w even are anchors, coded first with the hyperprior's parameters;
 * the others are coded second, with parameters that a context model
 * computes from the decoded anchors around them. Anchors and non-anchors
 * are each listed channel by channel in raster order.
 *
 * The trained context network is not available; a fixed stand-in takes its
 * place, defined here and nowhere in the paper: for a non-anchor with
 * in-bounds 4-neighbours (all anchors) of symbol sum ctx (64-bit integer)
 * and count cnt, each component keeps its weight, moves its mean toward the
 * neighbours, m_k = fmaf(-cnt, mu_k, (float)ctx), mu'_k = fmaf(0.125, m_k,
 * mu_k), and narrows its scale, sigma'_k = 0.75 sigma_k (each one FP32
 * rounding, in this order).
 * ------------------------------------------------------------------- */
static int64_t ckbd_count(int64_t C, int64_t H, int64_t W, int anchor)
{
    int64_t n = 0;
    for (int64_t h = 0; h < H; ++h)
        for (int64_t w = 0; w < W; ++w)
            if ((((h + w) & 1) == 0) == (anchor != 0)) ++n;
    return C * n;
}

/* params [3][K][N] and y[N] -> anchor and non-anchor parameters and
 * symbols; any output may be NULL. */
void or_ckbd_split(int K, int64_t C, int64_t H, int64_t W, const float *params, const int32_t *y, float *params_a,
                   int32_t *y_a, float *params_n, int32_t *y_n)
{
    const int64_t N = C * H * W, Na = ckbd_count(C, H, W, 1), Nn = N - Na;
    int64_t ia = 0, in = 0;
    for (int64_t c = 0; c < C; ++c)
        for (int64_t h = 0; h < H; ++h)
            for (int64_t w = 0; w < W; ++w) {
                const int64_t n = (c * H + h) * W + w;
                const int anchor = ((h + w) & 1) == 0;
                float *po = anchor ? params_a : params_n;
                int32_t *yo = anchor ? y_a : y_n;
                const int64_t i = anchor ? ia++ : in++, M = anchor ? Na : Nn;
                if (po)
                    for (int r = 0; r < 3 * K; ++r) po[r * M + i] = params[r * N + n];
                if (yo && y) yo[i] = y[n];
            }
}

/* Anchor and non-anchor symbols -> y[N] (y_n may be NULL: anchors only). */
void or_ckbd_merge(int64_t C, int64_t H, int64_t W, const int32_t *y_a, const int32_t *y_n, int32_t *y)
{
    int64_t ia = 0, in = 0;
    for (int64_t c = 0; c < C; ++c)
        for (int64_t h = 0; h < H; ++h)
            for (int64_t w = 0; w < W; ++w) {
                const int64_t n = (c * H + h) * W + w;
                if (((h + w) & 1) == 0) y[n] = y_a[ia++];
                else if (y_n) y[n] = y_n[in++];
                else ++in;
            }
}

/* Stand-in context: hyperprior params [3][K][N] and y[N] (anchors read) ->
 * non-anchor parameters [3][K][Nn]. */
void or_ckbd_context(int K, int64_t C, int64_t H, int64_t W, const float *params, const int32_t *y, float *params_n)
{
    const int64_t N = C * H * W, Nn = N - ckbd_count(C, H, W, 1);
    int64_t in = 0;
    for (int64_t c = 0; c < C; ++c)
        for (int64_t h = 0; h < H; ++h)
            for (int64_t w = 0; w < W; ++w) {
                if (((h + w) & 1) == 0) continue;
                const int64_t n = (c * H + h) * W + w;
                int64_t ctx = 0;
                int cnt = 0;
                if (h > 0) { ctx += y[n - W]; ++cnt; }
                if (h + 1 < H) { ctx += y[n + W]; ++cnt; }
                if (w > 0) { ctx += y[n - 1]; ++cnt; }
                if (w + 1 < W) { ctx += y[n + 1]; ++cnt; }
                for (int k = 0; k < K; ++k) {
                    const float wk = params[(0 * K + k) * N + n];
                    const float mu = params[(1 * K + k) * N + n];
                    const float sg = params[(2 * K + k) * N + n];
                    const float m = fmaf(-(float)cnt, mu, (float)ctx);
                    params_n[(0 * K + k) * Nn + in] = wk;
                    params_n[(1 * K + k) * Nn + in] = fmaf(0.125f, m, mu);
                    params_n[(2 * K + k) * Nn + in] = sg * 0.75f;
                }
                ++in;
            }
}
