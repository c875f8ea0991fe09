// fgmm_device.cuh -- device-side arithmetic of the table-free GMM coder.
//
// Everything here is the per-symbol quantised mixture CDF that the encoder
// evaluates at the coded symbol and the decoder searches (Sec. III-A), with
// the Gaussian CDF replaced by the Abramowitz & Stegun 26.2.17 approximation
// (Sec. III-B, Eq. 8). Every floating-point step is written with an explicit
// round-to-nearest intrinsic (__fmul_rn, __fsub_rn, __fmaf_rn, __frcp_rn) so
// that no contraction or reassociation can change a bit: the coded stream is
// a function of these exact IEEE operations, and any decoder that performs
// the same operations reproduces it.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace fgmm {

constexpr int kMaxK = 4;
constexpr uint32_t kProbBits = 16;
constexpr uint32_t kM = 1u << kProbBits;   // total frequency
constexpr uint32_t kL = 1u << 16;          // rANS lower bound / initial state
constexpr int kYmax = 255;                 // window clamp (alphabet [-255, 255])
constexpr float kR = 8.0f;                 // window half-width in scales
constexpr float kSigmaMin = 0.11f;         // scale floor

// Device error codes (the same numbers as fgmm_status).
constexpr int32_t kErrBadParams = 2;
constexpr int32_t kErrCapacity = 3;
constexpr int32_t kErrCorrupt = 4;
constexpr int32_t kErrTimeout = 5;

__device__ __forceinline__ void set_error(int32_t* err, int32_t code)
{
    if (*reinterpret_cast<volatile int32_t*>(err) == 0) atomicCAS(err, 0, code);
}

// exp(a), a in [-72, 0]: Cody-Waite reduction a = k ln2 + r (ln2 split into
// a high part whose product with any |k| <= 127 is short, and the rounding
// remainder), degree-7 Taylor polynomial of exp(r) with coefficients 1/i!,
// and the factor 2^k added into the exponent field.
__device__ __forceinline__ float exp_cw(float a)
{
    const float kLog2e = 0x1.715476p+0f;
    const float kLn2Hi = 0x1.62e4p-1f;
    const float kLn2Lo = 0x1.7f7d1cp-20f;
    // k = rint(a log2 e) by adding and removing 1.5 * 2^23 (round to nearest
    // even, exact for |a log2 e| < 2^22); the sum's low mantissa bits hold k
    // in two's complement, so (bits << 23) is k * 2^23 modulo 2^32.
    const float kMagic = 0x1.8p23f;
    const float tm = __fadd_rn(__fmul_rn(a, kLog2e), kMagic);
    const float k = __fsub_rn(tm, kMagic);
    float r = __fmaf_rn(-k, kLn2Hi, a);
    r = __fmaf_rn(-k, kLn2Lo, r);
    float p = 0x1.a01a02p-13f;           // fp32(1/7!)
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);  // fp32(1/6!)
    p = __fmaf_rn(p, r, 0x1.111112p-7f);   // fp32(1/5!)
    p = __fmaf_rn(p, r, 0x1.555556p-5f);   // fp32(1/4!)
    p = __fmaf_rn(p, r, 0x1.555556p-3f);   // fp32(1/3!)
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    return __uint_as_float(__float_as_uint(p) + (__float_as_uint(tm) << 23));
}

// 1/d, correctly rounded, for normal d with a normal reciprocal
// (2^-125 <= d <= 2^125): the hardware reciprocal approximation refined by
// one Newton-Raphson step, y1 = y0 + y0 (1 - d y0), with the residual and the
// update each a single fused multiply-add. fgmm_self_check compares it with
// __frcp_rn on every float of that range. Being inline, it lets the K
// component evaluations of a CDF probe overlap.
__device__ __forceinline__ float recip(float d)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
    const float e = __fmaf_rn(-d, y, 1.0f);
    return __fmaf_rn(y, e, y);
}

// 1/s for a floored scale s >= 0.11 (any finite value above): the inline
// reciprocal below 2^125; above, where 1/s may be subnormal, the correctly
// rounded division, kept out of line so that the common path carries none
// of its code.
static __device__ __noinline__ float recip_scale_slow(float s) { return __frcp_rn(s); }
__device__ __forceinline__ float recip_scale(float s) { return s < 0x1p125f ? recip(s) : recip_scale_slow(s); }

// Phi-hat(z): A&S 26.2.17, Phi(x) ~ 1 - Z(x) sum_i b_i t^i, t = 1/(1+px),
// x = |z|, mirrored for z < 0. p = 0.2316419 and b_1..b_5 are the handbook's;
// the 1/sqrt(2 pi) of the density Z is pre-multiplied into the b_i
// (c_i = fp32(b_i / sqrt(2 pi))). z is clamped to [-12, 12] and rounded to the
// grid 2^-22 (half to even), where this FP32 evaluation is monotone.
//
// phi_hat_s takes zs = z * 2^22 and works on the grid index r = x * 2^22
// (an integer below 2^26) with constants scaled by powers of two, which
// changes no rounding: fma(p 2^-22, r, 1) = fma(p, x, 1) and
// (r r) (-2^-45) = (x x) (-1/2) exactly, since every scaled value stays a
// normal float.
__device__ __forceinline__ float phi_hat_s(float zs)
{
    const float kP22 = 0x1.da6712p-25f;   // fp32(p) * 2^-22
    const float kC1 = 0x1.04f20cp-3f;
    const float kC2 = -0x1.23531cp-3f;
    const float kC3 = 0x1.6be1c6p-1f;
    const float kC4 = -0x1.7401c6p-1f;
    const float kC5 = 0x1.0fb844p-1f;
    // r = |rint(clamp(z) 2^22)| (rint is odd); the mirror below tests z's
    // sign, which agrees with the rounded value's except when that is +-0,
    // where both branches give 1/2 (Phi-hat(0) = 1 - q(0) = q(0) = 1/2
    // exactly).
    const float r = rintf(fminf(fabsf(zs), 0x1.8p25f));   // 12 * 2^22
    float d = __fmaf_rn(kP22, r, 1.0f);   // 1 + p x, in [1, 3.78]
    float t = recip(d);
    float h = __fmaf_rn(kC5, t, kC4);
    h = __fmaf_rn(h, t, kC3);
    h = __fmaf_rn(h, t, kC2);
    h = __fmaf_rn(h, t, kC1);
    float g = __fmul_rn(h, t);
    float a = __fmul_rn(__fmul_rn(r, r), -0x1p-45f);   // -x^2 / 2
    float q = __fmul_rn(exp_cw(a), g);
    return zs >= 0.0f ? __fsub_rn(1.0f, q) : q;
}

// The other two approximations of Sec. III-B (Sec. V, Table II), on the
// same clamp, grid and mirror; each gives the lower tail q = Phi-hat(-x):
//   logistic: Phi(x) ~ 1 / (1 + exp(-1.702 x)),   q = 1 / (1 + exp(1.702 x));
//   Polya:    Phi(x) ~ (1 + sqrt(1 - exp(-2 x^2 / pi))) / 2 (Polya's form,
//             with the factor 2/pi), q = (e/2) (1 / (1 + sqrt(1 - e))),
//             e = exp(max(-(2/pi) x^2, -72)).
// With x = r 2^-22 the constants are scaled by powers of two (1.702 2^-22,
// 2/pi 2^-44), which changes no rounding. Both are monotone on the grid.
enum { kPhiAS = 0, kPhiLogistic = 1, kPhiPolya = 2 };

template <int PHI>
__device__ __forceinline__ float phi_hat_v(float zs)
{
    if constexpr (PHI == kPhiAS) {
        return phi_hat_s(zs);
    } else {
        const float r = rintf(fminf(fabsf(zs), 0x1.8p25f));   // |z| 2^22 on the grid, clamp 12
        float q;
        if constexpr (PHI == kPhiLogistic) {
            const float E = exp_cw(__fmul_rn(0x1.b3b646p-22f, r));   // fp32(1.702) 2^-22
            q = recip(__fadd_rn(1.0f, E));
        } else {
            const float a = fmaxf(-__fmul_rn(0x1.45f306p-45f, __fmul_rn(r, r)), -72.0f);   // fp32(2/pi) 2^-44
            const float e = exp_cw(a);
            const float sq = __fsqrt_rn(__fsub_rn(1.0f, e));
            q = __fmul_rn(__fmul_rn(0.5f, e), recip(__fadd_rn(1.0f, sq)));
        }
        return zs >= 0.0f ? __fsub_rn(1.0f, q) : q;
    }
}

// Phi-hat(z) for any z: z * 2^22 is exact (or overflows to +-inf, which the
// clamp maps to 12 as it does z).
template <int PHI = kPhiAS>
__device__ __forceinline__ float phi_hat(float z) { return phi_hat_v<PHI>(__fmul_rn(z, 0x1p22f)); }

// Parameter loads from the planar [3][K][N] layout.
__device__ __forceinline__ float load_param(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_param(const __nv_bfloat16* p, int64_t i)
{
    const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

// One symbol's mixture, ready for CDF probes: weights, means, 2^22 times the
// reciprocal floored scales (1/sigma' scaled exactly, so that (b - mu) isg
// = z 2^22 with the same rounding as (b - mu) / sigma'), the window [lo, hi]
// and T' = 2^16 - W - 1.
template <int K>
struct Mix {
    float w[K], mu[K], isg[K];
    int lo, hi;
    float tp;
};

// Loads symbol n's parameters and prepares its window. Returns false (and
// neutralises the mixture: all weights 0) if a parameter is invalid
// (weight negative or non-finite, mean non-finite, scale non-finite or <= 0).
template <int K, typename T>
__device__ __forceinline__ bool load_mix(const T* params, int64_t N, int64_t n, Mix<K>& m)
{
    float a = __int_as_float(0xff800000);   // -inf
    float b = __int_as_float(0x7f800000);   // +inf
    float lo_f = b, hi_f = a;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float w = load_param(params, (int64_t)(0 * K + k) * N + n);
        float mu = load_param(params, (int64_t)(1 * K + k) * N + n);
        float s = load_param(params, (int64_t)(2 * K + k) * N + n);
        ok = ok && isfinite(w) && w >= 0.0f && isfinite(mu) && isfinite(s) && s > 0.0f;
        float sp = fmaxf(s, kSigmaMin);
        m.w[k] = w;
        m.mu[k] = mu;
        m.isg[k] = __fmul_rn(recip_scale(sp), 0x1p22f);
        lo_f = fminf(lo_f, __fmaf_rn(-kR, sp, mu));
        hi_f = fmaxf(hi_f, __fmaf_rn(kR, sp, mu));
    }
    if (!ok) {
#pragma unroll
        for (int k = 0; k < K; ++k) { m.w[k] = 0.0f; m.mu[k] = 0.0f; m.isg[k] = 0x1p22f; }
        lo_f = -1.0f;
        hi_f = 1.0f;
    }
    lo_f = fminf(fmaxf(floorf(lo_f), -(float)kYmax), (float)kYmax);
    hi_f = fminf(fmaxf(ceilf(hi_f), -(float)kYmax), (float)kYmax);
    // lo <= hi always: floor(a) <= ceil(b) for a <= b (a, b the extreme
    // window ends, both finite here), and clamping keeps the order, so the
    // coded definition's swap of lo and hi never applies
    m.lo = (int)lo_f;
    m.hi = (int)hi_f;
    m.tp = (float)(int)(kM - (uint32_t)(m.hi - m.lo + 1) - 1u);
    return ok;
}

// F-hat(j - 1/2) = sum_k w_k Phi-hat((b - mu_k) / sigma'_k), k ascending.
template <int K, int PHI = kPhiAS>
__device__ __forceinline__ float mix_cdf(const Mix<K>& m, int j)
{
    const float b = __fsub_rn((float)j, 0.5f);
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float zs = __fmul_rn(__fsub_rn(b, m.mu[k]), m.isg[k]);   // z 2^22
        acc = __fmaf_rn(m.w[k], phi_hat_v<PHI>(zs), acc);
    }
    return acc;
}

// Quantised CDF Q(j) for lo < j <= hi+1: (j - lo) + floor(T' min(F-hat, 1)).
// Q(lo) = 0 is not evaluated.
template <int K, int PHI = kPhiAS>
__device__ __forceinline__ uint32_t q_at(const Mix<K>& m, int j)
{
    const float v = fminf(mix_cdf<K, PHI>(m, j), 1.0f);
    return (uint32_t)(j - m.lo) + __float2uint_rd(__fmul_rn(m.tp, v));   // floor of a value >= 0
}

// The rANS interval of symbol s. Escape (s outside [lo, hi]) gets
// [Q(hi+1), 2^16); an interval is an escape iff start + freq == 2^16.
template <int K, int PHI = kPhiAS>
__device__ __forceinline__ void interval_of(const Mix<K>& m, int32_t s, uint32_t& start, uint32_t& freq)
{
    if (s >= m.lo && s <= m.hi) {
        const uint32_t a = (s == m.lo) ? 0u : q_at<K, PHI>(m, s);
        const uint32_t b = q_at<K, PHI>(m, s + 1);
        start = a;
        freq = b - a;
    } else {
        const uint32_t e = q_at<K, PHI>(m, m.hi + 1);
        start = e;
        freq = kM - e;
    }
}

// Decoder search: the symbol whose interval holds `slot`, by binary search
// over Q (Sec. III-A). The escape slot is searched as one more symbol: the
// range is [lo, hi + 2) with Q(hi + 2) = 2^16 standing in for the end of the
// escape interval (never evaluated), so landing on hi + 1 means escape and no
// separate escape test is needed. Returns true for the escape slot.
// `probes` counts CDF evaluations (ceil or floor of log2(W + 1)).
template <int K, int PHI = kPhiAS>
__device__ __forceinline__ bool search_slot(const Mix<K>& m, uint32_t slot, int32_t& s, uint32_t& start,
                                            uint32_t& freq, int& probes)
{
    int a = m.lo, b = m.hi + 2;
    uint32_t qa = 0, qb = kM;
    while (b - a > 1) {
        const int mid = a + ((b - a) >> 1);
        const uint32_t qm = q_at<K, PHI>(m, mid);
        ++probes;
        if (qm <= slot) { a = mid; qa = qm; }
        else { b = mid; qb = qm; }
    }
    s = a;
    start = qa;
    freq = qb - qa;
    return a == m.hi + 1;
}

// Fast steering evaluation of the mixture CDF at b for the decoder's
// search: the A&S form of phi_hat_s with the hardware reciprocal and base-2
// exponential, no clamp and no grid rounding (accurate to about 1e-6). It
// only decides where the search goes next; search_slot_guided confirms the
// symbol it reaches with the exact quantised CDF (q_at), so this function's
// rounding never reaches a decoded symbol or a frequency.
__device__ __forceinline__ float rcp_approx(float d)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d));
    return y;
}
__device__ __forceinline__ float ex2_approx(float a)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// One component of the fast evaluation at zs = z 2^22.
__device__ __forceinline__ float phi_fast_s(float zs)
{
    const float kP22 = 0x1.da6712p-25f;    // p 2^-22 (zs = z 2^22)
    const float kE = -0x1.715476p-45f;     // -log2(e) / 2 * 2^-44: exp(-z^2/2) = 2^(kE zs^2)
    const float t = rcp_approx(fmaf(kP22, fabsf(zs), 1.0f));
    float h = fmaf(0x1.0fb844p-1f, t, -0x1.7401c6p-1f);
    h = fmaf(h, t, 0x1.6be1c6p-1f);
    h = fmaf(h, t, -0x1.23531cp-3f);
    h = fmaf(h, t, 0x1.04f20cp-3f);
    const float q = ex2_approx((zs * kE) * zs) * (h * t);
    return zs >= 0.0f ? 1.0f - q : q;
}

// The fast evaluation's zs is the exact evaluation's (the same two
// roundings of the same operands), so the two differ only in phi_fast_s
// against phi_hat_s.
template <int K>
__device__ __forceinline__ float mix_cdf_fast(const Mix<K>& m, float b)
{
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float zs = (b - m.mu[k]) * m.isg[k];
        acc = fmaf(m.w[k], phi_fast_s(zs), acc);
    }
    return acc;
}

// Decoder search with a fast guide (Sec. III-A's binary search, steered by
// mix_cdf_fast): the binary search over [lo, hi + 2) runs on the fast
// evaluation, deciding Q(mid) <= slot as (mid - lo) + T' v < slot + 1;
// then the exact quantised CDF is evaluated at the symbol it reached and at
// its successor (Q(lo) = 0 and Q(hi + 2) = 2^16 need no evaluation) and
// must bracket the slot. If it does not (the fast evaluation decided a
// near-tie the other way), the exact binary search runs. The result is the
// exact search's in every case: the symbol whose exact interval holds the
// slot is unique. `probes` counts the search's probes (the evaluations the
// exact binary search makes on the same path), `fallbacks` the exact
// searches run after a failed check.
template <int K>
__device__ __forceinline__ bool search_slot_guided(const Mix<K>& m, uint32_t slot, int32_t& s, uint32_t& start,
                                                   uint32_t& freq, int& probes, int& fallbacks)
{
    int a = m.lo, b = m.hi + 2;
    const float thr = (float)(slot + 1u);
    while (b - a > 1) {
        const int mid = a + ((b - a) >> 1);
        const float v = fminf(mix_cdf_fast<K>(m, (float)mid - 0.5f), 1.0f);
        ++probes;
        if (fmaf(m.tp, v, (float)(mid - m.lo)) < thr) a = mid;
        else b = mid;
    }
    const uint32_t qa = a == m.lo ? 0u : q_at<K>(m, a);
    const uint32_t qb = a == m.hi + 1 ? kM : q_at<K>(m, a + 1);
    if (qa <= slot && slot < qb) {
        s = a;
        start = qa;
        freq = qb - qa;
        return a == m.hi + 1;
    }
    ++fallbacks;
    int extra = 0;
    return search_slot<K>(m, slot, s, start, freq, extra);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-level refill after a decode sub-phase (one lane per stream, 32
// streams per warp): the lanes (among `part`) whose state fell below 2^16
// take the last c unread words, the lane of rank r word ptr - c + r. A read
// below the segment start is never performed; it marks the stream bad.
__device__ __forceinline__ void refill_warp(uint32_t& x, bool part, const uint16_t* __restrict__ words,
                                            int64_t& ptr, int64_t beg, bool& bad, uint32_t lt)
{
    const bool need = part && x < kL;
    const uint32_t m = __ballot_sync(0xffffffffu, need);
    if (m) {
        const int c = __popc(m);
        if (need) {
            const int64_t idx = ptr - c + __popc(m & lt);
            uint32_t w = 0;
            if (idx >= beg) w = __ldg(words + idx);
            else bad = true;
            x = (x << 16) | w;
        }
        ptr -= c;
    }
}

}  // namespace fgmm
