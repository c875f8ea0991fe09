// fgmm_segment.cuh -- one 32-stream segment coded by one warp (lane = stream).
//
// Shared by the single-latent kernels and the persistent batch kernels:
//   enc_segment_fused: the table-free encoder of Sec. III-A for one segment,
//     with the quantised-CDF interval evaluated inline at the coded symbol
//     and fed straight to rANS (Eq. 3); parameters of the next step are
//     loaded one step ahead.
//   dec_segment: binary search over the on-the-fly quantised CDF (steered
//     by the fast evaluation and confirmed exactly for A&S), inverse rANS
//     step, ballot-ranked refill; end-of-segment integrity check.
#pragma once

#include "fgmm_device.cuh"

namespace fgmm {

template <int K>
struct RawParams {
    float v[3 * K];
};

template <int K, typename T>
__device__ __forceinline__ void load_raw_params(const T* __restrict__ params, int64_t N, int64_t n, RawParams<K>& r)
{
#pragma unroll
    for (int i = 0; i < 3 * K; ++i) r.v[i] = load_param(params, (int64_t)i * N + n);
}

// Prepares a Mix from raw (w, mu, sigma) values; the same arithmetic as
// load_mix. Returns false for invalid parameters (mixture neutralised).
template <int K>
__device__ __forceinline__ bool mix_from_params(const RawParams<K>& r, Mix<K>& m)
{
    float lo_f = __int_as_float(0x7f800000), hi_f = __int_as_float(0xff800000);
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float w = r.v[k], mu = r.v[K + k], s = r.v[2 * K + k];
        ok = ok && isfinite(w) && w >= 0.0f && isfinite(mu) && isfinite(s) && s > 0.0f;
        const float sp = fmaxf(s, kSigmaMin);
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

// Exact x / f and x mod f for x < f * 2^16 (the state after
// renormalisation), f in [1, 2^16). The FP32 estimate x * (1/f), with the
// hardware reciprocal (at most 1 ulp off), has relative error below 2^-21,
// so with the quotient below 2^16 it is off by less than 1/32 and its
// truncation by at most one; one correction step each way makes it exact
// (fgmm_self_check tests it at the remainders 0, 1 and f - 1).
__device__ __forceinline__ uint32_t divmod_small(uint32_t x, uint32_t f, uint32_t& r)
{
    const float rf = rcp_approx((float)f);
    uint32_t q = __float2uint_rz(__fmul_rn(__uint2float_rn(x), rf));
    int32_t rem = (int32_t)(x - q * f);
    if (rem < 0) { --q; rem += (int32_t)f; }
    else if (rem >= (int32_t)f) { ++q; rem -= (int32_t)f; }
    r = (uint32_t)rem;
    return q;
}

// rANS encode of (start, freq) on the lanes where `part` holds, with the
// sub-phase's renormalisation words appended in ascending lane order.
__device__ __forceinline__ void enc_put_warp(uint32_t& x, uint32_t start, uint32_t freq, bool part,
                                             uint16_t* __restrict__ out, int64_t& base, uint32_t lt)
{
    const bool need = part && x >= (freq << 16);
    const uint32_t m = __ballot_sync(0xffffffffu, need);
    if (need) {
        out[base + __popc(m & lt)] = (uint16_t)(x & 0xffffu);
        x >>= 16;
    }
    base += __popc(m);
    if (part) {
        uint32_t r;
        const uint32_t q = divmod_small(x, freq, r);
        x = (q << 16) + r + start;
    }
}

// Fused encode of segment g (streams 32g .. 32g+31) of a latent into
// out[0 .. *len_out). out must hold 3 * 32 * T + 64 words.
template <int K, typename T>
__device__ __forceinline__ void enc_segment_fused(const T* __restrict__ params, int64_t N, int32_t S, int64_t T_steps,
                                                  int64_t g, const int32_t* __restrict__ sym,
                                                  uint16_t* __restrict__ out, int64_t* len_out, int32_t* err)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    uint32_t x = kL;
    int64_t base = 0;
    bool badp = false;
    int64_t n = (T_steps - 1) * (int64_t)S + g * 32 + lane;
    RawParams<K> cur;
    int32_t scur = 0;
    if (T_steps > 0 && n < N) {
        load_raw_params<K, T>(params, N, n, cur);
        scur = __ldg(sym + n);
    }
    for (int64_t t = T_steps - 1; t >= 0; --t, n -= S) {
        const bool act = n < N;
        RawParams<K> nxt;
        int32_t snxt = 0;
        if (t > 0 && n - S < N) {   // next (lower) step: prefetch
            load_raw_params<K, T>(params, N, n - S, nxt);
            snxt = __ldg(sym + n - S);
        }
        uint32_t start = 0, freq = 0;
        if (act) {
            Mix<K> m;
            badp |= !mix_from_params<K>(cur, m);
            interval_of<K>(m, scur, start, freq);
        }
        const bool esc = act && (start + freq == kM);
        if (__ballot_sync(0xffffffffu, esc)) {
            const uint32_t raw = esc ? (uint32_t)scur : 0u;
            enc_put_warp(x, raw & 0xffffu, 1u, esc, out, base, lt);
            enc_put_warp(x, raw >> 16, 1u, esc, out, base, lt);
        }
        enc_put_warp(x, start, freq, act, out, base, lt);
        cur = nxt;
        scur = snxt;
    }
    out[base + 2 * lane] = (uint16_t)(x & 0xffffu);
    out[base + 2 * lane + 1] = (uint16_t)(x >> 16);
    if (lane == 0) *len_out = base + 64;
    if (__ballot_sync(0xffffffffu, badp) && lane == 0) set_error(err, kErrBadParams);
}

// Decode of segment g whose words are words[beg, end). Symbols go to out[n].
template <int K, typename T, int PHI = kPhiAS>
__device__ __forceinline__ void dec_segment(const T* __restrict__ params, int64_t N, int32_t S, int64_t T_steps,
                                            int64_t g, const uint16_t* __restrict__ words, int64_t beg, int64_t end,
                                            int32_t* __restrict__ out, int32_t* err, unsigned long long* stats)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    uint32_t x = (uint32_t)__ldg(words + end - 64 + 2 * lane) | ((uint32_t)__ldg(words + end - 63 + 2 * lane) << 16);
    int64_t ptr = end - 64;
    bool bad = false, badp = false;
    int probes = 0, decoded = 0, fallbacks = 0;
    int64_t n = g * 32 + lane;
    RawParams<K> cur;
    if (T_steps > 0 && n < N) load_raw_params<K, T>(params, N, n, cur);
    for (int64_t t = 0; t < T_steps; ++t, n += S) {
        const bool act = n < N;
        RawParams<K> nxt;
        if (t + 1 < T_steps && n + S < N) load_raw_params<K, T>(params, N, n + S, nxt);
        // the refill words of the next steps lie just below ptr (a segment
        // consumes a few words per step): pull their line into L1 ahead
        if (lane == 0 && ptr - 96 >= beg) asm volatile("prefetch.global.L1 [%0];" ::"l"(words + ptr - 96));
        int32_t s = 0;
        bool esc = false;
        if (act) {
            ++decoded;
            Mix<K> m;
            badp |= !mix_from_params<K>(cur, m);
            const uint32_t slot = x & 0xffffu;
            uint32_t st, fr;
            if constexpr (PHI == kPhiAS) esc = search_slot_guided<K>(m, slot, s, st, fr, probes, fallbacks);
            else esc = search_slot<K, PHI>(m, slot, s, st, fr, probes);
            x = fr * (x >> 16) + slot - st;
        }
        refill_warp(x, act, words, ptr, beg, bad, lt);
        if (__ballot_sync(0xffffffffu, esc)) {
            uint32_t hi16 = 0, lo16 = 0;
            if (esc) { hi16 = x & 0xffffu; x >>= 16; }
            refill_warp(x, esc, words, ptr, beg, bad, lt);
            if (esc) { lo16 = x & 0xffffu; x >>= 16; }
            refill_warp(x, esc, words, ptr, beg, bad, lt);
            if (esc) s = (int32_t)((hi16 << 16) | lo16);
        }
        if (act) out[n] = s;
        cur = nxt;
    }
    const bool fail = bad || x != kL || ptr != beg;
    if (__ballot_sync(0xffffffffu, fail) && lane == 0) set_error(err, kErrCorrupt);
    if (__ballot_sync(0xffffffffu, badp) && lane == 0) set_error(err, kErrBadParams);
    if (stats) {
        int p = probes, d = decoded, f = fallbacks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
            f += __shfl_xor_sync(0xffffffffu, f, o);
        }
        if (lane == 0) {
            atomicAdd(stats, (unsigned long long)p);
            atomicAdd(stats + 1, (unsigned long long)d);
            if (f) atomicAdd(stats + 3, (unsigned long long)f);
        }
    }
}

}  // namespace fgmm
