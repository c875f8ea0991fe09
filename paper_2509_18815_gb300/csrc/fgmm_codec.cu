// fgmm_codec.cu -- table-free GMM rANS encode / decode for sm_103a.
//
// Encode (Sec. III-A: evaluate the CDF at the coded symbol, then rANS, Eq. 3)
// runs in four launches:
//   1. fgmm_interval_kernel: one thread per symbol computes the symbol's
//      quantised-CDF interval (start, freq). Fully data-parallel over N.
//   2. fgmm_rans_enc_kernel: one CTA per 32-stream segment, one lane per
//      stream, steps T-1 .. 0: a warp prepares each step's interval data in
//      shared memory, a second runs the integer state chain; the
//      renormalisation words of a sub-phase are compacted with a warp ballot
//      and popc rank and appended to the segment's scratch buffer.
//   3. fgmm_scan_kernel: exclusive prefix sum of the segment lengths.
//   4. fgmm_compact_kernel: copies segments to their offsets.
// Decode (Sec. III-A: binary search over the same on-the-fly CDF) is one
// launch of a kernel in fgmm_decode.cu.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"
#include "fgmm_segment.cuh"

using namespace fgmm;

namespace {

constexpr uint32_t kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Phi-hat evaluation (tests and sweeps).
// ---------------------------------------------------------------------------
template <int PHI>
__global__ void phi_kernel(const float* __restrict__ z, float* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = phi_hat<PHI>(z[i]);
}

// Exhaustive check of recip() against __frcp_rn over [2^-125, 2^125]
// (every float), and a check of the encoder's exact division for every
// divisor f in [1, 2^16) at x = q f + r, r in {0, 1, f - 1}, for the 64
// smallest and 64 largest quotients and every 67th one in between.
__global__ void self_check_recip_kernel(unsigned long long* bad)
{
    unsigned long long nb = 0;
    const uint32_t lo = 0x01000000u, hi = 0x7e000000u;   // 2^-125 .. 2^125
    for (uint32_t u = lo + blockIdx.x * blockDim.x + threadIdx.x; u <= hi; u += gridDim.x * blockDim.x) {
        const float d = __uint_as_float(u);
        if (__float_as_uint(recip(d)) != __float_as_uint(__frcp_rn(d))) ++nb;
    }
    atomicAdd(bad, nb);
}

__global__ void self_check_div_kernel(unsigned long long* bad)
{
    unsigned long long nb = 0;
    constexpr uint32_t kQ = 128 + (65536 - 128) / 67;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < 65536ull * kQ;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t f = (uint32_t)(i / kQ), qi = (uint32_t)(i % kQ);
        const uint32_t q = qi < 64 ? qi : (qi < 128 ? 65535u - (qi - 64) : 64u + (qi - 128) * 67u);
        if (f == 0 || q > 65535u) continue;
        const uint32_t rs[3] = {0u, 1u % f, f - 1};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint64_t x64 = (uint64_t)q * f + rs[k];
            if (x64 >= ((uint64_t)f << 16)) continue;
            uint32_t r;
            const uint32_t qq = divmod_small((uint32_t)x64, f, r);
            if (qq != q || r != rs[k]) ++nb;
        }
    }
    atomicAdd(bad, nb);
}

// Largest |phi_fast_s(zs) - phi_hat_s(zs)| over every float zs that is not
// a NaN (infinities included: (b - mu) 2^22 / sigma' can overflow), as the
// bit pattern of a non-negative double (whose order is the integers').
__global__ void fast_phi_bound_kernel(unsigned long long* out)
{
    unsigned long long best = 0;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < (1ull << 32);
         u += (uint64_t)gridDim.x * blockDim.x) {
        const float zs = __uint_as_float((uint32_t)u);
        if (zs != zs) continue;
        const double d = fabs((double)phi_fast_s(zs) - (double)phi_hat_s(zs));
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        best = b > best ? b : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(kFull, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

template <int PHI>
__global__ void phi_grid_kernel(int64_t i0, float* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = phi_hat<PHI>(__fmul_rn((float)(i0 + i), 0x1p-22f));
}

// ---------------------------------------------------------------------------
// 1. Intervals: sf[n] = start | freq << 16.
// ---------------------------------------------------------------------------
template <int K, typename T, int PHI>
__global__ void __launch_bounds__(256) fgmm_interval_kernel(const T* __restrict__ params, int64_t N,
                                                            const int32_t* __restrict__ sym,
                                                            uint32_t* __restrict__ sf, int32_t* err)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        Mix<K> m;
        if (!load_mix<K>(params, N, n, m)) set_error(err, kErrBadParams);
        uint32_t st, fr;
        interval_of<K, PHI>(m, __ldg(sym + n), st, fr);
        sf[n] = st | (fr << 16);
    }
}

// ---------------------------------------------------------------------------
// 2. Interleaved rANS encoder, one segment per CTA of two warps.
// ---------------------------------------------------------------------------

// Step values of one interval: start, freq, freq << 16 (the renormalisation
// bound), 1/freq rounded toward zero and the escape test.
struct EncStep {
    uint32_t st, fr, fs;
    float rf;
    bool esc;
};

__device__ __forceinline__ EncStep enc_step(uint32_t v, bool act)
{
    EncStep e;
    e.st = v & 0xffffu;
    e.fr = v >> 16;
    e.fs = e.fr << 16;
    e.rf = __frcp_rz((float)(e.fr > 0u ? e.fr : 1u));
    e.esc = act && (e.st + e.fr == kM);
    return e;
}

// x -> C(x) for the interval of e, with the renormalisation word appended
// in ascending lane order (the rANS step of enc_put_warp with 1/freq known).
// y = x after renormalisation is below freq * 2^16, so q = floor(y / freq)
// is below 2^16. Every rounding of the estimate is toward zero (y, 1/freq,
// the product), so it is at most q and, with relative error below 3 * 2^-23,
// above q - 1: one upward correction makes it exact.
__device__ __forceinline__ void enc_put_pre(uint32_t& x, const EncStep& e, bool part, uint16_t* __restrict__ out,
                                            int64_t& base, uint32_t lt)
{
    const bool need = part && x >= e.fs;
    const uint32_t m = __ballot_sync(kFull, need);
    if (need) out[base + __popc(m & lt)] = (uint16_t)(x & 0xffffu);
    base += __popc(m);
    const uint32_t y = need ? x >> 16 : x;
    uint32_t q = __float2uint_rz(__fmul_rz(__uint2float_rz(y), e.rf));
    uint32_t rem = y - q * e.fr;
    if (rem >= e.fr) { ++q; rem -= e.fr; }
    if (part) x = (q << 16) + rem + e.st;
}

// Segment g of one latent, by a CTA of two warps. The preparing warp turns
// each step's interval into what the rANS step needs (start | freq << 16,
// 1/freq rounded toward zero, the escape vote of the warp, the raw symbol of
// an escape) and stores it in shared memory, kEncBlk steps at a time, one
// block ahead of the state warp; the state warp then runs only the state
// update and the word compaction. The two meet at a CTA barrier once per
// block. Steps k = 0 .. T-1 are the symbol steps T-1 .. 0.
constexpr int kEncBlk = 16;   // steps per hand-off block
constexpr int kEncThreads = 64;

struct EncPrepSlot {
    uint32_t sf[32];
    float rf[32];
    int32_t raw[32];
};

struct EncPrepRing {
    EncPrepSlot slot[2][kEncBlk];
    uint32_t esc[2][kEncBlk];   // escape votes (lane mask) of each step
};

__device__ __forceinline__ void rans_enc_segment(EncPrepRing& ring, const uint32_t* __restrict__ sf,
                                                 const int32_t* __restrict__ sym, int64_t N, int32_t S, int64_t T,
                                                 uint16_t* __restrict__ seg_words, int64_t seg_cap,
                                                 int64_t* __restrict__ seg_len, int64_t g)
{
    const int lane = threadIdx.x & 31;
    const bool prep = threadIdx.x >= 32;
    const int64_t n_top = (T - 1) * (int64_t)S + g * 32 + lane;   // step T-1; step T-1-k is n_top - k S
    const int64_t nblk = (T + kEncBlk - 1) / kEncBlk;
    // preparing warp: steps b kEncBlk .. of block b into buffer b & 1
    auto fill = [&](int64_t b) {
        const int buf = (int)(b & 1);
        int64_t k = b * kEncBlk;
        uint32_t v[kEncBlk];
#pragma unroll
        for (int i = 0; i < kEncBlk; ++i) {
            const int64_t n = n_top - (k + i) * S;
            v[i] = (k + i < T && n < N) ? __ldg(sf + n) : 0u;
        }
#pragma unroll
        for (int i = 0; i < kEncBlk; ++i) {
            const int64_t n = n_top - (k + i) * S;
            const bool act = k + i < T && n < N;
            const uint32_t st = v[i] & 0xffffu, fr = v[i] >> 16;
            const bool esc = act && st + fr == kM;
            ring.slot[buf][i].sf[lane] = v[i];
            ring.slot[buf][i].rf[lane] = __frcp_rz((float)(fr > 0u ? fr : 1u));
            ring.slot[buf][i].raw[lane] = esc ? __ldg(sym + n) : 0;
            const uint32_t m = __ballot_sync(kFull, esc);
            if (lane == 0) ring.esc[buf][i] = m;
        }
    };
    if (prep && nblk > 0) fill(0);
    __syncthreads();
    uint16_t* out = seg_words + g * seg_cap;
    const uint32_t lt = lanemask_lt();
    uint32_t x = kL;
    int64_t base = 0;
    const bool act0 = n_top < N;   // only step T-1 (k = 0) can hold lanes past N
    const EncStep one = enc_step(1u << 16, false);   // raw chunk: freq 1
    for (int64_t b = 0; b < nblk; ++b) {
        if (prep) {
            if (b + 1 < nblk) fill(b + 1);
        } else {
            const int buf = (int)(b & 1);
            const int nk = (int)min((int64_t)kEncBlk, T - b * kEncBlk);
#pragma unroll 4
            for (int i = 0; i < nk; ++i) {
                const bool act = act0 || b > 0 || i > 0;
                const uint32_t v = ring.slot[buf][i].sf[lane];
                const float rf = ring.slot[buf][i].rf[lane];
                const uint32_t em = ring.esc[buf][i];
                if (em) {
                    const bool esc = (em >> lane) & 1u;
                    const uint32_t raw = (uint32_t)ring.slot[buf][i].raw[lane];
                    enc_put_pre(x, EncStep{raw & 0xffffu, one.fr, one.fs, one.rf, false}, esc, out, base, lt);
                    enc_put_pre(x, EncStep{raw >> 16, one.fr, one.fs, one.rf, false}, esc, out, base, lt);
                }
                const uint32_t fr = v >> 16;
                enc_put_pre(x, EncStep{v & 0xffffu, fr, fr << 16, rf, false}, act, out, base, lt);
            }
        }
        __syncthreads();   // block b read, block b + 1 written
    }
    if (!prep) {
        out[base + 2 * lane] = (uint16_t)(x & 0xffffu);
        out[base + 2 * lane + 1] = (uint16_t)(x >> 16);
        if (lane == 0) seg_len[g] = base + 64;
    }
}

__global__ void __launch_bounds__(kEncThreads) fgmm_rans_enc_kernel(const uint32_t* __restrict__ sf,
                                                                    const int32_t* __restrict__ sym, int64_t N,
                                                                    int32_t S, int64_t T,
                                                                    uint16_t* __restrict__ seg_words, int64_t seg_cap,
                                                                    int64_t* __restrict__ seg_len, int64_t nseg)
{
    __shared__ EncPrepRing ring;
    const int64_t g = blockIdx.x;   // one segment per block
    if (g >= nseg) return;
    rans_enc_segment(ring, sf, sym, N, S, T, seg_words, seg_cap, seg_len, g);
}

// Two latents' segments in one launch (the checkerboard's two passes): the
// first a.nseg blocks encode latent a, the rest latent b.
struct EncLatentDev {
    const uint32_t* sf;
    const int32_t* sym;
    int64_t N;
    int32_t S;
    int64_t T;
    uint16_t* seg;
    int64_t cap;
    int64_t* len;
    int64_t nseg;
};

__global__ void __launch_bounds__(kEncThreads) fgmm_rans_enc2_kernel(EncLatentDev a, EncLatentDev b)
{
    __shared__ EncPrepRing ring;
    const int64_t g = blockIdx.x;
    if (g < a.nseg) rans_enc_segment(ring, a.sf, a.sym, a.N, a.S, a.T, a.seg, a.cap, a.len, g);
    else if (g - a.nseg < b.nseg) rans_enc_segment(ring, b.sf, b.sym, b.N, b.S, b.T, b.seg, b.cap, b.len, g - a.nseg);
}

// ---------------------------------------------------------------------------
// 3. Exclusive prefix sum of segment lengths (one block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) fgmm_scan_kernel(const int64_t* __restrict__ seg_len, int64_t nseg,
                                                         int64_t* __restrict__ offsets, int64_t* total_out,
                                                         int64_t cap, int32_t* err)
{
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nseg; base += blockDim.x) {
        const int64_t i = base + tid;
        const int64_t v = i < nseg ? seg_len[i] : 0;
        int64_t inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(kFull, inc, d);
            if (lane >= d) inc += o;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            const int nw = blockDim.x >> 5;
            int64_t w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t o = __shfl_up_sync(kFull, w, d);
                if (lane >= d) w += o;
            }
            if (lane < nw) warp_tot[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const int64_t before = carry + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (i < nseg) offsets[i] = before + inc - v;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = before + inc;
        __syncthreads();
    }
    if (tid == 0) {
        offsets[nseg] = carry;
        *total_out = carry;
        if (carry > cap) set_error(err, kErrCapacity);
    }
}

// ---------------------------------------------------------------------------
// 4. Segment compaction: one warp per segment.
// ---------------------------------------------------------------------------
// One warp per (segment, chunk of kCompactChunk words): 16-byte loads from
// the segment's 16-byte-aligned scratch, 2-byte stores to its offset.
constexpr int64_t kCompactChunk = 2048;

__global__ void __launch_bounds__(256) fgmm_compact_kernel(const uint16_t* __restrict__ seg_words, int64_t seg_cap,
                                                           const int64_t* __restrict__ seg_len,
                                                           const int64_t* __restrict__ offsets, int64_t nseg,
                                                           uint16_t* __restrict__ words, int64_t cap)
{
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t chunks = (seg_cap + kCompactChunk - 1) / kCompactChunk;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; item < nseg * chunks;
         item += nwarps) {
        const int64_t g = item / chunks, i0 = (item % chunks) * kCompactChunk;
        const int64_t len = seg_len[g], dst = offsets[g];
        if (dst + len > cap || i0 >= len) continue;   // capacity error already recorded / chunk past the end
        const int64_t n = len - i0 < kCompactChunk ? len - i0 : kCompactChunk;
        const uint16_t* src = seg_words + g * seg_cap + i0;
        uint16_t* d = words + dst + i0;
#pragma unroll 4
        for (int64_t i = 8 * lane; i < n; i += 256) {
            // i + 8 <= seg_cap - i0: segments hold a multiple of 8 words
            const uint4 v = *reinterpret_cast<const uint4*>(src + i);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (i + e < n) d[i + e] = (uint16_t)(w[e >> 1] >> (16 * (e & 1)));
        }
    }
}

// ---------------------------------------------------------------------------
// 3+4. Scan and compaction in one launch, for up to kScanCompactMax
// segments: block g sums the lengths of the segments before it (its offset)
// and of all of them (the total), writes offsets[g] (block 0 also
// offsets[nseg], the total and the capacity error) and copies its segment
// when it fits: the offsets, total, error and words of fgmm_scan_kernel
// followed by fgmm_compact_kernel, without the dependent round trips
// between the two launches.
// ---------------------------------------------------------------------------
constexpr int64_t kScanCompactMax = 1024;

__global__ void __launch_bounds__(256) fgmm_scan_compact_kernel(const uint16_t* __restrict__ seg_words,
                                                                int64_t seg_cap, const int64_t* __restrict__ seg_len,
                                                                int64_t nseg, int64_t* __restrict__ offsets,
                                                                int64_t* total_out, uint16_t* __restrict__ words,
                                                                int64_t cap, int32_t* err)
{
    __shared__ int64_t part[2][8];
    const int64_t g = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t before = 0, all = 0;
    for (int64_t i = tid; i < nseg; i += blockDim.x) {
        const int64_t v = seg_len[i];
        all += v;
        if (i < g) before += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(kFull, before, o);
        all += __shfl_xor_sync(kFull, all, o);
    }
    if (lane == 0) {
        part[0][wid] = before;
        part[1][wid] = all;
    }
    __syncthreads();
    before = 0;
    all = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        before += part[0][w];
        all += part[1][w];
    }
    const int64_t len = seg_len[g];
    if (tid == 0) {
        offsets[g] = before;
        if (g == 0) {
            offsets[nseg] = all;
            *total_out = all;
            if (all > cap) set_error(err, kErrCapacity);
        }
    }
    if (before + len > cap) return;   // the capacity error is recorded by block 0
    const uint16_t* src = seg_words + g * seg_cap;
    uint16_t* d = words + before;
    for (int64_t i = 8 * (int64_t)tid; i < len; i += 8 * (int64_t)blockDim.x) {
        // i + 8 <= seg_cap: segments hold a multiple of 8 words
        const uint4 v = *reinterpret_cast<const uint4*>(src + i);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (i + e < len) d[i + e] = (uint16_t)(w[e >> 1] >> (16 * (e & 1)));
    }
}

// ---------------------------------------------------------------------------
// Host-side dispatch helpers.
// ---------------------------------------------------------------------------
inline int grid_for(int64_t n, int threads, int max_blocks)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

template <int K, typename T, int PHI>
void launch_interval(const fgmm_latent* lat, const int32_t* sym, uint32_t* sf, int32_t* err, int sms,
                     cudaStream_t st)
{
    if (lat->N == 0) return;
    const int threads = 256;
    fgmm_interval_kernel<K, T, PHI><<<grid_for(lat->N, threads, sms * 16), threads, 0, st>>>(
        static_cast<const T*>(lat->params), lat->N, sym, sf, err);
}

template <typename T, int PHI>
void dispatch_interval(const fgmm_latent* lat, const int32_t* sym, uint32_t* sf, int32_t* err, int sms,
                       cudaStream_t st)
{
    switch (lat->K) {
    case 1: launch_interval<1, T, PHI>(lat, sym, sf, err, sms, st); break;
    case 2: launch_interval<2, T, PHI>(lat, sym, sf, err, sms, st); break;
    case 3: launch_interval<3, T, PHI>(lat, sym, sf, err, sms, st); break;
    default: launch_interval<4, T, PHI>(lat, sym, sf, err, sms, st); break;
    }
}

template <int PHI>
void launch_interval_phi(const fgmm_latent* lat, const int32_t* sym, uint32_t* sf, int32_t* err, int sms,
                         cudaStream_t st)
{
    if (lat->dtype == FGMM_DTYPE_BF16) dispatch_interval<__nv_bfloat16, PHI>(lat, sym, sf, err, sms, st);
    else dispatch_interval<float, PHI>(lat, sym, sf, err, sms, st);
}

// Intervals with approximation phi (kPhiAS, kPhiLogistic, kPhiPolya).
void launch_interval_any(const fgmm_latent* lat, const int32_t* sym, uint32_t* sf, int32_t* err, int sms,
                         cudaStream_t st, int phi = kPhiAS)
{
    if (phi == kPhiLogistic) launch_interval_phi<kPhiLogistic>(lat, sym, sf, err, sms, st);
    else if (phi == kPhiPolya) launch_interval_phi<kPhiPolya>(lat, sym, sf, err, sms, st);
    else launch_interval_phi<kPhiAS>(lat, sym, sf, err, sms, st);
}



// Per-segment scratch capacity: at most three words per lane and step (an
// escape emits for two chunks and the main symbol) plus the flush block;
// rounded to 8 words so that every segment starts 16-byte aligned.
inline int64_t seg_cap_words(int64_t T) { return (int64_t)align_up((size_t)(3 * 32 * T + 64), 8); }

// One warp per (segment, chunk) item of the compaction.
inline void launch_compact(const uint16_t* seg, int64_t cap, const int64_t* len, const int64_t* offsets,
                           int64_t nseg, uint16_t* words, int64_t words_cap, int sms, cudaStream_t st)
{
    const int64_t items = nseg * ((cap + kCompactChunk - 1) / kCompactChunk);
    fgmm_compact_kernel<<<grid_for(items * 32, 256, sms * 8), 256, 0, st>>>(seg, cap, len, offsets, nseg, words,
                                                                            words_cap);
}

// Offsets, total and compaction of nseg segments: one launch for up to
// kScanCompactMax segments, else the scan and the compaction kernels.
inline void launch_scan_compact(const uint16_t* seg, int64_t cap, const int64_t* len, int64_t nseg,
                                int64_t* offsets, int64_t* total, uint16_t* words, int64_t words_cap, int32_t* err,
                                int sms, cudaStream_t st)
{
    if (nseg >= 1 && nseg <= kScanCompactMax) {
        fgmm_scan_compact_kernel<<<(unsigned)nseg, 256, 0, st>>>(seg, cap, len, nseg, offsets, total, words,
                                                                 words_cap, err);
        return;
    }
    fgmm_scan_kernel<<<1, 1024, 0, st>>>(len, nseg, offsets, total, words_cap, err);
    launch_compact(seg, cap, len, offsets, nseg, words, words_cap, sms, st);
}

}  // namespace

// ===========================================================================
// Shared host helpers.
// ===========================================================================
namespace fgmm {

cudaError_t decode_planned(fgmm_handle* h, DecodeArgs& a, int K, int dtype, cudaStream_t st)
{
    a.err = h->d_err;
    a.stats = h->stats_on ? h->d_stats : nullptr;
    int lanes = 1, cluster = 1, round0 = 0, kernel = 0;
    decode_resolve(a.nseg, h->num_sms, h->decode_lanes, h->decode_cluster, h->decode_round0, h->phi, &lanes,
                   &cluster, &round0, &kernel);
    if (kernel == FGMM_DEC_WS && a.T >= ((int64_t)1 << 24)) {   // streams beyond the warp-specialised kernel's range
        lanes = 1;
        cluster = 1;
        round0 = 0;
        kernel = FGMM_DEC_LANE;
    }
    a.r0 = round0 > 0 ? round0 : 32;
    a.phi = h->phi;
    a.silent = h->test_silent_stream;
    return launch_decode(a, K, dtype, lanes, cluster, st);
}

fgmm_status ws_reserve(fgmm_handle* h, size_t bytes, cudaStream_t stream)
{
    if (bytes <= h->ws_bytes) return FGMM_OK;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "ws_reserve sync");
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    const size_t want = align_up(bytes + bytes / 4, (size_t)1 << 20);
    e = cudaMalloc(&h->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->ws = nullptr;
        return fail(h, FGMM_ERR_NO_MEMORY, "workspace allocation failed");
    }
    h->ws_bytes = want;
    return FGMM_OK;
}

fgmm_status encode_reserve(fgmm_handle* h, int64_t N, int32_t S, cudaStream_t st, EncodeWs* ws)
{
    const int64_t nseg = S / 32, T = steps_of(N, S);
    const int64_t cap = seg_cap_words(T);
    // workspace: intervals [N] u32 | segment scratch [nseg][cap] u16 | lengths [nseg] i64
    const size_t o_sf = 0;
    const size_t o_seg = align_up(o_sf + sizeof(uint32_t) * (size_t)N, 256);
    const size_t o_len = align_up(o_seg + sizeof(uint16_t) * (size_t)(nseg * cap), 256);
    const size_t bytes = o_len + sizeof(int64_t) * (size_t)nseg;
    fgmm_status s = ws_reserve(h, bytes, st);
    if (s != FGMM_OK) return s;
    char* base = static_cast<char*>(h->ws);
    ws->sf = reinterpret_cast<uint32_t*>(base + o_sf);
    ws->seg = reinterpret_cast<uint16_t*>(base + o_seg);
    ws->len = reinterpret_cast<int64_t*>(base + o_len);
    ws->cap = cap;
    return FGMM_OK;
}

void encode_from_intervals(const EncodeWs& ws, const int32_t* symbols, int64_t N, int32_t S, uint16_t* words,
                           int64_t words_cap, int64_t* offsets, int64_t* n_words_out, int32_t* err, int sms,
                           cudaStream_t st)
{
    const int64_t nseg = S / 32, T = steps_of(N, S);
    fgmm_rans_enc_kernel<<<(unsigned)nseg, kEncThreads, 0, st>>>(ws.sf, symbols, N, S, T, ws.seg,
                                                                                  ws.cap, ws.len, nseg);
    launch_scan_compact(ws.seg, ws.cap, ws.len, nseg, offsets, n_words_out, words, words_cap, err, sms, st);
}

void launch_scan(const int64_t* len, int64_t nseg, int64_t* offsets, int64_t* total_out, int64_t cap, int32_t* err,
                 cudaStream_t st)
{
    fgmm_scan_kernel<<<1, 1024, 0, st>>>(len, nseg, offsets, total_out, cap, err);
}

void encode2_from_intervals(const EncPass& a, const EncPass& b, int32_t* err, int sms, cudaStream_t st)
{
    const EncPass* p[2] = {&a, &b};
    EncLatentDev d[2];
    for (int i = 0; i < 2; ++i) {
        const int64_t nseg = p[i]->S / 32;
        d[i] = EncLatentDev{p[i]->sf, p[i]->sym, p[i]->N, p[i]->S, steps_of(p[i]->N, p[i]->S),
                            p[i]->seg, seg_cap_words(steps_of(p[i]->N, p[i]->S)), p[i]->len, nseg};
    }
    fgmm_rans_enc2_kernel<<<(unsigned)(d[0].nseg + d[1].nseg), kEncThreads, 0, st>>>(d[0], d[1]);
    for (int i = 0; i < 2; ++i) {
        launch_scan_compact(d[i].seg, d[i].cap, d[i].len, d[i].nseg, p[i]->offsets, p[i]->total, p[i]->words,
                            p[i]->words_cap, err, sms, st);
    }
}

int64_t encode_seg_cap(int64_t N, int32_t S) { return seg_cap_words(steps_of(N, S)); }

fgmm_status check_latent(fgmm_handle* h, const fgmm_latent* lat)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (!lat) return fail(h, FGMM_ERR_INVALID_ARG, "latent is NULL");
    if (lat->K < 1 || lat->K > FGMM_MAX_K) return fail(h, FGMM_ERR_INVALID_ARG, "K must be in [1, 4]");
    if (lat->dtype != FGMM_DTYPE_F32 && lat->dtype != FGMM_DTYPE_BF16)
        return fail(h, FGMM_ERR_INVALID_ARG, "dtype must be FGMM_DTYPE_F32 or FGMM_DTYPE_BF16");
    if (lat->N < 0 || lat->N > ((int64_t)1 << 40)) return fail(h, FGMM_ERR_INVALID_ARG, "N out of range");
    if (lat->N > 0 && !lat->params) return fail(h, FGMM_ERR_INVALID_ARG, "params is NULL");
    return FGMM_OK;
}

}  // namespace fgmm

// ===========================================================================
// C ABI.
// ===========================================================================
extern "C" {

fgmm_status fgmm_create(fgmm_handle** out)
{
    if (!out) return FGMM_ERR_INVALID_ARG;
    *out = nullptr;
    fgmm_handle* h = new fgmm_handle();
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_stats, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(h->d_stats, 0, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->d_err) cudaFree(h->d_err);
        if (h->d_stats) cudaFree(h->d_stats);
        delete h;
        return FGMM_ERR_CUDA;
    }
    *out = h;
    return FGMM_OK;
}

void fgmm_destroy(fgmm_handle* h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->ws) cudaFree(h->ws);
    if (h->d_err) cudaFree(h->d_err);
    if (h->d_stats) cudaFree(h->d_stats);
    delete h;
}

const char* fgmm_status_string(int32_t status)
{
    switch (status) {
    case FGMM_OK: return "ok";
    case FGMM_ERR_INVALID_ARG: return "invalid argument";
    case FGMM_ERR_BAD_PARAMS: return "invalid mixture parameter (NaN/Inf, negative weight, or scale <= 0)";
    case FGMM_ERR_CAPACITY: return "output buffer too small";
    case FGMM_ERR_CORRUPT: return "corrupt or truncated stream";
    case FGMM_ERR_TIMEOUT: return "bounded wait timed out";
    case FGMM_ERR_CUDA: return "CUDA error";
    case FGMM_ERR_NO_MEMORY: return "out of device memory";
    case FGMM_ERR_TOO_LARGE: return "request exceeds the fixed scratch of the allocation-free encoder";
    default: return "unknown status";
    }
}

const char* fgmm_last_error(const fgmm_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

fgmm_status fgmm_sync_status(fgmm_handle* h, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_sync_status");
    int32_t v = 0;
    e = cudaMemcpy(&v, h->d_err, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_sync_status read");
    if (v != 0) {
        e = cudaMemset(h->d_err, 0, sizeof(int32_t));
        if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_sync_status clear");
        h->last_error = fgmm_status_string(v);
    }
    return static_cast<fgmm_status>(v);
}

fgmm_status fgmm_stats_enable(fgmm_handle* h, int32_t on)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    h->stats_on = on != 0;
    return FGMM_OK;
}

fgmm_status fgmm_stats_read(fgmm_handle* h, uint64_t* out, void* stream)
{
    if (!h || !out) return FGMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    unsigned long long v[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(v, h->d_stats, sizeof v, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(h->d_stats, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_stats_read");
    for (int i = 0; i < 4; ++i) out[i] = v[i];
    return FGMM_OK;
}

fgmm_status fgmm_phi(fgmm_handle* h, const float* z, float* out, int64_t n, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!z || !out))) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_phi: bad arguments");
    if (n == 0) return FGMM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int g = grid_for(n, 256, h->num_sms * 16);
    if (h->phi == kPhiLogistic) phi_kernel<kPhiLogistic><<<g, 256, 0, st>>>(z, out, n);
    else if (h->phi == kPhiPolya) phi_kernel<kPhiPolya><<<g, 256, 0, st>>>(z, out, n);
    else phi_kernel<kPhiAS><<<g, 256, 0, st>>>(z, out, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_phi launch");
}

fgmm_status fgmm_phi_grid(fgmm_handle* h, int64_t i0, float* out, int64_t n, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && !out) || i0 < -(int64_t)(1 << 30) || i0 + n > (int64_t)(1 << 30))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_phi_grid: bad arguments");
    if (n == 0) return FGMM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int g = grid_for(n, 256, h->num_sms * 16);
    if (h->phi == kPhiLogistic) phi_grid_kernel<kPhiLogistic><<<g, 256, 0, st>>>(i0, out, n);
    else if (h->phi == kPhiPolya) phi_grid_kernel<kPhiPolya><<<g, 256, 0, st>>>(i0, out, n);
    else phi_grid_kernel<kPhiAS><<<g, 256, 0, st>>>(i0, out, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_phi_grid launch");
}

fgmm_status fgmm_self_check(fgmm_handle* h, uint64_t* out)
{
    if (!h || !out) return FGMM_ERR_INVALID_ARG;
    unsigned long long* d = h->d_stats + 4;   // spare counters
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        self_check_recip_kernel<<<h->num_sms * 8, 256>>>(d);
        self_check_div_kernel<<<h->num_sms * 8, 256>>>(d + 1);
        e = cudaDeviceSynchronize();
    }
    unsigned long long v[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(v, d, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_self_check");
    out[0] = v[0];
    out[1] = v[1];
    return FGMM_OK;
}

fgmm_status fgmm_fast_phi_bound(fgmm_handle* h, double* out)
{
    if (!h || !out) return FGMM_ERR_INVALID_ARG;
    unsigned long long* d = h->d_stats + 4;   // spare counter
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        fast_phi_bound_kernel<<<h->num_sms * 8, 256>>>(d);
        e = cudaDeviceSynchronize();
    }
    unsigned long long v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_fast_phi_bound");
    std::memcpy(out, &v, sizeof v);
    return FGMM_OK;
}

fgmm_status fgmm_freqs(fgmm_handle* h, const fgmm_latent* lat, const int32_t* symbols, uint32_t* sf, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (lat->N > 0 && (!symbols || !sf)) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_freqs: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    launch_interval_any(lat, symbols, sf, h->d_err, h->num_sms, st, h->phi);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_freqs launch");
}

int64_t fgmm_encode_bound_words(int64_t N, int32_t S)
{
    if (S <= 0 || S % 32 != 0 || N < 0) return -1;
    const int64_t T = steps_of(N, S);
    return (int64_t)(S / 32) * (3 * 32 * T + 64);
}

fgmm_status fgmm_encode(fgmm_handle* h, const fgmm_latent* lat, const int32_t* symbols, int32_t S, uint16_t* words,
                        int64_t words_cap, int64_t* offsets, int64_t* n_words_out, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || !n_words_out || words_cap < 0 || (words_cap > 0 && !words) || (lat->N > 0 && !symbols))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_encode: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EncodeWs ws;
    s = encode_reserve(h, lat->N, S, st, &ws);
    if (s != FGMM_OK) return s;
    launch_interval_any(lat, symbols, ws.sf, h->d_err, h->num_sms, st, h->phi);
    encode_from_intervals(ws, symbols, lat->N, S, words, words_cap, offsets, n_words_out, h->d_err, h->num_sms, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_encode launch");
}

fgmm_status fgmm_decode(fgmm_handle* h, const fgmm_latent* lat, const uint16_t* words, int64_t n_words,
                        const int64_t* offsets, int32_t S, int32_t* symbols_out, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || n_words < 0 || (n_words > 0 && !words) || (lat->N > 0 && !symbols_out))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_decode: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DecodeArgs a;
    a.params = lat->params;
    a.N = lat->N;
    a.S = S;
    a.T = steps_of(lat->N, S);
    a.words = words;
    a.n_words = n_words;
    a.offsets = offsets;
    a.nseg = S / 32;
    a.out = symbols_out;
    cudaError_t e = decode_planned(h, a, lat->K, lat->dtype, st);
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_decode launch");
}

fgmm_status fgmm_decode_plan(fgmm_handle* h, int32_t S, int32_t* out)
{
    if (!h || !out) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_decode_plan: NULL argument");
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    int lanes = 1, cluster = 1, round0 = 0, kernel = 0;
    decode_resolve(S / 32, h->num_sms, h->decode_lanes, h->decode_cluster, h->decode_round0, h->phi, &lanes,
                   &cluster, &round0, &kernel);
    out[0] = lanes;
    out[1] = cluster;
    out[2] = kernel;
    out[3] = round0;
    return FGMM_OK;
}

fgmm_status fgmm_set_option(fgmm_handle* h, int32_t option, int64_t value)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    switch (option) {
    case FGMM_OPT_DECODE_LANES:
        if (!(value == 0 || value == 1 || value == 2 || value == 4 || value == 8 || value == 16 || value == 32))
            return fail(h, FGMM_ERR_INVALID_ARG, "decode lanes must be 0 (auto), 1, 2, 4, 8, 16 or 32");
        h->decode_lanes = (int)value;
        return FGMM_OK;
    case FGMM_OPT_DECODE_CLUSTER:
        if (!(value == 0 || value == 1 || value == 2 || value == 4 || value == 8))
            return fail(h, FGMM_ERR_INVALID_ARG, "decode cluster must be 0 (auto), 1, 2, 4 or 8");
        h->decode_cluster = (int)value;
        return FGMM_OK;
    case FGMM_OPT_PHI:
        if (!(value == FGMM_PHI_AS || value == FGMM_PHI_LOGISTIC || value == FGMM_PHI_POLYA))
            return fail(h, FGMM_ERR_INVALID_ARG, "approximation must be FGMM_PHI_AS, _LOGISTIC or _POLYA");
        h->phi = (int)value;
        return FGMM_OK;
    case FGMM_OPT_TEST_SILENT_STREAM:
        if (value < -1 || value > 31) return fail(h, FGMM_ERR_INVALID_ARG, "silent stream must be -1 (off) or 0..31");
        h->test_silent_stream = (int)value;
        return FGMM_OK;
    case FGMM_OPT_MLP_ACT:
        if (!(value == FGMM_MLP_ACT_PL || value == FGMM_MLP_ACT_SIGMOID))
            return fail(h, FGMM_ERR_INVALID_ARG, "activation must be FGMM_MLP_ACT_PL or FGMM_MLP_ACT_SIGMOID");
        h->mlp_act = (int)value;
        return FGMM_OK;
    case FGMM_OPT_TEST_SILENT_ARRIVALS:
        if (value != 0 && value != 1) return fail(h, FGMM_ERR_INVALID_ARG, "silent arrivals must be 0 or 1");
        h->test_silent_arrivals = (int)value;
        return FGMM_OK;
    case FGMM_OPT_DECODE_ROUND0:
        if (!(value == 0 || value == 16 || value == 32))
            return fail(h, FGMM_ERR_INVALID_ARG, "decode first-round points must be 0 (auto), 16 or 32");
        h->decode_round0 = (int)value;
        return FGMM_OK;
    default:
        return fail(h, FGMM_ERR_INVALID_ARG, "unknown option");
    }
}

}  // extern "C"

// ===========================================================================
// Allocation-free encode: the same four kernels as fgmm_encode, with their
// scratch in a fixed static device array instead of handle workspace.
// ===========================================================================

// Fixed scratch for fgmm_encode_noalloc, resident on every GPU that loads
// this library until the process exits. Host code must not use this name as
// an address: it is a host-side stand-in. The device address comes from
// cudaGetSymbolAddress in noalloc_scratch_for_current_device().
static __device__ __align__(256) unsigned char fgmm_noalloc_scratch[FGMM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocMaxDevices = 128;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices];
int g_noalloc_sms[kNoAllocMaxDevices];
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices];   // context the address belongs to (0 = none yet)

// Unique id of the calling thread's current CUDA context (0 if none), from
// the driver entry points the runtime hands out (no link against the driver
// library). A context that replaces another (after cudaDeviceReset, for
// example) has a new id, and the array may have a new address in it.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Set-up per device and context, with that device current: look up (with
// cudaGetSymbolAddress, which also makes the device's context current if
// none is) and cache the device address of the scratch array and the SM
// count; look them up again whenever the current context is not the one
// the cached address was taken in.
cudaError_t noalloc_scratch_for_current_device(void** ptr, int* sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, fgmm_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
        g_noalloc_sms[dev] = n;
        g_noalloc_ctx[dev] = current_context_id();   // the context is current now
    }
    *ptr = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" fgmm_status fgmm_encode_noalloc(const fgmm_latent* lat, const int32_t* symbols, int32_t S,
                                           uint16_t* words, int64_t words_cap, int64_t* offsets,
                                           int64_t* n_words_out, int32_t* status_out, void* stream)
{
    if (!lat || lat->K < 1 || lat->K > FGMM_MAX_K || lat->N < 0 || lat->N > ((int64_t)1 << 40) ||
        (lat->dtype != FGMM_DTYPE_F32 && lat->dtype != FGMM_DTYPE_BF16) || (lat->N > 0 && !lat->params))
        return FGMM_ERR_INVALID_ARG;
    if (S <= 0 || S % 32 != 0) return FGMM_ERR_INVALID_ARG;
    if (!offsets || !n_words_out || !status_out || words_cap < 0 || (words_cap > 0 && !words) ||
        (lat->N > 0 && !symbols))
        return FGMM_ERR_INVALID_ARG;
    const int64_t N = lat->N, nseg = S / 32, T = steps_of(N, S);
    const int64_t cap = seg_cap_words(T);
    const size_t o_sf = 0;
    const size_t o_seg = align_up(o_sf + sizeof(uint32_t) * (size_t)N, 256);
    const size_t o_len = align_up(o_seg + sizeof(uint16_t) * (size_t)(nseg * cap), 256);
    const size_t bytes = o_len + sizeof(int64_t) * (size_t)nseg;
    if (bytes > (size_t)FGMM_NOALLOC_SCRATCH_BYTES) return FGMM_ERR_TOO_LARGE;

    void* base = nullptr;
    int sms = 0;
    cudaError_t e = noalloc_scratch_for_current_device(&base, &sms);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FGMM_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(base);
    uint32_t* sf = reinterpret_cast<uint32_t*>(ws + o_sf);
    uint16_t* seg = reinterpret_cast<uint16_t*>(ws + o_seg);
    int64_t* len = reinterpret_cast<int64_t*>(ws + o_len);

    e = cudaMemsetAsync(status_out, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FGMM_ERR_CUDA;
    }
    launch_interval_any(lat, symbols, sf, status_out, sms, st);
    fgmm_rans_enc_kernel<<<(unsigned)nseg, kEncThreads, 0, st>>>(sf, symbols, N, S, T, seg, cap,
                                                                                  len, nseg);
    fgmm_scan_kernel<<<1, 1024, 0, st>>>(len, nseg, offsets, n_words_out, words_cap, status_out);
    launch_compact(seg, cap, len, offsets, nseg, words, words_cap, sms, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : FGMM_ERR_CUDA;
}
