// fgmm_gsm.cu -- Gaussian single model coder with pre-built tables: the
// scheme of Sec. II-C that makes the GSM cheap. The quantiser has already
// shifted each latent by its mean, so the coder receives the integer
// residual q and the scale sigma only, and codes q with N(0, sigma). Sigma
// is quantised to the smallest of L <= 64 increasing levels at or above it
// (the last level above them all), so one CDF row per level is all the
// coder ever needs, built once ahead of coding.
//
// A level's row is this library's quantised CDF of N(0, level) -- the K = 1
// mixture (1, 0, level) with the same window, escape slot and scale floor as
// the table-free coder -- so a GSM stream is byte-identical to fgmm_encode
// of K = 1 parameters (1, 0, level of sigma).
//
// Tables blob (device, caller-owned, 16-byte aligned, kBlobBytes):
//   [0, 512)          header: int32 L at 0, float levels[64] at 16
//   [512, 66048)      uint16 rows[64][512], row[j] = Q(clamp(j - 255, lo, hi + 1)),
//                     0 left of the window (the table coder's row layout)
//   [66048, 198144)   uint2 buckets[64][258]: for b in [0, 256],
//                     J = the largest j in [0, 510] with row[j] <= 256 b,
//                     bucket = (J | row[J] << 16, row[J + 1]); entry 257 is 0
// Decoding slot v reads buckets b = v >> 8 and b + 1: row[J_b] <= v <
// row[J_{b+1} + 1], and v is an escape iff v >= row[J_{b+1} + 1] (then that
// value is the escape start); a short search over the row finishes the
// rare buckets that hold more than one symbol boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"
#include "fgmm_segment.cuh"

using namespace fgmm;

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kRow = 512;
constexpr int kLmax = 64;
constexpr int kBktStride = 258;                                         // 257 used + 1 pad (16-byte rows)
constexpr uint32_t kHdrBytes = 512;
constexpr uint32_t kRowsOff = kHdrBytes;
constexpr uint32_t kRowsBytes = kLmax * kRow * 2;                        // 65536
constexpr uint32_t kBktOff = kRowsOff + kRowsBytes;                     // 66048
constexpr uint32_t kBktBytes = kLmax * kBktStride * 8;                  // 132096
constexpr uint32_t kBlobBytes = kBktOff + kBktBytes;                    // 198144
constexpr uint32_t kDecSmem = kBlobBytes;                               // same layout in shared memory
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint64_t kWaitNs = 1000000000ull;                              // 1 s
constexpr int kRing = 8;                                                // scale prefetch depth (steps)

struct GsmLevels {
    float lv[kLmax];
    int L;
};

// Level search table: lvp[i] = level i for i < L - 1, +inf from L - 1 on, so
// that the count of entries below sigma is the smallest level >= sigma among
// the first L - 1, else L - 1.
__device__ __forceinline__ void load_levels(const unsigned char* __restrict__ blob, float* lvp, int i)
{
    int L = __ldg(reinterpret_cast<const int32_t*>(blob));
    L = L < 1 ? 1 : (L > kLmax ? kLmax : L);
    const float* lv = reinterpret_cast<const float*>(blob + 16);
    lvp[i] = i < L - 1 ? __ldg(lv + i) : __int_as_float(0x7f800000);
}

__device__ __forceinline__ int level_of(const float* lvp, float sg)
{
    int pos = 0;
#pragma unroll
    for (int step = 32; step > 0; step >>= 1)
        if (lvp[pos + step - 1] < sg) pos += step;
    return pos;
}

__device__ __forceinline__ bool scale_ok(float sg) { return isfinite(sg) && sg > 0.0f; }

// ---------------------------------------------------------------------------
// Build: one block per level, 256 threads, two row entries each, then the
// bucket index by binary search over the row in shared memory.
// ---------------------------------------------------------------------------
template <int PHI>
__global__ void __launch_bounds__(256) fgmm_gsm_build_kernel(GsmLevels p, unsigned char* __restrict__ blob)
{
    __shared__ uint16_t row[kRow];
    const int l = blockIdx.x;
    const int t = threadIdx.x;
    RawParams<1> r;
    r.v[0] = 1.0f;
    r.v[1] = 0.0f;
    r.v[2] = p.lv[l];
    Mix<1> m;
    mix_from_params<1>(r, m);   // levels are checked on the host
    uint32_t q[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int j = -kYmax + 2 * t + e;
        const int jc = j <= m.lo ? m.lo + 1 : (j > m.hi + 1 ? m.hi + 1 : j);
        const uint32_t v = q_at<1, PHI>(m, jc);
        q[e] = j <= m.lo ? 0u : v;
        row[2 * t + e] = (uint16_t)q[e];
    }
    reinterpret_cast<uint32_t*>(blob + kRowsOff + (size_t)l * kRow * 2)[t] = q[0] | (q[1] << 16);
    __syncthreads();
    uint2* bkt = reinterpret_cast<uint2*>(blob + kBktOff) + (size_t)l * kBktStride;
    for (int b = t; b < kBktStride; b += 256) {
        uint2 v = make_uint2(0u, 0u);
        if (b <= 256) {
            const uint32_t target = 256u * (uint32_t)b;
            int a = 0, c = kRow - 1;   // row[0] = 0 <= target; answer in [0, 510]
            while (c - a > 1) {
                const int mid = (a + c) >> 1;
                if ((uint32_t)row[mid] <= target) a = mid;
                else c = mid;
            }
            v = make_uint2((uint32_t)a | ((uint32_t)row[a] << 16), (uint32_t)row[a + 1]);
        }
        bkt[b] = v;
    }
    if (l == 0) {
        uint32_t* hdr = reinterpret_cast<uint32_t*>(blob);
        for (int i = t; i < (int)(kHdrBytes / 4); i += 256) {
            uint32_t w = 0;
            if (i == 0) w = (uint32_t)p.L;
            else if (i >= 4 && i < 4 + kLmax) w = __float_as_uint(i - 4 < p.L ? p.lv[i - 4] : 0.0f);
            hdr[i] = w;
        }
    }
}

// ---------------------------------------------------------------------------
// Intervals: sf[n] = start | freq << 16 from the row of the level of
// scales[n] at q = symbols[n].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) fgmm_gsm_interval_kernel(const T* __restrict__ scales, int64_t N,
                                                                const int32_t* __restrict__ sym,
                                                                const unsigned char* __restrict__ blob,
                                                                uint32_t* __restrict__ sf, int32_t* err)
{
    __shared__ float lvp[kLmax];
    if (threadIdx.x < kLmax) load_levels(blob, lvp, threadIdx.x);
    __syncthreads();
    const uint16_t* rows = reinterpret_cast<const uint16_t*>(blob + kRowsOff);
    bool bad = false;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float sg = load_param(scales, n);
        bad |= !scale_ok(sg);
        const uint16_t* row = rows + level_of(lvp, sg) * kRow;
        const int32_t q = __ldg(sym + n);
        uint32_t v = 0;
        bool in = false;
        if (q >= -kYmax && q <= kYmax) {
            const uint32_t a = __ldg(row + q + kYmax), b = __ldg(row + q + kYmax + 1);
            in = b > a;
            v = a | ((b - a) << 16);
        }
        if (!in) {
            const uint32_t e = __ldg(row + kRow - 1);
            v = e | ((kM - e) << 16);
        }
        sf[n] = v;
    }
    if (bad) set_error(err, kErrBadParams);
}

// ---------------------------------------------------------------------------
// Decoder: the whole tables blob staged in shared memory by one bulk copy
// (cp.async.bulk completing on an mbarrier, bounded wait), then one warp per
// 32-stream segment, one lane per stream, persistent over segments; each
// warp reads its segment's words through a shared-memory ring.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the mbarrier; gives up after `limit` tries or
// kWaitNs nanoseconds, whichever comes first (each try may suspend the
// thread for a hardware-defined time).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit)
{
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// Per-warp word ring: the segment's words are consumed downward from the
// top; a ring of kWRing words in shared memory holds the words at and above
// `fill` (slot = absolute index mod kWRing), refilled kWChunk words at a
// time by cp.async (8 bytes per lane) well before they are read. A chunk
// overwrites the slots of words kWRing above it, which are consumed once
// (first unread word + 1) - fill <= kWRing - kWChunk. One step reads at most
// 96 words (32 symbols plus two escape chunks each), fewer than kWChunk, so
// one issue per step keeps up. Pieces outside [0, n_words) are zero-filled,
// never read.
constexpr int kWRing = 512, kWChunk = 128, kWMaxStep = 96;

__device__ __forceinline__ void wring_issue(uint16_t* ring, const uint16_t* __restrict__ words, int64_t n_words,
                                            int64_t a0, int lane)
{
    const int64_t a = a0 + 4 * lane;
    int bytes = 0;
    if (a >= 0 && a < n_words) bytes = n_words - a >= 4 ? 8 : (int)(n_words - a) * 2;
    const uint16_t* src = bytes > 0 ? words + a : words;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(ring + (int)(a & (kWRing - 1)));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Level of every symbol's scale (uint8), and the scale check, ahead of the
// decoder: the search over the levels leaves the decoder's serial chain.
template <typename T>
__global__ void __launch_bounds__(256) fgmm_gsm_level_kernel(const T* __restrict__ scales, int64_t N,
                                                             const unsigned char* __restrict__ blob,
                                                             uint8_t* __restrict__ lev, int32_t* err)
{
    __shared__ float lvp[kLmax];
    if (threadIdx.x < kLmax) load_levels(blob, lvp, threadIdx.x);
    __syncthreads();
    bool bad = false;
    // four loads in flight per thread before the searches
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x * 4 + threadIdx.x; b < N; b += (int64_t)gridDim.x * blockDim.x * 4) {
        float sg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t n = b + (int64_t)u * blockDim.x;
            sg[u] = n < N ? load_param(scales, n) : 1.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t n = b + (int64_t)u * blockDim.x;
            if (n < N) {
                bad |= !scale_ok(sg[u]);
                lev[n] = (uint8_t)level_of(lvp, sg[u]);
            }
        }
    }
    if (bad) set_error(err, kErrBadParams);
}

__global__ void __launch_bounds__(1024, 1) fgmm_gsm_dec_kernel(const uint8_t* __restrict__ lev, int64_t N, int32_t S,
                                                               int64_t T_steps, const unsigned char* __restrict__ blob,
                                                               const uint16_t* __restrict__ words, int64_t n_words,
                                                               const int64_t* __restrict__ offsets, int64_t nseg,
                                                               int32_t* __restrict__ out, int32_t* err)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(8) unsigned long long mbar_s;
    const uint16_t* srow = reinterpret_cast<const uint16_t*>(sm + kRowsOff);
    const uint2* sbkt = reinterpret_cast<const uint2*>(sm + kBktOff);
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&mbar_s);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = kBlobBytes - kRowsOff;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(sm + kRowsOff);
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mbar),
                     "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
            "l"(blob + kRowsOff), "r"(bytes), "r"(mbar)
            : "memory");
    }
    if (!mbar_wait(mbar, 0, kWaitLimit)) {
        if (threadIdx.x == 0) set_error(err, kErrTimeout);
        mbar_wait(mbar, 0, kWaitLimit);   // let the copy land before the block leaves
        return;
    }

    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const uint32_t lt = lanemask_lt();
    uint16_t* ring = reinterpret_cast<uint16_t*>(sm + kBlobBytes) + (threadIdx.x >> 5) * kWRing;
    for (int64_t g = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); g < nseg; g += (int64_t)gridDim.x * wpb) {
        const int64_t beg = offsets[g], end = offsets[g + 1];
        // a stream of fewer than 2^24 steps has fewer than 2^31 words
        if (!(beg >= 0 && end <= n_words && end - beg >= 64 && end - beg < ((int64_t)1 << 31))) {
            if (lane == 0) set_error(err, kErrCorrupt);
            continue;
        }
        uint32_t x = (uint32_t)__ldg(words + end - 64 + 2 * lane) |
                     ((uint32_t)__ldg(words + end - 63 + 2 * lane) << 16);
        // word indices relative to beg (32-bit); ring slot (bmod + i) mod kWRing
        const int bmod = (int)(beg & (kWRing - 1));
        int rp = (int)(end - 64 - beg);
        // ring: the kWRing words below rp rounded up to 4 (absolute), loaded and waited for
        int rf = (int)((((end - 64 + 3) & ~(int64_t)3) - kWRing) - beg);
#pragma unroll
        for (int c = 0; c < kWRing / kWChunk; ++c) wring_issue(ring, words, n_words, beg + rf + c * kWChunk, lane);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncwarp();
        int rready = rf;
        int pending = 0;
        bool bad = false;
        const int64_t n0 = g * 32 + lane;
        // steps of this lane's stream with a symbol: t < tn
        const int tn = n0 < N ? (int)((N - n0 + S - 1) / S) : 0;
        const int Ts = (int)T_steps;
        const uint8_t* lnext = lev + n0 + (int64_t)kRing * S;   // level of step t + kRing
        int32_t* op = out + n0;                                 // symbol of step t
        // levels of steps t .. t + kRing - 1 in registers, each loaded
        // kRing steps before it is used
        uint32_t lring[kRing];
#pragma unroll
        for (int k = 0; k < kRing; ++k) lring[k] = k < tn ? (uint32_t)__ldg(lev + n0 + (int64_t)k * S) : 0u;
        auto refill = [&](bool part) {
            const bool need = part && x < kL;
            const uint32_t m = __ballot_sync(kFull, need);
            const int c = __popc(m);
            const int i = rp - c + __popc(m & lt);
            const uint32_t w = ring[(bmod + i) & (kWRing - 1)];
            bad |= need && i < 0;
            x = need ? (x << 16) | (i >= 0 ? w : 0u) : x;
            rp -= c;
        };
        auto step = [&](int t, uint32_t& lslot) {
            const bool act = t < tn;
            const int lvl = (int)min(lslot, (uint32_t)(kLmax - 1));
            lslot = t + kRing < tn ? (uint32_t)__ldg(lnext) : 0u;
            lnext += S;
            // words: issue the next chunk once its slots are consumed; wait
            // only if this step could read below what has landed
            if (rp - rf <= kWRing - kWChunk && rf > 0) {
                rf -= kWChunk;
                wring_issue(ring, words, n_words, beg + rf, lane);
                ++pending;
            }
            if (rp - kWMaxStep < rready) {
                if (pending >= 2) {
                    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                    rready = rf + kWChunk;
                    pending = 1;
                }
                if (rp - kWMaxStep < rready) {
                    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                    rready = rf;
                    pending = 0;
                }
                __syncwarp();
            }
            // the bucket pair decides most slots; the row search runs only
            // for lanes whose bucket holds more than one boundary
            const uint32_t slot = x & 0xffffu;
            const uint2* bk = sbkt + lvl * kBktStride + (slot >> 8);
            const uint2 P = bk[0], Pn = bk[1];
            // clamped so that a blob that was never built still reads inside
            // its row
            int j0 = min((int)(P.x & 0xffffu), kRow - 2);
            int j1 = min(max((int)(Pn.x & 0xffffu) + 1, j0 + 1), kRow - 1);
            uint32_t qa = P.x >> 16, qb = Pn.y;
            const bool esc = act && slot >= qb;
            bool srch = act && !esc && j1 - j0 > 1;
            if (__any_sync(kFull, srch)) {
                const uint16_t* row = srow + lvl * kRow;
                while (srch) {
                    const int mid = (j0 + j1) >> 1;
                    const uint32_t qm = row[mid];
                    if (qm <= slot) { j0 = mid; qa = qm; }
                    else { j1 = mid; qb = qm; }
                    srch = j1 - j0 > 1;
                }
            }
            const uint32_t st = esc ? qb : qa;
            const uint32_t fr = esc ? kM - qb : qb - qa;
            const uint32_t xn = fr * (x >> 16) + slot - st;
            x = act ? xn : x;
            int32_t s = j0 - kYmax;
            refill(act);
            if (__any_sync(kFull, esc)) {
                uint32_t hi16 = 0, lo16 = 0;
                if (esc) { hi16 = x & 0xffffu; x >>= 16; }
                refill(esc);
                if (esc) { lo16 = x & 0xffffu; x >>= 16; }
                refill(esc);
                if (esc) s = (int32_t)((hi16 << 16) | lo16);
            }
            if (act) *op = s;
            op += S;
        };
        int t = 0;
        for (; t + kRing <= Ts; t += kRing) {
#pragma unroll
            for (int k = 0; k < kRing; ++k) step(t + k, lring[k]);
        }
#pragma unroll
        for (int k = 0; k < kRing; ++k)
            if (t + k < Ts) step(t + k, lring[k]);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // the ring is reused by the next segment
        __syncwarp();
        const bool fail = bad || x != kL || rp != 0;
        if (__ballot_sync(kFull, fail) && lane == 0) set_error(err, kErrCorrupt);
    }
}

template <typename T>
void launch_interval(const void* scales, int64_t N, const int32_t* sym, const unsigned char* blob, uint32_t* sf,
                     int32_t* err, int sms, cudaStream_t st)
{
    const int64_t blocks = (N + 255) / 256 < (int64_t)sms * 16 ? (N + 255) / 256 : (int64_t)sms * 16;
    fgmm_gsm_interval_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const T*>(scales), N, sym, blob, sf,
                                                                   err);
}

void launch_interval_any(int32_t dtype, const void* scales, int64_t N, const int32_t* sym, const unsigned char* blob,
                         uint32_t* sf, int32_t* err, int sms, cudaStream_t st)
{
    if (N == 0) return;
    if (dtype == FGMM_DTYPE_BF16) launch_interval<__nv_bfloat16>(scales, N, sym, blob, sf, err, sms, st);
    else launch_interval<float>(scales, N, sym, blob, sf, err, sms, st);
}

// Decoder grid: one CTA per SM at most (the staged tables take ~194 KB of
// shared memory), ceil(nseg / SMs) warps per CTA up to 32, warps looping
// over segments beyond that.
cudaError_t launch_dec(int32_t dtype, const void* scales, int64_t N, int32_t S, const unsigned char* blob,
                       uint8_t* lev, const uint16_t* words, int64_t n_words, const int64_t* offsets, int32_t* out,
                       int32_t* err, int sms, cudaStream_t st)
{
    if (N > 0) {
        const int64_t blocks = (N + 1023) / 1024 < (int64_t)sms * 16 ? (N + 1023) / 1024 : (int64_t)sms * 16;
        if (dtype == FGMM_DTYPE_BF16)
            fgmm_gsm_level_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(
                static_cast<const __nv_bfloat16*>(scales), N, blob, lev, err);
        else
            fgmm_gsm_level_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const float*>(scales), N,
                                                                            blob, lev, err);
    }
    const int64_t nseg = S / 32;
    int64_t wpb = (nseg + sms - 1) / sms;
    if (wpb > 32) wpb = 32;
    int64_t grid = (nseg + wpb - 1) / wpb;
    if (grid > sms) grid = sms;
    const size_t smem = kDecSmem + (size_t)wpb * kWRing * sizeof(uint16_t);
    cudaError_t e = cudaFuncSetAttribute(fgmm_gsm_dec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kDecSmem + 32 * kWRing * sizeof(uint16_t)));
    if (e != cudaSuccess) return e;
    fgmm_gsm_dec_kernel<<<(unsigned)grid, (unsigned)(wpb * 32), smem, st>>>(lev, N, S, steps_of(N, S), blob, words,
                                                                             n_words, offsets, nseg, out, err);
    return cudaGetLastError();
}

fgmm_status check_gsm(fgmm_handle* h, int32_t dtype, int64_t N, const void* scales, const void* tables)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (dtype != FGMM_DTYPE_F32 && dtype != FGMM_DTYPE_BF16)
        return fail(h, FGMM_ERR_INVALID_ARG, "dtype must be FGMM_DTYPE_F32 or FGMM_DTYPE_BF16");
    if (N < 0 || N > ((int64_t)1 << 40)) return fail(h, FGMM_ERR_INVALID_ARG, "N out of range");
    if (N > 0 && !scales) return fail(h, FGMM_ERR_INVALID_ARG, "scales is NULL");
    if (!tables || (reinterpret_cast<uintptr_t>(tables) & 15u) != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "tables must be a 16-byte aligned device pointer");
    return FGMM_OK;
}

}  // namespace

extern "C" {

int64_t fgmm_gsm_tables_bytes(void) { return (int64_t)kBlobBytes; }

void fgmm_gsm_default_levels(float* out)
{
    if (!out) return;
    const double a = std::log(0.11), b = std::log(256.0);
    for (int i = 0; i < kLmax; ++i) out[i] = (float)std::exp(a + (b - a) * (double)i / 63.0);
}

fgmm_status fgmm_gsm_build(fgmm_handle* h, const float* levels, int32_t L, void* tables, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (!levels || L < 1 || L > kLmax) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_gsm_build: need 1..64 levels");
    if (!tables || (reinterpret_cast<uintptr_t>(tables) & 15u) != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "tables must be a 16-byte aligned device pointer");
    GsmLevels p{};
    for (int i = 0; i < L; ++i) {
        if (!std::isfinite(levels[i]) || !(levels[i] > 0.0f) || (i > 0 && !(levels[i] > levels[i - 1])))
            return fail(h, FGMM_ERR_INVALID_ARG, "levels must be finite, > 0 and strictly increasing");
        p.lv[i] = levels[i];
    }
    p.L = L;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* blob = static_cast<unsigned char*>(tables);
    switch (h->phi) {
    case FGMM_PHI_LOGISTIC: fgmm_gsm_build_kernel<kPhiLogistic><<<L, 256, 0, st>>>(p, blob); break;
    case FGMM_PHI_POLYA: fgmm_gsm_build_kernel<kPhiPolya><<<L, 256, 0, st>>>(p, blob); break;
    default: fgmm_gsm_build_kernel<kPhiAS><<<L, 256, 0, st>>>(p, blob); break;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_gsm_build launch");
}

fgmm_status fgmm_gsm_freqs(fgmm_handle* h, int32_t dtype, int64_t N, const void* scales, const int32_t* symbols,
                           const void* tables, uint32_t* sf, void* stream)
{
    fgmm_status s = check_gsm(h, dtype, N, scales, tables);
    if (s != FGMM_OK) return s;
    if (N > 0 && (!symbols || !sf)) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_gsm_freqs: NULL buffer");
    launch_interval_any(dtype, scales, N, symbols, static_cast<const unsigned char*>(tables), sf, h->d_err,
                        h->num_sms, static_cast<cudaStream_t>(stream));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_gsm_freqs launch");
}

fgmm_status fgmm_gsm_encode(fgmm_handle* h, int32_t dtype, int64_t N, const void* scales, const int32_t* symbols,
                            int32_t S, const void* tables, uint16_t* words, int64_t words_cap, int64_t* offsets,
                            int64_t* n_words_out, void* stream)
{
    fgmm_status s = check_gsm(h, dtype, N, scales, tables);
    if (s != FGMM_OK) return s;
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || !n_words_out || words_cap < 0 || (words_cap > 0 && !words) || (N > 0 && !symbols))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_gsm_encode: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EncodeWs ws;
    s = encode_reserve(h, N, S, st, &ws);
    if (s != FGMM_OK) return s;
    launch_interval_any(dtype, scales, N, symbols, static_cast<const unsigned char*>(tables), ws.sf, h->d_err,
                        h->num_sms, st);
    encode_from_intervals(ws, symbols, N, S, words, words_cap, offsets, n_words_out, h->d_err, h->num_sms, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_gsm_encode launch");
}

fgmm_status fgmm_gsm_decode(fgmm_handle* h, int32_t dtype, int64_t N, const void* scales, const void* tables,
                            const uint16_t* words, int64_t n_words, const int64_t* offsets, int32_t S,
                            int32_t* symbols_out, void* stream)
{
    fgmm_status s = check_gsm(h, dtype, N, scales, tables);
    if (s != FGMM_OK) return s;
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || n_words < 0 || (n_words > 0 && !words) || (N > 0 && !symbols_out))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_gsm_decode: NULL buffer");
    if (n_words > 0 && (reinterpret_cast<uintptr_t>(words) & 7u) != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_gsm_decode: words must be 8-byte aligned");
    if (steps_of(N, S) >= ((int64_t)1 << 24))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_gsm_decode: at most 2^24 - 1 steps per stream");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // workspace: one level byte per symbol
    s = ws_reserve(h, (size_t)(N > 0 ? N : 1), st);
    if (s != FGMM_OK) return s;
    cudaError_t e = launch_dec(dtype, scales, N, S, static_cast<const unsigned char*>(tables),
                               static_cast<uint8_t*>(h->ws), words, n_words, offsets, symbols_out, h->d_err,
                               h->num_sms, st);
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_gsm_decode launch");
}

}  // extern "C"
