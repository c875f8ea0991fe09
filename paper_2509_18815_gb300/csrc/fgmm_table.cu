// fgmm_table.cu -- table-based GMM coder: the comparison for the table-free
// path. It is the algorithm of Sec. II-C (Eqs. 4-5): for every symbol, the
// quantised CDF is evaluated at every point of the alphabet, j in
// [-255, 256], into a table row (O(K |Y|) per symbol), and coding then looks
// intervals up in the table; decoding binary-searches the table row. The
// table holds the same quantised CDF as the on-the-fly coder (same window,
// escape and FP32 operation order), so both produce byte-identical streams.
//
// Table layout: uint16 [N][512], row n entry j + 255 = Q(clamp(j, lo, hi+1)).
// Q(hi+1) <= 65535 fits; entries left of the window are 0 and entries right
// of it repeat Q(hi+1). In-window symbols have row[s+256] > row[s+255]; any
// other value is an escape with interval [row[511], 2^16).
#include <cuda_runtime.h>

#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"

using namespace fgmm;

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kRow = 512;

// One block per row: 256 threads, two adjacent entries each (one 32-bit
// store). Every entry costs one mixture-CDF evaluation, the table approach's
// O(K |Y|) work per symbol.
template <int K, typename T>
__global__ void __launch_bounds__(256) fgmm_table_build_kernel(const T* __restrict__ params, int64_t N,
                                                               uint16_t* __restrict__ table, int32_t* err)
{
    for (int64_t n = blockIdx.x; n < N; n += gridDim.x) {
        Mix<K> m;
        const bool ok = load_mix<K>(params, N, n, m);
        if (!ok && threadIdx.x == 0) set_error(err, kErrBadParams);
        uint32_t q[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int j = -kYmax + 2 * (int)threadIdx.x + e;
            const int jc = j <= m.lo ? m.lo + 1 : (j > m.hi + 1 ? m.hi + 1 : j);
            const uint32_t v = q_at<K>(m, jc);
            q[e] = j <= m.lo ? 0u : v;
        }
        reinterpret_cast<uint32_t*>(table + n * kRow)[threadIdx.x] = q[0] | (q[1] << 16);
    }
}

// Intervals by table lookup.
__global__ void __launch_bounds__(256) fgmm_table_interval_kernel(const uint16_t* __restrict__ table, int64_t N,
                                                                  const int32_t* __restrict__ sym,
                                                                  uint32_t* __restrict__ sf)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const uint16_t* row = table + n * kRow;
        const int32_t s = __ldg(sym + n);
        if (s >= -kYmax && s <= kYmax) {
            const uint32_t a = __ldg(row + s + kYmax), b = __ldg(row + s + kYmax + 1);
            if (b > a) {
                sf[n] = a | ((b - a) << 16);
                continue;
            }
        }
        const uint32_t e = __ldg(row + kRow - 1);
        sf[n] = e | ((kM - e) << 16);
    }
}

// Decoder: binary search over the table row, one lane per stream.
__global__ void __launch_bounds__(32) fgmm_table_dec_kernel(const uint16_t* __restrict__ table, int64_t N,
                                                             int32_t S, int64_t T_steps,
                                                             const uint16_t* __restrict__ words, int64_t n_words,
                                                             const int64_t* __restrict__ offsets, int64_t nseg,
                                                             int32_t* __restrict__ out, int32_t* err)
{
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= nseg) return;
    const int64_t beg = offsets[g], end = offsets[g + 1];
    if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
        if (lane == 0) set_error(err, kErrCorrupt);
        return;
    }
    const uint32_t lt = lanemask_lt();
    uint32_t x = (uint32_t)__ldg(words + end - 64 + 2 * lane) | ((uint32_t)__ldg(words + end - 63 + 2 * lane) << 16);
    int64_t ptr = end - 64;
    bool bad = false;
    int64_t n = g * 32 + lane;
    for (int64_t t = 0; t < T_steps; ++t, n += S) {
        const bool act = n < N;
        int32_t s = 0;
        bool esc = false;
        if (act) {
            const uint16_t* row = table + n * kRow;
            const uint32_t slot = x & 0xffffu;
            const uint32_t e = __ldg(row + kRow - 1);
            uint32_t start, freq;
            if (slot >= e) {
                esc = true;
                start = e;
                freq = kM - e;
            } else {
                int a = 0, b = kRow - 1;   // row[0] = Q(lo) = 0 <= slot < row[511]
                uint32_t qa = 0, qb = e;
                while (b - a > 1) {
                    const int mid = (a + b) >> 1;
                    const uint32_t qm = __ldg(row + mid);
                    if (qm <= slot) { a = mid; qa = qm; }
                    else { b = mid; qb = qm; }
                }
                s = a - kYmax;
                start = qa;
                freq = qb - qa;
            }
            x = freq * (x >> 16) + slot - start;
        }
        refill_warp(x, act, words, ptr, beg, bad, lt);
        if (__ballot_sync(kFull, esc)) {
            uint32_t hi16 = 0, lo16 = 0;
            if (esc) { hi16 = x & 0xffffu; x >>= 16; }
            refill_warp(x, esc, words, ptr, beg, bad, lt);
            if (esc) { lo16 = x & 0xffffu; x >>= 16; }
            refill_warp(x, esc, words, ptr, beg, bad, lt);
            if (esc) s = (int32_t)((hi16 << 16) | lo16);
        }
        if (act) out[n] = s;
    }
    const bool fail = bad || x != kL || ptr != beg;
    if (__ballot_sync(kFull, fail) && lane == 0) set_error(err, kErrCorrupt);
}

template <int K, typename T>
void launch_build_kt(const fgmm_latent* lat, uint16_t* table, int32_t* err, int sms, cudaStream_t st)
{
    const int64_t blocks = lat->N < (int64_t)sms * 64 ? lat->N : (int64_t)sms * 64;
    fgmm_table_build_kernel<K, T><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const T*>(lat->params), lat->N, table,
                                                                    err);
}

template <typename T>
void launch_build_t(const fgmm_latent* lat, uint16_t* table, int32_t* err, int sms, cudaStream_t st)
{
    switch (lat->K) {
    case 1: launch_build_kt<1, T>(lat, table, err, sms, st); break;
    case 2: launch_build_kt<2, T>(lat, table, err, sms, st); break;
    case 3: launch_build_kt<3, T>(lat, table, err, sms, st); break;
    default: launch_build_kt<4, T>(lat, table, err, sms, st); break;
    }
}

void launch_build(const fgmm_latent* lat, uint16_t* table, int32_t* err, int sms, cudaStream_t st)
{
    if (lat->N == 0) return;
    if (lat->dtype == FGMM_DTYPE_BF16) launch_build_t<__nv_bfloat16>(lat, table, err, sms, st);
    else launch_build_t<float>(lat, table, err, sms, st);
}

}  // namespace

extern "C" {

int64_t fgmm_table_bytes(int64_t N)
{
    if (N < 0) return -1;
    return N * kRow * (int64_t)sizeof(uint16_t);
}

fgmm_status fgmm_table_build(fgmm_handle* h, const fgmm_latent* lat, uint16_t* table, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (h->phi != FGMM_PHI_AS) return fail(h, FGMM_ERR_INVALID_ARG, "the table coder takes FGMM_PHI_AS only");
    if (lat->N > 0 && !table) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_table_build: NULL table");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    launch_build(lat, table, h->d_err, h->num_sms, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_table_build launch");
}

fgmm_status fgmm_table_encode(fgmm_handle* h, const fgmm_latent* lat, const int32_t* symbols, int32_t S,
                              uint16_t* table, uint16_t* words, int64_t words_cap, int64_t* offsets,
                              int64_t* n_words_out, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (h->phi != FGMM_PHI_AS) return fail(h, FGMM_ERR_INVALID_ARG, "the table coder takes FGMM_PHI_AS only");
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || !n_words_out || words_cap < 0 || (words_cap > 0 && !words) ||
        (lat->N > 0 && (!symbols || !table)))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_table_encode: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EncodeWs ws;
    s = encode_reserve(h, lat->N, S, st, &ws);
    if (s != FGMM_OK) return s;
    launch_build(lat, table, h->d_err, h->num_sms, st);
    if (lat->N > 0) {
        const int64_t blocks = (lat->N + 255) / 256 < (int64_t)h->num_sms * 16 ? (lat->N + 255) / 256
                                                                               : (int64_t)h->num_sms * 16;
        fgmm_table_interval_kernel<<<(unsigned)blocks, 256, 0, st>>>(table, lat->N, symbols, ws.sf);
    }
    encode_from_intervals(ws, symbols, lat->N, S, words, words_cap, offsets, n_words_out, h->d_err, h->num_sms, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_table_encode launch");
}

fgmm_status fgmm_table_decode(fgmm_handle* h, const fgmm_latent* lat, uint16_t* table, const uint16_t* words,
                              int64_t n_words, const int64_t* offsets, int32_t S, int32_t* symbols_out, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (h->phi != FGMM_PHI_AS) return fail(h, FGMM_ERR_INVALID_ARG, "the table coder takes FGMM_PHI_AS only");
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || n_words < 0 || (n_words > 0 && !words) || (lat->N > 0 && (!symbols_out || !table)))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_table_decode: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    launch_build(lat, table, h->d_err, h->num_sms, st);
    const int64_t nseg = S / 32;
    const int64_t blocks = nseg;
    fgmm_table_dec_kernel<<<(unsigned)blocks, 32, 0, st>>>(table, lat->N, S, steps_of(lat->N, S), words, n_words,
                                                            offsets, nseg, symbols_out, h->d_err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_table_decode launch");
}

}  // extern "C"
