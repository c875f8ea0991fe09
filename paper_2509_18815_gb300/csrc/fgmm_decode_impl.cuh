// fgmm_decode_impl.cuh -- decoder kernels (included by the fp32 and bf16
// instantiation units fgmm_decode.cu and fgmm_decode_bf16.cu).
//
// Decoders: binary search over the on-the-fly quantised
// CDF (Sec. III-A), inverse rANS step (Eq. 3), ballot-ranked refill.
//
// Two kernels produce identical symbols (the search result is unique
// because Q is strictly increasing); they differ in how the search is
// spread over lanes:
//
// * fgmm_dec_kernel (G = 1): one lane per stream, 32 streams (a segment) per
//   warp, plain binary search (one CDF evaluation per round). Least work per
//   symbol; the choice when there are enough segments to fill the GPU. The
//   next step's parameters are loaded one step ahead into registers.
//
// * fgmm_dec_ws_kernel (G = 8, 16 or 32, clusters of 2-8 CTAs; its own
//   units, fgmm_decode_ws.cuh): consumer warps run the state-dependent
//   chain; producer warps prepare the mixture and the first search round two
//   steps ahead.
//
// * fgmm_dec_coop_kernel (G = 2 .. 16): G lanes cooperate on one stream and
//   evaluate G points of the quantised CDF per round (G-ary search), so a
//   step needs ~log_{G+1}(W) dependent rounds instead of ~log_2(W). A CTA of
//   G warps holds one segment; parameters are staged through a cp.async ring
//   in shared memory PF steps ahead, the segment's words are copied to
//   shared memory when they fit, and the refill ranks of the 32 streams are
//   combined through shared memory with one CTA barrier per step. The choice
//   when the streams alone cannot fill the GPU (few streams, long streams).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"
#include "fgmm_segment.cuh"

using namespace fgmm;

namespace {

constexpr uint32_t kFull = 0xffffffffu;

// Q(j) <= slot for lo < j <= hi + 1, decided on the fast steering
// evaluation of the CDF (thr = slot + 1); see search_slot_guided.
template <int K>
__device__ __forceinline__ bool fast_le(const Mix<K>& m, int j, float thr)
{
    const float v = fminf(mix_cdf_fast<K>(m, (float)j - 0.5f), 1.0f);
    return fmaf(m.tp, v, (float)(j - m.lo)) < thr;
}

// ---------------------------------------------------------------------------
// G = 1: binary search, one lane per stream.
// ---------------------------------------------------------------------------
template <int K, typename T, int PHI>
__global__ void __launch_bounds__(32) fgmm_dec_kernel(const T* __restrict__ params, int64_t N, int32_t S,
                                                       int64_t T_steps, const uint16_t* __restrict__ words,
                                                       int64_t n_words, const int64_t* __restrict__ offsets,
                                                       int64_t nseg, int32_t* __restrict__ out, int32_t* err,
                                                       unsigned long long* stats)
{
    const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (g >= nseg) return;
    const int64_t beg = offsets[g], end = offsets[g + 1];
    if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
        if ((threadIdx.x & 31) == 0) set_error(err, kErrCorrupt);
        return;
    }
    dec_segment<K, T, PHI>(params, N, S, T_steps, g, words, beg, end, out, err, stats);
}

// ---------------------------------------------------------------------------
// G = 2 .. 32: cooperative G-ary search, one CTA of G warps per segment.
// ---------------------------------------------------------------------------
constexpr int kPF = 4;            // parameter prefetch distance (steps)
constexpr int kRing = 8;          // ring slots (>= kPF + 2, power of two)
constexpr int kWordCap = 16384;   // segment words staged in shared memory if they fit

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem, int src_bytes)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem, int src_bytes)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(n)); }

// Copies step t's parameters of COLS consecutive streams (3K rows x COLS
// symbols) into ring slot `dst` ([3K][COLS] of T). Elements at n >= N are zero-filled and
// never read from global memory. mode 2: 16-byte cp.async (rows 16-byte
// aligned); mode 1: 4-byte cp.async (rows 4-byte aligned); mode 0: plain
// loads and shared stores (any alignment), visible after the next barrier.
template <int K, typename T, int COLS>
__device__ __forceinline__ void stage_params(T* dst, const T* __restrict__ params, int64_t N, int64_t n0, int tid,
                                             int nthreads, int mode)
{
    if (mode == 2) {
        constexpr int per_chunk = 16 / (int)sizeof(T);
        constexpr int chunks_per_row = COLS / per_chunk > 0 ? COLS / per_chunk : 1;
        constexpr int total = 3 * K * chunks_per_row;
        for (int c = tid; c < total; c += nthreads) {
            const int row = c / chunks_per_row, col = (c % chunks_per_row) * per_chunk;
            const int64_t n = n0 + col;
            int64_t valid = N - n;
            valid = valid < 0 ? 0 : (valid > per_chunk ? per_chunk : valid);
            const T* src = valid > 0 ? params + (int64_t)row * N + n : params;
            cp_async_16(dst + row * COLS + col, src, (int)(valid * sizeof(T)));
        }
    } else if (mode == 1) {
        constexpr int per_chunk = 4 / (int)sizeof(T);
        constexpr int chunks_per_row = COLS / per_chunk;
        constexpr int total = 3 * K * chunks_per_row;
        for (int c = tid; c < total; c += nthreads) {
            const int row = c / chunks_per_row, col = (c % chunks_per_row) * per_chunk;
            const int64_t n = n0 + col;
            int64_t valid = N - n;
            valid = valid < 0 ? 0 : (valid > per_chunk ? per_chunk : valid);
            const T* src = valid > 0 ? params + (int64_t)row * N + n : params;
            cp_async_4(dst + row * COLS + col, src, (int)(valid * sizeof(T)));
        }
    } else {
        constexpr int total = 3 * K * COLS;
        for (int c = tid; c < total; c += nthreads) {
            const int row = c / COLS, col = c % COLS;
            const int64_t n = n0 + col;
            dst[row * COLS + col] = n < N ? params[(int64_t)row * N + n] : T(0.0f);
        }
    }
}

template <typename T>
__device__ __forceinline__ float smem_param(const T* p);
template <>
__device__ __forceinline__ float smem_param<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float smem_param<__nv_bfloat16>(const __nv_bfloat16* p)
{
    return __uint_as_float((uint32_t)(*reinterpret_cast<const unsigned short*>(p)) << 16);
}

// Barrier over the CTAs that share a segment: the CTA itself (CL = 1) or
// the thread-block cluster (CL > 1, release/acquire at cluster scope).
template <int CL>
__device__ __forceinline__ void seg_sync()
{
    if constexpr (CL == 1) {
        __syncthreads();
    } else {
        asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    }
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Stores v at `local` in the shared memory of every CTA of the cluster.
template <int CL>
__device__ __forceinline__ void publish(uint32_t* local, uint32_t v)
{
    if constexpr (CL == 1) {
        *local = v;
    } else {
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
#pragma unroll
        for (uint32_t r = 0; r < (uint32_t)CL; ++r) {
            uint32_t ra;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
            asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
        }
    }
}

// Segment-wide refill for one sub-phase. need: this stream needs a word.
// Each of the segment's G warps publishes the need bits of its 32/G streams;
// after the barrier every thread forms the segment's 32-bit mask and the
// stream's rank.
template <int G, int CL>
__device__ __forceinline__ void refill_coop(uint32_t& x, bool need, uint32_t* pub, int wseg, int grp, int sub,
                                            const uint16_t* wsrc, int64_t wbase, int64_t& ptr, int64_t beg,
                                            bool& bad)
{
    constexpr int SPW = 32 / G;    // streams per warp
    const uint32_t b = __ballot_sync(kFull, need && sub == 0);
    uint32_t part = 0;
#pragma unroll
    for (int i = 0; i < SPW; ++i) part |= ((b >> (i * G)) & 1u) << i;
    if ((threadIdx.x & 31) == 0) publish<CL>(pub + wseg, part);
    seg_sync<CL>();
    uint32_t M = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) M |= pub[i] << (i * SPW);
    if (M) {
        const int w = wseg * SPW + grp;   // stream index within the segment
        const int c = __popc(M);
        if (need) {
            const int64_t idx = ptr - c + __popc(M & ((1u << w) - 1u));
            uint32_t v = 0;
            if (idx >= beg) v = wsrc[idx - wbase];
            else bad = true;
            x = (x << 16) | v;
        }
        ptr -= c;
    }
}

// One segment per CL CTAs (a cluster when CL > 1); each CTA holds 32/CL
// streams, G lanes per stream, G/CL warps.
template <int K, typename T, int G, int CL>
__global__ void __launch_bounds__(32 * G / CL) fgmm_dec_coop_kernel(const T* __restrict__ params, int64_t N,
                                                                    int32_t S, int64_t T_steps,
                                                                    const uint16_t* __restrict__ words,
                                                                    int64_t n_words,
                                                                    const int64_t* __restrict__ offsets,
                                                                    int32_t* __restrict__ out, int32_t* err,
                                                                    unsigned long long* stats, int mode)
{
    constexpr int SPW = 32 / G;        // streams per warp
    constexpr int SPC = 32 / CL;       // streams per CTA
    constexpr int WPC = G / CL;        // warps per CTA
    constexpr int NT = 32 * WPC;
    extern __shared__ __align__(16) unsigned char smem[];
    T* ring = reinterpret_cast<T*>(smem);                                              // [kRing][3K][SPC]
    uint32_t* pubs = reinterpret_cast<uint32_t*>(smem + sizeof(T) * kRing * 3 * K * SPC);   // [6][G]
    uint16_t* wsm = reinterpret_cast<uint16_t*>(pubs + 6 * G);                         // [kWordCap]

    const int rank = CL > 1 ? (int)cluster_rank() : 0;
    const int tid = threadIdx.x, lane = tid & 31, grp = lane / G, sub = lane % G;
    const int wseg = rank * WPC + (tid >> 5);          // warp index within the segment
    const int wstream = wseg * SPW + grp;              // stream index within the segment
    const int wcol = wstream - rank * SPC;             // column in this CTA's parameter slots
    const int64_t g = blockIdx.x / CL;
    const int64_t beg = offsets[g], end = offsets[g + 1];
    if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
        if (tid == 0 && rank == 0) set_error(err, kErrCorrupt);
        return;   // uniform over the segment's CTAs, before any barrier
    }
    const int64_t seg_len = end - beg;
    const bool staged = seg_len <= kWordCap;
    const uint16_t* wsrc = staged ? wsm : words;
    const int64_t wbase = staged ? beg : 0;

    // prologue: parameters of steps 0 .. PF-1, then the segment's words
    const int64_t nbase = g * 32 + rank * SPC;
#pragma unroll
    for (int p = 0; p < kPF; ++p) {
        if (p < T_steps)
            stage_params<K, T, SPC>(ring + (p % kRing) * 3 * K * SPC, params, N, p * (int64_t)S + nbase, tid, NT, mode);
        cp_async_commit();
    }
    if (staged)
        for (int64_t i = tid; i < seg_len; i += NT) wsm[i] = __ldg(words + beg + i);
    cp_async_wait<kPF - 1>();
    seg_sync<CL>();   // all CTAs of the cluster are running before any remote store

    uint32_t x = (uint32_t)wsrc[end - 64 + 2 * wstream - wbase] | ((uint32_t)wsrc[end - 63 + 2 * wstream - wbase] << 16);
    int64_t ptr = end - 64;
    bool bad = false, badp = false;
    int probes = 0, decoded = 0;
    const unsigned gshift = grp * G;

    for (int64_t t = 0; t < T_steps; ++t) {
        // prefetch step t + PF into its ring slot (the slot of step t + PF - kRing,
        // read before the previous barrier)
        if (t + kPF < T_steps)
            stage_params<K, T, SPC>(ring + ((t + kPF) % kRing) * 3 * K * SPC, params, N,
                                    (t + kPF) * (int64_t)S + nbase, tid, NT, mode);
        cp_async_commit();

        const int64_t n = t * (int64_t)S + g * 32 + wstream;
        const bool act = n < N;
        int32_t s = 0;
        bool esc = false;
        uint32_t start = 0, freq = 1;
        Mix<K> m;
        {
            const T* slot_p = ring + (t % kRing) * 3 * K * SPC;
            RawParams<K> r;
#pragma unroll
            for (int i = 0; i < 3 * K; ++i) r.v[i] = smem_param<T>(slot_p + i * SPC + wcol);
            const bool ok = mix_from_params<K>(r, m);
            badp |= act && !ok;
        }
        const uint32_t slot = x & 0xffffu;
        const uint32_t gm = (G == 32) ? kFull : ((1u << G) - 1u);
        const int W = m.hi - m.lo + 1;
        // G-ary search over [lo, hi + 2) steered by the fast evaluation of
        // the CDF (fast_le); Q(hi + 2) = 2^16 is never evaluated. Round 0:
        // G points p_i = lo + ceil((i+1) W / G), p_{G-1} = hi + 1.
        const float thr = (float)(slot + 1u);
        int a = m.lo, b = m.hi + 2;
        {
            const int p = m.lo + ((sub + 1) * W + G - 1) / G;
            const bool le = act && fast_le<K>(m, p, thr);
            probes += act;
            const int c = __popc((__ballot_sync(kFull, le) >> gshift) & gm);
            if (c > 0) a = m.lo + (c * W + G - 1) / G;
            if (c < G) b = m.lo + ((c + 1) * W + G - 1) / G;
        }
        // further rounds: G points strictly inside (a, b)
        while (__any_sync(kFull, act && b - a > 1)) {
            const bool live = act && b - a > 1;
            const int L = b - a;
            const bool fine = L - 1 <= G;
            const int p = fine ? a + 1 + sub : a + ((sub + 1) * L) / (G + 1);
            const bool valid = live && (fine ? sub < L - 1 : true);
            const bool le = valid && fast_le<K>(m, p, thr);
            probes += valid;
            const int c = __popc((__ballot_sync(kFull, le) >> gshift) & gm);
            const int nvalid = fine ? min(L - 1, G) : G;
            if (live) {
                const int na = c > 0 ? (fine ? a + c : a + (c * L) / (G + 1)) : a;
                if (c < nvalid) b = fine ? a + 1 + c : a + ((c + 1) * L) / (G + 1);
                a = na;
            }
        }
        // exact check: lane 0 of the group evaluates Q(a), lane 1 Q(a + 1)
        // (Q(lo) = 0 and Q(hi + 2) = 2^16 need no evaluation), together
        uint32_t qa, qb;
        {
            const int jv = sub == 1 ? a + 1 : a;
            uint32_t qv = jv <= m.lo ? 0u : kM;
            if (act && sub < 2 && jv > m.lo && jv <= m.hi + 1) qv = q_at<K>(m, jv);
            qa = __shfl_sync(kFull, qv, grp * G);
            qb = __shfl_sync(kFull, qv, grp * G + 1);
        }
        bool ok = !act || (qa <= slot && slot < qb);
        if (__any_sync(kFull, !ok)) {
            // a near-tie the fast evaluation decided the other way: the exact
            // G-ary search over [lo, hi + 2) for the streams concerned
            const bool redo = !ok;
            int ea = m.lo, eb = m.hi + 2;
            uint32_t eqa = 0, eqb = kM;
            while (__any_sync(kFull, redo && eb - ea > 1)) {
                const bool live = redo && eb - ea > 1;
                const int L = eb - ea;
                const bool fine = L - 1 <= G;
                const int p = fine ? ea + 1 + sub : ea + ((sub + 1) * L) / (G + 1);
                const bool valid = live && (fine ? sub < L - 1 : true);
                const uint32_t q = valid ? q_at<K>(m, p) : 0u;
                const int c = __popc((__ballot_sync(kFull, valid && q <= slot) >> gshift) & gm);
                const uint32_t q_c = __shfl_sync(kFull, q, grp * G + (c < G ? c : G - 1));
                const uint32_t q_c1 = __shfl_sync(kFull, q, grp * G + (c > 0 ? c - 1 : 0));
                const int nvalid = fine ? min(L - 1, G) : G;
                if (live) {
                    const int na = c > 0 ? (fine ? ea + c : ea + (c * L) / (G + 1)) : ea;
                    const uint32_t nqa = c > 0 ? q_c1 : eqa;
                    if (c < nvalid) { eb = fine ? ea + 1 + c : ea + ((c + 1) * L) / (G + 1); eqb = q_c; }
                    ea = na;
                    eqa = nqa;
                }
            }
            if (redo) { a = ea; qa = eqa; qb = eqb; }
        }
        if (act) {
            s = a;
            esc = a == m.hi + 1;
            start = qa;
            freq = qb - qa;
        }
        if (act) {
            x = freq * (x >> 16) + slot - start;
            decoded += (sub == 0);
        }
        // wait for step t+1's parameters before the barrier that publishes them
        cp_async_wait<kPF - 1>();
        const int par = (int)(t & 1);
        // publish the escape bits with the refill bits
        const uint32_t be = __ballot_sync(kFull, act && esc && sub == 0);
        uint32_t epart = 0;
#pragma unroll
        for (int i = 0; i < SPW; ++i) epart |= ((be >> (i * G)) & 1u) << i;
        if (lane == 0) publish<CL>(pubs + (2 + par) * G + wseg, epart);
        refill_coop<G, CL>(x, act && x < kL, pubs + par * G, wseg, grp, sub, wsrc, wbase, ptr, beg, bad);
        uint32_t E = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) E |= pubs[(2 + par) * G + i] << (i * SPW);
        if (E) {   // uniform over the segment's CTAs
            uint32_t hi16 = 0, lo16 = 0;
            if (esc) { hi16 = x & 0xffffu; x >>= 16; }
            refill_coop<G, CL>(x, esc && x < kL, pubs + 4 * G, wseg, grp, sub, wsrc, wbase, ptr, beg, bad);
            if (esc) { lo16 = x & 0xffffu; x >>= 16; }
            refill_coop<G, CL>(x, esc && x < kL, pubs + 5 * G, wseg, grp, sub, wsrc, wbase, ptr, beg, bad);
            if (esc) s = (int32_t)((hi16 << 16) | lo16);
            seg_sync<CL>();   // escape buffers are reused by the next escape step
        }
        if (act && sub == 0) out[n] = s;
    }
    cp_async_wait<0>();
    const bool fail = bad || x != kL || ptr != beg;
    if (__syncthreads_or(fail) && tid == 0) set_error(err, kErrCorrupt);
    if (__syncthreads_or(badp) && tid == 0) set_error(err, kErrBadParams);
    if (stats) {
        int p = probes, d = decoded;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(kFull, p, o);
            d += __shfl_xor_sync(kFull, d, o);
        }
        if (lane == 0) {
            atomicAdd(stats, (unsigned long long)p);
            atomicAdd(stats + 1, (unsigned long long)d);
        }
    }
    seg_sync<CL>();   // no CTA leaves while another may still address its shared memory
}

// Warp-specialised decoder (fgmm_decode_ws.cuh), compiled in its own units.
template <typename T>
cudaError_t launch_ws_any(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st)
{
    if constexpr (sizeof(T) == 2) return launch_ws_bf16(a, K, CL, SPW, st);
    else return launch_ws_f32(a, K, CL, SPW, st);
}


template <int K, typename T, int G, int CL>
cudaError_t launch_coop(const DecodeArgs& a, cudaStream_t st)
{
    constexpr int SPC = 32 / CL;
    const size_t smem = sizeof(T) * kRing * 3 * K * SPC + sizeof(uint32_t) * 6 * G + sizeof(uint16_t) * kWordCap;
    auto kern = fgmm_dec_coop_kernel<K, T, G, CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // copy mode: rows start at params + r * N (elements), so the row
    // alignment follows from the base pointer and N
    const uintptr_t base = reinterpret_cast<uintptr_t>(a.params);
    int mode = 0;
    if (base % 16 == 0 && (a.N * (int64_t)sizeof(T)) % 16 == 0 && SPC * sizeof(T) >= 16) mode = 2;
    else if (base % 4 == 0 && (a.N * (int64_t)sizeof(T)) % 4 == 0) mode = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.nseg * CL));
    cfg.blockDim = dim3(32 * G / CL);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = CL > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const T*>(a.params), a.N, a.S, a.T, a.words, a.n_words,
                              a.offsets, a.out, a.err, a.stats, mode);
}

template <int K, typename T, int G>
cudaError_t launch_coop_cl(const DecodeArgs& a, int CL, cudaStream_t st)
{
    if constexpr (G >= 4) {
        if (CL == 4) return launch_coop<K, T, G, 4>(a, st);
    }
    if constexpr (G >= 2) {
        if (CL == 2) return launch_coop<K, T, G, 2>(a, st);
    }
    return launch_coop<K, T, G, 1>(a, st);
}

template <int K, typename T>
cudaError_t launch_k(const DecodeArgs& a, int G, int CL, cudaStream_t st)
{
    switch (G) {
    case 2: return launch_coop_cl<K, T, 2>(a, CL, st);
    case 4: return launch_coop_cl<K, T, 4>(a, CL, st);
    case 8: return CL >= 2 ? launch_ws_any<T>(a, K, CL, 4, st) : launch_coop_cl<K, T, 8>(a, 1, st);
    case 16: return CL >= 2 ? launch_ws_any<T>(a, K, CL, 2, st) : launch_coop_cl<K, T, 16>(a, 1, st);
    case 32: return launch_ws_any<T>(a, K, CL < 2 ? 2 : CL, 1, st);
    default: {
        const int threads = 32;   // one warp (segment) per block: segments spread over all SMs
        const int64_t blocks = (a.nseg * 32 + threads - 1) / threads;
        auto kern = a.phi == kPhiLogistic ? fgmm_dec_kernel<K, T, kPhiLogistic>
                    : (a.phi == kPhiPolya ? fgmm_dec_kernel<K, T, kPhiPolya> : fgmm_dec_kernel<K, T, kPhiAS>);
        kern<<<(unsigned)blocks, threads, 0, st>>>(static_cast<const T*>(a.params), a.N, a.S, a.T, a.words, a.n_words,
                                                   a.offsets, a.nseg, a.out, a.err, a.stats);
        return cudaGetLastError();
    }
    }
}

template <typename T>
cudaError_t launch_t(const DecodeArgs& a, int K, int G, int CL, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_k<1, T>(a, G, CL, st);
    case 2: return launch_k<2, T>(a, G, CL, st);
    case 3: return launch_k<3, T>(a, G, CL, st);
    default: return launch_k<4, T>(a, G, CL, st);
    }
}

}  // namespace

// Launch entry for one parameter type (defined in the instantiation units).
template <typename T>
cudaError_t launch_decode_t(const DecodeArgs& a, int K, int G, int CL, cudaStream_t st)
{
    return launch_t<T>(a, K, G, CL, st);
}
