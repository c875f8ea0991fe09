// fgmm_batch.cu -- many latents of uneven sizes in one persistent launch.
//
// A batch plan binds n latents (parameters, symbols, output buffers) and
// their stream counts S_i (given, or chosen by fgmm_autotune). All segments
// of all latents form one work list, ordered longest first; a persistent
// grid of warps pulls segments from an atomic counter (no inter-CTA waits)
// and codes each with the one-warp segment coder of fgmm_segment.cuh:
//   encode: one persistent launch of the fused encoder (quantised-CDF
//           interval inline, then rANS), then the offset scan and the
//           compaction over all segments;
//   decode: one persistent launch of the binary-search decoder.
// The launch sequence of each direction can be captured once into a CUDA
// graph and replayed. Latent i's stream is words[offsets[b_i] ..
// offsets[b_i + S_i/32]) with b_i its first segment, byte-identical to
// fgmm_encode of that latent alone with S_i streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"
#include "fgmm_segment.cuh"

using namespace fgmm;

namespace {

using WorkItem = BatchWorkItem;

constexpr int kBatchThreads = 32;        // one warp per block: warps spread over all SMs
constexpr int kTargetWarpsPerSM = 16;    // enough resident warps to keep the issue slots busy

template <int K, typename T>
__device__ __forceinline__ void enc_item(const BatchLatentDev& L, int32_t g, uint16_t* scratch, int64_t* len,
                                         int32_t* err)
{
    enc_segment_fused<K, T>(static_cast<const T*>(L.params), L.N, L.S, L.T, g, L.symbols,
                            scratch + L.scr_base + (int64_t)g * L.scr_cap, len + L.seg_base + g, err);
}

template <typename T>
__device__ __forceinline__ void enc_item_t(const BatchLatentDev& L, int32_t g, uint16_t* scratch, int64_t* len,
                                           int32_t* err)
{
    switch (L.K) {
    case 1: enc_item<1, T>(L, g, scratch, len, err); break;
    case 2: enc_item<2, T>(L, g, scratch, len, err); break;
    case 3: enc_item<3, T>(L, g, scratch, len, err); break;
    default: enc_item<4, T>(L, g, scratch, len, err); break;
    }
}

__global__ void __launch_bounds__(kBatchThreads) fgmm_batch_enc_kernel(const BatchLatentDev* __restrict__ lats,
                                                                       const WorkItem* __restrict__ work,
                                                                       int64_t nwork, unsigned long long* counter,
                                                                       uint16_t* __restrict__ scratch,
                                                                       int64_t* __restrict__ len, int32_t* err)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(counter, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= (unsigned long long)nwork) break;
        const WorkItem w = work[i];
        const BatchLatentDev L = lats[w.latent];
        if (L.dtype == FGMM_DTYPE_BF16) enc_item_t<__nv_bfloat16>(L, w.g, scratch, len, err);
        else enc_item_t<float>(L, w.g, scratch, len, err);
    }
}

template <int K, typename T>
__device__ __forceinline__ void dec_item(const BatchLatentDev& L, int32_t g, const uint16_t* words, int64_t n_words,
                                         const int64_t* offsets, int32_t* err, unsigned long long* stats)
{
    const int64_t gg = L.seg_base + g;
    const int64_t beg = offsets[gg], end = offsets[gg + 1];
    if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
        if ((threadIdx.x & 31) == 0) set_error(err, kErrCorrupt);
        return;
    }
    dec_segment<K, T>(static_cast<const T*>(L.params), L.N, L.S, L.T, g, words, beg, end, L.decoded, err, stats);
}

template <typename T>
__device__ __forceinline__ void dec_item_t(const BatchLatentDev& L, int32_t g, const uint16_t* words, int64_t n_words,
                                           const int64_t* offsets, int32_t* err, unsigned long long* stats)
{
    switch (L.K) {
    case 1: dec_item<1, T>(L, g, words, n_words, offsets, err, stats); break;
    case 2: dec_item<2, T>(L, g, words, n_words, offsets, err, stats); break;
    case 3: dec_item<3, T>(L, g, words, n_words, offsets, err, stats); break;
    default: dec_item<4, T>(L, g, words, n_words, offsets, err, stats); break;
    }
}

__global__ void __launch_bounds__(kBatchThreads) fgmm_batch_dec_kernel(const BatchLatentDev* __restrict__ lats,
                                                                       const WorkItem* __restrict__ work,
                                                                       int64_t nwork, unsigned long long* counter,
                                                                       const uint16_t* __restrict__ words,
                                                                       int64_t n_words,
                                                                       const int64_t* __restrict__ offsets,
                                                                       int32_t* err, unsigned long long* stats)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(counter, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= (unsigned long long)nwork) break;
        const WorkItem w = work[i];
        const BatchLatentDev L = lats[w.latent];
        if (L.dtype == FGMM_DTYPE_BF16) dec_item_t<__nv_bfloat16>(L, w.g, words, n_words, offsets, err, stats);
        else dec_item_t<float>(L, w.g, words, n_words, offsets, err, stats);
    }
}

// Specialised persistent kernels for batches whose latents share K and the
// parameter type (fewer registers than the mixed kernels above).
template <int K, typename T>
__global__ void __launch_bounds__(kBatchThreads) fgmm_batch_enc_kt_kernel(const BatchLatentDev* __restrict__ lats,
                                                                          const WorkItem* __restrict__ work,
                                                                          int64_t nwork, unsigned long long* counter,
                                                                          uint16_t* __restrict__ scratch,
                                                                          int64_t* __restrict__ len, int32_t* err)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(counter, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= (unsigned long long)nwork) break;
        const WorkItem w = work[i];
        enc_item<K, T>(lats[w.latent], w.g, scratch, len, err);
    }
}

template <int K, typename T>
__global__ void __launch_bounds__(kBatchThreads) fgmm_batch_dec_kt_kernel(const BatchLatentDev* __restrict__ lats,
                                                                          const WorkItem* __restrict__ work,
                                                                          int64_t nwork, unsigned long long* counter,
                                                                          const uint16_t* __restrict__ words,
                                                                          int64_t n_words,
                                                                          const int64_t* __restrict__ offsets,
                                                                          int32_t* err, unsigned long long* stats)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(counter, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= (unsigned long long)nwork) break;
        const WorkItem w = work[i];
        dec_item<K, T>(lats[w.latent], w.g, words, n_words, offsets, err, stats);
    }
}

using EncKernel = void (*)(const BatchLatentDev*, const WorkItem*, int64_t, unsigned long long*, uint16_t*, int64_t*,
                           int32_t*);
using DecKernel = void (*)(const BatchLatentDev*, const WorkItem*, int64_t, unsigned long long*, const uint16_t*,
                           int64_t, const int64_t*, int32_t*, unsigned long long*);

template <typename T>
void pick_kt(int K, EncKernel* e, DecKernel* d)
{
    switch (K) {
    case 1: *e = fgmm_batch_enc_kt_kernel<1, T>; *d = fgmm_batch_dec_kt_kernel<1, T>; break;
    case 2: *e = fgmm_batch_enc_kt_kernel<2, T>; *d = fgmm_batch_dec_kt_kernel<2, T>; break;
    case 3: *e = fgmm_batch_enc_kt_kernel<3, T>; *d = fgmm_batch_dec_kt_kernel<3, T>; break;
    default: *e = fgmm_batch_enc_kt_kernel<4, T>; *d = fgmm_batch_dec_kt_kernel<4, T>; break;
    }
}

// Kernels for a batch: specialised when all latents share K and dtype.
void pick_kernels(const std::vector<int>& Ks, const std::vector<int>& dts, EncKernel* e, DecKernel* d)
{
    bool same = true;
    for (size_t i = 1; i < Ks.size(); ++i) same = same && Ks[i] == Ks[0] && dts[i] == dts[0];
    if (Ks.empty() || !same) {
        *e = fgmm_batch_enc_kernel;
        *d = fgmm_batch_dec_kernel;
        return;
    }
    if (dts[0] == FGMM_DTYPE_BF16) pick_kt<__nv_bfloat16>(Ks[0], e, d);
    else pick_kt<float>(Ks[0], e, d);
}

// Compaction of all segments: warp per segment, 16-bit copies.
__global__ void __launch_bounds__(256) fgmm_batch_compact_kernel(const uint16_t* __restrict__ scratch,
                                                                 const int64_t* __restrict__ scr_off,
                                                                 const int64_t* __restrict__ len,
                                                                 const int64_t* __restrict__ offsets, int64_t nseg,
                                                                 uint16_t* __restrict__ words, int64_t cap)
{
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nseg; g += nwarps) {
        const int64_t n = len[g], dst = offsets[g];
        if (dst + n > cap) continue;   // capacity error recorded by the scan
        const uint16_t* src = scratch + scr_off[g];
        for (int64_t i = lane; i < n; i += 32) words[dst + i] = src[i];
    }
}

}  // namespace

struct fgmm_batch {
    int n = 0;
    std::vector<int32_t> S;
    int64_t nseg = 0;
    BatchLatentDev* d_lats = nullptr;
    WorkItem* d_work = nullptr;
    uint16_t* d_scratch = nullptr;
    int64_t* d_scr_off = nullptr;      // scratch word offset of each global segment
    int64_t* d_len = nullptr;
    unsigned long long* d_counters = nullptr;   // [0] encode queue, [1] decode queue
    uint16_t* words = nullptr;
    int64_t words_cap = 0;
    int64_t* offsets = nullptr;
    int64_t* n_words_out = nullptr;
    int grid_enc = 0, grid_dec = 0;
    EncKernel enc_kernel = nullptr;
    DecKernel dec_kernel = nullptr;
    std::vector<int> Ks, dts;          // per latent, host copies
    cudaGraphExec_t g_enc = nullptr, g_dec = nullptr;
    fgmm_handle* h = nullptr;
};

namespace {

void enqueue_encode(fgmm_batch* b, cudaStream_t st)
{
    fgmm_handle* h = b->h;
    cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned long long), st);
    b->enc_kernel<<<b->grid_enc, kBatchThreads, 0, st>>>(b->d_lats, b->d_work, b->nseg, b->d_counters, b->d_scratch,
                                                          b->d_len, h->d_err);
    // offsets over all segments, then compaction into the output
    launch_scan(b->d_len, b->nseg, b->offsets, b->n_words_out, b->words_cap, h->d_err, st);
    const int64_t cblocks = std::min<int64_t>((int64_t)h->num_sms * 8, (b->nseg * 32 + 255) / 256);
    if (b->nseg > 0)
        fgmm_batch_compact_kernel<<<(unsigned)std::max<int64_t>(cblocks, 1), 256, 0, st>>>(
            b->d_scratch, b->d_scr_off, b->d_len, b->offsets, b->nseg, b->words, b->words_cap);
}

void enqueue_decode(fgmm_batch* b, cudaStream_t st)
{
    fgmm_handle* h = b->h;
    cudaMemsetAsync(b->d_counters + 1, 0, sizeof(unsigned long long), st);
    b->dec_kernel<<<b->grid_dec, kBatchThreads, 0, st>>>(b->d_lats, b->d_work, b->nseg, b->d_counters + 1, b->words,
                                                          b->words_cap, b->offsets, h->d_err,
                                                          h->stats_on ? h->d_stats : nullptr);
}

void free_plan(fgmm_batch* b)
{
    if (b->g_enc) cudaGraphExecDestroy(b->g_enc);
    if (b->g_dec) cudaGraphExecDestroy(b->g_dec);
    cudaFree(b->d_lats);
    cudaFree(b->d_work);
    cudaFree(b->d_scratch);
    cudaFree(b->d_scr_off);
    cudaFree(b->d_len);
    cudaFree(b->d_counters);
    delete b;
}

}  // namespace

extern "C" {

fgmm_status fgmm_autotune(fgmm_handle* h, const int64_t* N, int32_t n, double max_overhead, double bits_per_symbol,
                          int32_t* S_out)
{
    if (!h || !N || !S_out || n < 0 || !(max_overhead > 0.0) || !(bits_per_symbol > 0.0))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_autotune: bad arguments");
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (N[i] < 0) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_autotune: negative N");
        total += N[i];
    }
    // Warps the batch decoder keeps resident: occupancy of the K = 3 fp32
    // decoder, capped at kTargetWarpsPerSM per SM (beyond that the SM's
    // issue slots are full and more streams only add container bits).
    int blocks_per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm,
                                                                  fgmm_batch_dec_kt_kernel<3, float>, kBatchThreads, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_autotune occupancy");
    const int64_t warps_per_sm = std::max(1, std::min(blocks_per_sm * (kBatchThreads / 32), kTargetWarpsPerSM));
    const int64_t max_segments = std::max<int64_t>(1, (int64_t)h->num_sms * warps_per_sm);
    // Each stream ends with a 32-bit flushed state: keeping that below
    // max_overhead of the payload needs T >= 32 / (max_overhead * bps).
    const double t_min = std::ceil(32.0 / (max_overhead * bits_per_symbol));
    double t_star = std::max(t_min, std::ceil((double)total / (32.0 * (double)max_segments)));
    for (int iter = 0; iter < 200; ++iter) {
        int64_t segs = 0;
        for (int i = 0; i < n; ++i) {
            int64_t s = (int64_t)std::ceil((double)N[i] / t_star);
            s = (s + 31) / 32 * 32;
            if (s < 32) s = 32;
            const int64_t smax = std::max<int64_t>(32, (N[i] + 31) / 32 * 32);
            if (s > smax) s = smax;
            if (s > (int64_t)1 << 30) s = (int64_t)1 << 30;
            S_out[i] = (int32_t)s;
            segs += s / 32;
        }
        // one wave: every segment resident at once (a second wave of a few
        // segments would double the time)
        if (segs <= max_segments || t_star >= (double)total) break;
        t_star = std::ceil(t_star * 1.03) + 1.0;
    }
    return FGMM_OK;
}

fgmm_status fgmm_batch_create(fgmm_handle* h, const fgmm_batch_latent* lats, int32_t n, const int32_t* S_in,
                              uint16_t* words, int64_t words_cap, int64_t* offsets, int64_t* n_words_out,
                              fgmm_batch** out)
{
    if (!h || !out || n < 0 || (n > 0 && !lats) || !offsets || !n_words_out || words_cap < 0 ||
        (words_cap > 0 && !words))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_batch_create: bad arguments");
    if (h->phi != FGMM_PHI_AS) return fail(h, FGMM_ERR_INVALID_ARG, "batches take FGMM_PHI_AS only");
    *out = nullptr;
    std::vector<int32_t> S(n);
    std::vector<int64_t> Ns(n);
    for (int i = 0; i < n; ++i) {
        fgmm_latent l{lats[i].K, lats[i].dtype, lats[i].N, lats[i].params};
        fgmm_status s = check_latent(h, &l);
        if (s != FGMM_OK) return s;
        Ns[i] = lats[i].N;
    }
    if (S_in) {
        for (int i = 0; i < n; ++i) {
            if (S_in[i] <= 0 || S_in[i] % 32 != 0)
                return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_batch_create: S must be positive multiples of 32");
            S[i] = S_in[i];
        }
    } else {
        fgmm_status s = fgmm_autotune(h, Ns.data(), n, 0.01, 3.5, S.data());
        if (s != FGMM_OK) return s;
    }
    fgmm_batch* b = new fgmm_batch();
    b->h = h;
    b->n = n;
    b->S = S;
    std::vector<BatchLatentDev> L(n);
    int64_t seg = 0, scr = 0;
    for (int i = 0; i < n; ++i) {
        L[i].params = lats[i].params;
        L[i].symbols = lats[i].symbols;
        L[i].decoded = lats[i].decoded;
        L[i].N = lats[i].N;
        L[i].S = S[i];
        L[i].T = steps_of(lats[i].N, S[i]);
        L[i].K = lats[i].K;
        L[i].dtype = lats[i].dtype;
        L[i].seg_base = seg;
        L[i].scr_base = scr;
        L[i].scr_cap = (3 * 32 * L[i].T + 64 + 7) / 8 * 8;
        seg += S[i] / 32;
        scr += (int64_t)(S[i] / 32) * L[i].scr_cap;
    }
    b->nseg = seg;
    // work list: every segment, longest latent first (balances the tail)
    std::vector<WorkItem> work;
    work.reserve((size_t)seg);
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return L[a].T > L[c].T; });
    for (int i : order)
        for (int32_t g = 0; g < S[i] / 32; ++g) work.push_back(WorkItem{i, g});
    std::vector<int64_t> scr_off((size_t)seg);
    for (int i = 0; i < n; ++i)
        for (int64_t g = 0; g < S[i] / 32; ++g) scr_off[(size_t)(L[i].seg_base + g)] = L[i].scr_base + g * L[i].scr_cap;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&b->d_scr_off, sizeof(int64_t) * std::max<int64_t>(seg, 1));
    if (e == cudaSuccess && seg > 0)
        e = cudaMemcpy(b->d_scr_off, scr_off.data(), sizeof(int64_t) * seg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_lats, sizeof(BatchLatentDev) * std::max(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_work, sizeof(WorkItem) * std::max<int64_t>(seg, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_scratch, sizeof(uint16_t) * std::max<int64_t>(scr, 8));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_len, sizeof(int64_t) * std::max<int64_t>(seg, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpy(b->d_lats, L.data(), sizeof(BatchLatentDev) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && seg > 0)
        e = cudaMemcpy(b->d_work, work.data(), sizeof(WorkItem) * seg, cudaMemcpyHostToDevice);
    {
        std::vector<int> Ks(n), dts(n);
        for (int i = 0; i < n; ++i) { Ks[i] = lats[i].K; dts[i] = lats[i].dtype; }
        pick_kernels(Ks, dts, &b->enc_kernel, &b->dec_kernel);
        b->Ks = Ks;
        b->dts = dts;
    }
    int bpm_e = 0, bpm_d = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpm_e, b->enc_kernel, kBatchThreads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpm_d, b->dec_kernel, kBatchThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(b);
        return fail(h, FGMM_ERR_NO_MEMORY, "fgmm_batch_create: device allocation failed");
    }
    const int64_t warps_needed = std::max<int64_t>(seg, 1);
    b->grid_enc = (int)std::min<int64_t>((int64_t)h->num_sms * std::max(bpm_e, 1),
                                         (warps_needed + kBatchThreads / 32 - 1) / (kBatchThreads / 32));
    b->grid_dec = (int)std::min<int64_t>((int64_t)h->num_sms * std::max(bpm_d, 1),
                                         (warps_needed + kBatchThreads / 32 - 1) / (kBatchThreads / 32));
    b->words = words;
    b->words_cap = words_cap;
    b->offsets = offsets;
    b->n_words_out = n_words_out;
    *out = b;
    return FGMM_OK;
}

void fgmm_batch_destroy(fgmm_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    free_plan(b);
}

int64_t fgmm_batch_segments(const fgmm_batch* b) { return b ? b->nseg : -1; }

fgmm_status fgmm_batch_streams(const fgmm_batch* b, int32_t* S_out)
{
    if (!b || (!S_out && b->n > 0)) return FGMM_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) S_out[i] = b->S[i];
    return FGMM_OK;
}

fgmm_status fgmm_batch_capture(fgmm_batch* b)
{
    if (!b) return FGMM_ERR_INVALID_ARG;
    fgmm_handle* h = b->h;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_batch_capture stream");
    for (int dir = 0; dir < 2 && e == cudaSuccess; ++dir) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        if (dir == 0) enqueue_encode(b, cs);
        else enqueue_decode(b, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess) break;
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) break;
        if (dir == 0) b->g_enc = exec;
        else b->g_dec = exec;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(h, e, "fgmm_batch_capture");
    }
    return FGMM_OK;
}

fgmm_status fgmm_batch_encode(fgmm_batch* b, void* stream)
{
    if (!b) return FGMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->g_enc) {
        cudaError_t e = cudaGraphLaunch(b->g_enc, st);
        return e == cudaSuccess ? FGMM_OK : cuda_fail(b->h, e, "fgmm_batch_encode graph");
    }
    enqueue_encode(b, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(b->h, e, "fgmm_batch_encode launch");
}

fgmm_status fgmm_batch_decode(fgmm_batch* b, void* stream)
{
    if (!b) return FGMM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->g_dec && !b->h->stats_on) {
        cudaError_t e = cudaGraphLaunch(b->g_dec, st);
        return e == cudaSuccess ? FGMM_OK : cuda_fail(b->h, e, "fgmm_batch_decode graph");
    }
    enqueue_decode(b, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(b->h, e, "fgmm_batch_decode launch");
}

fgmm_status fgmm_batch_decode_proposal(fgmm_batch* b, const void* packed, void* stream)
{
    if (!b) return FGMM_ERR_INVALID_ARG;
    fgmm_handle* h = b->h;
    for (int i = 0; i < b->n; ++i)
        if (b->Ks[i] != 3 || b->dts[i] != b->dts[0])
            return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_batch_decode_proposal: latents must be K = 3 of one dtype");
    if (packed && reinterpret_cast<uintptr_t>(packed) % 16 != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_batch_decode_proposal: packed must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b->d_counters + 1, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && b->nseg > 0)
        e = launch_batch_prop(b->d_lats, b->d_work, b->nseg, b->d_counters + 1, b->words, b->words_cap, b->offsets,
                              packed, b->n > 0 ? b->dts[0] : FGMM_DTYPE_F32, h->mlp_act, h->d_err,
                              h->stats_on ? h->d_stats : nullptr, h->num_sms, st);
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_batch_decode_proposal launch");
}

}  // extern "C"
