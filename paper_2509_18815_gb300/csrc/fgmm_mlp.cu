// fgmm_mlp.cu -- learned decode proposal (no counterpart in the paper).
//
// A 10 -> 64 -> 64 -> 1 MLP maps a symbol's mixture parameters and its rANS
// slot to a guess of the symbol. The decoder evaluates the exact quantised
// CDF at the guess and its successor; if the slot falls between them the
// symbol is found with two CDF evaluations, otherwise a galloping search
// from the guess brackets the symbol and a binary search (Sec. III-A)
// finishes it. Decoded symbols therefore never depend on the network.
//
// Features (K = 3): weights, means and log-scales standardised by the
// mixture's own mean m0 and standard deviation s0 (components sorted by
// mean), and u - 1/2 with u = (slot + 1/2) / 2^16; target (s - m0) / s0
// clipped to [-8, 8]; guess round(m0 + s0 y). Activation: z * sat(1/2 + c z),
// c = 1.702 / 4 (GELU with the logistic CDF of Eq. 9 replaced by its tangent
// at 0, saturated to [0, 1]).
//
// Training (FP32): per 64-sample block the forward pass, the loss and the
// hand-written backward pass run in shared memory; per-block gradient
// partials are reduced in a fixed order by the Adam kernel (deterministic).
// Inference in the decoder: BF16 weights, FP32 accumulation, mma.sync
// m16n8k16 over the 32 queries of a warp (one per stream); the layer-1
// accumulators become the layer-2 A fragments without leaving registers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"
#include "fgmm_segment.cuh"

using namespace fgmm;

namespace {

constexpr int kIn = 10, kHid = 64;
constexpr int kNP = kIn * kHid + kHid + kHid * kHid + kHid + kHid + 1;   // 4929
constexpr int oW1 = 0, oB1 = kIn * kHid, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid;
constexpr float kActC = 1.702f / 4.0f;
constexpr int kTS = 64;            // samples per training block
constexpr int kTrainThreads = 128;

// Activations (FGMM_MLP_ACT_*): ACT 0, z * sat(1/2 + c z), the GELU
// z Phi(z) with the logistic CDF of Eq. 9 replaced by its tangent at 0;
// ACT 1, z * sigma(1.702 z), the GELU with Phi replaced by the logistic CDF
// of Eq. 9 itself. FAST uses the hardware exponential (inference only).
template <int ACT, bool FAST = false>
__device__ __forceinline__ float act(float z)
{
    if constexpr (ACT == 0) {
        return z * __saturatef(fmaf(kActC, z, 0.5f));
    } else if constexpr (FAST) {
        return __fdividef(z, 1.0f + __expf(-1.702f * z));
    } else {
        return z / (1.0f + expf(-1.702f * z));
    }
}
template <int ACT>
__device__ __forceinline__ float act_grad(float z)
{
    if constexpr (ACT == 0) {
        const float r = fmaf(kActC, z, 0.5f);
        if (r <= 0.0f) return 0.0f;
        if (r >= 1.0f) return 1.0f;
        return r + kActC * z;
    } else {
        const float sg = 1.0f / (1.0f + expf(-1.702f * z));
        return sg + 1.702f * z * sg * (1.0f - sg);
    }
}

// Standardised features of one query (see the file comment). FAST selects
// the hardware approximations of sqrt, reciprocal and log (the decoder's
// guess needs no exactness; training data uses the accurate forms).
template <bool FAST = false>
__device__ __forceinline__ void features(const float* w_in, const float* mu_in, const float* sg_in, uint32_t slot,
                                         float* x, float& m0, float& s0)
{
    float w[3] = {w_in[0], w_in[1], w_in[2]};
    float mu[3] = {mu_in[0], mu_in[1], mu_in[2]};
    float sp[3] = {fmaxf(sg_in[0], kSigmaMin), fmaxf(sg_in[1], kSigmaMin), fmaxf(sg_in[2], kSigmaMin)};
    // stable 3-element sort by mean
#define FGMM_CSWAP(i, j)                                                        \
    if (mu[i] > mu[j]) {                                                        \
        float t_ = mu[i]; mu[i] = mu[j]; mu[j] = t_;                            \
        t_ = w[i]; w[i] = w[j]; w[j] = t_;                                      \
        t_ = sp[i]; sp[i] = sp[j]; sp[j] = t_;                                  \
    }
    FGMM_CSWAP(0, 1)
    FGMM_CSWAP(1, 2)
    FGMM_CSWAP(0, 1)
#undef FGMM_CSWAP
    m0 = w[0] * mu[0] + w[1] * mu[1] + w[2] * mu[2];
    float v = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) v += w[k] * (sp[k] * sp[k] + (mu[k] - m0) * (mu[k] - m0));
    float inv;
    if (FAST) {
        inv = rsqrtf(fmaxf(v, 1e-4f));
        s0 = fmaxf(v, 1e-4f) * inv;
    } else {
        s0 = sqrtf(fmaxf(v, 1e-4f));
        inv = 1.0f / s0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        x[k] = w[k];
        x[3 + k] = (mu[k] - m0) * inv;
        x[6 + k] = FAST ? __logf(sp[k] * inv) : logf(sp[k] * inv);
    }
    x[9] = ((float)slot + 0.5f) * (1.0f / 65536.0f) - 0.5f;
}

// ---------------------------------------------------------------------------
// Training data: (features, target) from (params, symbol, uniform draw).
// The slot is drawn uniformly inside the symbol's interval of the coder's
// quantised CDF: slot = start + min(freq - 1, floor(v * freq)).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) mlp_data_kernel(const T* __restrict__ params, int64_t N,
                                                       const int32_t* __restrict__ sym, const float* __restrict__ uni,
                                                       float* __restrict__ X, float* __restrict__ tgt,
                                                       int32_t* __restrict__ slots, int32_t* err)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        Mix<3> m;
        if (!load_mix<3>(params, N, n, m)) set_error(err, kErrBadParams);
        const int32_t s = sym[n];
        uint32_t st, fr;
        interval_of<3>(m, s, st, fr);
        uint32_t off = (uint32_t)(uni[n] * (float)fr);
        if (off > fr - 1) off = fr - 1;
        const uint32_t slot = st + off;
        float w[3], mu[3], sg[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            w[k] = load_param(params, (int64_t)k * N + n);
            mu[k] = load_param(params, (int64_t)(3 + k) * N + n);
            sg[k] = load_param(params, (int64_t)(6 + k) * N + n);
        }
        float x[kIn], m0, s0;
        features(w, mu, sg, slot, x, m0, s0);
#pragma unroll
        for (int i = 0; i < kIn; ++i) X[n * kIn + i] = x[i];
        tgt[n] = fminf(fmaxf(((float)s - m0) / s0, -8.0f), 8.0f);
        if (slots) slots[n] = (int32_t)slot;
    }
}

// ---------------------------------------------------------------------------
// Loss and gradient of one block of kTS samples; partial sums per block.
// ---------------------------------------------------------------------------
template <int ACT>
__global__ void __launch_bounds__(kTrainThreads) mlp_grad_kernel(const float* __restrict__ X,
                                                                 const float* __restrict__ tgt, int64_t B,
                                                                 const float* __restrict__ theta,
                                                                 float* __restrict__ partial)
{
    extern __shared__ float sm[];
    float* th = sm;                         // [kNP] (padded to 4932)
    float* xs = th + 4932;                  // [kTS][kIn]
    float* z1 = xs + kTS * kIn;             // [kTS][kHid]
    float* z2 = z1 + kTS * kHid;            // [kTS][kHid]
    float* dy = z2 + kTS * kHid;            // [kTS]
    float* red = dy + kTS;                  // [kTrainThreads]
    const int tid = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * kTS;
    const int64_t rem = B - s0;
    const int ns = rem < kTS ? (int)rem : kTS;
    float* out = partial + (int64_t)blockIdx.x * (kNP + 1);
    for (int i = tid; i < kNP; i += kTrainThreads) th[i] = theta[i];
    for (int i = tid; i < kTS * kIn; i += kTrainThreads) xs[i] = (i / kIn) < ns ? X[s0 * kIn + i] : 0.0f;
    __syncthreads();
    // forward, layer 1 and 2 (pre-activations kept)
    for (int e = tid; e < kTS * kHid; e += kTrainThreads) {
        const int s = e / kHid, j = e % kHid;
        float a = th[oB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) a = fmaf(xs[s * kIn + k], th[oW1 + k * kHid + j], a);
        z1[e] = a;
    }
    __syncthreads();
    for (int e = tid; e < kTS * kHid; e += kTrainThreads) {
        const int s = e / kHid, j = e % kHid;
        float a = th[oB2 + j];
        for (int i = 0; i < kHid; ++i) a = fmaf(act<ACT>(z1[s * kHid + i]), th[oW2 + i * kHid + j], a);
        z2[e] = a;
    }
    __syncthreads();
    float lsum = 0.0f;
    if (tid < kTS) {
        float y = th[oB3];
        for (int j = 0; j < kHid; ++j) y = fmaf(act<ACT>(z2[tid * kHid + j]), th[oW3 + j], y);
        float r = 0.0f;
        if (tid < ns) r = y - tgt[s0 + tid];
        dy[tid] = 2.0f * r / (float)B;
        lsum = r * r;
    }
    red[tid] = lsum;
    __syncthreads();
    // output layer gradients
    if (tid < kHid) {
        float g = 0.0f;
        for (int s = 0; s < kTS; ++s) g = fmaf(act<ACT>(z2[s * kHid + tid]), dy[s], g);
        out[oW3 + tid] = g;
    }
    if (tid == 0) {
        float g = 0.0f, l = 0.0f;
        for (int s = 0; s < kTS; ++s) g += dy[s];
        for (int i = 0; i < kTrainThreads; ++i) l += red[i];
        out[oB3] = g;
        out[kNP] = l;
    }
    __syncthreads();
    for (int e = tid; e < kTS * kHid; e += kTrainThreads) {
        const int s = e / kHid, j = e % kHid;
        z2[e] = dy[s] * th[oW3 + j] * act_grad<ACT>(z2[e]);   // d2
    }
    __syncthreads();
    for (int e = tid; e < kHid * kHid; e += kTrainThreads) {
        const int i = e / kHid, j = e % kHid;
        float g = 0.0f;
        for (int s = 0; s < kTS; ++s) g = fmaf(act<ACT>(z1[s * kHid + i]), z2[s * kHid + j], g);
        out[oW2 + e] = g;
    }
    if (tid < kHid) {
        float g = 0.0f;
        for (int s = 0; s < kTS; ++s) g += z2[s * kHid + tid];
        out[oB2 + tid] = g;
    }
    __syncthreads();
    for (int e = tid; e < kTS * kHid; e += kTrainThreads) {
        const int s = e / kHid, i = e % kHid;
        float a = 0.0f;
        for (int j = 0; j < kHid; ++j) a = fmaf(th[oW2 + i * kHid + j], z2[s * kHid + j], a);
        z1[e] = a * act_grad<ACT>(z1[e]);   // d1
    }
    __syncthreads();
    for (int e = tid; e < kIn * kHid; e += kTrainThreads) {
        const int k = e / kHid, i = e % kHid;
        float g = 0.0f;
        for (int s = 0; s < kTS; ++s) g = fmaf(xs[s * kIn + k], z1[s * kHid + i], g);
        out[oW1 + e] = g;
    }
    if (tid < kHid) {
        float g = 0.0f;
        for (int s = 0; s < kTS; ++s) g += z1[s * kHid + tid];
        out[oB1 + tid] = g;
    }
}

// Sums the per-block partials in block order (deterministic); optionally
// applies one Adam step. grad_out may be NULL; loss_out receives the mean
// squared error of the batch.
__global__ void __launch_bounds__(256) mlp_reduce_adam_kernel(const float* __restrict__ partial, int nblocks,
                                                              int64_t B, float* __restrict__ theta,
                                                              float* __restrict__ grad_out, float* __restrict__ m,
                                                              float* __restrict__ v, int64_t step, float lr,
                                                              float* loss_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNP) return;
    float g = 0.0f;
    for (int b = 0; b < nblocks; ++b) g += partial[(int64_t)b * (kNP + 1) + p];
    if (p == kNP) {
        if (loss_out) *loss_out = g / (float)B;
        return;
    }
    if (grad_out) grad_out[p] = g;
    if (m) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float mt = b1 * m[p] + (1.0f - b1) * g;
        const float vt = b2 * v[p] + (1.0f - b2) * g * g;
        m[p] = mt;
        v[p] = vt;
        const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
        theta[p] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// BF16 inference: packed fragments and the warp-level forward pass.
// ---------------------------------------------------------------------------
struct MlpPacked {
    uint2 w1f[8][32];        // B fragments of W1 (k padded 10 -> 16), per n-tile and lane
    uint2 w2f[4][8][32];     // B fragments of W2, per k-tile, n-tile and lane
    float b1[kHid], b2[kHid], w3[kHid];
    float b3, pad[3];
};
static_assert(sizeof(MlpPacked) == 11024, "packed MLP layout");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__global__ void mlp_pack_kernel(const float* __restrict__ theta, MlpPacked* __restrict__ P)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid < 8 * 32) {
        const int nt = tid / 32, lane = tid % 32, g = lane >> 2, t = lane & 3;
        const int n = 8 * nt + g;
        auto w1 = [&](int k) { return k < kIn ? theta[oW1 + k * kHid + n] : 0.0f; };
        P->w1f[nt][lane] = make_uint2(pack_bf16(w1(2 * t), w1(2 * t + 1)), pack_bf16(w1(2 * t + 8), w1(2 * t + 9)));
    }
    if (tid < 4 * 8 * 32) {
        const int kt = tid / 256, nt = (tid / 32) % 8, lane = tid % 32, g = lane >> 2, t = lane & 3;
        const int n = 8 * nt + g, k0 = 16 * kt + 2 * t;
        auto w2 = [&](int k) { return theta[oW2 + k * kHid + n]; };
        P->w2f[kt][nt][lane] = make_uint2(pack_bf16(w2(k0), w2(k0 + 1)), pack_bf16(w2(k0 + 8), w2(k0 + 9)));
    }
    if (tid < kHid) {
        P->b1[tid] = theta[oB1 + tid];
        P->b2[tid] = theta[oB2 + tid];
        P->w3[tid] = theta[oW3 + tid];
    }
    if (tid == 0) {
        P->b3 = theta[oB3];
        P->pad[0] = P->pad[1] = P->pad[2] = 0.0f;
    }
}

__device__ __forceinline__ void mma_bf16(float& c0, float& c1, float& c2, float& c3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b.x), "r"(b.y));
}

// Forward pass for the 32 queries of a warp; x: this lane's 10 features.
// xs: per-warp shared scratch of 32 x 12 words. Returns this lane's y.
template <int ACT>
__device__ __forceinline__ float mlp_warp_forward(const MlpPacked* __restrict__ P, const float* x, uint32_t* xs)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    __syncwarp();
    uint32_t* row = xs + lane * 12;
    row[0] = pack_bf16(x[0], x[1]);
    row[1] = pack_bf16(x[2], x[3]);
    row[2] = pack_bf16(x[4], x[5]);
    row[3] = pack_bf16(x[6], x[7]);
    row[4] = pack_bf16(x[8], x[9]);
    row[5] = row[6] = row[7] = 0u;
    __syncwarp();
    float ys[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        const uint32_t a0 = xs[r0 * 12 + t], a1 = xs[r1 * 12 + t], a2 = xs[r0 * 12 + t + 4], a3 = xs[r1 * 12 + t + 4];
        uint32_t h[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float bb0 = P->b1[8 * nt + 2 * t], bb1 = P->b1[8 * nt + 2 * t + 1];
            float c0 = bb0, c1 = bb1, c2 = bb0, c3 = bb1;
            mma_bf16(c0, c1, c2, c3, a0, a1, a2, a3, P->w1f[nt][lane]);
            const uint32_t lo = pack_bf16(act<ACT, true>(c0), act<ACT, true>(c1)), hi = pack_bf16(act<ACT, true>(c2), act<ACT, true>(c3));
            if (nt & 1) { h[nt >> 1][2] = lo; h[nt >> 1][3] = hi; }
            else { h[nt >> 1][0] = lo; h[nt >> 1][1] = hi; }
        }
        float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float bb0 = P->b2[8 * nt + 2 * t], bb1 = P->b2[8 * nt + 2 * t + 1];
            float c0 = bb0, c1 = bb1, c2 = bb0, c3 = bb1;
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) mma_bf16(c0, c1, c2, c3, h[kt][0], h[kt][1], h[kt][2], h[kt][3], P->w2f[kt][nt][lane]);
            const float w0 = P->w3[8 * nt + 2 * t], w1 = P->w3[8 * nt + 2 * t + 1];
            y0 = fmaf(act<ACT, true>(c0), w0, fmaf(act<ACT, true>(c1), w1, y0));
            y1 = fmaf(act<ACT, true>(c2), w0, fmaf(act<ACT, true>(c3), w1, y1));
        }
        y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
        y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
        y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
        y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
        ys[mt][0] = y0 + P->b3;
        ys[mt][1] = y1 + P->b3;
    }
    const int r = lane & 15, src = 4 * (r & 7);
    const float v00 = __shfl_sync(0xffffffffu, ys[0][0], src), v01 = __shfl_sync(0xffffffffu, ys[0][1], src);
    const float v10 = __shfl_sync(0xffffffffu, ys[1][0], src), v11 = __shfl_sync(0xffffffffu, ys[1][1], src);
    return (lane < 16) ? ((r < 8) ? v00 : v01) : ((r < 8) ? v10 : v11);
}

template <int ACT>
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ X, int64_t B,
                                                          const MlpPacked* __restrict__ Pg, float* __restrict__ y)
{
    __shared__ MlpPacked P;
    __shared__ uint32_t xs[4][32 * 12];
    for (int i = threadIdx.x; i < (int)(sizeof(MlpPacked) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&P)[i] = reinterpret_cast<const uint32_t*>(Pg)[i];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 4;
    for (int64_t base = ((int64_t)blockIdx.x * 4 + w) * 32; base < B; base += nw * 32) {
        const int64_t q = base + lane;
        float x[kIn];
#pragma unroll
        for (int i = 0; i < kIn; ++i) x[i] = q < B ? X[q * kIn + i] : 0.0f;
        const float v = mlp_warp_forward<ACT>(&P, x, xs[w]);
        if (q < B) y[q] = v;
    }
}

// ---------------------------------------------------------------------------
// Proposal-bracketed decoder (K = 3), one warp per segment. The guess comes
// from the network, or (ANALYTIC) from the inverse of the logistic
// approximation of Phi (Sec. III-B) on the component of largest weight:
// mu + sigma' ln(u / (1 - u)) / 1.702, u = (slot + 1/2) / 2^16.
//
// The search from the guess g (clamped to [lo, hi + 1], hi + 1 the escape
// slot) runs on the fast steering evaluation of the CDF (mix_cdf_fast):
// two probes decide whether Q(g) <= slot < Q(g + 1); otherwise a gallop of
// steps 1, 2, 4, ... away from g brackets the slot and a binary search
// finishes it. The symbol reached is then confirmed with the exact
// quantised CDF at it and its successor, as in search_slot_guided; a failed
// check runs the exact binary search. Decoded symbols therefore never
// depend on the network or on the fast evaluation. Counters: probes (fast
// evaluations of the search), hits (g was the symbol), fallbacks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool fast_le(const Mix<3>& m, int j, float thr)
{
    const float v = fminf(mix_cdf_fast<3>(m, (float)j - 0.5f), 1.0f);
    return fmaf(m.tp, v, (float)(j - m.lo)) < thr;   // Q(j) <= slot, decided on the fast evaluation
}

__device__ __forceinline__ bool search_from_guess(const Mix<3>& m, uint32_t slot, int gi, int32_t& s,
                                                  uint32_t& start, uint32_t& freq, int& probes, int& hits,
                                                  int& fallbacks)
{
    const float thr = (float)(slot + 1u);
    const int top = m.hi + 2;   // Q(hi + 2) = 2^16 > slot
    int a, b;
    ++probes;
    if (gi == m.lo || fast_le(m, gi, thr)) {
        a = gi;   // Q(a) <= slot: gallop up for b with Q(b) > slot
        int step = 1;
        for (;;) {
            b = a + step;
            if (b >= top) { b = top; break; }
            ++probes;
            if (!fast_le(m, b, thr)) break;
            a = b;
            step <<= 1;
        }
    } else {
        b = gi;   // Q(b) > slot: gallop down for a with Q(a) <= slot
        int step = 1;
        for (;;) {
            a = b - step;
            if (a <= m.lo) { a = m.lo; break; }
            ++probes;
            if (fast_le(m, a, thr)) break;
            b = a;
            step <<= 1;
        }
    }
    while (b - a > 1) {
        const int mid = a + ((b - a) >> 1);
        ++probes;
        if (fast_le(m, mid, thr)) a = mid;
        else b = mid;
    }
    const uint32_t qa = a == m.lo ? 0u : q_at<3>(m, a);
    const uint32_t qb = a == m.hi + 1 ? kM : q_at<3>(m, a + 1);
    if (qa <= slot && slot < qb) {
        s = a;
        start = qa;
        freq = qb - qa;
        hits += a == gi;
        return a == m.hi + 1;
    }
    ++fallbacks;
    int extra = 0;
    return search_slot<3>(m, slot, s, start, freq, extra);
}

// Decodes segment g of a K = 3 latent (words[beg, end)) with the proposal;
// all 32 lanes of the warp must call it (the network runs warp-wide).
template <typename T, bool ANALYTIC, int ACT>
__device__ __forceinline__ void dec_segment_prop(const T* __restrict__ params, int64_t N, int32_t S, int64_t T_steps,
                                                 int64_t g, const uint16_t* __restrict__ words, int64_t beg,
                                                 int64_t end, const MlpPacked* __restrict__ P, uint32_t* xs,
                                                 int32_t* __restrict__ out, int32_t* err, unsigned long long* stats)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    uint32_t x = (uint32_t)__ldg(words + end - 64 + 2 * lane) | ((uint32_t)__ldg(words + end - 63 + 2 * lane) << 16);
    int64_t ptr = end - 64;
    bool bad = false, badp = false;
    int probes = 0, decoded = 0, hits = 0, fallbacks = 0;
    int64_t n = g * 32 + lane;
    RawParams<3> cur;
    if (T_steps > 0 && n < N) load_raw_params<3, T>(params, N, n, cur);
    for (int64_t t = 0; t < T_steps; ++t, n += S) {
        const bool act_l = n < N;
        RawParams<3> nxt;
        if (t + 1 < T_steps && n + S < N) load_raw_params<3, T>(params, N, n + S, nxt);
        Mix<3> m;
        if (act_l) badp |= !mix_from_params<3>(cur, m);
        else {
#pragma unroll
            for (int i = 0; i < 9; ++i) cur.v[i] = 1.0f;
            mix_from_params<3>(cur, m);
        }
        const uint32_t slot = x & 0xffffu;
        float guess;
        if constexpr (ANALYTIC) {
            int kd = cur.v[1] > cur.v[0] ? 1 : 0;
            kd = cur.v[2] > cur.v[kd] ? 2 : kd;
            const float u = ((float)slot + 0.5f) * 0x1p-16f;
            guess = cur.v[3 + kd] + fmaxf(cur.v[6 + kd], kSigmaMin) * (__logf(__fdividef(u, 1.0f - u)) * (1.0f / 1.702f));
        } else {
            float f[kIn], m0, s0;
            features<true>(&cur.v[0], &cur.v[3], &cur.v[6], slot, f, m0, s0);
            const float yv = mlp_warp_forward<ACT>(P, f, xs);   // all lanes take part
            guess = fmaf(s0, yv, m0);
        }
        int32_t s = 0;
        bool esc = false;
        if (act_l) {
            ++decoded;
            float gf = rintf(guess);
            gf = isfinite(gf) ? fminf(fmaxf(gf, (float)m.lo), (float)(m.hi + 1)) : (float)m.lo;
            uint32_t start, freq;
            esc = search_from_guess(m, slot, (int)gf, s, start, freq, probes, hits, fallbacks);
            x = freq * (x >> 16) + slot - start;
        }
        refill_warp(x, act_l, words, ptr, beg, bad, lt);
        if (__ballot_sync(0xffffffffu, esc)) {
            uint32_t hi16 = 0, lo16 = 0;
            if (esc) { hi16 = x & 0xffffu; x >>= 16; }
            refill_warp(x, esc, words, ptr, beg, bad, lt);
            if (esc) { lo16 = x & 0xffffu; x >>= 16; }
            refill_warp(x, esc, words, ptr, beg, bad, lt);
            if (esc) s = (int32_t)((hi16 << 16) | lo16);
        }
        if (act_l) out[n] = s;
        cur = nxt;
    }
    const bool fail = bad || x != kL || ptr != beg;
    if (__ballot_sync(0xffffffffu, fail) && lane == 0) set_error(err, kErrCorrupt);
    if (__ballot_sync(0xffffffffu, badp) && lane == 0) set_error(err, kErrBadParams);
    if (stats) {
        int p = probes, d = decoded, hh = hits, fb = fallbacks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
            hh += __shfl_xor_sync(0xffffffffu, hh, o);
            fb += __shfl_xor_sync(0xffffffffu, fb, o);
        }
        if (lane == 0) {
            atomicAdd(stats, (unsigned long long)p);
            atomicAdd(stats + 1, (unsigned long long)d);
            atomicAdd(stats + 2, (unsigned long long)hh);
            if (fb) atomicAdd(stats + 3, (unsigned long long)fb);
        }
    }
}

// Single latent: one warp (one segment) per block, so that segments spread
// over all SMs.
template <typename T, bool ANALYTIC, int ACT>
__global__ void __launch_bounds__(32) fgmm_dec_prop_kernel(const T* __restrict__ params, int64_t N, int32_t S,
                                                            int64_t T_steps, const uint16_t* __restrict__ words,
                                                            int64_t n_words, const int64_t* __restrict__ offsets,
                                                            int64_t nseg, const MlpPacked* __restrict__ Pg,
                                                            int32_t* __restrict__ out, int32_t* err,
                                                            unsigned long long* stats)
{
    __shared__ MlpPacked P;
    __shared__ uint32_t xs[32 * 12];
    if constexpr (!ANALYTIC) {
        for (int i = threadIdx.x; i < (int)(sizeof(MlpPacked) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t*>(&P)[i] = reinterpret_cast<const uint32_t*>(Pg)[i];
        __syncthreads();
    }
    const int64_t g = blockIdx.x;
    if (g >= nseg) return;   // after the block-wide load; no block barrier follows
    const int64_t beg = offsets[g], end = offsets[g + 1];
    if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
        if ((threadIdx.x & 31) == 0) set_error(err, kErrCorrupt);
        return;
    }
    dec_segment_prop<T, ANALYTIC, ACT>(params, N, S, T_steps, g, words, beg, end, &P, xs, out, err, stats);
}

// Batch: persistent CTAs of 4 warps sharing one copy of the packed network
// in shared memory; each warp takes (latent, segment) items from the queue.
constexpr int kPropWarps = 4;

template <typename T, bool ANALYTIC, int ACT>
__global__ void __launch_bounds__(32 * kPropWarps) fgmm_batch_dec_prop_kernel(
    const BatchLatentDev* __restrict__ lats, const BatchWorkItem* __restrict__ work, int64_t nwork,
    unsigned long long* counter, const uint16_t* __restrict__ words, int64_t n_words,
    const int64_t* __restrict__ offsets, const MlpPacked* __restrict__ Pg, int32_t* err, unsigned long long* stats)
{
    __shared__ MlpPacked P;
    __shared__ uint32_t xs[kPropWarps][32 * 12];
    if constexpr (!ANALYTIC) {
        for (int i = threadIdx.x; i < (int)(sizeof(MlpPacked) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t*>(&P)[i] = reinterpret_cast<const uint32_t*>(Pg)[i];
        __syncthreads();
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(counter, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= (unsigned long long)nwork) break;
        const BatchWorkItem it = work[i];
        const BatchLatentDev L = lats[it.latent];
        const int64_t gg = L.seg_base + it.g;
        const int64_t beg = offsets[gg], end = offsets[gg + 1];
        if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
            if (lane == 0) set_error(err, kErrCorrupt);
            continue;
        }
        dec_segment_prop<T, ANALYTIC, ACT>(static_cast<const T*>(L.params), L.N, L.S, L.T, it.g, words, beg, end, &P,
                                           xs[w], L.decoded, err, stats);
    }
}

template <typename T, bool ANALYTIC, int ACT>
cudaError_t launch_batch_prop_t(const BatchLatentDev* lats, const BatchWorkItem* work, int64_t nwork,
                                unsigned long long* counter, const uint16_t* words, int64_t n_words,
                                const int64_t* offsets, const MlpPacked* P, int32_t* err, unsigned long long* stats,
                                int num_sms, cudaStream_t st)
{
    auto kern = fgmm_batch_dec_prop_kernel<T, ANALYTIC, ACT>;
    int bpm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpm, kern, 32 * kPropWarps, 0);
    if (e != cudaSuccess) return e;
    const int64_t blocks_needed = (nwork + kPropWarps - 1) / kPropWarps;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * std::max(bpm, 1), blocks_needed));
    kern<<<(unsigned)grid, 32 * kPropWarps, 0, st>>>(lats, work, nwork, counter, words, n_words, offsets, P, err,
                                                     stats);
    return cudaGetLastError();
}

constexpr size_t grad_smem_bytes()
{
    return sizeof(float) * (4932 + kTS * kIn + 2 * kTS * kHid + kTS + kTrainThreads);
}

fgmm_status launch_grad(fgmm_handle* h, const float* X, const float* tgt, int64_t B, const float* theta,
                        float** partial_out, int* nblocks_out, cudaStream_t st)
{
    const int64_t nb = (B + kTS - 1) / kTS;
    fgmm_status s = ws_reserve(h, sizeof(float) * (size_t)(nb * (kNP + 1)), st);
    if (s != FGMM_OK) return s;
    float* partial = static_cast<float*>(h->ws);
    const size_t smem = grad_smem_bytes();
    auto kern = h->mlp_act == FGMM_MLP_ACT_SIGMOID ? mlp_grad_kernel<1> : mlp_grad_kernel<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp grad attribute");
    kern<<<(unsigned)nb, kTrainThreads, smem, st>>>(X, tgt, B, theta, partial);
    *partial_out = partial;
    *nblocks_out = (int)nb;
    return FGMM_OK;
}

}  // namespace

extern "C" {

fgmm_status fgmm_mlp_data(fgmm_handle* h, const fgmm_latent* lat, const int32_t* symbols, const float* uniforms,
                          float* X, float* target, int32_t* slots, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (lat->K != 3) return fail(h, FGMM_ERR_INVALID_ARG, "the proposal network takes K = 3 mixtures");
    if (h->phi != FGMM_PHI_AS) return fail(h, FGMM_ERR_INVALID_ARG, "the proposal path takes FGMM_PHI_AS only");
    if (lat->N > 0 && (!symbols || !uniforms || !X || !target))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_mlp_data: NULL buffer");
    if (lat->N == 0) return FGMM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t blocks = std::min<int64_t>((lat->N + 255) / 256, (int64_t)h->num_sms * 16);
    if (lat->dtype == FGMM_DTYPE_BF16)
        mlp_data_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(
            static_cast<const __nv_bfloat16*>(lat->params), lat->N, symbols, uniforms, X, target, slots, h->d_err);
    else
        mlp_data_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const float*>(lat->params), lat->N,
                                                                  symbols, uniforms, X, target, slots, h->d_err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_mlp_data launch");
}

fgmm_status fgmm_mlp_loss_grad(fgmm_handle* h, const float* X, const float* target, int64_t B, const float* theta,
                               float* grad, float* loss, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (B <= 0 || !X || !target || !theta || !grad || !loss)
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_mlp_loss_grad: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* partial = nullptr;
    int nb = 0;
    fgmm_status s = launch_grad(h, X, target, B, theta, &partial, &nb, st);
    if (s != FGMM_OK) return s;
    mlp_reduce_adam_kernel<<<(kNP + 1 + 255) / 256, 256, 0, st>>>(partial, nb, B, nullptr, grad, nullptr, nullptr, 0,
                                                                   0.0f, loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_mlp_loss_grad launch");
}

fgmm_status fgmm_mlp_train(fgmm_handle* h, const float* X, const float* target, int64_t N, float* theta,
                           float* adam_m, float* adam_v, int64_t step0, int64_t steps, int64_t batch, float lr,
                           float* loss_trace, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (N <= 0 || batch <= 0 || batch > N || steps < 0 || step0 < 0 || !X || !target || !theta || !adam_m ||
        !adam_v || !loss_trace)
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_mlp_train: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nbatches = N / batch;
    for (int64_t i = 0; i < steps; ++i) {
        const int64_t k = step0 + i;
        const int64_t off = (k % nbatches) * batch;
        float* partial = nullptr;
        int nb = 0;
        fgmm_status s = launch_grad(h, X + off * kIn, target + off, batch, theta, &partial, &nb, st);
        if (s != FGMM_OK) return s;
        mlp_reduce_adam_kernel<<<(kNP + 1 + 255) / 256, 256, 0, st>>>(partial, nb, batch, theta, nullptr, adam_m,
                                                                       adam_v, k + 1, lr, loss_trace + i);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_mlp_train launch");
}

fgmm_status fgmm_mlp_pack(fgmm_handle* h, const float* theta, void* packed, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (!theta || !packed || reinterpret_cast<uintptr_t>(packed) % 16 != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_mlp_pack: bad arguments (packed must be 16-byte aligned)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mlp_pack_kernel<<<4, 256, 0, st>>>(theta, static_cast<MlpPacked*>(packed));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_mlp_pack launch");
}

fgmm_status fgmm_mlp_forward(fgmm_handle* h, const float* X, int64_t B, const void* packed, float* y, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    if (B < 0 || (B > 0 && (!X || !y)) || !packed) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_mlp_forward: bad arguments");
    if (B == 0) return FGMM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t blocks = std::min<int64_t>((B + 127) / 128, (int64_t)h->num_sms * 8);
    auto kern = h->mlp_act == FGMM_MLP_ACT_SIGMOID ? mlp_forward_kernel<1> : mlp_forward_kernel<0>;
    kern<<<(unsigned)blocks, 128, 0, st>>>(X, B, static_cast<const MlpPacked*>(packed), y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_mlp_forward launch");
}

fgmm_status fgmm_decode_proposal(fgmm_handle* h, const fgmm_latent* lat, const void* packed, const uint16_t* words,
                                 int64_t n_words, const int64_t* offsets, int32_t S, int32_t* symbols_out,
                                 void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (lat->K != 3) return fail(h, FGMM_ERR_INVALID_ARG, "the proposal network takes K = 3 mixtures");
    if (h->phi != FGMM_PHI_AS) return fail(h, FGMM_ERR_INVALID_ARG, "the proposal path takes FGMM_PHI_AS only");
    if (S <= 0 || S % 32 != 0) return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets || n_words < 0 || (n_words > 0 && !words) || (lat->N > 0 && !symbols_out))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_decode_proposal: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nseg = S / 32, T = steps_of(lat->N, S);
    const int64_t blocks = nseg;
    unsigned long long* stats = h->stats_on ? h->d_stats : nullptr;
    const MlpPacked* P = static_cast<const MlpPacked*>(packed);
    const bool sig = h->mlp_act == FGMM_MLP_ACT_SIGMOID;
    if (lat->dtype == FGMM_DTYPE_BF16) {
        auto kern = !P ? fgmm_dec_prop_kernel<__nv_bfloat16, true, 0>
                       : (sig ? fgmm_dec_prop_kernel<__nv_bfloat16, false, 1> : fgmm_dec_prop_kernel<__nv_bfloat16, false, 0>);
        kern<<<(unsigned)blocks, 32, 0, st>>>(static_cast<const __nv_bfloat16*>(lat->params), lat->N, S, T, words,
                                              n_words, offsets, nseg, P, symbols_out, h->d_err, stats);
    } else {
        auto kern = !P ? fgmm_dec_prop_kernel<float, true, 0>
                       : (sig ? fgmm_dec_prop_kernel<float, false, 1> : fgmm_dec_prop_kernel<float, false, 0>);
        kern<<<(unsigned)blocks, 32, 0, st>>>(static_cast<const float*>(lat->params), lat->N, S, T, words, n_words,
                                              offsets, nseg, P, symbols_out, h->d_err, stats);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_decode_proposal launch");
}

}  // extern "C"

namespace fgmm {

cudaError_t launch_batch_prop(const BatchLatentDev* lats, const BatchWorkItem* work, int64_t nwork,
                              unsigned long long* counter, const uint16_t* words, int64_t n_words,
                              const int64_t* offsets, const void* packed, int dtype, int act, int32_t* err,
                              unsigned long long* stats, int num_sms, cudaStream_t st)
{
    const MlpPacked* P = static_cast<const MlpPacked*>(packed);
    if (dtype == FGMM_DTYPE_BF16) {
        if (!P)
            return launch_batch_prop_t<__nv_bfloat16, true, 0>(lats, work, nwork, counter, words, n_words, offsets,
                                                              P, err, stats, num_sms, st);
        if (act == FGMM_MLP_ACT_SIGMOID)
            return launch_batch_prop_t<__nv_bfloat16, false, 1>(lats, work, nwork, counter, words, n_words, offsets,
                                                               P, err, stats, num_sms, st);
        return launch_batch_prop_t<__nv_bfloat16, false, 0>(lats, work, nwork, counter, words, n_words, offsets, P,
                                                           err, stats, num_sms, st);
    }
    if (!P)
        return launch_batch_prop_t<float, true, 0>(lats, work, nwork, counter, words, n_words, offsets, P, err, stats,
                                                  num_sms, st);
    if (act == FGMM_MLP_ACT_SIGMOID)
        return launch_batch_prop_t<float, false, 1>(lats, work, nwork, counter, words, n_words, offsets, P, err,
                                                   stats, num_sms, st);
    return launch_batch_prop_t<float, false, 0>(lats, work, nwork, counter, words, n_words, offsets, P, err, stats,
                                               num_sms, st);
}

}  // namespace fgmm
