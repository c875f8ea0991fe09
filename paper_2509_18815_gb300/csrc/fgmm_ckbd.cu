// fgmm_ckbd.cu -- checkerboard two-pass coding around the coder (the context
// model of the paper's codecs, Sec. IV-A). In every channel of a C x H x W
// latent the positions with h + w even are anchors, coded first with the
// hyperprior's parameters; the others are coded second with parameters a
// context model computes from the decoded anchors. These kernels move
// symbols and parameters between the latent and the two passes, and run a
// fixed stand-in for the trained context network.
//
// Listing: anchors (non-anchors) channel by channel in raster order. Row h
// of a channel holds ceil(W/2) anchors when h is even, floor(W/2) when odd
// (the reverse for non-anchors), so position (c, h, w) of its class has
// index c * per_channel + (h / 2) * W + (h & 1) * first_row + (w >> 1),
// first_row = ceil(W/2) for anchors, floor(W/2) for non-anchors.
//
// Stand-in context (a fixed function in place of the trained network): for
// a non-anchor with in-bounds 4-neighbours of symbol sum ctx (64-bit) and
// count cnt, each component keeps w_k and takes
//   m_k = fmaf(-cnt, mu_k, float(ctx)),  mu'_k = fmaf(0.125, m_k, mu_k),
//   sigma'_k = 0.75 sigma_k,
// each one FP32 rounding in this order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"

using namespace fgmm;

namespace {

struct Geom {
    int64_t C, H, W, N;
    int64_t per_a, per_n;   // anchors / non-anchors per channel
};

__host__ __device__ inline Geom make_geom(int64_t C, int64_t H, int64_t W)
{
    Geom g;
    g.C = C;
    g.H = H;
    g.W = W;
    g.N = C * H * W;
    g.per_a = (H * W + 1) / 2;
    g.per_n = H * W - g.per_a;
    return g;
}

// Class (anchor?) and index within the class of position n.
__device__ __forceinline__ bool ckbd_index(const Geom& g, int64_t n, int64_t& i)
{
    const int64_t hw = g.H * g.W;
    const int64_t c = n / hw, r = n - c * hw;
    const int64_t h = r / g.W, w = r - h * g.W;
    const bool anchor = ((h + w) & 1) == 0;
    const int64_t first = anchor ? (g.W + 1) / 2 : g.W / 2;
    i = c * (anchor ? g.per_a : g.per_n) + (h >> 1) * g.W + (h & 1) * first + (w >> 1);
    return anchor;
}

// Parameters are moved as raw elements of their dtype (E = 4 or 2 bytes).
template <typename E>
__global__ void __launch_bounds__(256) fgmm_ckbd_split_kernel(Geom g, int K, const E* __restrict__ params,
                                                              const int32_t* __restrict__ y, E* __restrict__ pa,
                                                              int32_t* __restrict__ ya, E* __restrict__ pn,
                                                              int32_t* __restrict__ yn)
{
    const int64_t Na = g.C * g.per_a, Nn = g.C * g.per_n;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < g.N; n += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        const bool anchor = ckbd_index(g, n, i);
        E* po = anchor ? pa : pn;
        int32_t* yo = anchor ? ya : yn;
        const int64_t M = anchor ? Na : Nn;
        if (po)
            for (int r = 0; r < 3 * K; ++r) po[r * M + i] = params[r * g.N + n];
        if (yo && y) yo[i] = __ldg(y + n);
    }
}

__global__ void __launch_bounds__(256) fgmm_ckbd_merge_kernel(Geom g, const int32_t* __restrict__ ya,
                                                              const int32_t* __restrict__ yn,
                                                              int32_t* __restrict__ y)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < g.N; n += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        if (ckbd_index(g, n, i)) y[n] = __ldg(ya + i);
        else if (yn) y[n] = __ldg(yn + i);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) fgmm_ckbd_context_kernel(Geom g, int K, const T* __restrict__ params,
                                                                const int32_t* __restrict__ y,
                                                                float* __restrict__ pn)
{
    const int64_t Nn = g.C * g.per_n;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < g.N; n += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        if (ckbd_index(g, n, i)) continue;
        const int64_t r = n % (g.H * g.W), h = r / g.W, w = r - h * g.W;
        int64_t ctx = 0;
        int cnt = 0;
        if (h > 0) { ctx += __ldg(y + n - g.W); ++cnt; }
        if (h + 1 < g.H) { ctx += __ldg(y + n + g.W); ++cnt; }
        if (w > 0) { ctx += __ldg(y + n - 1); ++cnt; }
        if (w + 1 < g.W) { ctx += __ldg(y + n + 1); ++cnt; }
        const float fc = __ll2float_rn(ctx), fn = -(float)cnt;
        for (int k = 0; k < K; ++k) {
            const float wk = load_param(params, (int64_t)(0 * K + k) * g.N + n);
            const float mu = load_param(params, (int64_t)(1 * K + k) * g.N + n);
            const float sg = load_param(params, (int64_t)(2 * K + k) * g.N + n);
            const float m = __fmaf_rn(fn, mu, fc);
            pn[(0 * K + k) * Nn + i] = wk;
            pn[(1 * K + k) * Nn + i] = __fmaf_rn(0.125f, m, mu);
            pn[(2 * K + k) * Nn + i] = __fmul_rn(sg, 0.75f);
        }
    }
}

unsigned grid_for(int64_t N, int sms)
{
    const int64_t b = (N + 255) / 256;
    return (unsigned)(b < (int64_t)sms * 16 ? (b > 0 ? b : 1) : (int64_t)sms * 16);
}

fgmm_status check_geom(fgmm_handle* h, int64_t C, int64_t H, int64_t W)
{
    if (C < 0 || H < 0 || W < 0 || (H > 0 && W > 0 && C > ((int64_t)1 << 40) / (H * W)) || H > ((int64_t)1 << 30) ||
        W > ((int64_t)1 << 30))
        return fail(h, FGMM_ERR_INVALID_ARG, "checkerboard: bad C, H, W");
    return FGMM_OK;
}

}  // namespace

extern "C" {

int64_t fgmm_ckbd_anchors(int64_t C, int64_t H, int64_t W)
{
    if (C < 0 || H < 0 || W < 0) return -1;
    return C * ((H * W + 1) / 2);
}

fgmm_status fgmm_ckbd_split(fgmm_handle* h, const fgmm_latent* lat, int64_t C, int64_t H, int64_t W,
                            const int32_t* y, void* params_a, int32_t* y_a, void* params_n, int32_t* y_n,
                            void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    s = check_geom(h, C, H, W);
    if (s != FGMM_OK) return s;
    if (lat->N != C * H * W) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_split: N != C * H * W");
    if (lat->N > 0 && (y_a || y_n) && !y) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_split: NULL y");
    if (lat->N == 0) return FGMM_OK;
    const Geom g = make_geom(C, H, W);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = grid_for(g.N, h->num_sms);
    if (lat->dtype == FGMM_DTYPE_BF16)
        fgmm_ckbd_split_kernel<uint16_t><<<grid, 256, 0, st>>>(g, lat->K, static_cast<const uint16_t*>(lat->params),
                                                               y, static_cast<uint16_t*>(params_a), y_a,
                                                               static_cast<uint16_t*>(params_n), y_n);
    else
        fgmm_ckbd_split_kernel<uint32_t><<<grid, 256, 0, st>>>(g, lat->K, static_cast<const uint32_t*>(lat->params),
                                                               y, static_cast<uint32_t*>(params_a), y_a,
                                                               static_cast<uint32_t*>(params_n), y_n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_ckbd_split launch");
}

fgmm_status fgmm_ckbd_merge(fgmm_handle* h, int64_t C, int64_t H, int64_t W, const int32_t* y_a,
                            const int32_t* y_n, int32_t* y, void* stream)
{
    if (!h) return FGMM_ERR_INVALID_ARG;
    fgmm_status s = check_geom(h, C, H, W);
    if (s != FGMM_OK) return s;
    const Geom g = make_geom(C, H, W);
    if (g.N == 0) return FGMM_OK;
    if (!y_a || !y) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_merge: NULL buffer");
    fgmm_ckbd_merge_kernel<<<grid_for(g.N, h->num_sms), 256, 0, static_cast<cudaStream_t>(stream)>>>(g, y_a, y_n, y);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_ckbd_merge launch");
}

fgmm_status fgmm_ckbd_context(fgmm_handle* h, const fgmm_latent* lat, int64_t C, int64_t H, int64_t W,
                              const int32_t* y, float* params_n, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    s = check_geom(h, C, H, W);
    if (s != FGMM_OK) return s;
    if (lat->N != C * H * W) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_context: N != C * H * W");
    const Geom g = make_geom(C, H, W);
    if (g.C * g.per_n == 0) return FGMM_OK;
    if (!y || !params_n) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_context: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = grid_for(g.N, h->num_sms);
    if (lat->dtype == FGMM_DTYPE_BF16)
        fgmm_ckbd_context_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(
            g, lat->K, static_cast<const __nv_bfloat16*>(lat->params), y, params_n);
    else
        fgmm_ckbd_context_kernel<float><<<grid, 256, 0, st>>>(g, lat->K, static_cast<const float*>(lat->params), y,
                                                              params_n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_ckbd_context launch");
}

}  // extern "C"
