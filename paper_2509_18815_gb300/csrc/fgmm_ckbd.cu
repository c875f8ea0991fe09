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
//
// fgmm_ckbd_encode computes both passes' intervals in one kernel and runs
// both rANS encoders in one launch; fgmm_ckbd_decode runs both passes in one
// launch of the warp-specialised decoder when the plan allows, so that the
// non-anchors decode a few steps behind the anchors they depend on.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"
#include "fgmm_segment.cuh"

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

// Both passes' intervals in one pass over the latent (the split, the
// stand-in context and the interval kernel of the separate calls): symbol n
// of class c at index i gets sf_c[i] = start | freq << 16 of its quantised-
// CDF interval under the anchors' hyperprior parameters, or under the
// context's parameters for a non-anchor (computed from the hyperprior
// parameters widened to fp32 and the neighbours in y, as the context kernel
// does), and y_c[i] = y[n].
template <int K, typename T, int PHI>
__global__ void __launch_bounds__(256) fgmm_ckbd_interval_kernel(Geom g, const T* __restrict__ params,
                                                                 const int32_t* __restrict__ y,
                                                                 uint32_t* __restrict__ sf_a, int32_t* __restrict__ y_a,
                                                                 uint32_t* __restrict__ sf_n, int32_t* __restrict__ y_n,
                                                                 int32_t* err)
{
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < g.N; n += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        const bool anchor = ckbd_index(g, n, i);
        RawParams<K> r;
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) r.v[q] = load_param(params, (int64_t)q * g.N + n);
        const int32_t s = __ldg(y + n);
        if (!anchor) {
            const int64_t rr = n % (g.H * g.W), h = rr / g.W, w = rr - h * g.W;
            int64_t ctx = 0;
            int cnt = 0;
            if (h > 0) { ctx += __ldg(y + n - g.W); ++cnt; }
            if (h + 1 < g.H) { ctx += __ldg(y + n + g.W); ++cnt; }
            if (w > 0) { ctx += __ldg(y + n - 1); ++cnt; }
            if (w + 1 < g.W) { ctx += __ldg(y + n + 1); ++cnt; }
            const float fc = __ll2float_rn(ctx), fn = -(float)cnt;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float mu = r.v[K + k];
                r.v[K + k] = __fmaf_rn(0.125f, __fmaf_rn(fn, mu, fc), mu);
                r.v[2 * K + k] = __fmul_rn(r.v[2 * K + k], 0.75f);
            }
        }
        Mix<K> m;
        if (!mix_from_params<K>(r, m)) set_error(err, kErrBadParams);
        uint32_t st, fr;
        interval_of<K, PHI>(m, s, st, fr);
        (anchor ? sf_a : sf_n)[i] = st | (fr << 16);
        (anchor ? y_a : y_n)[i] = s;
    }
}

template <typename T, int PHI>
void launch_ckbd_interval_t(const Geom& g, int K, const void* params, const int32_t* y, uint32_t* sf_a, int32_t* y_a,
                            uint32_t* sf_n, int32_t* y_n, int32_t* err, unsigned grid, cudaStream_t st)
{
    const T* p = static_cast<const T*>(params);
    switch (K) {
    case 1: fgmm_ckbd_interval_kernel<1, T, PHI><<<grid, 256, 0, st>>>(g, p, y, sf_a, y_a, sf_n, y_n, err); break;
    case 2: fgmm_ckbd_interval_kernel<2, T, PHI><<<grid, 256, 0, st>>>(g, p, y, sf_a, y_a, sf_n, y_n, err); break;
    case 3: fgmm_ckbd_interval_kernel<3, T, PHI><<<grid, 256, 0, st>>>(g, p, y, sf_a, y_a, sf_n, y_n, err); break;
    default: fgmm_ckbd_interval_kernel<4, T, PHI><<<grid, 256, 0, st>>>(g, p, y, sf_a, y_a, sf_n, y_n, err); break;
    }
}

template <typename T>
void launch_ckbd_interval(const Geom& g, int K, int phi, const void* params, const int32_t* y, uint32_t* sf_a,
                          int32_t* y_a, uint32_t* sf_n, int32_t* y_n, int32_t* err, unsigned grid, cudaStream_t st)
{
    if (phi == FGMM_PHI_LOGISTIC)
        launch_ckbd_interval_t<T, kPhiLogistic>(g, K, params, y, sf_a, y_a, sf_n, y_n, err, grid, st);
    else if (phi == FGMM_PHI_POLYA)
        launch_ckbd_interval_t<T, kPhiPolya>(g, K, params, y, sf_a, y_a, sf_n, y_n, err, grid, st);
    else
        launch_ckbd_interval_t<T, kPhiAS>(g, K, params, y, sf_a, y_a, sf_n, y_n, err, grid, st);
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

// Whether fgmm_ckbd_decode runs both passes in one launch: the A&S
// approximation, no decoder option or test hook, the
// automatic plan of the combined segments is the fused kernel's (16 lanes,
// clusters of 4, 16-point first round), every cluster resident at once,
// fewer than 2^24 steps per pass and C H W < 2^31.
fgmm_status ckbd_fusable(fgmm_handle* h, int K, int dtype, int64_t C, int64_t H, int64_t W, int32_t Sa, int32_t Sn,
                         bool* fuse)
{
    *fuse = false;
    const Geom g = make_geom(C, H, W);
    const int64_t Na = g.C * g.per_a, Nn = g.C * g.per_n;
    if (h->phi != FGMM_PHI_AS || h->decode_lanes != 0 || h->decode_cluster != 0 ||
        h->decode_round0 != 0 || h->test_silent_stream >= 0 || Na == 0 || Nn == 0 ||
        steps_of(Na, Sa) >= ((int64_t)1 << 24) || steps_of(Nn, Sn) >= ((int64_t)1 << 24) ||
        g.N >= ((int64_t)1 << 31))
        return FGMM_OK;
    const int64_t nseg = Sa / 32 + Sn / 32;
    int lanes = 1, cluster = 1, round0 = 0, kernel = 0;
    decode_resolve(nseg, h->num_sms, 0, 0, 0, FGMM_PHI_AS, &lanes, &cluster, &round0, &kernel);
    if (!(kernel == FGMM_DEC_WS && lanes == 16 && cluster == 4 && round0 == 16)) return FGMM_OK;
    const int di = dtype == FGMM_DTYPE_BF16 ? 1 : 0;
    if (h->ckbd_clusters[di][K] < 0) {
        int n = 0;
        cudaError_t e = ws_ckbd_capacity(K, dtype, &n);
        if (e != cudaSuccess) return cuda_fail(h, e, "checkerboard decode: occupancy query");
        h->ckbd_clusters[di][K] = n;
    }
    *fuse = nseg <= h->ckbd_clusters[di][K];
    return FGMM_OK;
}

}  // namespace

extern "C" {

fgmm_status fgmm_ckbd_encode(fgmm_handle* h, const fgmm_latent* lat, int64_t C, int64_t H, int64_t W,
                             const int32_t* y, int32_t Sa, uint16_t* words_a, int64_t words_cap_a, int64_t* offsets_a,
                             int64_t* n_words_a, int32_t Sn, uint16_t* words_n, int64_t words_cap_n,
                             int64_t* offsets_n, int64_t* n_words_n, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    s = check_geom(h, C, H, W);
    if (s != FGMM_OK) return s;
    if (lat->N != C * H * W) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_encode: N != C * H * W");
    if (Sa <= 0 || Sa % 32 != 0 || Sn <= 0 || Sn % 32 != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets_a || !offsets_n || !n_words_a || !n_words_n || words_cap_a < 0 || words_cap_n < 0 ||
        (words_cap_a > 0 && !words_a) || (words_cap_n > 0 && !words_n) || (lat->N > 0 && !y))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_encode: NULL buffer");
    const Geom g = make_geom(C, H, W);
    const int64_t Na = g.C * g.per_a, Nn = g.C * g.per_n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // workspace: intervals [Na] | [Nn] | symbols [Na] | [Nn] | segment scratch
    // of pass 1 | of pass 2 | segment lengths of pass 1 | of pass 2
    const int64_t ga = Sa / 32, gn = Sn / 32;
    const int64_t cap_a = encode_seg_cap(Na, Sa), cap_n = encode_seg_cap(Nn, Sn);
    size_t off[9];
    off[0] = 0;
    off[1] = align_up(off[0] + 4 * (size_t)Na, 256);
    off[2] = align_up(off[1] + 4 * (size_t)Nn, 256);
    off[3] = align_up(off[2] + 4 * (size_t)Na, 256);
    off[4] = align_up(off[3] + 4 * (size_t)Nn, 256);
    off[5] = align_up(off[4] + 2 * (size_t)(ga * cap_a), 256);
    off[6] = align_up(off[5] + 2 * (size_t)(gn * cap_n), 256);
    off[7] = align_up(off[6] + 8 * (size_t)ga, 256);
    off[8] = off[7] + 8 * (size_t)gn;
    s = ws_reserve(h, off[8], st);
    if (s != FGMM_OK) return s;
    char* base = static_cast<char*>(h->ws);
    uint32_t* sf_a = reinterpret_cast<uint32_t*>(base + off[0]);
    uint32_t* sf_n = reinterpret_cast<uint32_t*>(base + off[1]);
    int32_t* y_a = reinterpret_cast<int32_t*>(base + off[2]);
    int32_t* y_n = reinterpret_cast<int32_t*>(base + off[3]);
    if (g.N > 0) {
        const unsigned grid = grid_for(g.N, h->num_sms);
        if (lat->dtype == FGMM_DTYPE_BF16)
            launch_ckbd_interval<__nv_bfloat16>(g, lat->K, h->phi, lat->params, y, sf_a, y_a, sf_n, y_n, h->d_err,
                                                grid, st);
        else
            launch_ckbd_interval<float>(g, lat->K, h->phi, lat->params, y, sf_a, y_a, sf_n, y_n, h->d_err, grid, st);
    }
    EncPass pa{sf_a, y_a, Na, Sa, reinterpret_cast<uint16_t*>(base + off[4]), reinterpret_cast<int64_t*>(base + off[6]),
               words_a, words_cap_a, offsets_a, n_words_a};
    EncPass pn{sf_n, y_n, Nn, Sn, reinterpret_cast<uint16_t*>(base + off[5]), reinterpret_cast<int64_t*>(base + off[7]),
               words_n, words_cap_n, offsets_n, n_words_n};
    encode2_from_intervals(pa, pn, h->d_err, h->num_sms, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_ckbd_encode launch");
}

fgmm_status fgmm_ckbd_decode_plan(fgmm_handle* h, int32_t K, int32_t dtype, int64_t C, int64_t H, int64_t W,
                                  int32_t Sa, int32_t Sn, int32_t* fused)
{
    if (!h || !fused) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_decode_plan: NULL argument");
    if (K < 1 || K > 4 || (dtype != FGMM_DTYPE_F32 && dtype != FGMM_DTYPE_BF16))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_decode_plan: bad K or dtype");
    if (Sa <= 0 || Sa % 32 != 0 || Sn <= 0 || Sn % 32 != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    fgmm_status s = check_geom(h, C, H, W);
    if (s != FGMM_OK) return s;
    bool f = false;
    s = ckbd_fusable(h, K, dtype, C, H, W, Sa, Sn, &f);
    if (s != FGMM_OK) return s;
    *fused = f ? 1 : 0;
    return FGMM_OK;
}

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

fgmm_status fgmm_ckbd_decode(fgmm_handle* h, const fgmm_latent* lat, int64_t C, int64_t H, int64_t W,
                             const uint16_t* words_a, int64_t n_words_a, const int64_t* offsets_a, int32_t Sa,
                             const uint16_t* words_n, int64_t n_words_n, const int64_t* offsets_n, int32_t Sn,
                             int32_t* y, void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    s = check_geom(h, C, H, W);
    if (s != FGMM_OK) return s;
    if (lat->N != C * H * W) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_decode: N != C * H * W");
    if (Sa <= 0 || Sa % 32 != 0 || Sn <= 0 || Sn % 32 != 0)
        return fail(h, FGMM_ERR_INVALID_ARG, "S must be a positive multiple of 32");
    if (!offsets_a || !offsets_n || n_words_a < 0 || n_words_n < 0 || (n_words_a > 0 && !words_a) ||
        (n_words_n > 0 && !words_n) || (lat->N > 0 && !y))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_ckbd_decode: NULL buffer");
    const Geom g = make_geom(C, H, W);
    const int64_t Na = g.C * g.per_a, Nn = g.C * g.per_n;
    const int K = lat->K;
    const size_t esz = lat->dtype == FGMM_DTYPE_BF16 ? 2 : 4;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // workspace: anchor params [3K][Na] | non-anchor params [3K][Nn] (room
    // for fp32: lat's dtype in one launch, the context's fp32 otherwise) |
    // anchors [Na] | non-anchors [Nn] | pass-0 step arrivals [steps]
    const size_t b_pa = align_up(3 * (size_t)K * Na * esz, 256), b_pn = align_up(3 * (size_t)K * Nn * 4, 256);
    const size_t b_ya = align_up(4 * (size_t)Na, 256), b_yn = align_up(4 * (size_t)Nn, 256);
    const size_t b_pr = align_up(4 * (size_t)steps_of(Na, Sa), 256);
    s = ws_reserve(h, b_pa + b_pn + b_ya + b_yn + b_pr, st);
    if (s != FGMM_OK) return s;
    unsigned char* base = static_cast<unsigned char*>(h->ws);
    void* pa = base;
    float* pn = reinterpret_cast<float*>(base + b_pa);
    int32_t* ya = reinterpret_cast<int32_t*>(base + b_pa + b_pn);
    int32_t* yn = reinterpret_cast<int32_t*>(base + b_pa + b_pn + b_ya);
    uint32_t* arrivals = reinterpret_cast<uint32_t*>(base + b_pa + b_pn + b_ya + b_yn);
    DecodeArgs da, dn;
    da.params = pa;
    da.N = Na;
    da.S = Sa;
    da.T = steps_of(Na, Sa);
    da.words = words_a;
    da.n_words = n_words_a;
    da.offsets = offsets_a;
    da.nseg = Sa / 32;
    da.out = ya;
    dn.params = pn;
    dn.N = Nn;
    dn.S = Sn;
    dn.T = steps_of(Nn, Sn);
    dn.words = words_n;
    dn.n_words = n_words_n;
    dn.offsets = offsets_n;
    dn.nseg = Sn / 32;
    dn.out = yn;

    bool fuse = false;
    s = ckbd_fusable(h, K, lat->dtype, C, H, W, Sa, Sn, &fuse);
    if (s != FGMM_OK) return s;
    const unsigned grid = grid_for(g.N, h->num_sms);
    cudaError_t e;
    if (fuse) {   // the hyperprior parameters of both classes, in lat's dtype
        if (lat->dtype == FGMM_DTYPE_BF16)
            fgmm_ckbd_split_kernel<uint16_t><<<grid, 256, 0, st>>>(g, K, static_cast<const uint16_t*>(lat->params),
                                                                   nullptr, static_cast<uint16_t*>(pa), nullptr,
                                                                   reinterpret_cast<uint16_t*>(pn), nullptr);
        else
            fgmm_ckbd_split_kernel<uint32_t><<<grid, 256, 0, st>>>(g, K, static_cast<const uint32_t*>(lat->params),
                                                                   nullptr, static_cast<uint32_t*>(pa), nullptr,
                                                                   reinterpret_cast<uint32_t*>(pn), nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(arrivals, 0, 4 * (size_t)da.T, st);
        if (e == cudaSuccess) {
            CkbdFuseArgs fa;
            da.err = dn.err = h->d_err;
            da.stats = dn.stats = h->stats_on ? h->d_stats : nullptr;
            da.r0 = dn.r0 = 16;
            fa.pass[0] = da;
            fa.pass[1] = dn;
            fa.C = C;
            fa.H = H;
            fa.W = W;
            fa.arrivals = arrivals;
            fa.silent_arrivals = h->test_silent_arrivals;
            e = launch_ws_ckbd(fa, K, lat->dtype, st);
        }
        if (e == cudaSuccess) {
            fgmm_ckbd_merge_kernel<<<grid, 256, 0, st>>>(g, ya, yn, y);
            e = cudaGetLastError();
        }
        return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_ckbd_decode launch");
    }
    // the passes one after the other
    if (g.N == 0) return FGMM_OK;
    if (lat->dtype == FGMM_DTYPE_BF16)
        fgmm_ckbd_split_kernel<uint16_t><<<grid, 256, 0, st>>>(g, K, static_cast<const uint16_t*>(lat->params),
                                                               nullptr, static_cast<uint16_t*>(pa), nullptr,
                                                               nullptr, nullptr);
    else
        fgmm_ckbd_split_kernel<uint32_t><<<grid, 256, 0, st>>>(g, K, static_cast<const uint32_t*>(lat->params),
                                                               nullptr, static_cast<uint32_t*>(pa), nullptr,
                                                               nullptr, nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = decode_planned(h, da, K, lat->dtype, st);
    if (e == cudaSuccess) {
        fgmm_ckbd_merge_kernel<<<grid, 256, 0, st>>>(g, ya, nullptr, y);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && Nn > 0) {
        if (lat->dtype == FGMM_DTYPE_BF16)
            fgmm_ckbd_context_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(
                g, K, static_cast<const __nv_bfloat16*>(lat->params), y, pn);
        else
            fgmm_ckbd_context_kernel<float><<<grid, 256, 0, st>>>(g, K, static_cast<const float*>(lat->params), y,
                                                                  pn);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = decode_planned(h, dn, K, FGMM_DTYPE_F32, st);
        if (e == cudaSuccess) {
            fgmm_ckbd_merge_kernel<<<grid, 256, 0, st>>>(g, ya, yn, y);
            e = cudaGetLastError();
        }
    }
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_ckbd_decode launch");
}

}  // extern "C"
