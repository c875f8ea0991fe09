// fgmm_audit.cu -- FP64 rate audit of the FP32 coder against the exact
// mixture (the "no approximation" reference of Sec. V, which uses erfc).
//
// Per symbol s of a latent:
//   ideal bits  -log2 p64(s), p64(s) = sum_k w_k [Phi(z_k(s+1/2)) - Phi(z_k(s-1/2))]
//               in FP64, each difference taken on the component's tail side
//               (erfc of the smaller |z|) so that it does not cancel;
//   coded bits  -log2(freq / 2^16) of the interval the coder uses, plus 32
//               raw bits for an escape;
//   CDF error   |F-hat32(b) - F64(b)| at the boundaries the encoder evaluates
//               (s - 1/2 if s > lo, and s + 1/2; hi + 1/2 for an escape).
// This is the only FP64 code in the library; no coding step depends on it.
// Per-block partial results are reduced in a fixed order by a second
// one-block kernel, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cstdint>

#include "fgmm_device.cuh"
#include "fgmm_internal.h"

using namespace fgmm;

namespace {

constexpr int kAuditThreads = 256;

__device__ __forceinline__ double ncdf64(double z) { return 0.5 * erfc(-z * 0.70710678118654752440); }

// Phi(b) - Phi(a) for a <= b without cancellation.
__device__ __forceinline__ double nmass64(double a, double b)
{
    const double r = 0.70710678118654752440;   // 1/sqrt(2)
    if (a >= 0.0) return 0.5 * (erfc(a * r) - erfc(b * r));
    if (b <= 0.0) return 0.5 * (erfc(-b * r) - erfc(-a * r));
    return 1.0 - 0.5 * erfc(b * r) - 0.5 * erfc(-a * r);
}

template <int K>
__device__ __forceinline__ double mix_cdf64(const float* w, const float* mu, const float* sp, double b)
{
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) acc += (double)w[k] * ncdf64((b - (double)mu[k]) / (double)sp[k]);
    return acc;
}

struct AuditPart {
    double ideal, coded, maxerr, nesc;
};

template <int K, typename T, int PHI>
__global__ void __launch_bounds__(kAuditThreads) fgmm_audit_kernel(const T* __restrict__ params, int64_t N,
                                                                   const int32_t* __restrict__ sym,
                                                                   AuditPart* __restrict__ parts, int32_t* err)
{
    double ideal = 0.0, coded = 0.0, maxerr = 0.0, nesc = 0.0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        Mix<K> m;
        if (!load_mix<K>(params, N, n, m)) set_error(err, kErrBadParams);
        float w[K], mu[K], sp[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            w[k] = load_param(params, (int64_t)k * N + n);
            mu[k] = load_param(params, (int64_t)(K + k) * N + n);
            sp[k] = fmaxf(load_param(params, (int64_t)(2 * K + k) * N + n), kSigmaMin);
        }
        const int32_t s = __ldg(sym + n);
        uint32_t st, fr;
        interval_of<K, PHI>(m, s, st, fr);
        const bool esc = st + fr == kM;
        // FP64 mass of the symbol under the exact mixture
        double p = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const double a = ((double)s - 0.5 - (double)mu[k]) / (double)sp[k];
            const double b = ((double)s + 0.5 - (double)mu[k]) / (double)sp[k];
            p += (double)w[k] * nmass64(a, b);
        }
        p = fmax(p, 2.2250738585072014e-308);
        ideal += -log2(p);
        coded += 16.0 - log2((double)fr) + (esc ? 32.0 : 0.0);
        nesc += esc ? 1.0 : 0.0;
        // CDF error at the evaluated boundaries (j - 1/2)
        int j0 = esc ? m.hi + 1 : s + 1;
        const double e0 = fabs((double)mix_cdf<K, PHI>(m, j0) - mix_cdf64<K>(w, mu, sp, (double)j0 - 0.5));
        maxerr = fmax(maxerr, e0);
        if (!esc && s > m.lo) {
            const double e1 = fabs((double)mix_cdf<K, PHI>(m, s) - mix_cdf64<K>(w, mu, sp, (double)s - 0.5));
            maxerr = fmax(maxerr, e1);
        }
    }
    // block reduction in a fixed order
    __shared__ AuditPart sm[kAuditThreads];
    sm[threadIdx.x] = AuditPart{ideal, coded, maxerr, nesc};
    __syncthreads();
    for (int off = kAuditThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            AuditPart a = sm[threadIdx.x], b = sm[threadIdx.x + off];
            sm[threadIdx.x] = AuditPart{a.ideal + b.ideal, a.coded + b.coded, fmax(a.maxerr, b.maxerr), a.nesc + b.nesc};
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(kAuditThreads) fgmm_audit_reduce_kernel(const AuditPart* __restrict__ parts,
                                                                          int nparts, double* out)
{
    __shared__ AuditPart sm[kAuditThreads];
    AuditPart acc{0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const AuditPart p = parts[i];
        acc = AuditPart{acc.ideal + p.ideal, acc.coded + p.coded, fmax(acc.maxerr, p.maxerr), acc.nesc + p.nesc};
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kAuditThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            AuditPart a = sm[threadIdx.x], b = sm[threadIdx.x + off];
            sm[threadIdx.x] = AuditPart{a.ideal + b.ideal, a.coded + b.coded, fmax(a.maxerr, b.maxerr), a.nesc + b.nesc};
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sm[0].ideal;
        out[1] = sm[0].coded;
        out[2] = sm[0].maxerr;
        out[3] = sm[0].nesc;
    }
}

template <int K, typename T, int PHI>
void launch_audit_kt(const fgmm_latent* lat, const int32_t* sym, AuditPart* parts, int nblocks, int32_t* err,
                     cudaStream_t st)
{
    fgmm_audit_kernel<K, T, PHI><<<nblocks, kAuditThreads, 0, st>>>(static_cast<const T*>(lat->params), lat->N, sym,
                                                                    parts, err);
}

template <typename T, int PHI>
void launch_audit_t(const fgmm_latent* lat, const int32_t* sym, AuditPart* parts, int nblocks, int32_t* err,
                    cudaStream_t st)
{
    switch (lat->K) {
    case 1: launch_audit_kt<1, T, PHI>(lat, sym, parts, nblocks, err, st); break;
    case 2: launch_audit_kt<2, T, PHI>(lat, sym, parts, nblocks, err, st); break;
    case 3: launch_audit_kt<3, T, PHI>(lat, sym, parts, nblocks, err, st); break;
    default: launch_audit_kt<4, T, PHI>(lat, sym, parts, nblocks, err, st); break;
    }
}

template <int PHI>
void launch_audit_phi(const fgmm_latent* lat, const int32_t* sym, AuditPart* parts, int nblocks, int32_t* err,
                      cudaStream_t st)
{
    if (lat->dtype == FGMM_DTYPE_BF16) launch_audit_t<__nv_bfloat16, PHI>(lat, sym, parts, nblocks, err, st);
    else launch_audit_t<float, PHI>(lat, sym, parts, nblocks, err, st);
}

}  // namespace

extern "C" fgmm_status fgmm_rate_audit(fgmm_handle* h, const fgmm_latent* lat, const int32_t* symbols, double* out,
                                       void* stream)
{
    fgmm_status s = check_latent(h, lat);
    if (s != FGMM_OK) return s;
    if (!out || (lat->N > 0 && !symbols)) return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_rate_audit: NULL buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t nb = (lat->N + kAuditThreads - 1) / kAuditThreads;
    if (nb > (int64_t)h->num_sms * 8) nb = (int64_t)h->num_sms * 8;
    if (nb < 1) nb = 1;
    s = ws_reserve(h, sizeof(AuditPart) * (size_t)nb, st);
    if (s != FGMM_OK) return s;
    AuditPart* parts = static_cast<AuditPart*>(h->ws);
    if (h->phi == kPhiLogistic) launch_audit_phi<kPhiLogistic>(lat, symbols, parts, (int)nb, h->d_err, st);
    else if (h->phi == kPhiPolya) launch_audit_phi<kPhiPolya>(lat, symbols, parts, (int)nb, h->d_err, st);
    else launch_audit_phi<kPhiAS>(lat, symbols, parts, (int)nb, h->d_err, st);
    fgmm_audit_reduce_kernel<<<1, kAuditThreads, 0, st>>>(parts, (int)nb, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FGMM_OK : cuda_fail(h, e, "fgmm_rate_audit launch");
}
