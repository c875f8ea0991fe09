// fgmm_peak.cu -- throughput probes for the roofline denominators.
//
// The coder's decode is bound by FP32 arithmetic (quantised-CDF
// evaluations) and its encode by HBM and FP32 arithmetic. The FP32 peak the
// benchmark divides by is measured here rather than derived from unit counts:
// a grid of 4 CTAs x 256 threads per SM runs independent chains of FP32
// fused multiply-adds (or of the XU reciprocal approximation that the
// reciprocal in every CDF evaluation starts from, each followed by one FMA),
// 8 chains per thread, so
// every SM sub-partition has enough independent instructions to issue one
// per cycle. The caller times the launch with CUDA events; ops counts one
// FMA (or one reciprocal) per lane as one operation.
#include <cuda_runtime.h>

#include <cstdint>

#include "fgmm_internal.h"

using namespace fgmm;

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 16;   // chain steps per loop iteration

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) fgmm_peak_kernel(int64_t iters, float a, float b, float* sink)
{
    float v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = 1.0f + (float)(threadIdx.x & 7) * 0x1p-10f + (float)i * 0x1p-6f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                if constexpr (KIND == 0) {
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(v[i]) : "f"(a), "f"(b));
                } else {
                    // x <- a / x + b: the reciprocal (XU) plus one FMA, so
                    // no pair of steps can cancel; the XU pipe, 1/8 the FMA
                    // rate, sets the time
                    asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(v[i]));
                    asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(v[i]) : "f"(a), "f"(b));
                }
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += v[i];
    // the values stay near 1 (x -> a x + b with a + b = 1, or x -> a / x + b
    // with a = 1/2, b = 1), so this
    // store never happens; it only keeps the chains alive
    if (s == -1.0f) *sink = s;
}

}  // namespace

extern "C" fgmm_status fgmm_peak_probe(fgmm_handle* h, int32_t kind, int64_t iters, float* sink, double* ops_out,
                                       void* stream)
{
    if (!h || !sink || !ops_out || iters < 1 || (kind != FGMM_PEAK_FMA && kind != FGMM_PEAK_RCP))
        return fail(h, FGMM_ERR_INVALID_ARG, "fgmm_peak_probe: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = h->num_sms * kPeakBlocksPerSM;
    if (kind == FGMM_PEAK_FMA) fgmm_peak_kernel<0><<<grid, kPeakThreads, 0, st>>>(iters, 0.999f, 0.001f, sink);
    else fgmm_peak_kernel<1><<<grid, kPeakThreads, 0, st>>>(iters, 0.5f, 1.0f, sink);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "fgmm_peak_probe launch");
    *ops_out = (double)grid * kPeakThreads * (double)iters * kUnroll * kChains;
    return FGMM_OK;
}
