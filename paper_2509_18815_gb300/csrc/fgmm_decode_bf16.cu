// fgmm_decode_bf16.cu -- decoder instantiations for bf16 parameters
// (kernels in fgmm_decode_impl.cuh).
#include "fgmm_decode_impl.cuh"

namespace fgmm {

cudaError_t launch_decode_bf16(const DecodeArgs& a, int K, int G, int CL, cudaStream_t st)
{
    return launch_decode_t<__nv_bfloat16>(a, K, G, CL, st);
}

}  // namespace fgmm
