// fgmm_decode_ws.cu -- warp-specialised decoder, fp32 parameters (kernel in
// fgmm_decode_ws.cuh).
#include "fgmm_decode_ws.cuh"

namespace fgmm {

cudaError_t launch_ws_f32(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st)
{
    return launch_ws_t<float>(a, K, CL, SPW, st);
}

}  // namespace fgmm
