// fgmm_decode_ws_bf16.cu -- warp-specialised decoder, bf16 parameters
// (kernel in fgmm_decode_ws.cuh).
#include "fgmm_decode_ws.cuh"

namespace fgmm {

cudaError_t launch_ws_bf16(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st)
{
    return launch_ws_t<__nv_bfloat16>(a, K, CL, SPW, st);
}

cudaError_t ws_ckbd_capacity_bf16(int K, int* clusters) { return ws_ckbd_capacity_t<__nv_bfloat16>(K, clusters); }

cudaError_t launch_ws_ckbd_bf16(const CkbdFuseArgs& a, int K, cudaStream_t st)
{
    return launch_ws_ckbd_t<__nv_bfloat16>(a, K, st);
}

}  // namespace fgmm
