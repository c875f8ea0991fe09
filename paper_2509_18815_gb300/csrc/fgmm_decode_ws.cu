// fgmm_decode_ws.cu -- warp-specialised decoder, fp32 parameters (kernel in
// fgmm_decode_ws.cuh).
#include "fgmm_decode_ws.cuh"

namespace fgmm {

cudaError_t launch_ws_f32(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st)
{
    return launch_ws_t<float>(a, K, CL, SPW, st);
}

cudaError_t ws_ckbd_capacity(int K, int dtype, int* clusters)
{
    return dtype == FGMM_DTYPE_BF16 ? ws_ckbd_capacity_bf16(K, clusters) : ws_ckbd_capacity_t<float>(K, clusters);
}

cudaError_t launch_ws_ckbd(const CkbdFuseArgs& a, int K, int dtype, cudaStream_t st)
{
    return dtype == FGMM_DTYPE_BF16 ? launch_ws_ckbd_bf16(a, K, st) : launch_ws_ckbd_t<float>(a, K, st);
}

}  // namespace fgmm
