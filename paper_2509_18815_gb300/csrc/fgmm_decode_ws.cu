// fgmm_decode_ws.cu -- warp-specialised decoder, fp32 parameters (kernel in
// fgmm_decode_ws.cuh).
#include "fgmm_decode_ws.cuh"

namespace fgmm {

cudaError_t launch_ws_f32(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st)
{
    return launch_ws_t<float>(a, K, CL, SPW, st);
}

cudaError_t ws_ckbd_capacity(int K, int* clusters)
{
    switch (K) {
    case 1: return ws_ckbd_capacity_k<1>(clusters);
    case 2: return ws_ckbd_capacity_k<2>(clusters);
    case 3: return ws_ckbd_capacity_k<3>(clusters);
    default: return ws_ckbd_capacity_k<4>(clusters);
    }
}

cudaError_t launch_ws_ckbd(const CkbdFuseArgs& a, int K, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_ws_ckbd_k<1>(a, st);
    case 2: return launch_ws_ckbd_k<2>(a, st);
    case 3: return launch_ws_ckbd_k<3>(a, st);
    default: return launch_ws_ckbd_k<4>(a, st);
    }
}

}  // namespace fgmm
