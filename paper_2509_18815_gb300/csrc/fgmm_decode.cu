// fgmm_decode.cu -- decoder dispatch and the fp32-parameter instantiations
// (kernels in fgmm_decode_impl.cuh).
#include "fgmm_decode_impl.cuh"

namespace fgmm {

cudaError_t launch_decode_bf16(const DecodeArgs& a, int K, int G, int CL, cudaStream_t st);

void decode_config_auto(int64_t nseg, int num_sms, int* lanes, int* cluster, int* round0)
{
    // Enough segments to give every SM several warps: one lane per stream,
    // binary search (least work). Fewer: G lanes per stream, and a cluster of
    // CTAs per segment when the segments leave most SMs idle; the fewer the
    // segments, the more lanes per stream. With 16 lanes per stream a
    // 16-point first round (two streams per producer warp) halves the
    // producers' issue slots. Measured on GB300 (152 SMs): 1-8 segments ->
    // 32 lanes x clusters of 8; 16-32 -> 16 lanes x clusters of 4; 48 -> 16
    // lanes x clusters of 8; 68-100 -> 16 lanes x clusters of 4; 152 -> 8
    // lanes; 200-304 -> 4 lanes; 608 -> 1 lane.
    const int64_t sms = num_sms;
    *round0 = 32;
    if (nseg >= 4 * sms) { *lanes = 1; *cluster = 1; return; }
    if (nseg * 16 <= sms) { *lanes = 32; *cluster = 8; return; }
    *round0 = 16;
    if (nseg * 4 <= sms) { *lanes = 16; *cluster = 4; return; }
    if (nseg * 8 <= sms * 3) { *lanes = 16; *cluster = 8; return; }
    if (nseg * 3 <= sms * 2) { *lanes = 16; *cluster = 4; return; }
    *round0 = 32;
    if (nseg * 4 <= sms * 5) { *lanes = 8; *cluster = 1; return; }
    *lanes = 4;
    *cluster = 1;
}

void decode_resolve(int64_t nseg, int num_sms, int opt_lanes, int opt_cluster, int opt_round0, int phi, int* lanes,
                    int* cluster, int* round0, int* kernel)
{
    if (phi != FGMM_PHI_AS) {   // the other approximations run on the lane decoder only
        *lanes = 1;
        *cluster = 1;
        *round0 = 0;
        *kernel = FGMM_DEC_LANE;
        return;
    }
    int G = 1, CL = 1, R0 = 32;
    decode_config_auto(nseg, num_sms, &G, &CL, &R0);
    if (opt_lanes > 0) {
        G = opt_lanes;
        CL = 1;
        R0 = 32;
    }
    if (opt_cluster > 0) CL = opt_cluster;
    if (G < 2) CL = 1;
    if (G < 8 && CL > 4) CL = 4;   // the G-ary kernel takes clusters of up to 4
    if (CL > G) CL = G;
    if (G == 32 && CL < 2) CL = 2;   // 32 lanes per stream: the warp-specialised kernel, clusters of 2 or more
    *lanes = G;
    *cluster = CL;
    // G >= 8 with a cluster: the warp-specialised kernel (32 / G streams per
    // consumer warp; a 16-point first round only with 16 lanes per stream)
    if (G == 1) *kernel = FGMM_DEC_LANE;
    else if (CL >= 2 && G >= 8) *kernel = FGMM_DEC_WS;
    else *kernel = FGMM_DEC_COOP;
    if (opt_round0 > 0) R0 = opt_round0;
    *round0 = *kernel == FGMM_DEC_WS ? (G == 16 ? R0 : 32) : 0;
}

cudaError_t launch_decode(const DecodeArgs& a, int K, int dtype, int G, int CL, cudaStream_t st)
{
    if (a.nseg == 0) return cudaSuccess;
    if (dtype == FGMM_DTYPE_BF16) return launch_decode_bf16(a, K, G, CL, st);
    return launch_decode_t<float>(a, K, G, CL, st);
}

}  // namespace fgmm
