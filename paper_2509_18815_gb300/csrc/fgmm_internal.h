// fgmm_internal.h -- host-side handle shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/fgmm.h"

struct fgmm_handle {
    int device = 0;
    int32_t* d_err = nullptr;          // sticky device error word
    unsigned long long* d_stats = nullptr;  // [0] cdf evaluations, [1] symbols decoded
    bool stats_on = false;
    void* ws = nullptr;                // reusable workspace
    size_t ws_bytes = 0;
    int num_sms = 0;
    int decode_lanes = 0;              // 0 = automatic; else lanes per stream (1, 2, 4, 8, 16, 32)
    int decode_cluster = 0;            // 0 = automatic; else CTAs per segment (1, 2, 4, 8)
    int decode_round0 = 0;             // 0 = automatic; else first-round points of the ws decoder (16, 32)
    int test_silent_stream = -1;       // test hook: a stream of segment 0 that posts no refill flags
    int phi = 0;                       // Phi approximation (FGMM_PHI_*)
    int mlp_act = 0;                   // activation of the proposal network (FGMM_MLP_ACT_*)
    int ckbd_clusters[2][5] = {{-1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1}};   // fused two-pass decode: resident
                                                                              // clusters per dtype and K (-1 unknown)
    int test_silent_arrivals = 0;      // test hook: the fused two-pass decode's anchor CTAs count no steps
    std::string last_error;
};

namespace fgmm {

inline fgmm_status fail(fgmm_handle* h, fgmm_status st, const char* msg)
{
    if (h) h->last_error = msg;
    return st;
}

inline fgmm_status cuda_fail(fgmm_handle* h, cudaError_t e, const char* where)
{
    if (h) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
        h->last_error = buf;
    }
    return FGMM_ERR_CUDA;
}

// Ensures the workspace holds at least `bytes` (256-byte aligned base).
// Growing synchronises `stream` first so that no queued kernel still uses
// the old buffer.
fgmm_status ws_reserve(fgmm_handle* h, size_t bytes, cudaStream_t stream);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Checks the latent descriptor on the host.
fgmm_status check_latent(fgmm_handle* h, const fgmm_latent* lat);

// Encode stages shared by fgmm_encode and the table coder (fgmm_codec.cu):
// workspace for per-symbol intervals, per-segment word buffers and lengths;
// then rANS encode of the intervals, offset scan and compaction.
struct EncodeWs {
    uint32_t* sf;
    uint16_t* seg;
    int64_t* len;
    int64_t cap;
};
fgmm_status encode_reserve(fgmm_handle* h, int64_t N, int32_t S, cudaStream_t st, EncodeWs* ws);
// One latent of a two-latent encode: its intervals (sf[n] = start | freq <<
// 16) and symbols, S streams, segment scratch seg ([S/32][encode_seg_cap]
// words) and lengths len ([S/32]), and the caller's outputs.
struct EncPass {
    const uint32_t* sf;
    const int32_t* sym;
    int64_t N;
    int32_t S;
    uint16_t* seg;
    int64_t* len;
    uint16_t* words;
    int64_t words_cap;
    int64_t* offsets;
    int64_t* total;
};
int64_t encode_seg_cap(int64_t N, int32_t S);
// rANS encode of both latents' segments in one launch, then each latent's
// scan and compaction (the outputs of two fgmm_encode calls).
void encode2_from_intervals(const EncPass& a, const EncPass& b, int32_t* err, int sms, cudaStream_t st);
void encode_from_intervals(const EncodeWs& ws, const int32_t* symbols, int64_t N, int32_t S, uint16_t* words,
                           int64_t words_cap, int64_t* offsets, int64_t* n_words_out, int32_t* err, int sms,
                           cudaStream_t st);
// Exclusive scan of nseg segment lengths into offsets[0..nseg], total into
// *total_out; records FGMM_ERR_CAPACITY if the total exceeds cap.
void launch_scan(const int64_t* len, int64_t nseg, int64_t* offsets, int64_t* total_out, int64_t cap, int32_t* err,
                 cudaStream_t st);
inline int64_t steps_of(int64_t N, int32_t S) { return N > 0 ? (N + S - 1) / S : 0; }

// Decoder launch (fgmm_decode.cu).
struct DecodeArgs {
    const void* params;
    int64_t N;
    int32_t S;
    int64_t T;
    const uint16_t* words;
    int64_t n_words;
    const int64_t* offsets;
    int64_t nseg;
    int32_t* out;
    int32_t* err;
    unsigned long long* stats;
    int r0 = 32;                       // first-round points of the warp-specialised decoder
    int silent = -1;                   // test hook: stream of segment 0 that posts no refill flags
    int phi = 0;                       // Phi approximation (FGMM_PHI_*); non-A&S only on the lane decoder
};
void decode_config_auto(int64_t nseg, int num_sms, int* lanes, int* cluster, int* round0);
// Checkerboard two-pass decode in one launch of the warp-specialised decoder
// (fp32 or bf16 parameters, 16 lanes per stream, clusters of 4 CTAs,
// 16-point first round): clusters 0 .. nseg0-1 decode the anchors (pass[0], parameters
// = the anchors' hyperprior parameters), the rest the non-anchors (pass[1],
// parameters = the non-anchors' hyperprior parameters, to which the
// stand-in context is applied on the fly from pass 0's decoded anchors,
// once every pass-0 CTA has completed the steps that hold those anchors).
// arrivals: one word per pass-0 step, zero before the launch; C H W < 2^31.
struct CkbdFuseArgs {
    DecodeArgs pass[2];
    int64_t C, H, W;
    uint32_t* arrivals;
    int silent_arrivals = 0;   // test hook: the anchor CTAs count no steps
};
cudaError_t launch_ws_ckbd(const CkbdFuseArgs& a, int K, int dtype, cudaStream_t st);
cudaError_t launch_ws_ckbd_bf16(const CkbdFuseArgs& a, int K, cudaStream_t st);
// Clusters of launch_ws_ckbd's kernel that the current device holds at once:
// the fused launch runs only when all of them fit, so that every pass-1
// cluster's wait is on pass-0 clusters that are resident.
cudaError_t ws_ckbd_capacity(int K, int dtype, int* clusters);
cudaError_t ws_ckbd_capacity_bf16(int K, int* clusters);
// Warp-specialised decoder for fp32 / bf16 parameters: CL CTAs per segment,
// SPW streams per consumer warp (1, 2 or 4).
cudaError_t launch_ws_f32(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st);
cudaError_t launch_ws_bf16(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st);
// Final decoder choice: automatic plan, then the handle's options, then the
// limits of each kernel (clusters only with G >= 2, at most 4 below G = 32).
void decode_resolve(int64_t nseg, int num_sms, int opt_lanes, int opt_cluster, int opt_round0, int phi, int* lanes,
                    int* cluster, int* round0, int* kernel);
cudaError_t launch_decode(const DecodeArgs& a, int K, int dtype, int lanes, int cluster, cudaStream_t st);
// Fills a's error word, statistics and test hook from the handle, picks the
// decoder as fgmm_decode does (the handle's options, else the automatic plan)
// and launches it.
cudaError_t decode_planned(fgmm_handle* h, DecodeArgs& a, int K, int dtype, cudaStream_t st);

// Batch plan records shared by the batch coder (fgmm_batch.cu) and the
// batched proposal decoder (fgmm_mlp.cu).
struct BatchLatentDev {
    const void* params;
    const int32_t* symbols;
    int32_t* decoded;
    int64_t N;
    int64_t T;          // steps = ceil(N / S)
    int64_t seg_base;   // first global segment
    int64_t scr_base;   // first scratch word of the latent's segments
    int64_t scr_cap;    // scratch words per segment of this latent
    int32_t K, dtype, S, pad;
};

struct BatchWorkItem {
    int32_t latent;
    int32_t g;          // segment within the latent
};

// Persistent proposal-bracketed decode of a batch (all latents K = 3, one
// dtype): warps take work items from *counter (zeroed by the caller).
// packed == nullptr selects the analytic proposal.
cudaError_t launch_batch_prop(const BatchLatentDev* lats, const BatchWorkItem* work, int64_t nwork,
                              unsigned long long* counter, const uint16_t* words, int64_t n_words,
                              const int64_t* offsets, const void* packed, int dtype, int act, int32_t* err,
                              unsigned long long* stats, int num_sms, cudaStream_t st);

}  // namespace fgmm
