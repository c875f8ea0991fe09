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

}  // namespace fgmm
