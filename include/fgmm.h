/*
 * fgmm.h -- C ABI of the table-free Gaussian-mixture rANS coder for GB300.
 *
 * The coder implements FlashGMM's hot path (Sec. III-A): for every symbol of
 * a latent, the quantised CDF of its K-component Gaussian mixture (Sec. II-A,
 * Eq. 2) is evaluated on the fly at the coded symbol and fed to rANS
 * (Sec. II-B, Eq. 3); the decoder finds each symbol by binary search over
 * the same on-the-fly CDF. No CDF table is built. The Gaussian CDF is the
 * Abramowitz & Stegun 26.2.17 approximation (Sec. III-B, Eq. 8) evaluated in
 * FP32 with a fixed operation order, so every decoder that follows that
 * order reproduces the encoder's frequencies bit for bit.
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" are CUDA device pointers owned by the caller;
 *    the library never frees them. Pointers marked "host" are host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls are asynchronous on that stream unless stated.
 *  - A handle owns reusable device workspace (grown with cudaMalloc on
 *    demand, before any launch of the call) and a sticky device error word.
 *    Use one handle per stream; calls on one handle must not overlap on the
 *    device.
 *  - Host-side argument errors are returned immediately; data-dependent
 *    errors found by a kernel (bad parameters, corrupt stream, capacity) are
 *    recorded in the device error word and returned by fgmm_sync_status().
 *    Kernels never trap: they record the error and finish with bounded work.
 *
 * Latent layout: N symbols with planar parameters params[3][K][N]
 * (row 0 weights w_k, row 1 means mu_k, row 2 scales sigma_k), fp32 or bf16.
 * Valid parameters: w_k finite and >= 0, mu_k finite, sigma_k finite and > 0.
 * Scales are floored at 0.11 before use.
 *
 * Stream format (S streams per latent, S a positive multiple of 32):
 * symbol n belongs to stream n mod S at step n div S; streams are grouped 32
 * to a segment. A segment's 16-bit words are: the renormalisation words in
 * the order the encoder emitted them (steps T-1 .. 0, and within a step the
 * low escape chunk, high escape chunk and main symbol sub-phases, lanes in
 * ascending order), then the 32 final states as (low, high) word pairs.
 * offsets[g] is the word offset of segment g, offsets[S/32] the total.
 */
#ifndef FGMM_H
#define FGMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FGMM_OK = 0,
    FGMM_ERR_INVALID_ARG = 1, /* host-side argument check failed */
    FGMM_ERR_BAD_PARAMS = 2,  /* a mixture parameter is NaN/Inf/negative weight/scale <= 0 */
    FGMM_ERR_CAPACITY = 3,    /* output buffer too small */
    FGMM_ERR_CORRUPT = 4,     /* stream fails the end-of-decode check or would read out of its segment */
    FGMM_ERR_TIMEOUT = 5,     /* a bounded wait gave up (reserved; no kernel here waits) */
    FGMM_ERR_CUDA = 6,        /* a CUDA runtime call or launch failed */
    FGMM_ERR_NO_MEMORY = 7,   /* workspace allocation failed */
    FGMM_ERR_TOO_LARGE = 8    /* request exceeds the fixed scratch of fgmm_encode_noalloc */
} fgmm_status;

enum { FGMM_DTYPE_F32 = 0, FGMM_DTYPE_BF16 = 1 };

#define FGMM_MAX_K 4

/* One latent: K mixture components (1..FGMM_MAX_K), N symbols, parameters
 * in `dtype` at device pointer `params` with layout [3][K][N]. */
typedef struct {
    int32_t K;
    int32_t dtype;
    int64_t N;
    const void *params;
} fgmm_latent;

typedef struct fgmm_handle fgmm_handle;

/* Creates a handle on the current CUDA device. *out receives it. */
fgmm_status fgmm_create(fgmm_handle **out);

/* Frees the handle's workspace (after synchronising its last stream). */
void fgmm_destroy(fgmm_handle *h);

/* Static description of a status code. */
const char *fgmm_status_string(int32_t status);

/* Text of the last host-side error on this handle ("" if none). */
const char *fgmm_last_error(const fgmm_handle *h);

/* Synchronises `stream`, then returns and clears the first device error
 * recorded since the last call (FGMM_OK if none), or FGMM_ERR_CUDA. */
fgmm_status fgmm_sync_status(fgmm_handle *h, void *stream);

/* Phi-hat (Sec. III-B, Eq. 8, A&S 26.2.17) at n points: out[i] =
 * Phi-hat(z[i]). z and out are device float arrays of length n. */
fgmm_status fgmm_phi(fgmm_handle *h, const float *z, float *out, int64_t n, void *stream);

/* Phi-hat on the grid: out[i] = Phi-hat((i0 + i) * 2^-22), i < n (device). */
fgmm_status fgmm_phi_grid(fgmm_handle *h, int64_t i0, float *out, int64_t n, void *stream);

/* Per-symbol rANS intervals (the on-the-fly quantised CDF at the symbol,
 * Sec. III-A): sf[n] = start | freq << 16 (device uint32[N]); symbols is a
 * device int32[N]. An interval is the escape slot iff start + freq == 2^16. */
fgmm_status fgmm_freqs(fgmm_handle *h, const fgmm_latent *lat, const int32_t *symbols, uint32_t *sf,
                       void *stream);

/* Worst-case number of 16-bit words fgmm_encode can produce for N symbols
 * in S streams (host-only, no CUDA call). Negative if S is invalid. */
int64_t fgmm_encode_bound_words(int64_t N, int32_t S);

/* Encodes one latent (Sec. III-A encode: CDF at the symbol, then rANS,
 * Eq. 3) into S interleaved streams.
 *   symbols      device int32[N]
 *   S            streams, a positive multiple of 32
 *   words        device uint16[words_cap] output
 *   offsets      device int64[S/32 + 1] output (segment word offsets)
 *   n_words_out  device int64[1] output (total words)
 * If the stream does not fit in words_cap, FGMM_ERR_CAPACITY is recorded
 * and `words` is left incomplete. */
fgmm_status fgmm_encode(fgmm_handle *h, const fgmm_latent *lat, const int32_t *symbols, int32_t S,
                        uint16_t *words, int64_t words_cap, int64_t *offsets, int64_t *n_words_out,
                        void *stream);

/* Decodes one latent coded by fgmm_encode with the same parameters and S
 * (Sec. III-A decode: binary search over the on-the-fly CDF).
 *   words       device uint16[n_words]
 *   offsets     device int64[S/32 + 1]; every segment must lie inside
 *               [0, n_words) and hold at least its 64 flush words
 *   symbols_out device int32[N]
 * A segment whose offsets are out of range, a stream that would read
 * outside its segment, or one that does not end in the initial state with
 * all words consumed records FGMM_ERR_CORRUPT (no out-of-range access). */
fgmm_status fgmm_decode(fgmm_handle *h, const fgmm_latent *lat, const uint16_t *words, int64_t n_words,
                        const int64_t *offsets, int32_t S, int32_t *symbols_out, void *stream);

/* Optional counters. When enabled, decoders add the number of quantised-CDF
 * evaluations they make to a device counter; fgmm_stats_read synchronises
 * `stream` and copies {cdf_evals, symbols_decoded} to host out[2], then
 * zeroes the counters. */
fgmm_status fgmm_stats_enable(fgmm_handle *h, int32_t on);
fgmm_status fgmm_stats_read(fgmm_handle *h, uint64_t *out, void *stream);

/* Size of the fixed device scratch array used by fgmm_encode_noalloc. */
#define FGMM_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Allocation-free variant of fgmm_encode. The paper has no counterpart: it
 * exists for callers that cannot allocate device memory at the time they
 * encode, for example code running inside a host callback or a real-time
 * loop where cudaMalloc would block or is forbidden, or a plugin in a host
 * application that owns all device allocations. It needs no handle and
 * never calls cudaMalloc, cudaFree or any allocating routine; it produces
 * exactly the words, offsets and total of fgmm_encode.
 *
 * Its scratch (per-symbol intervals, per-segment word buffers and lengths)
 * lives in one static device array of FGMM_NOALLOC_SCRATCH_BYTES (16 MiB)
 * that every GPU which loads this library holds until the process exits.
 * A request fits when
 *   align256(4 N) + align256(2 (S/32) align8(96 ceil(N/S) + 64)) + 8 (S/32)
 * is at most that size (about 1.5 M symbols); larger requests return
 * FGMM_ERR_TOO_LARGE without launching anything.
 *
 * All calls in the process share the one array, and it keeps whatever the
 * last call left there (every scratch element is written before it is read,
 * so nothing in it needs clearing). Calls whose work overlaps on the GPU
 * (on different streams, or from different threads without ordering) race
 * on the array and corrupt each other's output: serialise them.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture on the device.
 *
 * Arguments are those of fgmm_encode (all device pointers, caller-owned),
 * without the handle, plus
 *   status_out  device int32[1]: set to 0 at the start of the call, then to
 *               the first data-dependent error the kernels find
 *               (FGMM_ERR_BAD_PARAMS, FGMM_ERR_CAPACITY); read it after the
 *               stream has synchronised.
 * The call is asynchronous on `stream`; the return value covers host-side
 * checks and launch errors only. */
fgmm_status fgmm_encode_noalloc(const fgmm_latent *lat, const int32_t *symbols, int32_t S, uint16_t *words,
                                int64_t words_cap, int64_t *offsets, int64_t *n_words_out, int32_t *status_out,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FGMM_H */
