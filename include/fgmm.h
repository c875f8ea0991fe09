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
 *    device. A CUDA graph that captured a call holds the workspace's
 *    address: a later call on the same handle that needs more workspace
 *    frees it, and the graph must not be replayed after that.
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
    FGMM_ERR_TIMEOUT = 5,     /* a bounded wait in a decoder gave up (the refill exchange of fgmm_dec_ws_kernel,
                                 the two-pass decode's wait for decoded anchors) */
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

/* Exhaustive check, on the current GPU, of the fast exact arithmetic the
 * kernels rely on: out[0] = number of floats d in [2^-125, 2^125] whose
 * Newton-refined reciprocal differs from the correctly rounded 1/d;
 * out[1] = number of failures of the encoder's division x / f (f in
 * [1, 2^16), quotient below 2^16) at the remainders 0, 1 and f - 1.
 * Both must be 0. Synchronous; takes about a second. */
fgmm_status fgmm_self_check(fgmm_handle *h, uint64_t *out);

/* Exhaustive measurement, on the current GPU, of how far the decoders'
 * fast steering evaluation of one component (hardware reciprocal and exp2,
 * no clamp or grid) can be from the coded Phi-hat at the same argument:
 * *out = the largest |fast(zs) - Phi-hat(zs)| over every float zs = z 2^22
 * that is not a NaN. Synchronous; a few milliseconds. */
fgmm_status fgmm_fast_phi_bound(fgmm_handle *h, double *out);

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

/* ---- Table-based comparison coder (Sec. II-C, Eqs. 4-5) -----------------
 * The conventional GMM coder the paper speeds up: the quantised CDF of every
 * symbol is evaluated at every point of the alphabet j in [-255, 256] into a
 * table (512 uint16 per symbol, O(K |Y|) work per symbol), and coding reads
 * intervals from it; decoding binary-searches the table row. The table holds
 * the same quantised CDF as the table-free coder, so the streams are
 * byte-identical to fgmm_encode's.
 * Table layout: device uint16 [N][512], 4-byte aligned, caller-owned;
 * entry [n][j + 255] = Q_n(clamp(j, lo_n, hi_n + 1)). */

/* Bytes of the table for N symbols (host-only). */
int64_t fgmm_table_bytes(int64_t N);

/* Builds the table of a latent. */
fgmm_status fgmm_table_build(fgmm_handle *h, const fgmm_latent *lat, uint16_t *table, void *stream);

/* Builds the table, then encodes from it; arguments as fgmm_encode plus the
 * table buffer (fgmm_table_bytes(N) bytes). */
fgmm_status fgmm_table_encode(fgmm_handle *h, const fgmm_latent *lat, const int32_t *symbols, int32_t S,
                              uint16_t *table, uint16_t *words, int64_t words_cap, int64_t *offsets,
                              int64_t *n_words_out, void *stream);

/* Builds the table, then decodes by binary search over each table row;
 * arguments as fgmm_decode plus the table buffer. */
fgmm_status fgmm_table_decode(fgmm_handle *h, const fgmm_latent *lat, uint16_t *table, const uint16_t *words,
                              int64_t n_words, const int64_t *offsets, int32_t S, int32_t *symbols_out,
                              void *stream);

/* ---- Gaussian single model with pre-built tables (Sec. II-C) ------------
 * The scheme that makes the GSM cheap: the quantiser has already shifted
 * each latent by its mean, so the coder receives the integer residual q and
 * the scale sigma only and codes q with N(0, sigma); sigma is quantised to
 * the smallest of L increasing levels at or above it (the last level above
 * them all; by default 64 levels spaced evenly in log between 0.11 and 256),
 * so one quantised-CDF row per level, built once, serves every symbol.
 * A level's row is this library's quantised CDF of N(0, level) (K = 1, same
 * window, escape slot and 0.11 scale floor, the handle's FGMM_OPT_PHI at
 * build time), so a GSM stream is byte-identical to fgmm_encode of the K = 1
 * parameters (w, mu, sigma) = (1, 0, level of sigma); the stream format is
 * fgmm_encode's.
 *
 * Tables: a device blob of fgmm_gsm_tables_bytes() bytes, 16-byte aligned,
 * caller-owned, written by fgmm_gsm_build and read-only afterwards:
 *   [0, 512)        int32 L at byte 0, float levels[64] at byte 16;
 *   [512, 66048)    uint16 rows[64][512], rows[l][j + 255] =
 *                   Q_l(clamp(j, lo_l, hi_l + 1)), 0 left of the window;
 *   [66048, 198144) uint32 pairs buckets[64][258]: for b in [0, 256],
 *                   J = the largest j in [0, 510] with rows[l][j] <= 256 b,
 *                   bucket = (J | rows[l][J] << 16, rows[l][J + 1]); entry
 *                   257 is 0. The decoder's slot index.
 * Scales: device fp32 or bf16 [N] (dtype FGMM_DTYPE_*); a scale must be
 * finite and > 0 (else FGMM_ERR_BAD_PARAMS through fgmm_sync_status). */

/* Bytes of the tables blob (host-only). */
int64_t fgmm_gsm_tables_bytes(void);

/* The 64 default levels, float(exp(ln 0.11 + i (ln 256 - ln 0.11) / 63))
 * for i = 0..63 computed in double; out is host float[64]. */
void fgmm_gsm_default_levels(float *out);

/* Builds the tables of L (1..64) levels given in host memory (finite, > 0,
 * strictly increasing; else FGMM_ERR_INVALID_ARG) into `tables`. */
fgmm_status fgmm_gsm_build(fgmm_handle *h, const float *levels, int32_t L, void *tables, void *stream);

/* Per-symbol intervals start | freq << 16 into device uint32 sf[N] (as
 * fgmm_freqs for the K = 1 parameters above). */
fgmm_status fgmm_gsm_freqs(fgmm_handle *h, int32_t dtype, int64_t N, const void *scales, const int32_t *symbols,
                           const void *tables, uint32_t *sf, void *stream);

/* Encodes residuals symbols[N] (device int32) with their scales; other
 * arguments and the output as fgmm_encode. */
fgmm_status fgmm_gsm_encode(fgmm_handle *h, int32_t dtype, int64_t N, const void *scales, const int32_t *symbols,
                            int32_t S, const void *tables, uint16_t *words, int64_t words_cap, int64_t *offsets,
                            int64_t *n_words_out, void *stream);

/* Decodes N residuals into device int32 symbols_out[N]; arguments and
 * errors as fgmm_decode, except that `words` must be 8-byte aligned and a
 * stream may hold at most 2^24 - 1 symbols (ceil(N / S) < 2^24; both
 * FGMM_ERR_INVALID_ARG otherwise). The decoder stages the tables in shared memory
 * (cp.async.bulk on an mbarrier whose wait is bounded: FGMM_ERR_TIMEOUT if
 * it gives up) and runs one lane per stream. */
fgmm_status fgmm_gsm_decode(fgmm_handle *h, int32_t dtype, int64_t N, const void *scales, const void *tables,
                            const uint16_t *words, int64_t n_words, const int64_t *offsets, int32_t S,
                            int32_t *symbols_out, void *stream);

/* ---- Checkerboard two-pass coding (the context model, Sec. IV-A) ---------
 * In every channel of a C x H x W latent (N = C H W, n = (c H + h) W + w)
 * the positions with h + w even are anchors: pass 1 codes them with the
 * hyperprior's parameters; pass 2 codes the others with parameters that a
 * context model computes from the decoded anchors. Anchors (non-anchors)
 * are listed channel by channel in raster order, C ceil(HW/2) (C floor(HW/2))
 * of them; each pass is an ordinary latent for fgmm_encode / fgmm_decode.
 * Decoding: pass 1, fgmm_ckbd_merge of the anchors, the context, pass 2,
 * fgmm_ckbd_merge of both. */

/* Anchors of a C x H x W latent (host-only; -1 for negative sizes). */
int64_t fgmm_ckbd_anchors(int64_t C, int64_t H, int64_t W);

/* Gathers the anchors' and non-anchors' parameters ([3][K][Na], [3][K][Nn],
 * lat's dtype) and symbols (int32) out of lat (N = C H W) and y (device
 * int32 [N]). Any output may be NULL; y may be NULL when both symbol
 * outputs are. */
fgmm_status fgmm_ckbd_split(fgmm_handle *h, const fgmm_latent *lat, int64_t C, int64_t H, int64_t W,
                            const int32_t *y, void *params_a, int32_t *y_a, void *params_n, int32_t *y_n,
                            void *stream);

/* Scatters anchor symbols y_a (and non-anchor symbols y_n, unless NULL) into
 * y (device int32 [N]); positions of a NULL class are left unchanged. */
fgmm_status fgmm_ckbd_merge(fgmm_handle *h, int64_t C, int64_t H, int64_t W, const int32_t *y_a,
                            const int32_t *y_n, int32_t *y, void *stream);

/* The stand-in context model (no trained network is available; this fixed
 * function takes its place): from the hyperprior parameters lat (N = C H W)
 * and the anchors of y, the non-anchors' parameters params_n (device fp32
 * [3][K][Nn]): for a non-anchor whose in-bounds 4-neighbours sum to ctx
 * (64-bit) over cnt of them, w'_k = w_k, mu'_k = fmaf(0.125, fmaf(-cnt, mu_k,
 * float(ctx)), mu_k), sigma'_k = 0.75 sigma_k (FP32, round to nearest). */
fgmm_status fgmm_ckbd_context(fgmm_handle *h, const fgmm_latent *lat, int64_t C, int64_t H, int64_t W,
                              const int32_t *y, float *params_n, void *stream);

/* The whole two-pass encode in one call: from the hyperprior parameters lat
 * (N = C H W) and the symbols y (device int32 [N]), the anchors' streams
 * (Sa streams, coded with the anchors' hyperprior parameters) into
 * words_a / offsets_a / *n_words_a, and the non-anchors' (Sn streams, coded
 * with fgmm_ckbd_context's parameters) into words_n / offsets_n /
 * *n_words_n, each as fgmm_encode writes them (the same bytes as
 * fgmm_ckbd_split, fgmm_ckbd_context and two fgmm_encode calls). One kernel
 * computes both passes' intervals (the split and the context included),
 * one launch runs both passes' rANS encoders. Capacities and errors as for
 * fgmm_encode; honours FGMM_OPT_PHI. Uses the handle's workspace. */
fgmm_status fgmm_ckbd_encode(fgmm_handle *h, const fgmm_latent *lat, int64_t C, int64_t H, int64_t W,
                             const int32_t *y, int32_t Sa, uint16_t *words_a, int64_t words_cap_a, int64_t *offsets_a,
                             int64_t *n_words_a, int32_t Sn, uint16_t *words_n, int64_t words_cap_n,
                             int64_t *offsets_n, int64_t *n_words_n, void *stream);

/* The whole two-pass decode in one call: from the hyperprior parameters lat
 * (N = C H W) and the two passes' streams (words_a / offsets_a of the
 * anchors coded with Sa streams from the anchors' hyperprior parameters;
 * words_n / offsets_n of the non-anchors coded with Sn streams from
 * fgmm_ckbd_context's parameters; the layout of fgmm_decode), writes the
 * latent's symbols to y (device int32 [N]). The same symbols as fgmm_ckbd_split,
 * fgmm_decode of the anchors, fgmm_ckbd_merge, fgmm_ckbd_context,
 * fgmm_decode of the non-anchors and fgmm_ckbd_merge, which it runs when it
 * cannot do better. It does better (fp32 or bf16 parameters, the A&S
 * approximation) when the automatic decoder plan of the Sa / 32 + Sn / 32
 * segments is the warp-specialised decoder with 16 lanes per stream,
 * clusters of 4 and a 16-point first round, every cluster fits on the
 * device at once, each pass has fewer than 2^24 steps, C H W < 2^31, and
 * no decoder option or test hook is set (fgmm_ckbd_decode_plan): then one
 * launch decodes both passes, the non-anchors' streams starting as soon as
 * the anchors next to their symbols are decoded, with the context applied
 * as their parameters are loaded. Each wait for anchors gives up after
 * about 2 s (FGMM_ERR_TIMEOUT from fgmm_sync_status): work on other streams
 * that keeps the anchor clusters off the GPU that long makes the decode
 * fail, so give it a GPU that can hold all its clusters. Uses the handle's
 * workspace (anchor parameters, non-anchor parameters, the two passes'
 * symbols). Stream errors are reported as by fgmm_decode. */
fgmm_status fgmm_ckbd_decode(fgmm_handle *h, const fgmm_latent *lat, int64_t C, int64_t H, int64_t W,
                             const uint16_t *words_a, int64_t n_words_a, const int64_t *offsets_a, int32_t Sa,
                             const uint16_t *words_n, int64_t n_words_n, const int64_t *offsets_n, int32_t Sn,
                             int32_t *y, void *stream);

/* *fused = 1 if fgmm_ckbd_decode on this handle decodes a K-component
 * latent of parameter type dtype and shape C x H x W, coded with Sa and Sn
 * streams, in one launch, else 0 (host-only; may query the device's
 * occupancy once per K). */
fgmm_status fgmm_ckbd_decode_plan(fgmm_handle *h, int32_t K, int32_t dtype, int64_t C, int64_t H, int64_t W,
                                  int32_t Sa, int32_t Sn, int32_t *fused);

/* ---- FP64 rate audit (Sec. V "no approximation" reference) --------------
 * For a latent and its symbols, computes in FP64 on the GPU:
 *   out[0] = sum over symbols of -log2 p64(s), p64 the exact mixture mass of
 *            [s - 1/2, s + 1/2) with erfc (the ideal code length);
 *   out[1] = sum of -log2(freq / 2^16) of the coder's intervals, plus 32 bits
 *            for each escape (the coder's code length without container);
 *   out[2] = max |F-hat32(b) - F64(b)| over the boundaries the encoder
 *            evaluates;
 *   out[3] = number of escapes.
 * out is device double[4]. Rate overhead = out[1] / out[0] - 1. */
fgmm_status fgmm_rate_audit(fgmm_handle *h, const fgmm_latent *lat, const int32_t *symbols, double *out,
                            void *stream);

/* ---- Batches: many latents in one persistent launch ---------------------
 * A plan binds n latents and their buffers. All segments of all latents
 * form one work list (longest latents first) that a persistent grid of warps
 * drains through an atomic counter; encode is one such launch (the interval
 * of each symbol evaluated inline, then rANS) followed by the offset scan and
 * compaction over all segments, decode is one such launch. Latent i's stream
 * is words[offsets[b_i] .. offsets[b_i + S_i/32]), b_i = sum_{j<i} S_j/32,
 * byte-identical to fgmm_encode of that latent with S_i streams.
 * fgmm_batch_capture records both launch sequences into CUDA graphs once;
 * later fgmm_batch_encode/decode calls replay them. */
typedef struct {
    int32_t K;
    int32_t dtype;
    int64_t N;
    const void *params;      /* device [3][K][N] */
    const int32_t *symbols;  /* device int32[N]: encoder input */
    int32_t *decoded;        /* device int32[N]: decoder output */
} fgmm_batch_latent;

typedef struct fgmm_batch fgmm_batch;

/* Stream counts for a batch: the most parallel choice whose container cost
 * (a 32-bit flushed state per stream) stays within max_overhead of the
 * payload at bits_per_symbol, without more streams than the batch decoder
 * runs concurrently on this GPU:
 *   T* = max(ceil(32 / (max_overhead * bits_per_symbol)),
 *            ceil(sum N / concurrent streams)),
 *   S_i = clamp(roundup32(ceil(N_i / T*)), 32, roundup32(N_i)).
 * N is host int64[n]; S_out host int32[n]. Host-only (queries occupancy). */
fgmm_status fgmm_autotune(fgmm_handle *h, const int64_t *N, int32_t n, double max_overhead, double bits_per_symbol,
                          int32_t *S_out);

/* Creates a plan. lats: host array of n latents (device pointers inside).
 * S_in: host int32[n] stream counts (multiples of 32), or NULL for
 * fgmm_autotune with max_overhead 1% at 3.5 bits/symbol. words (device,
 * words_cap entries), offsets (device int64[total segments + 1]) and
 * n_words_out (device int64[1]) receive the encoded batch and are read by
 * the decoder. The plan allocates its own device work list and encode
 * scratch (about 6 bytes per symbol) here, never later. */
fgmm_status fgmm_batch_create(fgmm_handle *h, const fgmm_batch_latent *lats, int32_t n, const int32_t *S_in,
                              uint16_t *words, int64_t words_cap, int64_t *offsets, int64_t *n_words_out,
                              fgmm_batch **out);
void fgmm_batch_destroy(fgmm_batch *b);
/* Total segments (offsets has this many + 1 entries). */
int64_t fgmm_batch_segments(const fgmm_batch *b);
/* Copies the stream count of every latent to host S_out[n]. */
fgmm_status fgmm_batch_streams(const fgmm_batch *b, int32_t *S_out);
/* Captures the encode and decode launch sequences into CUDA graphs. */
fgmm_status fgmm_batch_capture(fgmm_batch *b);
/* Encodes / decodes the whole batch on `stream` (graph replay if captured). */
fgmm_status fgmm_batch_encode(fgmm_batch *b, void *stream);
fgmm_status fgmm_batch_decode(fgmm_batch *b, void *stream);
/* Decodes the whole batch with the decode proposal (see the proposal
 * section below) in one persistent launch of 4-warp CTAs that each hold one
 * copy of the packed network in shared memory: packed (device,
 * FGMM_MLP_PACKED_BYTES, from fgmm_mlp_pack) or NULL for the analytic
 * proposal; the activation is the plan handle's FGMM_OPT_MLP_ACT. Every
 * latent must have K = 3 and all the same dtype (FGMM_ERR_INVALID_ARG
 * otherwise). Output and errors as fgmm_batch_decode; not captured in the
 * plan's graphs. */
fgmm_status fgmm_batch_decode_proposal(fgmm_batch *b, const void *packed, void *stream);

/* ---- Learned decode proposal (no counterpart in the paper) --------------
 * A 10 -> 64 -> 64 -> 1 MLP guesses a symbol from its mixture (K = 3) and
 * its rANS slot; fgmm_decode_proposal searches from the guess (two probes
 * decide whether the guess is the symbol, else a gallop of growing steps
 * and a binary search; the probes use a fast evaluation of the CDF) and
 * confirms the symbol reached with the exact quantised CDF (an exact binary
 * search if that check fails), so decoded symbols equal fgmm_decode's for
 * any network weights. Features: weights, means and log-scales standardised
 * by the mixture mean m0 and standard deviation s0 (components sorted by
 * mean), and (slot + 1/2)/2^16 - 1/2; output y, guess round(m0 + s0 y).
 * Activation (FGMM_OPT_MLP_ACT, used by training, fgmm_mlp_forward and the
 * proposal decoders): FGMM_MLP_ACT_PL, z * sat(1/2 + (1.702/4) z) (default),
 * or FGMM_MLP_ACT_SIGMOID, z / (1 + exp(-1.702 z)); packed weights must be
 * used with the activation they were trained with.
 * Parameter vector theta (device fp32[FGMM_MLP_PARAMS]): W1[10][64], b1[64],
 * W2[64][64], b2[64], w3[64], b3. */
#define FGMM_MLP_PARAMS 4929
#define FGMM_MLP_PACKED_BYTES 11024

/* Training triples: for each symbol (K = 3 latent), the slot drawn
 * uniformly inside its interval, slot = start + min(freq - 1,
 * floor(uniforms[n] * freq)), its features X (device fp32[N][10]), target
 * (device fp32[N]: (s - m0)/s0 clipped to [-8, 8]) and, if slots is not
 * NULL, the slot (device int32[N]). uniforms: device fp32[N] in [0, 1). */
fgmm_status fgmm_mlp_data(fgmm_handle *h, const fgmm_latent *lat, const int32_t *symbols, const float *uniforms,
                          float *X, float *target, int32_t *slots, void *stream);

/* Mean squared error of the network on B samples and its gradient (FP32;
 * per-block partial sums reduced in a fixed order, so the result is
 * deterministic). grad: device fp32[FGMM_MLP_PARAMS]; loss: device fp32[1]. */
fgmm_status fgmm_mlp_loss_grad(fgmm_handle *h, const float *X, const float *target, int64_t B, const float *theta,
                               float *grad, float *loss, void *stream);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) over
 * consecutive minibatches of `batch` samples from X/target (N samples,
 * batch k = (step0 + i) mod (N / batch)); theta, adam_m, adam_v (device
 * fp32[FGMM_MLP_PARAMS]) are updated in place; loss_trace (device
 * fp32[steps]) receives each step's loss. Deterministic. */
fgmm_status fgmm_mlp_train(fgmm_handle *h, const float *X, const float *target, int64_t N, float *theta,
                           float *adam_m, float *adam_v, int64_t step0, int64_t steps, int64_t batch, float lr,
                           float *loss_trace, void *stream);

/* Converts theta to the BF16 fragment layout of the inference kernels
 * (device, FGMM_MLP_PACKED_BYTES, 16-byte aligned). */
fgmm_status fgmm_mlp_pack(fgmm_handle *h, const float *theta, void *packed, void *stream);

/* Inference (BF16 mma.sync, FP32 accumulation) on B feature rows:
 * y[b] = network(X[b]); X device fp32[B][10], y device fp32[B]. */
fgmm_status fgmm_mlp_forward(fgmm_handle *h, const float *X, int64_t B, const void *packed, float *y, void *stream);

/* fgmm_decode with the proposal (K = 3 latents); same arguments plus the
 * packed network. packed == NULL selects the analytic proposal instead: the
 * inverse of the logistic approximation of Phi (Sec. III-B) on the
 * component of largest weight, mu + sigma' ln(u / (1 - u)) / 1.702 with
 * u = (slot + 1/2) / 2^16 -- a comparison point for the network. */
fgmm_status fgmm_decode_proposal(fgmm_handle *h, const fgmm_latent *lat, const void *packed, const uint16_t *words,
                                 int64_t n_words, const int64_t *offsets, int32_t S, int32_t *symbols_out,
                                 void *stream);

/* Tuning options (fgmm_set_option). FGMM_OPT_DECODE_LANES: lanes that
 * cooperate on one stream in fgmm_decode: 1 (binary search, one lane per
 * stream), 2, 4, 8, 16 or 32 (G-ary search, G lanes per stream), or 0 to
 * choose from the number of segments (default). FGMM_OPT_DECODE_CLUSTER:
 * CTAs (a thread-block cluster, one SM each) sharing one segment when G > 1:
 * 1, 2 or 4 (at most G), 8 for G >= 8, or 0 for automatic; G = 32 takes at
 * least 2. FGMM_OPT_DECODE_ROUND0: points of the first search round that producer
 * warps of the warp-specialised decoder evaluate ahead of the state chain
 * when G = 16: 16 (two streams per producer warp) or 32, or 0 for
 * automatic; G = 8 and 32 always take 32. The decoded symbols depend on
 * none of these. */
enum { FGMM_OPT_DECODE_LANES = 1, FGMM_OPT_DECODE_CLUSTER = 2, FGMM_OPT_DECODE_ROUND0 = 3 };

/* Test hook for the bounded waits of the warp-specialised decoder
 * (FGMM_DEC_WS): stream `value` (0..31) of segment 0 posts no refill flags,
 * so the other streams' waits run out; the decode then records
 * FGMM_ERR_TIMEOUT, releases every wait through an abort flag, and returns.
 * -1 (default) turns it off. The paper has no counterpart. */
enum { FGMM_OPT_TEST_SILENT_STREAM = 4 };

/* FGMM_OPT_PHI selects the approximation of the Gaussian CDF in the coded
 * quantised CDF (Sec. III-B; the comparison of Sec. V, Table II):
 *   FGMM_PHI_AS        Abramowitz & Stegun 26.2.17 (default);
 *   FGMM_PHI_LOGISTIC  1 / (1 + exp(-1.702 z));
 *   FGMM_PHI_POLYA     (1 + sqrt(1 - exp(-2 z^2 / pi))) / 2 for z >= 0
 *                      (Polya's form; mirrored for z < 0).
 * All three are evaluated in FP32 on the clamp |z| <= 12 and the grid
 * 2^-22 with a fixed operation order, so encoder and decoder agree bit for
 * bit. A stream must be decoded with the approximation it was encoded
 * with. Honoured by fgmm_phi, fgmm_phi_grid, fgmm_freqs, fgmm_encode,
 * fgmm_decode (which then runs FGMM_DEC_LANE) and fgmm_rate_audit; the
 * table coder, batches, the proposal and fgmm_encode_noalloc take A&S only
 * and return FGMM_ERR_INVALID_ARG otherwise. */
enum { FGMM_OPT_PHI = 5 };
enum { FGMM_PHI_AS = 0, FGMM_PHI_LOGISTIC = 1, FGMM_PHI_POLYA = 2 };

/* FGMM_OPT_MLP_ACT: activation of the proposal network (see the proposal
 * section): FGMM_MLP_ACT_PL (0, default) or FGMM_MLP_ACT_SIGMOID (1). */
enum { FGMM_OPT_MLP_ACT = 6 };
enum { FGMM_MLP_ACT_PL = 0, FGMM_MLP_ACT_SIGMOID = 1 };

/* Test hook for the bounded wait of the one-launch two-pass decode
 * (fgmm_ckbd_decode): with value 1 the anchor CTAs count none of their
 * steps, so every non-anchor wait for them runs out (after about two
 * seconds); the decode then records FGMM_ERR_TIMEOUT, releases the other
 * waits through the clusters' abort flags, and returns. 0 (default) turns
 * it off. The paper has no counterpart. */
enum { FGMM_OPT_TEST_SILENT_ARRIVALS = 7 };
fgmm_status fgmm_set_option(fgmm_handle *h, int32_t option, int64_t value);

/* The decoder fgmm_decode would run for S streams (S / 32 segments) under
 * the handle's current options; host only, no GPU work, nothing allocated.
 * out (host, 4 entries): out[0] = lanes per stream, out[1] = CTAs per
 * segment (cluster size), out[3] = first-round points (FGMM_DEC_WS and
 * FGMM_DEC_WIDE; 0 for the others), out[2] = the kernel:
 *   FGMM_DEC_LANE  one lane per stream, binary search over the window
 *                  (Sec. III-B), one warp per segment;
 *   FGMM_DEC_COOP  G = 2..16 lanes per stream, G-ary search (clusters of
 *                  up to 4 CTAs for G = 2, 4; one CTA for G = 8, 16);
 *   FGMM_DEC_WIDE  32 lanes per stream, 32-point search, one CTA per segment;
 *   FGMM_DEC_WS    (streams of fewer than 2^24 steps, ceil(N / S) < 2^24;
 *                  fgmm_decode runs FGMM_DEC_LANE for longer ones)
 *                  G = 8, 16 or 32 with a cluster of 2, 4 or 8 CTAs per
 *                  segment: producer warps evaluate a 32-point first round
 *                  two steps ahead, consumer warps (32 / G streams each,
 *                  G lanes per stream) search inside the bracket.
 * The paper has no counterpart: it decodes with one thread per stream.
 * Errors: FGMM_ERR_INVALID_ARG for a NULL argument or S not a positive
 * multiple of 32. */
enum { FGMM_DEC_LANE = 0, FGMM_DEC_COOP = 1, FGMM_DEC_WIDE = 2, FGMM_DEC_WS = 3 };
fgmm_status fgmm_decode_plan(fgmm_handle *h, int32_t S, int32_t out[4]);

/* Optional counters. When enabled, decoders add the number of quantised-CDF
 * evaluations they make to a device counter (for the one-lane binary search:
 * its probes, the evaluations of the plain binary search on the same path);
 * fgmm_stats_read synchronises `stream` and copies {cdf_evals,
 * symbols_decoded, proposal_hits, guide_fallbacks} to host out[4], then
 * zeroes the counters. guide_fallbacks counts the symbols for which the
 * one-lane decoder's fast-steered search reached a symbol that the exact
 * check rejected, so that the exact binary search ran instead. */
fgmm_status fgmm_stats_enable(fgmm_handle *h, int32_t on);
fgmm_status fgmm_stats_read(fgmm_handle *h, uint64_t *out, void *stream);

/* Throughput probe for the roofline denominators (a measurement aid; the
 * paper has no counterpart). Launches, asynchronously on `stream`, a grid of
 * 4 CTAs of 256 threads per SM in which every thread runs 8 independent
 * chains of `iters` x 16 steps of one instruction:
 *   FGMM_PEAK_FMA  fma.rn.f32 (the FP32 pipe the CDF evaluations run on);
 *   FGMM_PEAK_RCP  rcp.approx.ftz.f32, each followed by one fma.rn.f32 so
 *                  that no two steps cancel (the XU pipe the reciprocals
 *                  use sets the time; ops counts the reciprocals).
 * *ops_out (host) receives the number of per-lane operations the launch
 * performs; the caller times the launch (CUDA events on `stream`) and
 * divides; a launch should run for a millisecond or more (iters ~2048 for
 * FMA, ~256 for RCP) so that the launch overhead does not count. sink:
 * device float[1], never written in practice (it keeps the chains from
 * being optimised away). iters >= 1. */
enum { FGMM_PEAK_FMA = 0, FGMM_PEAK_RCP = 1 };
fgmm_status fgmm_peak_probe(fgmm_handle *h, int32_t kind, int64_t iters, float *sink, double *ops_out,
                            void *stream);

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
 * (cudaGetSymbolAddress, with that device current) and caches it with the
 * id of the CUDA context it belongs to; make that first call before any
 * stream capture on the device. A call in another context of the device
 * (after cudaDeviceReset, which reloads the library's device code) looks the
 * address up again, so make the first call after a reset outside stream
 * capture too.
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
