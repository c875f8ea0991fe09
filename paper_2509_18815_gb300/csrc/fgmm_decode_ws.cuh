// fgmm_decode_ws.cuh -- warp-specialised decoder (included by the fp32 and
// bf16 instantiation units fgmm_decode_ws.cu and fgmm_decode_ws_bf16.cu).
//
// Binary search over the on-the-fly quantised CDF (Sec. III-A) split into a
// state-independent part and a state-dependent chain. Per stream, a producer
// warp prepares, kLead steps ahead, the stream's mixture (reciprocal scales,
// window) and evaluates Q at R0 (16 or 32) points spread over the window
// (round 0); a producer warp serves 32/R0 streams. Consumer warps run the
// chain of each step: a count of the round-0 values at or below the slot
// brackets the symbol between two round-0 points, the points inside the
// bracket (at most ceil(W/R0) - 1) are evaluated, then the inverse rANS step
// (Eq. 3) and the segment's refill exchange. A consumer warp serves SPW
// streams with 32/SPW lanes each (one bracket round when the bracket
// interior always fits the lanes, rounds of 32/SPW points otherwise).
//
// The exchange is a flag per stream, not a barrier: each stream writes
// (exchange number, refill bit, escape bit) into a double-buffered slot of
// every CTA of the cluster, then polls its own CTA's copies until all 32
// streams of the segment have posted that exchange. A slot is reused two
// exchanges later, by which time every stream has read it (a stream posts
// exchange e + 1 only after its wait for exchange e has ended). Producers
// and consumers of one CTA meet at a CTA barrier once per step. Every wait
// is bounded: a consumer that gives up records an error and raises an abort
// flag in all CTAs, after which no wait blocks.
//
// A second mode decodes the checkerboard's two passes in one launch (the
// anchors' clusters first, then the non-anchors'), with one more warp per
// CTA that counts the anchor steps done or, for the non-anchors, waits for
// the anchors next to its columns and loads them for the stand-in context
// (see fgmm_dec_ws_kernel and launch_ws_ckbd_k).
#pragma once

#include "fgmm_decode_impl.cuh"

namespace {

constexpr int kLead = 2;                     // producer lead (steps)
constexpr int kPre = 4;                      // precomputed-step slots (>= kLead + 2)
constexpr uint32_t kSpinLimit = 1u << 24;    // polls before a wait gives up

template <int K>
struct __align__(16) PreStep {
    uint32_t q0[32];              // Q at the 32 round-0 points
    float w[K], mu[K], isg[K];
    int lo, hi;
    float tp;
};

// Stores v at `local` in the CTA of cluster rank r.
__device__ __forceinline__ void store_rank(uint32_t* local, uint32_t r, uint32_t v)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(r));
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

// One refill exchange of the segment, called by every lane of every
// consumer warp, in two halves so that work can run between them. Post: lane
// j (< CL) of the group of stream ws posts that stream's flags (bit 0
// refill, bit 1 escape) to CTA j; posts is false only for the stream that
// the FGMM_OPT_TEST_SILENT_STREAM hook silences, to make the others' waits
// run out in a test. Wait: returns, in lane q, stream q's flags for
// exchange e.
template <int CL>
__device__ __forceinline__ void exchange_post(uint32_t* xflag, uint32_t e, int ws, int j, uint32_t bits, bool posts)
{
    uint32_t* slot = xflag + (e & 1u) * 32;
    const uint32_t tag = e & 0x3fffffffu;
    if (posts && j < CL) store_rank(slot + ws, (uint32_t)j, (tag << 2) | bits);
}

template <int CL>
__device__ __forceinline__ uint32_t exchange_wait(uint32_t* xflag, uint32_t* abort_flag, uint32_t e, int lane,
                                                  int32_t* err)
{
    uint32_t* slot = xflag + (e & 1u) * 32;
    const uint32_t tag = e & 0x3fffffffu;
    const volatile uint32_t* vs = slot;
    const volatile uint32_t* va = abort_flag;
    for (uint32_t spin = 0;; ++spin) {
        const uint32_t f = vs[lane];
        if (__all_sync(kFull, (f >> 2) == tag)) return f & 3u;
        if (__any_sync(kFull, *va != 0u)) return 0u;
        if (spin >= kSpinLimit) {
            if (lane == 0) set_error(err, kErrTimeout);
            if (lane < CL) store_rank(abort_flag, (uint32_t)lane, 1u);
            return 0u;
        }
    }
}

template <int CL>
__device__ __forceinline__ uint32_t exchange(uint32_t* xflag, uint32_t* abort_flag, uint32_t e, int ws, int j,
                                             int lane, uint32_t bits, int32_t* err, bool posts)
{
    exchange_post<CL>(xflag, e, ws, j, bits, posts);
    return exchange_wait<CL>(xflag, abort_flag, e, lane, err);
}

// Refill of one sub-step: M holds the segment's refill bits (stream q at
// bit q); streams read in rank order from the words just below rp, the read
// position relative to the segment's first word wseg[0] (32-bit: a segment
// holds fewer than 2^31 words, see launch_ws).
__device__ __forceinline__ void ws_refill(uint32_t& x, bool need, uint32_t M, uint32_t below,
                                          const uint16_t* wseg, int32_t& rp, bool& bad)
{
    if (M) {
        const int cnt = __popc(M);
        if (need) {
            const int32_t idx = rp - cnt + __popc(M & below);
            uint32_t v = 0;
            if (idx >= 0) v = wseg[idx];
            else bad = true;
            x = (x << 16) | v;
        }
        rp -= cnt;
    }
}

// Round-0 point i of R0 over the window [lo, hi]: the (i+1)/R0 quantile of
// the positions lo+1 .. hi+1 (point R0-1 is hi+1, the escape boundary).
template <int K, int R0>
__device__ __forceinline__ int round0_point(const Mix<K>& m, int i)
{
    const int W = m.hi - m.lo + 1;
    return m.lo + ((i + 1) * W + R0 - 1) / R0;
}

// ---------------------------------------------------------------------------
// Checkerboard two-pass decode in one launch (MODE 1 of the kernel below).
// Anchors are positions with h + w even; both classes are listed channel by
// channel in raster order (the layout of fgmm_ckbd.cu), so the anchors a
// non-anchor needs lie at most one row ahead of it, and the second pass can
// run a few steps behind the first instead of after it.
// ---------------------------------------------------------------------------
struct WsPassDev {
    const void* params;
    int64_t N;
    int32_t S, mode;
    int64_t T;
    const uint16_t* words;
    int64_t n_words;
    const int64_t* offsets;
    int32_t* out;
};

struct WsFuseDev {
    WsPassDev pass[2];
    int64_t nseg0;          // clusters of pass 0
    uint32_t H, W;          // C H W < 2^31 (the host checks)
    uint32_t per_a, per_n;  // anchors / non-anchors per channel
    uint32_t pq, pr;        // per_n = pq W + pr
    uint32_t adv_c, adv_h, adv_r;   // pass 1's S = adv_c per_n + adv_h W + adv_r
    const int32_t* ya;      // pass 0's output: the decoded anchors
    uint32_t* arrivals;     // [pass 0's steps]: pass-0 CTAs that completed the step
    int silent_arrivals;    // test hook: pass-0 CTAs count no steps
};

// The context warp's lane q follows column i = u S + nbase + q of pass 1
// from step to step as (c, hp, rem): channel c, and i's index within the
// channel, k = hp W + rem (rem < W). Rows alternate floor(W/2) and
// ceil(W/2) non-anchors, floor(W/2) first, so k sits in row 2 hp at w =
// 2 rem + 1 when rem < floor(W/2), else in row 2 hp + 1 at w = 2 (rem -
// floor(W/2)). Advancing by S adds the precomputed (adv_c, adv_h, adv_r)
// with one carry and at most one wrap into the next channel (k < per_n).
struct CkbdPos {
    uint32_t c, hp, rem;
};

__device__ __forceinline__ CkbdPos ckbd_pos(const WsFuseDev& fz, uint32_t i)
{
    CkbdPos p;
    p.c = i / fz.per_n;
    const uint32_t k = i - p.c * fz.per_n;
    p.hp = k / fz.W;
    p.rem = k - p.hp * fz.W;
    return p;
}

__device__ __forceinline__ void ckbd_advance(const WsFuseDev& fz, CkbdPos& p)
{
    p.c += fz.adv_c;
    p.hp += fz.adv_h;
    p.rem += fz.adv_r;
    if (p.rem >= fz.W) { p.rem -= fz.W; ++p.hp; }
    if (p.hp > fz.pq || (p.hp == fz.pq && p.rem >= fz.pr)) {   // k >= per_n = pq W + pr
        if (p.rem >= fz.pr) { p.rem -= fz.pr; p.hp -= fz.pq; }
        else { p.rem += fz.W - fz.pr; p.hp -= fz.pq + 1; }
        ++p.c;
    }
}

__device__ __forceinline__ uint32_t ckbd_row(const WsFuseDev& fz, const CkbdPos& p)
{
    return p.rem < fz.W / 2 ? 2 * p.hp : 2 * p.hp + 1;
}

// Index of the anchor at (c, h, w), h + w even.
__device__ __forceinline__ uint32_t anchor_index(const WsFuseDev& fz, uint32_t c, uint32_t h, uint32_t w)
{
    return c * fz.per_a + (h >> 1) * fz.W + (h & 1) * ((fz.W + 1) / 2) + (w >> 1);
}

// A cursor of the context warp over pass 1's steps: at step u, lane q's
// column u S + nbase + q (pos), and need, the pass-0 steps that must be
// complete before the warp reads the neighbours of the step's columns: 0
// when no column is below Nn, all of pass 0 when some but not all are,
// else the steps that hold the anchors of channel c's rows 0 .. min(h + 2,
// H) - 1 and of the earlier channels, (c, h) the last column's position
// (lane SPC - 1), among them every neighbour of the columns. That bound
// only grows from step to step, so need follows it by additions (needb =
// need Sa >= bound).
struct CkbdCursor {
    CkbdPos pos;
    uint32_t u, need, needb;
};

template <int SPC>
__device__ __forceinline__ void cursor_need(const WsFuseDev& fz, CkbdCursor& k, uint32_t nbase)
{
    const uint32_t Nn = (uint32_t)fz.pass[1].N, n0 = k.u * (uint32_t)fz.pass[1].S + nbase;
    const uint32_t rows = min(ckbd_row(fz, k.pos) + 2, fz.H);
    const uint32_t bound = __shfl_sync(kFull, k.pos.c * fz.per_a + (rows >> 1) * fz.W + (rows & 1) * ((fz.W + 1) / 2),
                                       SPC - 1);
    if (n0 >= Nn) {
        k.need = 0u;
    } else if (n0 + SPC > Nn) {
        k.need = (uint32_t)fz.pass[0].T;
    } else {
        const uint32_t Sa = (uint32_t)fz.pass[0].S;
        while (k.needb < bound) {
            k.needb += Sa;
            ++k.need;
        }
    }
}

template <int SPC>
__device__ __forceinline__ void cursor_next(const WsFuseDev& fz, CkbdCursor& k, uint32_t nbase)
{
    ckbd_advance(fz, k.pos);
    ++k.u;
    cursor_need<SPC>(fz, k, nbase);
}

// Polls read pass 0's arrival counts with acquire loads (measured faster
// here than a relaxed read and a fence) and, when a poll is needed, ask for
// the count of a step kPollAhead beyond the next one, so that one poll
// covers several steps.
constexpr int kPollAhead = 4;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kArrivalWaitNs = 2000000000ull;   // a wait for anchors gives up after 2 s

// Waits (warp-wide, bounded) until pass 0 has completed `need` steps, seen
// being the count already established. The acquire is lane 0's read of the
// step's arrival count; __syncwarp then orders the other lanes' later reads
// of the anchors after it. A wait gives up after kArrivalWaitNs of the
// global timer (polls go to L2, so a poll count would bound the time less
// well): FGMM_ERR_TIMEOUT and the cluster's abort flag.
template <int CL>
__device__ __forceinline__ void ckbd_wait(const WsFuseDev& fz, uint32_t need, uint32_t& seen, uint32_t nprog,
                                          uint32_t* abort_flag, int32_t* err, int lane)
{
    if (need <= seen) return;
    const volatile uint32_t* va = abort_flag;
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t v = 0;
        if (lane == 0) v = ld_acquire_u32(fz.arrivals + (need - 1));
        v = __shfl_sync(kFull, v, 0);
        if (v >= nprog) {
            __syncwarp();
            seen = need;
            return;
        }
        if (__any_sync(kFull, *va != 0u)) return;
        if (__shfl_sync(kFull, global_ns() - t0 > kArrivalWaitNs, 0)) {
            if (lane == 0) set_error(err, kErrTimeout);
            if (lane < CL) store_rank(abort_flag, (uint32_t)lane, 1u);
            return;
        }
    }
}

// Issues the loads of the in-bounds 4-neighbour anchors of the non-anchor
// at p when `take` (L2, never L1: pass 0 writes them during the launch);
// fixed slots (up, down, left, right; zero when out of bounds) keep v in
// registers.
__device__ __forceinline__ void ckbd_load(const WsFuseDev& fz, bool take, const CkbdPos& p, int32_t (&v)[4], int& cnt)
{
    v[0] = v[1] = v[2] = v[3] = 0;
    cnt = 0;
    if (!take) return;
    const uint32_t h = ckbd_row(fz, p), w = p.rem < fz.W / 2 ? 2 * p.rem + 1 : 2 * (p.rem - fz.W / 2);
    if (h > 0) v[0] = __ldcg(fz.ya + anchor_index(fz, p.c, h - 1, w));
    if (h + 1 < fz.H) v[1] = __ldcg(fz.ya + anchor_index(fz, p.c, h + 1, w));
    if (w > 0) v[2] = __ldcg(fz.ya + anchor_index(fz, p.c, h, w - 1));
    if (w + 1 < fz.W) v[3] = __ldcg(fz.ya + anchor_index(fz, p.c, h, w + 1));
    cnt = (h > 0) + (h + 1 < fz.H) + (w > 0) + (w + 1 < fz.W);
}

// float(ctx) and -cnt of the loaded neighbours (ctx summed in 64 bits).
__device__ __forceinline__ float2 ckbd_ctx(const int32_t (&v)[4], int cnt)
{
    const int64_t ctx = (int64_t)v[0] + (int64_t)v[1] + (int64_t)v[2] + (int64_t)v[3];
    return make_float2(__ll2float_rn(ctx), -(float)cnt);
}

// MODE 0: one latent (the arguments). MODE 1: the checkerboard's two passes
// in one launch (fz; the other arguments except err, stats and silent are
// unused), with one more warp per CTA, the context warp: clusters below
// fz.nseg0 decode the anchors, their context warp counting each completed
// step in fz.arrivals; the others decode the non-anchors, their context
// warp running a pipeline for the step the producers stage: it waits until
// pass 0 has completed the steps that hold the columns' neighbours (polled
// an iteration ahead, for a step kPollAhead further on), loads the
// neighbours into registers, and an iteration later turns them into
// (float(ctx), -cnt) in shared memory. The producers apply the stand-in
// context to the staged hyperprior parameters as they set the step's
// mixtures up: w' = w, mu' = fmaf(0.125, fmaf(-cnt, mu, float(ctx)), mu),
// sigma' = 0.75 sigma, each one FP32 rounding.
template <int K, typename T, int CL, int SPW, int R0, int MODE = 0>
__global__ void __launch_bounds__(32 * (32 / CL / SPW + 32 / CL * R0 / 32) + (MODE == 1 ? 32 : 0))
    fgmm_dec_ws_kernel(const T* __restrict__ params_a, int64_t N_a, int32_t S_a, int64_t T_a,
                       const uint16_t* __restrict__ words_a, int64_t n_words_a, const int64_t* __restrict__ offsets_a,
                       int32_t* __restrict__ out_a, int32_t* err, unsigned long long* stats, int mode_a, int silent,
                       WsFuseDev fz)
{
    constexpr int SPC = 32 / CL;              // streams per CTA
    constexpr int LPS = 32 / SPW;             // consumer lanes per stream
    constexpr int VPL = R0 / LPS;             // round-0 values per consumer lane
    constexpr int CW = SPC / SPW;             // consumer warps
    constexpr int SPP = 32 / R0;              // streams per producer warp
    constexpr int PW = SPC / SPP;             // producer warps
    constexpr int NT = 32 * (CW + PW) + (MODE == 1 ? 32 : 0);   // threads (MODE 1: + the context warp)
    constexpr int PNT = 32 * PW;              // producer threads
    // W <= 511, so the bracket interior has at most ceil(511 / R0) - 1 points
    constexpr bool kOneRound = LPS >= (511 + R0 - 1) / R0 - 1;
    static_assert(SPC % SPW == 0 && SPC % SPP == 0 && LPS >= CL && VPL >= 1, "stream groups lie in one CTA");
    extern __shared__ __align__(16) unsigned char smem[];
    PreStep<K>* pre = reinterpret_cast<PreStep<K>*>(smem);                                  // [kPre][SPC]
    T* ring = reinterpret_cast<T*>(smem + sizeof(PreStep<K>) * kPre * SPC);               // [kRing][3K][SPC]
    uint32_t* xflag = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(ring) +
                                                  sizeof(T) * kRing * 3 * K * SPC);     // [2][32]
    uint32_t* abort_flag = xflag + 64;                                                      // [1] (+3 pad)
    uint16_t* wsm = reinterpret_cast<uint16_t*>(xflag + 68);                                // [kWordCap]
    float2* ctxb = reinterpret_cast<float2*>(wsm + kWordCap);   // MODE 1, pass 1: (float(ctx), -cnt) [kRing][SPC]

    const int rank = (int)cluster_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool xwarp = MODE == 1 && warp == CW + PW;   // the context warp
    const bool producer = warp >= CW && !xwarp, consumer = warp < CW;
    const int grp = lane / LPS, j = lane % LPS;       // consumer: stream group, lane in group
    const int pi = lane % R0;                         // producer: round-0 point of this lane
    const int wl = producer ? (warp - CW) * SPP + lane / R0 : consumer ? warp * SPW + grp : 0;   // stream slot
    const int ws = rank * SPC + wl;                   // stream within the segment
    const uint32_t bit = 1u << ws;
    const int gbase = grp * LPS;
    const uint32_t gmask = LPS == 32 ? kFull : (((1u << LPS) - 1u) << gbase);
    const int ptid = tid - 32 * CW;                   // producer thread index
    int64_t g = blockIdx.x / CL;
    int pass = 0;
    const T* params = params_a;
    int64_t N = N_a, T_steps = T_a, n_words = n_words_a;
    int32_t S = S_a;
    int mode = mode_a;
    const uint16_t* words = words_a;
    const int64_t* offsets = offsets_a;
    int32_t* out = out_a;
    if constexpr (MODE == 1) {
        if (g >= fz.nseg0) {
            pass = 1;
            g -= fz.nseg0;
        }
        const WsPassDev& P = fz.pass[pass];
        params = static_cast<const T*>(P.params);
        N = P.N;
        S = P.S;
        T_steps = P.T;
        mode = P.mode;
        words = P.words;
        n_words = P.n_words;
        offsets = P.offsets;
        out = P.out;
    }
    const bool counts = MODE == 1 && pass == 0;   // pass 0 of MODE 1: counts each step's completion
    const bool ctxw = MODE == 1 && pass == 1 && xwarp;   // pass 1's context warp
    const bool posts = !(g == 0 && ws == silent);
    const int64_t beg = offsets[g], end = offsets[g + 1];
    if (!(beg >= 0 && end <= n_words && end - beg >= 64)) {
        if (tid == 0 && rank == 0) set_error(err, kErrCorrupt);
        if (counts && !fz.silent_arrivals)   // every step counted once for this CTA, so that no wait on it runs out
            for (int64_t u = tid; u < T_steps; u += NT) atomicAdd(fz.arrivals + u, 1u);
        return;
    }
    const int64_t seg_len = end - beg;
    const bool staged = seg_len <= kWordCap;
    const uint16_t* wseg = staged ? wsm : words + beg;   // the segment's words
    const int64_t nbase = g * 32 + rank * SPC;

    // producer: prepare step u of this warp's stream into pre[u % kPre]
    bool badp = false;
    int probes = 0;
    auto produce = [&](int64_t u) {
        const T* slot_p = ring + (u % kRing) * 3 * K * SPC;
        RawParams<K> r;
#pragma unroll
        for (int i = 0; i < 3 * K; ++i) r.v[i] = smem_param<T>(slot_p + i * SPC + wl);
        if (MODE == 1 && pass == 1) {   // the stand-in context
            const float2 cx = ctxb[(u % kRing) * SPC + wl];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                r.v[K + k] = __fmaf_rn(0.125f, __fmaf_rn(cx.y, r.v[K + k], cx.x), r.v[K + k]);
                r.v[2 * K + k] = __fmul_rn(r.v[2 * K + k], 0.75f);
            }
        }
        Mix<K> m;
        const bool ok = mix_from_params<K>(r, m);
        const bool act = u * (int64_t)S + g * 32 + ws < N;
        badp |= act && !ok;
        PreStep<K>& P = pre[(u % kPre) * SPC + wl];
        P.q0[pi] = q_at<K>(m, round0_point<K, R0>(m, pi));
        probes += act;
        if (pi == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) { P.w[k] = m.w[k]; P.mu[k] = m.mu[k]; P.isg[k] = m.isg[k]; }
            P.lo = m.lo;
            P.hi = m.hi;
            P.tp = m.tp;
        }
    };
    // consumer: step u's mixture and this lane's VPL round-0 values (round-0
    // point i at lane i / VPL, element i % VPL), into registers
    auto fetch = [&](int64_t u, Mix<K>& m, uint32_t (&q0)[VPL]) {
        const PreStep<K>& P = pre[(u % kPre) * SPC + wl];
#pragma unroll
        for (int k = 0; k < K; ++k) { m.w[k] = P.w[k]; m.mu[k] = P.mu[k]; m.isg[k] = P.isg[k]; }
        m.lo = P.lo;
        m.hi = P.hi;
        m.tp = P.tp;
        if constexpr (VPL == 1) {
            q0[0] = P.q0[j];
        } else if constexpr (VPL == 2) {
            const uint2 v = reinterpret_cast<const uint2*>(P.q0)[j];
            q0[0] = v.x;
            q0[1] = v.y;
        } else {
            const uint4 v = reinterpret_cast<const uint4*>(P.q0)[j];
            q0[0] = v.x;
            q0[1] = v.y;
            q0[2] = v.z;
            q0[3] = v.w;
        }
    };

    // prologue: exchange flags, parameters of steps 0 .. kLead+1, words,
    // round 0 of steps 0 .. kLead-1
    if (tid < 68) xflag[tid] = tid == 64 ? 0u : 0xffffffffu;   // tags no exchange number reaches; abort flag 0
    // pass 1 of MODE 1: (float(ctx), -cnt) per step slot and column, after the words
    uint32_t seen = 0, poll_k = 0, poll_v = 0;   // context warp: pass-0 steps known complete; poll in flight
    int32_t nb[4] = {0, 0, 0, 0};                 // context warp: neighbours loaded for the next slot
    int nbc = 0;
    CkbdCursor cur = {}, far = {};                // context warp: the next step to load; kPollAhead steps on
    const uint32_t nprog = (uint32_t)(fz.nseg0 * CL);
    // context warp: waits for and loads the neighbours of step cur.u, then moves both cursors on a step
    auto ctx_load = [&]() {
        ckbd_wait<CL>(fz, cur.need, seen, nprog, abort_flag, err, lane);
        ckbd_load(fz, lane < SPC && cur.u * (uint32_t)S + (uint32_t)nbase + lane < (uint32_t)N, cur.pos, nb, nbc);
        cursor_next<SPC>(fz, cur, (uint32_t)nbase);
        cursor_next<SPC>(fz, far, (uint32_t)nbase);
    };
    if constexpr (MODE == 1) {
        seg_sync<CL>();   // flags initialised in every CTA before a context wait may raise abort
        if (ctxw) {
            cur.pos = ckbd_pos(fz, (uint32_t)nbase + lane);
            cursor_need<SPC>(fz, cur, (uint32_t)nbase);
            far = cur;
            for (int d = 0; d < kPollAhead; ++d) cursor_next<SPC>(fz, far, (uint32_t)nbase);
            for (int64_t p = 0; p < kLead + 2 && p < T_steps; ++p) {
                ctx_load();
                if (lane < SPC) ctxb[(p % kRing) * SPC + lane] = ckbd_ctx(nb, nbc);
            }
        }
    }
    for (int p = 0; p < kLead + 2; ++p) {
        if (producer && p < T_steps)
            stage_params<K, T, SPC>(ring + (p % kRing) * 3 * K * SPC, params, N, p * (int64_t)S + nbase, ptid,
                                    PNT, mode);
        cp_async_commit();
    }
    if (staged)
        for (int64_t i = tid; i < seg_len; i += NT) wsm[i] = __ldg(words + beg + i);
    cp_async_wait<1>();   // steps 0 .. kLead resident
    __syncthreads();
    if (producer)
        for (int64_t u = 0; u < kLead && u < T_steps; ++u) produce(u);
    seg_sync<CL>();       // flags initialised in every CTA before any exchange

    int32_t rp = (int32_t)(seg_len - 64);   // read position in the segment
    uint32_t x = (uint32_t)wseg[rp + 2 * ws] | ((uint32_t)wseg[rp + 2 * ws + 1] << 16);
    int64_t n = g * 32 + ws;                  // this stream's symbol at step t (consumers)
    bool bad = false;
    int decoded = 0;
    uint32_t e = 0;       // exchange number (the same in every stream)
    Mix<K> m;
    uint32_t q0[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) q0[v] = 0;
    if (consumer && T_steps > 0) fetch(0, m, q0);

    for (int64_t t = 0; t < T_steps; ++t) {
        if (producer) {
            if (t + kLead + 2 < T_steps)
                stage_params<K, T, SPC>(ring + ((t + kLead + 2) % kRing) * 3 * K * SPC, params, N,
                                        (t + kLead + 2) * (int64_t)S + nbase, ptid, PNT, mode);
            cp_async_commit();
            // two-pass mode: the producers wait until the consumers have posted
            // this step's refill flags, so that the bracket round's CDF
            // evaluations do not share the sub-partitions' issue slots with
            // them (measured: the two-pass launch 3% faster, the one-pass
            // decoder 5% slower, where the producers' later work lengthens
            // the step)
            if constexpr (MODE == 1) asm volatile("bar.sync 1, %0;" ::"r"(32 * (CW + PW)) : "memory");
            if (t + kLead < T_steps) produce(t + kLead);
            cp_async_wait<1>();   // step t + kLead + 1 resident for the next iteration
        } else if (xwarp) {
            if (ctxw) {
                // neighbours of step t + kLead + 1 (loaded an iteration ago) into its slot
                if (t > 0 && t + kLead + 1 < T_steps && lane < SPC)
                    ctxb[((t + kLead + 1) % kRing) * SPC + lane] = ckbd_ctx(nb, nbc);
                if (poll_k != 0) {   // the poll issued an iteration ago
                    if (__shfl_sync(kFull, poll_v, 0) >= nprog) {   // lane 0's acquire saw the count
                        __syncwarp();
                        seen = poll_k;
                    }
                    poll_k = 0;
                }
                if (t + kLead + 2 < T_steps) {
                    ctx_load();   // step t + kLead + 2
                    // a poll for the next step's count, or the larger one kPollAhead steps on
                    if (t + kLead + 3 < T_steps && cur.need > seen) {
                        poll_k = max(cur.need, far.need);
                        if (lane == 0) poll_v = ld_acquire_u32(fz.arrivals + (poll_k - 1));
                    }
                }
            }
        } else {
            const bool act = n < N;
            int32_t s = 0;
            bool esc = false;
            uint32_t start = 0, freq = 1;
            const uint32_t slot = x & 0xffffu;
            // round 0: c = number of round-0 points with Q <= slot
            int c = 0;
#pragma unroll
            for (int v = 0; v < VPL; ++v) c += __popc(__ballot_sync(kFull, act && q0[v] <= slot) & gmask);
            uint32_t qa0, qb0;   // Q at the round-0 points that bracket the symbol
            if constexpr (VPL == 1) {
                const uint32_t qc1 = __shfl_sync(kFull, q0[0], gbase + (c > 0 ? c - 1 : 0));
                qa0 = c > 0 ? qc1 : 0u;
                qb0 = __shfl_sync(kFull, q0[0], gbase + (c < R0 ? c : R0 - 1));
            } else {
                const PreStep<K>& P = pre[(t % kPre) * SPC + wl];   // rewritten two steps later
                qb0 = P.q0[c < R0 ? c : R0 - 1];
                qa0 = c > 0 ? P.q0[c - 1] : 0u;
            }
            if (act && c == R0) {   // Q(hi+1) <= slot: escape
                esc = true;
                start = qa0;
                freq = kM - start;
            }
            const int W = m.hi - m.lo + 1;
            const int a = c > 0 ? m.lo + (c * W + R0 - 1) / R0 : m.lo;
            const int b = m.lo + ((min(c, R0 - 1) + 1) * W + R0 - 1) / R0;
            const int L = b - a;   // the symbol lies in [a, b); its L - 1 inner points are evaluated
            // inner points a+1 .. b-1: a first round of up to LPS points,
            // then (only when the interior exceeds the group) rounds of LPS
            {
                const bool valid = act && !esc && j < L - 1;
                const uint32_t q1 = q_at<K>(m, min(a + 1 + j, m.hi + 1));
                probes += valid;
                int c1 = __popc(__ballot_sync(kFull, valid && q1 <= slot) & gmask);
                const uint32_t q1a = __shfl_sync(kFull, q1, gbase + (c1 > 0 ? c1 - 1 : 0));
                const uint32_t q1b = __shfl_sync(kFull, q1, gbase + (c1 < LPS ? c1 : LPS - 1));
                uint32_t lastq = c1 > 0 ? q1a : qa0;
                uint32_t endq = c1 < min(LPS, L - 1) ? q1b : qb0;
                if constexpr (!kOneRound) {
                    // every first-round point <= slot and more inner points left
                    bool open = act && !esc && c1 == LPS && L - 1 > LPS;
                    for (int base = LPS; __any_sync(kFull, open); base += LPS) {
                        const int idx = base + j;
                        const bool v2 = open && idx < L - 1;
                        const uint32_t q2 = q_at<K>(m, min(a + 1 + idx, m.hi + 1));
                        probes += v2;
                        const int cnt = __popc(__ballot_sync(kFull, v2 && q2 <= slot) & gmask);
                        const uint32_t qlo = __shfl_sync(kFull, q2, gbase + (cnt > 0 ? cnt - 1 : 0));
                        const uint32_t qhi = __shfl_sync(kFull, q2, gbase + (cnt < LPS ? cnt : LPS - 1));
                        if (open) {
                            c1 += cnt;
                            if (cnt > 0) lastq = qlo;
                            if (cnt < min(LPS, L - 1 - base)) {
                                endq = qhi;
                                open = false;
                            } else if (base + LPS >= L - 1) {
                                open = false;   // every inner point <= slot: the bracket's end bounds the symbol
                            }
                        }
                    }
                }
                if (act && !esc) {
                    s = a + c1;
                    start = lastq;
                    freq = endq - start;
                }
            }
            if (act) {
                x = freq * (x >> 16) + slot - start;
                decoded += (j == 0);
            }
            // post this step's flags, then fetch step t + 1's round
            // (produced two barriers ago) while they travel
            const bool need = act && x < kL;
            const uint32_t below = bit - 1u;
            exchange_post<CL>(xflag, e, ws, j, (need ? 1u : 0u) | (esc ? 2u : 0u), posts);
            if constexpr (MODE == 1) asm volatile("bar.arrive 1, %0;" ::"r"(32 * (CW + PW)) : "memory");
            if (t + 1 < T_steps) fetch(t + 1, m, q0);
            const uint32_t f = exchange_wait<CL>(xflag, abort_flag, e++, lane, err);
            const uint32_t M = __ballot_sync(kFull, f & 1u), E = __ballot_sync(kFull, f & 2u);
            ws_refill(x, need, M, below, wseg, rp, bad);
            if (E) {   // the same in every stream of the segment
                uint32_t hi16 = 0, lo16 = 0;
                if (esc) { hi16 = x & 0xffffu; x >>= 16; }
                const bool n2 = esc && x < kL;
                const uint32_t M2 =
                    __ballot_sync(kFull, exchange<CL>(xflag, abort_flag, e++, ws, j, lane, n2 ? 1u : 0u, err, posts) & 1u);
                ws_refill(x, n2, M2, below, wseg, rp, bad);
                if (esc) { lo16 = x & 0xffffu; x >>= 16; }
                const bool n3 = esc && x < kL;
                const uint32_t M3 =
                    __ballot_sync(kFull, exchange<CL>(xflag, abort_flag, e++, ws, j, lane, n3 ? 1u : 0u, err, posts) & 1u);
                ws_refill(x, n3, M3, below, wseg, rp, bad);
                if (esc) s = (int32_t)((hi16 << 16) | lo16);
            }
            if (act && j == 0) out[n] = s;
            n += S;
        }
        __syncthreads();   // producers' round for step t + 2 visible; slots read
        if (counts && xwarp && lane == 0 && !fz.silent_arrivals) {   // the step's symbols stored by every consumer
            __threadfence();
            atomicAdd(fz.arrivals + t, 1u);
        }
    }
    cp_async_wait<0>();
    const bool fail = consumer && (bad || x != kL || rp != 0);
    if (__syncthreads_or(fail) && tid == 0) set_error(err, kErrCorrupt);
    if (__syncthreads_or(badp) && tid == 0) set_error(err, kErrBadParams);
    if (stats) {
        int p = probes, d = decoded;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(kFull, p, o);
            d += __shfl_xor_sync(kFull, d, o);
        }
        if (lane == 0) {
            atomicAdd(stats, (unsigned long long)p);
            atomicAdd(stats + 1, (unsigned long long)d);
        }
    }
    seg_sync<CL>();       // no CTA leaves while another may still write its flags
}

template <int K, typename T, int CL, int SPW, int R0>
cudaError_t launch_ws(const DecodeArgs& a, cudaStream_t st)
{
    constexpr int SPC = 32 / CL;
    constexpr int NT = 32 * (SPC / SPW + SPC * R0 / 32);
    const size_t smem = sizeof(PreStep<K>) * kPre * SPC + sizeof(T) * kRing * 3 * K * SPC + sizeof(uint32_t) * 68 +
                        sizeof(uint16_t) * kWordCap;
    // exchange numbers stay below 2^30, and a segment (at most 96 T + 64
    // words) below 2^31 words for the 32-bit read position
    if (a.T >= ((int64_t)1 << 24)) return cudaErrorInvalidValue;
    auto kern = fgmm_dec_ws_kernel<K, T, CL, SPW, R0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uintptr_t base = reinterpret_cast<uintptr_t>(a.params);
    int mode = 0;
    if (base % 16 == 0 && (a.N * (int64_t)sizeof(T)) % 16 == 0 && SPC * sizeof(T) >= 16) mode = 2;
    else if (base % 4 == 0 && (a.N * (int64_t)sizeof(T)) % 4 == 0 && SPC * sizeof(T) >= 4) mode = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.nseg * CL));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    WsFuseDev none = {};
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const T*>(a.params), a.N, a.S, a.T, a.words, a.n_words,
                              a.offsets, a.out, a.err, a.stats, mode, a.silent, none);
}

// Staging mode of stage_params for fp32 or bf16 rows of N elements at base.
template <typename T, int SPC>
int ws_stage_mode(const void* p, int64_t N)
{
    const uintptr_t base = reinterpret_cast<uintptr_t>(p);
    if (base % 16 == 0 && (N * (int64_t)sizeof(T)) % 16 == 0 && SPC * sizeof(T) >= 16) return 2;
    if (base % 4 == 0 && (N * (int64_t)sizeof(T)) % 4 == 0 && SPC * sizeof(T) >= 4) return 1;
    return 0;
}

// The checkerboard's two passes in one launch: 16 lanes per stream,
// clusters of 4, a 16-point first round, fp32 or bf16 hyperprior
// parameters (the context is applied to their fp32 values); pass 1's
// context slots follow the words in shared memory. The host runs it only
// when every cluster fits on the device at once (ws_ckbd_capacity).
template <int K, typename T>
struct WsCkbdShape {
    static constexpr int CL = 4, SPW = 2, R0 = 16, SPC = 32 / CL;
    static constexpr int NT = 32 * (SPC / SPW + SPC * R0 / 32) + 32;   // + the context warp
    static constexpr size_t smem = sizeof(PreStep<K>) * kPre * SPC + sizeof(T) * kRing * 3 * K * SPC +
                                   sizeof(uint32_t) * 68 + sizeof(uint16_t) * kWordCap + sizeof(float2) * kRing * SPC;
    static_assert((sizeof(PreStep<K>) * kPre * SPC + sizeof(T) * kRing * 3 * K * SPC + sizeof(uint32_t) * 68 +
                   sizeof(uint16_t) * kWordCap) % 8 == 0, "context slots 8-byte aligned");
};

// Clusters of the fused launch that the current device holds at once.
template <int K, typename T>
cudaError_t ws_ckbd_capacity_k(int* clusters)
{
    using Sh = WsCkbdShape<K, T>;
    auto kern = fgmm_dec_ws_kernel<K, T, Sh::CL, Sh::SPW, Sh::R0, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(Sh::CL);
    cfg.blockDim = dim3(Sh::NT);
    cfg.dynamicSmemBytes = Sh::smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Sh::CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
}

template <int K, typename T>
cudaError_t launch_ws_ckbd_k(const CkbdFuseArgs& a, cudaStream_t st)
{
    using Sh = WsCkbdShape<K, T>;
    constexpr int CL = Sh::CL, SPW = Sh::SPW, R0 = Sh::R0, SPC = Sh::SPC, NT = Sh::NT;
    constexpr size_t smem = Sh::smem;
    for (int p = 0; p < 2; ++p)
        if (a.pass[p].T >= ((int64_t)1 << 24)) return cudaErrorInvalidValue;
    auto kern = fgmm_dec_ws_kernel<K, T, CL, SPW, R0, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.C * a.H * a.W >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    WsFuseDev fz = {};
    for (int p = 0; p < 2; ++p) {
        const DecodeArgs& d = a.pass[p];
        fz.pass[p] = WsPassDev{d.params, d.N, d.S, ws_stage_mode<T, SPC>(d.params, d.N), d.T, d.words, d.n_words,
                               d.offsets, d.out};
    }
    fz.nseg0 = a.pass[0].nseg;
    fz.H = (uint32_t)a.H;
    fz.W = (uint32_t)a.W;
    fz.per_a = (uint32_t)((a.H * a.W + 1) / 2);
    fz.per_n = (uint32_t)(a.H * a.W) - fz.per_a;
    if (fz.per_n == 0) return cudaErrorInvalidValue;
    fz.pq = fz.per_n / fz.W;
    fz.pr = fz.per_n % fz.W;
    const uint32_t Sn = (uint32_t)a.pass[1].S, rs = Sn % fz.per_n;
    fz.adv_c = Sn / fz.per_n;
    fz.adv_h = rs / fz.W;
    fz.adv_r = rs % fz.W;
    fz.ya = a.pass[0].out;
    fz.arrivals = a.arrivals;
    fz.silent_arrivals = a.silent_arrivals;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((a.pass[0].nseg + a.pass[1].nseg) * CL));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const DecodeArgs& d0 = a.pass[0];
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const T*>(d0.params), d0.N, d0.S, d0.T, d0.words,
                              d0.n_words, d0.offsets, d0.out, d0.err, d0.stats, 0, d0.silent, fz);
}

template <typename T>
cudaError_t ws_ckbd_capacity_t(int K, int* clusters)
{
    switch (K) {
    case 1: return ws_ckbd_capacity_k<1, T>(clusters);
    case 2: return ws_ckbd_capacity_k<2, T>(clusters);
    case 3: return ws_ckbd_capacity_k<3, T>(clusters);
    default: return ws_ckbd_capacity_k<4, T>(clusters);
    }
}

template <typename T>
cudaError_t launch_ws_ckbd_t(const CkbdFuseArgs& a, int K, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_ws_ckbd_k<1, T>(a, st);
    case 2: return launch_ws_ckbd_k<2, T>(a, st);
    case 3: return launch_ws_ckbd_k<3, T>(a, st);
    default: return launch_ws_ckbd_k<4, T>(a, st);
    }
}

template <int K, typename T, int SPW, int R0>
cudaError_t launch_ws_cl(const DecodeArgs& a, int CL, cudaStream_t st)
{
    switch (CL) {
    case 8: return launch_ws<K, T, 8, SPW, R0>(a, st);
    case 4: return launch_ws<K, T, 4, SPW, R0>(a, st);
    default: return launch_ws<K, T, 2, SPW, R0>(a, st);
    }
}

// Round-0 width: 32 points for 32 and 8 lanes per stream; 16 lanes per
// stream take 16 (two streams per producer warp) or 32, as a.r0 says.
template <int K, typename T>
cudaError_t launch_ws_k(const DecodeArgs& a, int CL, int SPW, cudaStream_t st)
{
    switch (SPW) {
    case 4: return launch_ws_cl<K, T, 4, 32>(a, CL, st);
    case 2: return a.r0 == 16 ? launch_ws_cl<K, T, 2, 16>(a, CL, st) : launch_ws_cl<K, T, 2, 32>(a, CL, st);
    default: return launch_ws_cl<K, T, 1, 32>(a, CL, st);
    }
}

template <typename T>
cudaError_t launch_ws_t(const DecodeArgs& a, int K, int CL, int SPW, cudaStream_t st)
{
    if (a.nseg == 0) return cudaSuccess;
    switch (K) {
    case 1: return launch_ws_k<1, T>(a, CL, SPW, st);
    case 2: return launch_ws_k<2, T>(a, CL, SPW, st);
    case 3: return launch_ws_k<3, T>(a, CL, SPW, st);
    default: return launch_ws_k<4, T>(a, CL, SPW, st);
    }
}

}  // namespace
