"""GPU encode/decode parity with the CPU oracle: frequencies, bitstreams,
offsets and decoded symbols must be identical (bit-exact), on the seeded
synthetic workloads, across tile edges and ragged tails, with escapes and
extreme parameters; damage and bad input are reported through the status
word, never by a fault."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, host_u16, host_u32, need_gpu, oracle_params

pytestmark = pytest.mark.gpu


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


def _check_latent(params, syms, S, bf16=False, check_oracle_decode=True):
    codec = _codec()
    op = oracle_params(params, bf16)
    dp = dev_params(params, bf16)
    ds = dev_i32(syms)
    # frequencies
    sf_g = host_u32(codec.freqs(dp, ds))
    sf_c = oracle.freqs(op, syms)
    np.testing.assert_array_equal(sf_g, sf_c)
    # bitstream
    words_g, off_g = codec.encode(dp, ds, S)
    words_c, off_c = oracle.encode(op, syms, S)
    np.testing.assert_array_equal(off_g.cpu().numpy(), off_c)
    np.testing.assert_array_equal(host_u16(words_g), words_c)
    # decode
    out = codec.decode(dp, words_g, off_g, S).cpu().numpy()
    np.testing.assert_array_equal(out, syms)
    if check_oracle_decode:
        out_c, st = oracle.decode(op, words_c, off_c, S)
        assert st == oracle.OK
        np.testing.assert_array_equal(out_c, syms)


def test_workload_latent_192x16x16_k3_s32():
    lat = synth.make_latent(192, 16, 16, 3, seed=1001)
    _check_latent(lat.params, lat.symbols, 32)


def test_workload_latent_192x32x48_k3_s1024():
    lat = synth.make_latent(192, 32, 48, 3, seed=1002)
    _check_latent(lat.params, lat.symbols, 1024)


@pytest.mark.parametrize("N", [0, 1, 31, 32, 33, 1000, 4097, 70001])
@pytest.mark.parametrize("S", [32, 64, 1024])
def test_sizes(N, S):
    lat = synth.make_latent(1, 1, max(N, 1), 3, seed=N + 3 * S)
    _check_latent(np.ascontiguousarray(lat.params[:, :, :N]), np.ascontiguousarray(lat.symbols[:N]), S)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
@pytest.mark.parametrize("bf16", [False, True])
def test_components_and_dtypes(K, bf16):
    lat = synth.make_latent(16, 16, 16, K, seed=200 + K)
    _check_latent(lat.params, lat.symbols, 256, bf16=bf16)


def test_escapes():
    lat = synth.make_latent(8, 32, 32, 3, seed=300, escape_stress=0.02)
    s = lat.symbols.copy()
    s[:6] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, -256, 256, -1, 65536]
    _check_latent(lat.params, s, 128)


@pytest.mark.parametrize("T", [2, 15, 16, 17, 31, 33])
def test_step_counts_around_encoder_blocks_with_escapes(T):
    """The rANS encoder's preparing warp hands steps to its state warp 16 at
    a time: step counts on both sides of those blocks, a ragged last step,
    and whole steps of escapes at both ends of the encode (step T-1, coded
    first, and step 0, coded last), against the oracle."""
    S = 64
    N = T * S - 7
    lat = synth.make_latent(1, 1, N, 3, seed=700 + T, escape_stress=0.05)
    s = lat.symbols.copy()
    s[:S] = 70000 + np.arange(S)          # step 0
    s[(T - 1) * S:] = -70000               # step T-1 (57 symbols)
    _check_latent(lat.params, s, S)


def test_extreme_params():
    lat = synth.make_latent(4, 32, 32, 4, seed=301, sigma_max=64.0)
    p = lat.params.copy()
    p[2, :, ::5] = 0.11
    p[2, 1, 1::5] = 1e7
    p[1, 2, 2::5] = -3e4
    p[0, :, 3::5] = 0.0
    p[0, 0, 4::5] = 3.0
    p[1, 0, 6::11] = 3e38
    _check_latent(p, lat.symbols, 64)


def test_scales_at_and_beyond_2_to_125():
    """Scales of 2^125 and more take the correctly rounded reciprocal (the
    inverse may be subnormal); with means up to the float range the
    frequencies and the stream still match the oracle bit for bit."""
    lat = synth.make_latent(4, 16, 16, 3, seed=303)
    p = lat.params.copy()
    big = np.array([2.0 ** 125, 2.0 ** 126, 1e38, 3.4e38], dtype=np.float32)
    p[2, 1, ::3] = np.resize(big, p[2, 1, ::3].shape)
    p[2, 2, 1::7] = 3.4e38
    p[1, 1, ::6] = 1e38
    p[1, 2, 2::9] = -3e38
    _check_latent(p, lat.symbols, 64)


def test_large_scales_workload_distribution():
    lat = synth.make_latent(32, 32, 32, 3, seed=302, sigma_max=64.0)
    _check_latent(lat.params, lat.symbols, 512)


@pytest.mark.parametrize("K,bf16", [(3, False), (4, False), (3, True), (4, True)])
def test_workload_latent_320x64x96(K, bf16):
    """Full-size 1,966,080-symbol latent: GPU stream identical to the oracle's
    (the oracle encodes it in about a second); GPU round trip exact."""
    lat = synth.make_latent(320, 64, 96, K, seed=1003)
    codec = _codec()
    S = 4096
    op = oracle_params(lat.params, bf16)
    dp = dev_params(lat.params, bf16)
    ds = dev_i32(lat.symbols)
    words_g, off_g = codec.encode(dp, ds, S)
    words_c, off_c = oracle.encode(op, lat.symbols, S)
    np.testing.assert_array_equal(off_g.cpu().numpy(), off_c)
    np.testing.assert_array_equal(host_u16(words_g), words_c)
    out = codec.decode(dp, words_g, off_g, S).cpu().numpy()
    np.testing.assert_array_equal(out, lat.symbols)


# ---------------------------------------------------------------------------
# Errors are reported, not faulted.
# ---------------------------------------------------------------------------

def test_corrupt_streams_report_corrupt():
    codec = _codec()
    from paper_2509_18815_gb300._abi import FGMM_ERR_CORRUPT, FgmmError
    lat = synth.make_latent(4, 16, 16, 3, seed=400)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    S = 64
    words, off = codec.encode(dp, ds, S)
    bad = words.clone()
    bad[int(off[1].item()) - 64] ^= 0x1234
    with pytest.raises(FgmmError) as e:
        codec.decode(dp, bad, off, S)
    assert e.value.status == FGMM_ERR_CORRUPT
    # truncated: offsets beyond the words buffer
    with pytest.raises(FgmmError) as e:
        codec.decode(dp, words[:-5], off, S)
    assert e.value.status == FGMM_ERR_CORRUPT
    # segment shorter than its flush block
    off2 = off.clone()
    off2[1] = off2[0] + 10
    with pytest.raises(FgmmError) as e:
        codec.decode(dp, words, off2, S)
    assert e.value.status == FGMM_ERR_CORRUPT
    # garbage words: every read stays inside the segment
    junk = torch.randint(-32768, 32767, words.shape, dtype=torch.int16, device="cuda")
    with pytest.raises(FgmmError) as e:
        codec.decode(dp, junk, off, S)
    assert e.value.status == FGMM_ERR_CORRUPT
    # the handle is still usable afterwards
    out = codec.decode(dp, words, off, S).cpu().numpy()
    np.testing.assert_array_equal(out, lat.symbols)


def test_bad_params_and_capacity():
    codec = _codec()
    from paper_2509_18815_gb300._abi import FGMM_ERR_BAD_PARAMS, FGMM_ERR_CAPACITY, FGMM_ERR_INVALID_ARG, FgmmError
    lat = synth.make_latent(2, 16, 16, 3, seed=401)
    ds = dev_i32(lat.symbols)
    for c, v in [(0, -1.0), (0, float("nan")), (1, float("inf")), (2, 0.0), (2, -2.0)]:
        p = lat.params.copy()
        p[c, 1, 17] = v
        with pytest.raises(FgmmError) as e:
            codec.encode(dev_params(p), ds, 32)
        assert e.value.status == FGMM_ERR_BAD_PARAMS
    dp = dev_params(lat.params)
    with pytest.raises(FgmmError) as e:
        codec.encode(dp, ds, 32, words_cap=100)
    assert e.value.status == FGMM_ERR_CAPACITY
    with pytest.raises(ValueError):
        codec.encode(dp, ds, 48)
    from paper_2509_18815_gb300 import _abi
    import ctypes
    h = codec.handle()
    bad = codec.latent(dp)
    bad.K = 5
    st = _abi.fgmm_freqs(h.ptr, ctypes.byref(bad), ds.data_ptr(), ds.data_ptr(), None)
    assert st == FGMM_ERR_INVALID_ARG
    words, off = codec.encode(dp, ds, 32)
    np.testing.assert_array_equal(codec.decode(dp, words, off, 32).cpu().numpy(), lat.symbols)


def _set_lanes(G):
    from paper_2509_18815_gb300 import _abi
    codec = _codec()
    h = codec.handle()
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, G))


DECODE_CASES = [
    # (C, H, W, K, seed, escape_stress, sigma_max, S, bf16, N_cut)
    (8, 32, 32, 3, 500, 0.02, 16.0, 128, False, None),    # escapes, 16-byte staging
    (1, 1, 70001, 4, 501, 0.001, 64.0, 64, True, None),   # bf16, odd N: plain staging
    (1, 1, 4097, 2, 502, 0.0, 16.0, 1024, False, None),   # N % 4 = 1: 4-byte staging, mostly idle lanes
    (192, 32, 48, 3, 1002, 0.0, 16.0, 1024, False, None),  # the bench latent
    (4, 16, 16, 1, 503, 0.01, 16.0, 32, True, 1002),      # K = 1, bf16, 2N % 16 = 4: 4-byte staging
]


@pytest.mark.parametrize("case", range(len(DECODE_CASES)))
@pytest.mark.parametrize("G", [1, 2, 4, 8, 16, 32])
def test_decode_lanes_give_identical_symbols(case, G):
    codec = _codec()
    C, H, W, K, seed, esc, smax, S, bf16, cut = DECODE_CASES[case]
    lat = synth.make_latent(C, H, W, K, seed=seed, escape_stress=esc, sigma_max=smax)
    p, s = lat.params, lat.symbols
    if cut is not None:
        p, s = np.ascontiguousarray(p[:, :, :cut]), np.ascontiguousarray(s[:cut])
    dp, ds = dev_params(p, bf16), dev_i32(s)
    words, off = codec.encode(dp, ds, S)
    try:
        _set_lanes(G)
        out = codec.decode(dp, words, off, S).cpu().numpy()
    finally:
        _set_lanes(0)
    np.testing.assert_array_equal(out, s)


def _set_cluster(CL):
    from paper_2509_18815_gb300 import _abi
    codec = _codec()
    h = codec.handle()
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_CLUSTER, CL))


@pytest.mark.parametrize("case", range(len(DECODE_CASES)))
@pytest.mark.parametrize("G,CL", [(2, 2), (4, 4), (8, 2), (8, 4), (8, 8), (16, 2), (16, 4), (16, 8), (32, 1), (32, 2),
                                  (32, 4), (32, 8)])
def test_decode_clusters_give_identical_symbols(case, G, CL):
    """A segment spread over a cluster of CL CTAs (refill ranks exchanged
    through distributed shared memory) decodes the same symbols."""
    codec = _codec()
    C, H, W, K, seed, esc, smax, S, bf16, cut = DECODE_CASES[case]
    lat = synth.make_latent(C, H, W, K, seed=seed, escape_stress=esc, sigma_max=smax)
    p, s = lat.params, lat.symbols
    if cut is not None:
        p, s = np.ascontiguousarray(p[:, :, :cut]), np.ascontiguousarray(s[:cut])
    dp, ds = dev_params(p, bf16), dev_i32(s)
    words, off = codec.encode(dp, ds, S)
    try:
        _set_lanes(G)
        _set_cluster(CL)
        out = codec.decode(dp, words, off, S).cpu().numpy()
    finally:
        _set_lanes(0)
        _set_cluster(0)
    np.testing.assert_array_equal(out, s)


def test_decode_plan_follows_segments_and_options():
    """The plan names the decoder fgmm_decode runs: one lane per stream when
    segments fill the SMs several times over, 32 lanes and a cluster per
    segment when segments are few, and the options override both (with the
    cluster clamped to what each kernel takes)."""
    codec = _codec()
    from paper_2509_18815_gb300._abi import FgmmError
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    many = 32 * 4 * sms
    assert codec.decode_plan(many) == {"lanes": 1, "cluster": 1, "round0": 0, "kernel": "fgmm_dec_kernel"}
    assert codec.decode_plan(32) == {"lanes": 32, "cluster": 8, "round0": 32, "kernel": "fgmm_dec_ws_kernel"}
    few = 32 * max(1, sms // 4)
    assert codec.decode_plan(few) == {"lanes": 16, "cluster": 4, "round0": 16, "kernel": "fgmm_dec_ws_kernel"}
    try:
        _set_lanes(4)
        assert codec.decode_plan(few) == {"lanes": 4, "cluster": 1, "round0": 0, "kernel": "fgmm_dec_coop_kernel"}
        _set_lanes(32)
        assert codec.decode_plan(few) == {"lanes": 32, "cluster": 2, "round0": 32, "kernel": "fgmm_dec_ws_kernel"}
        _set_lanes(4)
        _set_cluster(8)
        assert codec.decode_plan(few) == {"lanes": 4, "cluster": 4, "round0": 0, "kernel": "fgmm_dec_coop_kernel"}
        _set_lanes(8)
        assert codec.decode_plan(few) == {"lanes": 8, "cluster": 8, "round0": 32, "kernel": "fgmm_dec_ws_kernel"}
        _set_lanes(16)
        _set_cluster(1)
        assert codec.decode_plan(few) == {"lanes": 16, "cluster": 1, "round0": 0, "kernel": "fgmm_dec_coop_kernel"}
        _set_cluster(8)
        _set_lanes(1)
        assert codec.decode_plan(few) == {"lanes": 1, "cluster": 1, "round0": 0, "kernel": "fgmm_dec_kernel"}
        _set_lanes(32)
        _set_cluster(1)
        assert codec.decode_plan(few) == {"lanes": 32, "cluster": 2, "round0": 32, "kernel": "fgmm_dec_ws_kernel"}
        _set_lanes(0)
        _set_cluster(0)
        _set_round0(32)
        assert codec.decode_plan(few) == {"lanes": 16, "cluster": 4, "round0": 32, "kernel": "fgmm_dec_ws_kernel"}
        _set_lanes(8)
        _set_cluster(8)
        assert codec.decode_plan(few) == {"lanes": 8, "cluster": 8, "round0": 32, "kernel": "fgmm_dec_ws_kernel"}
    finally:
        _set_lanes(0)
        _set_cluster(0)
        _set_round0(0)
    for bad in (8, 64, -1):
        with pytest.raises(FgmmError):
            _set_round0(bad)
    for bad in (0, -32, 33):
        with pytest.raises(FgmmError):
            codec.decode_plan(bad)


def _set_round0(R0):
    from paper_2509_18815_gb300 import _abi
    codec = _codec()
    h = codec.handle()
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_ROUND0, R0))


@pytest.mark.parametrize("case", range(len(DECODE_CASES)))
@pytest.mark.parametrize("CL", [2, 4, 8])
@pytest.mark.parametrize("R0", [16, 32])
def test_decode_round0_widths_give_identical_symbols(case, CL, R0):
    """16 lanes per stream with a 16- or 32-point first round (two or one
    streams per producer warp; with 16 points a wide window's bracket can
    need two rounds of 16 inner points) decode the same symbols."""
    codec = _codec()
    C, H, W, K, seed, esc, smax, S, bf16, cut = DECODE_CASES[case]
    lat = synth.make_latent(C, H, W, K, seed=seed, escape_stress=esc, sigma_max=smax)
    p, s = lat.params, lat.symbols
    if cut is not None:
        p, s = np.ascontiguousarray(p[:, :, :cut]), np.ascontiguousarray(s[:cut])
    dp, ds = dev_params(p, bf16), dev_i32(s)
    words, off = codec.encode(dp, ds, S)
    try:
        _set_lanes(16)
        _set_cluster(CL)
        _set_round0(R0)
        assert codec.decode_plan(S)["round0"] == R0
        out = codec.decode(dp, words, off, S).cpu().numpy()
    finally:
        _set_lanes(0)
        _set_cluster(0)
        _set_round0(0)
    np.testing.assert_array_equal(out, s)


@pytest.mark.parametrize("G,CL", [(16, 4), (32, 8)])
def test_decode_wait_times_out_and_recovers(G, CL):
    """A stream that never posts its refill flags makes the other streams'
    bounded waits run out: the warp-specialised decoder records
    FGMM_ERR_TIMEOUT, every wait is released through the abort flag, the
    kernel returns, and the next decode on the same context is exact. Four
    steps of one segment bound the time even if the abort did not spread."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    from paper_2509_18815_gb300._abi import FGMM_ERR_TIMEOUT, FgmmError
    lat = synth.make_latent(1, 1, 128, 3, seed=506)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    words, off = codec.encode(dp, ds, 32)
    h = codec.handle()
    try:
        _set_lanes(G)
        _set_cluster(CL)
        assert codec.decode_plan(32)["kernel"] == "fgmm_dec_ws_kernel"
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_STREAM, 5))
        with pytest.raises(FgmmError) as e:
            codec.decode(dp, words, off, 32)
        assert e.value.status == FGMM_ERR_TIMEOUT
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_STREAM, -1))
        out = codec.decode(dp, words, off, 32).cpu().numpy()
    finally:
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_STREAM, -1))
        _set_lanes(0)
        _set_cluster(0)
    np.testing.assert_array_equal(out, lat.symbols)
    with pytest.raises(FgmmError):
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_STREAM, 32))


@pytest.mark.parametrize("G,CL", [(1, 1), (8, 1), (32, 1), (8, 4), (8, 8), (16, 2), (32, 8)])
def test_decode_lanes_report_corruption(G, CL):
    codec = _codec()
    from paper_2509_18815_gb300._abi import FGMM_ERR_CORRUPT, FgmmError
    lat = synth.make_latent(4, 16, 16, 3, seed=504)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    words, off = codec.encode(dp, ds, 64)
    junk = torch.randint(-32768, 32767, words.shape, dtype=torch.int16, device="cuda")
    try:
        _set_lanes(G)
        _set_cluster(CL)
        with pytest.raises(FgmmError) as e:
            codec.decode(dp, junk, off, 64)
        assert e.value.status == FGMM_ERR_CORRUPT
        with pytest.raises(FgmmError) as e:
            codec.decode(dp, words[:-3], off, 64)
        assert e.value.status == FGMM_ERR_CORRUPT
        out = codec.decode(dp, words, off, 64).cpu().numpy()
    finally:
        _set_lanes(0)
        _set_cluster(0)
    np.testing.assert_array_equal(out, lat.symbols)


def test_decode_counts_cdf_evaluations():
    codec = _codec()
    lat = synth.make_latent(8, 16, 16, 3, seed=402)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    words, off = codec.encode(dp, ds, 64)
    codec.stats_enable(True)
    codec.stats_read()
    _set_lanes(1)
    try:
        codec.decode(dp, words, off, 64)
    finally:
        _set_lanes(0)
    evals, nsym = codec.stats_read()
    codec.stats_enable(False)
    assert nsym == lat.N
    lo, hi = oracle.window(lat.params)
    W = (hi - lo + 1).astype(np.float64)
    # bisection of [lo, hi + 2) (the escape slot searched as symbol hi + 1):
    # floor or ceil of log2(W + 1) CDF evaluations per symbol
    assert np.sum(np.floor(np.log2(W + 1))) <= evals <= np.sum(np.ceil(np.log2(W + 1)))


def test_guided_search_fallbacks_decode_exactly():
    """The one-lane decoder steers its binary search with a fast evaluation
    of the CDF and confirms the symbol with the exact quantised CDF. On a
    1,966,080-symbol latent (scales up to 64) the check rejects the steered
    symbol a few hundred times (near-ties, where the fast evaluation falls on
    the other side of a boundary); the exact search then decodes those
    symbols, and the whole latent round-trips. The search still probes as
    many points as the plain binary search."""
    codec = _codec()
    lat = synth.make_latent(320, 64, 96, 3, seed=1003, sigma_max=64.0)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    S = 4096
    words, off = codec.encode(dp, ds, S)
    codec.stats_enable(True)
    codec.stats_read()
    _set_lanes(1)
    try:
        out = codec.decode(dp, words, off, S)
    finally:
        _set_lanes(0)
    evals, nsym, _, fallbacks = codec.stats_read(with_hits=True, with_fallbacks=True)
    codec.stats_enable(False)
    assert torch.equal(out, ds)
    assert nsym == lat.N
    assert 0 < fallbacks < lat.N // 1000
    lo, hi = oracle.window(lat.params)
    W = (hi - lo + 1).astype(np.float64)
    assert np.sum(np.floor(np.log2(W + 1))) <= evals <= np.sum(np.ceil(np.log2(W + 1)))
