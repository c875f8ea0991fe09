"""Checkerboard two-pass coding on the GPU against the oracle: the split of
parameters and symbols into anchors and non-anchors, the merge back, the
stand-in context (bit-exact, fp32 and bf16 hyperprior parameters), the two
streams of the two-pass encode (byte-identical) and the two-pass decode,
both as one fused launch and as separate calls."""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, host_u16, need_gpu, oracle_params

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (2, 1, 5), (3, 4, 1), (2, 5, 7), (4, 6, 8), (8, 16, 24)]


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_split_merge_context_match_oracle(shape, bf16):
    codec = _codec()
    lat = synth.make_ckbd_latent(*shape, 3, seed=900 + sum(shape))
    lat.symbols[::23] = -77777   # large anchors and non-anchors
    dp, dy = dev_params(lat.params, bf16), dev_i32(lat.symbols)
    po = oracle_params(lat.params, bf16)
    pa, ya, pn, yn = codec.ckbd_split(dp, dy, shape)
    pa_o, ya_o, pn_o, yn_o = oracle.ckbd_split(po, lat.symbols, shape)
    np.testing.assert_array_equal(pa.float().cpu().numpy(), pa_o)
    np.testing.assert_array_equal(pn.float().cpu().numpy(), pn_o)
    np.testing.assert_array_equal(ya.cpu().numpy(), ya_o)
    np.testing.assert_array_equal(yn.cpu().numpy(), yn_o)
    np.testing.assert_array_equal(codec.ckbd_merge(ya, yn, shape).cpu().numpy(), lat.symbols)
    ctx = codec.ckbd_context(dp, dy, shape).cpu().numpy()
    np.testing.assert_array_equal(ctx.view(np.uint32), oracle.ckbd_context(po, lat.symbols, shape).view(np.uint32))


@pytest.mark.parametrize("shape,Sa,Sn,bf16", [((4, 16, 16), 32, 64, False), ((3, 9, 13), 64, 32, True),
                                               ((1, 1, 1), 32, 32, False), ((16, 32, 48), 512, 512, False)])
def test_two_pass_streams_and_decode(shape, Sa, Sn, bf16):
    codec = _codec()
    lat = synth.make_ckbd_latent(*shape, 3, seed=950 + Sa)
    dp, dy = dev_params(lat.params, bf16), dev_i32(lat.symbols)
    po = oracle_params(lat.params, bf16)
    (wa, oa), (wn, on) = codec.ckbd_encode(dp, dy, shape, Sa, Sn)
    (wa_o, oa_o), (wn_o, on_o) = oracle.ckbd_encode(po, lat.symbols, shape, Sa, Sn)
    np.testing.assert_array_equal(host_u16(wa), wa_o)
    np.testing.assert_array_equal(oa.cpu().numpy(), oa_o)
    np.testing.assert_array_equal(host_u16(wn), wn_o)
    np.testing.assert_array_equal(on.cpu().numpy(), on_o)
    y = codec.ckbd_decode(dp, (wa, oa), (wn, on), shape, Sa, Sn).cpu().numpy()
    np.testing.assert_array_equal(y, lat.symbols)


def test_full_size_latent():
    """320 x 64 x 96, K = 3: context bit-exact over the whole latent, exact
    two-pass round trip, and the context's rate gain on the second pass."""
    codec = _codec()
    shape = (320, 64, 96)
    lat = synth.make_ckbd_latent(*shape, 3, seed=1003)
    dp, dy = dev_params(lat.params), dev_i32(lat.symbols)
    ctx = codec.ckbd_context(dp, dy, shape).cpu().numpy()
    np.testing.assert_array_equal(ctx.view(np.uint32),
                                  oracle.ckbd_context(lat.params, lat.symbols, shape).view(np.uint32))
    S = 4096
    first, second = codec.ckbd_encode(dp, dy, shape, S, S)
    y = codec.ckbd_decode(dp, first, second, shape, S, S)
    assert torch.equal(y, dy)
    _, _, pn_h, yn = codec.ckbd_split(dp, dy, shape)
    _, bits_h, _, _ = codec.rate_audit(pn_h, yn)
    _, bits_c, _, _ = codec.rate_audit(torch.from_numpy(ctx).cuda(), yn)
    assert bits_c < 0.8 * bits_h


def test_errors_are_reported():
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    from paper_2509_18815_gb300._abi import FGMM_ERR_INVALID_ARG
    h = codec.handle()
    lat = synth.make_latent(2, 4, 4, 3, seed=990)
    dp = dev_params(lat.params)
    desc = codec.latent(dp)
    buf = torch.empty(1024, dtype=torch.float32, device="cuda")
    assert _abi.fgmm_ckbd_split(h.ptr, ctypes.byref(desc), 2, 4, 5, None, buf.data_ptr(), None, buf.data_ptr(),
                                None, None) == FGMM_ERR_INVALID_ARG
    assert _abi.fgmm_ckbd_context(h.ptr, ctypes.byref(desc), 2, 4, 4, None, buf.data_ptr(),
                                  None) == FGMM_ERR_INVALID_ARG
    assert _abi.fgmm_ckbd_merge(h.ptr, -1, 4, 4, None, None, None, None) == FGMM_ERR_INVALID_ARG
    assert _abi.fgmm_ckbd_anchors(3, 5, 5) == 39


@pytest.mark.parametrize("bf16", [False, True])
def test_two_pass_from_cuda_graphs(bf16):
    """The two-pass encode and decode captured into CUDA graphs replay to
    the oracle's streams and the exact symbols, twice in a row, and again
    after the input buffers were overwritten with a second latent."""
    codec = _codec()
    shape, Sa, Sn = (8, 16, 24), 64, 96
    lat = synth.make_ckbd_latent(*shape, 3, seed=961)
    dp, dy = dev_params(lat.params, bf16), dev_i32(lat.symbols)
    po = oracle_params(lat.params, bf16)
    gr = codec.CkbdGraphs(dp, shape, Sa, Sn)
    gr.capture_encode(dy)
    (wa_o, oa_o), (wn_o, on_o) = oracle.ckbd_encode(po, lat.symbols, shape, Sa, Sn)
    for _ in range(2):
        (wa, oa, ta), (wn, on, tn) = gr.encode()
        np.testing.assert_array_equal(host_u16(wa[: int(ta.item())]), wa_o)
        np.testing.assert_array_equal(oa.cpu().numpy(), oa_o)
        np.testing.assert_array_equal(host_u16(wn[: int(tn.item())]), wn_o)
        np.testing.assert_array_equal(on.cpu().numpy(), on_o)
    gr.capture_decode((wa[: int(ta.item())].clone(), oa.clone()), (wn[: int(tn.item())].clone(), on.clone()))
    for _ in range(2):
        gr.y.fill_(-3)
        np.testing.assert_array_equal(gr.decode().cpu().numpy(), lat.symbols)
    # new symbols and parameters in the captured input buffers: the encode
    # replay codes the new latent
    lat2 = synth.make_ckbd_latent(*shape, 3, seed=962)
    gr.params.copy_(dev_params(lat2.params, bf16))
    gr._y_in.copy_(dev_i32(lat2.symbols))
    (wa, oa, ta), (wn, on, tn) = gr.encode()
    (wa_o, _), (wn_o, _) = oracle.ckbd_encode(oracle_params(lat2.params, bf16), lat2.symbols, shape, Sa, Sn)
    np.testing.assert_array_equal(host_u16(wa[: int(ta.item())]), wa_o)
    np.testing.assert_array_equal(host_u16(wn[: int(tn.item())]), wn_o)


def _oracle_streams(lat, shape, Sa, Sn, bf16=False):
    po = oracle_params(lat.params, bf16)
    (wa, oa), (wn, on) = oracle.ckbd_encode(po, lat.symbols, shape, Sa, Sn)
    dev = lambda w, o: (torch.from_numpy(w.view(np.int16).copy()).cuda(), torch.from_numpy(o.copy()).cuda())
    return dev(wa, oa), dev(wn, on)


# (shape, Sa, Sn): 10 to 38 segments in all take the fused launch on a GPU
# of 152 SMs; odd sizes, one-column and one-row channels, one-step passes
FUSED = [((16, 32, 48), 512, 512), ((8, 16, 24), 160, 192), ((5, 9, 13), 320, 320), ((3, 7, 1), 160, 160),
         ((2, 1, 5), 160, 160), ((24, 20, 30), 64, 1088), ((64, 64, 96), 1024, 1024)]


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("shape,Sa,Sn", FUSED)
def test_fused_two_pass_decode(shape, Sa, Sn, bf16):
    """fgmm_ckbd_decode of the oracle's two streams gives the latent's
    symbols, in one launch where its plan says so, and the same symbols as
    the separate calls (integer output: equality); fp32 and bf16
    hyperprior parameters."""
    codec = _codec()
    lat = synth.make_ckbd_latent(*shape, 3, seed=970 + Sa + Sn + sum(shape))
    dp = dev_params(lat.params, bf16)
    first, second = _oracle_streams(lat, shape, Sa, Sn, bf16)
    nseg = Sa // 32 + Sn // 32
    fused = codec.ckbd_decode_fused(3, torch.bfloat16 if bf16 else torch.float32, shape, Sa, Sn)
    if 10 <= nseg <= 32 and torch.cuda.get_device_properties(0).multi_processor_count >= 128:
        assert fused
    for _ in range(2):
        y = codec.ckbd_decode(dp, first, second, shape, Sa, Sn)
        np.testing.assert_array_equal(y.cpu().numpy(), lat.symbols)
    y2 = codec.ckbd_decode_steps(dp, first, second, shape, Sa, Sn)
    np.testing.assert_array_equal(y2.cpu().numpy(), lat.symbols)


@pytest.mark.parametrize("K", [1, 2, 4])
def test_fused_two_pass_decode_components(K):
    codec = _codec()
    shape, Sa, Sn = (12, 16, 20), 256, 320
    lat = synth.make_ckbd_latent(*shape, K, seed=990 + K)
    dp = dev_params(lat.params)
    first, second = _oracle_streams(lat, shape, Sa, Sn)
    if torch.cuda.get_device_properties(0).multi_processor_count >= 128:
        assert codec.ckbd_decode_fused(K, torch.float32, shape, Sa, Sn)
    y = codec.ckbd_decode(dp, first, second, shape, Sa, Sn)
    np.testing.assert_array_equal(y.cpu().numpy(), lat.symbols)


def test_two_pass_decode_plan():
    """Cases outside the fused launch: too few segments for its plan, a
    decoder option set, another Phi approximation; and argument errors."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    from paper_2509_18815_gb300._abi import FGMM_ERR_INVALID_ARG
    assert codec.ckbd_decode_fused(3, torch.bfloat16, (16, 32, 48), 512, 512)
    assert not codec.ckbd_decode_fused(3, torch.float32, (4, 16, 16), 32, 64)
    hp = codec.Handle()
    hp.check(_abi.fgmm_set_option(hp.ptr, _abi.FGMM_OPT_PHI, _abi.FGMM_PHI_LOGISTIC))
    assert not codec.ckbd_decode_fused(3, torch.float32, (16, 32, 48), 512, 512, h=hp)
    hp.close()
    h = codec.Handle()
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 16))
    assert not codec.ckbd_decode_fused(3, torch.float32, (16, 32, 48), 512, 512, h=h)
    lat = synth.make_ckbd_latent(16, 32, 48, 3, seed=999)
    dp = dev_params(lat.params)
    first, second = _oracle_streams(lat, (16, 32, 48), 512, 512)
    y = codec.ckbd_decode(dp, first, second, (16, 32, 48), 512, 512, h=h)
    np.testing.assert_array_equal(y.cpu().numpy(), lat.symbols)
    h.close()
    out = ctypes.c_int32(-1)
    hd = codec.handle()
    assert _abi.fgmm_ckbd_decode_plan(hd.ptr, 3, 0, 2, 4, 4, 48, 32, ctypes.byref(out)) == FGMM_ERR_INVALID_ARG
    assert _abi.fgmm_ckbd_decode_plan(hd.ptr, 5, 0, 2, 4, 4, 32, 32, ctypes.byref(out)) == FGMM_ERR_INVALID_ARG
    desc = codec.latent(dp)
    assert _abi.fgmm_ckbd_decode(hd.ptr, ctypes.byref(desc), 16, 32, 47, None, 0, None, 512, None, 0, None, 512,
                                 None, None) == FGMM_ERR_INVALID_ARG


@pytest.mark.parametrize("which", ["anchors", "non_anchors", "anchor_offsets"])
def test_fused_two_pass_decode_reports_corrupt_streams(which):
    """Damaged words of either pass, or an anchor segment shorter than its
    final states, end the fused launch with an error (no wait runs out: a
    pass-0 segment that cannot be decoded still counts its steps), and the
    handle decodes the intact streams afterwards."""
    codec = _codec()
    from paper_2509_18815_gb300._abi import FgmmError
    shape, Sa, Sn = (16, 32, 48), 512, 512
    lat = synth.make_ckbd_latent(*shape, 3, seed=1010)
    dp = dev_params(lat.params)
    first, second = _oracle_streams(lat, shape, Sa, Sn)
    assert codec.ckbd_decode_fused(3, torch.float32, shape, Sa, Sn)
    (wa, oa), (wn, on) = first, second
    wa2, oa2, wn2 = wa.clone(), oa.clone(), wn.clone()
    if which == "anchors":
        wa2[int(oa[3]) : int(oa[4]) - 64] ^= 0x5A5A
    elif which == "non_anchors":
        wn2[int(on[7]) : int(on[8]) - 64] ^= 0x3C3C
    else:
        oa2[1] = oa2[0] + 10
    with pytest.raises(FgmmError):
        codec.ckbd_decode(dp, (wa2, oa2), (wn2, on), shape, Sa, Sn)
    y = codec.ckbd_decode(dp, first, second, shape, Sa, Sn)
    np.testing.assert_array_equal(y.cpu().numpy(), lat.symbols)


def test_fused_two_pass_decode_from_cuda_graph():
    """The fused decode captured into a CUDA graph replays to the exact
    symbols, and again after the captured stream buffers were overwritten
    with a second latent's streams of the same lengths' bound."""
    codec = _codec()
    shape, Sa, Sn = (16, 32, 48), 512, 512
    lat = synth.make_ckbd_latent(*shape, 3, seed=1020)
    dp = dev_params(lat.params)
    first, second = _oracle_streams(lat, shape, Sa, Sn)
    gr = codec.CkbdGraphs(dp, shape, Sa, Sn)
    gr.capture_decode(first, second)
    for _ in range(2):
        gr.y.fill_(-3)
        np.testing.assert_array_equal(gr.decode().cpu().numpy(), lat.symbols)


def test_fused_two_pass_decode_wait_times_out_and_recovers():
    """With the anchor CTAs counting none of their steps (a test hook), the
    non-anchor waits for decoded anchors run out after about two seconds:
    the launch records FGMM_ERR_TIMEOUT, releases the other waits and
    returns, and the next decode on the same handle is exact."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    from paper_2509_18815_gb300._abi import FGMM_ERR_TIMEOUT, FgmmError
    shape, Sa, Sn = (5, 9, 13), 320, 320   # 20 segments: the fused launch, one step per pass
    lat = synth.make_ckbd_latent(*shape, 3, seed=1030)
    dp = dev_params(lat.params)
    first, second = _oracle_streams(lat, shape, Sa, Sn)
    h = codec.Handle()
    try:
        assert codec.ckbd_decode_fused(3, torch.float32, shape, Sa, Sn, h=h)
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_ARRIVALS, 1))
        t0 = time.monotonic()
        with pytest.raises(FgmmError) as e:
            codec.ckbd_decode(dp, first, second, shape, Sa, Sn, h=h)
        assert e.value.status == FGMM_ERR_TIMEOUT
        assert time.monotonic() - t0 < 30.0
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_ARRIVALS, 0))
        y = codec.ckbd_decode(dp, first, second, shape, Sa, Sn, h=h)
        np.testing.assert_array_equal(y.cpu().numpy(), lat.symbols)
        with pytest.raises(FgmmError):
            h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_TEST_SILENT_ARRIVALS, 2))
    finally:
        h.close()


@pytest.mark.parametrize("phi", ["as", "logistic", "polya"])
@pytest.mark.parametrize("K,bf16", [(1, False), (3, True), (4, False)])
def test_two_pass_encode_in_one_call_matches_separate_calls(K, bf16, phi):
    """fgmm_ckbd_encode (intervals of both passes in one kernel, both rANS
    encoders in one launch) writes the same bytes as the split, the context
    and two fgmm_encode calls, under each Phi approximation (integer output:
    equality); with A&S both equal the oracle's streams."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    shape, Sa, Sn = (6, 10, 14), 96, 128
    lat = synth.make_ckbd_latent(*shape, K, seed=1040 + K)
    lat.symbols[::37] = 70000   # escapes in both classes
    dp, dy = dev_params(lat.params, bf16), dev_i32(lat.symbols)
    h = codec.Handle()
    try:
        code = {"as": _abi.FGMM_PHI_AS, "logistic": _abi.FGMM_PHI_LOGISTIC, "polya": _abi.FGMM_PHI_POLYA}[phi]
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_PHI, code))
        (wa, oa), (wn, on) = codec.ckbd_encode(dp, dy, shape, Sa, Sn, h=h)
        (wa2, oa2), (wn2, on2) = codec.ckbd_encode_steps(dp, dy, shape, Sa, Sn, h=h)
    finally:
        h.close()
    np.testing.assert_array_equal(host_u16(wa), host_u16(wa2))
    np.testing.assert_array_equal(oa.cpu().numpy(), oa2.cpu().numpy())
    np.testing.assert_array_equal(host_u16(wn), host_u16(wn2))
    np.testing.assert_array_equal(on.cpu().numpy(), on2.cpu().numpy())
    if phi == "as":
        (wa_o, oa_o), (wn_o, on_o) = oracle.ckbd_encode(oracle_params(lat.params, bf16), lat.symbols, shape, Sa, Sn)
        np.testing.assert_array_equal(host_u16(wa), wa_o)
        np.testing.assert_array_equal(host_u16(wn), wn_o)


def test_two_pass_encode_errors():
    """Argument errors are refused before any launch; a words buffer too
    small for a pass is reported as FGMM_ERR_CAPACITY; invalid parameters as
    FGMM_ERR_BAD_PARAMS; the handle stays usable."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    from paper_2509_18815_gb300._abi import FGMM_ERR_BAD_PARAMS, FGMM_ERR_CAPACITY, FGMM_ERR_INVALID_ARG, FgmmError
    shape, Sa, Sn = (4, 8, 8), 64, 64
    lat = synth.make_ckbd_latent(*shape, 3, seed=1050)
    dp, dy = dev_params(lat.params), dev_i32(lat.symbols)
    h = codec.handle()
    desc = codec.latent(dp)
    buf = torch.zeros(4096, dtype=torch.int64, device="cuda")
    p = buf.data_ptr()
    assert _abi.fgmm_ckbd_encode(h.ptr, ctypes.byref(desc), 4, 8, 9, dy.data_ptr(), Sa, p, 16, p, p, Sn, p, 16, p, p,
                                 None) == FGMM_ERR_INVALID_ARG
    assert _abi.fgmm_ckbd_encode(h.ptr, ctypes.byref(desc), 4, 8, 8, dy.data_ptr(), 48, p, 16, p, p, Sn, p, 16, p, p,
                                 None) == FGMM_ERR_INVALID_ARG
    assert _abi.fgmm_ckbd_encode(h.ptr, ctypes.byref(desc), 4, 8, 8, dy.data_ptr(), Sa, p, 16, None, p, Sn, p, 16,
                                 p, p, None) == FGMM_ERR_INVALID_ARG
    words = torch.empty(8, dtype=torch.int16, device="cuda")
    offs = torch.empty(3, dtype=torch.int64, device="cuda")
    tot = torch.empty(2, dtype=torch.int64, device="cuda")
    h.check(_abi.fgmm_ckbd_encode(h.ptr, ctypes.byref(desc), 4, 8, 8, dy.data_ptr(), Sa, words.data_ptr(), 8,
                                  offs.data_ptr(), tot.data_ptr(), Sn, words.data_ptr(), 8, offs.data_ptr(),
                                  tot[1:].data_ptr(), None))
    with pytest.raises(FgmmError) as e:
        h.sync()
    assert e.value.status == FGMM_ERR_CAPACITY
    bad = lat.params.copy()
    bad[2, 0, 5] = -1.0   # a non-anchor's scale (position 5 of row 0: h + w odd)
    with pytest.raises(FgmmError) as e:
        codec.ckbd_encode(dev_params(bad), dy, shape, Sa, Sn)
    assert e.value.status == FGMM_ERR_BAD_PARAMS
    (wa, oa), (wn, on) = codec.ckbd_encode(dp, dy, shape, Sa, Sn)
    y = codec.ckbd_decode(dp, (wa, oa), (wn, on), shape, Sa, Sn)
    np.testing.assert_array_equal(y.cpu().numpy(), lat.symbols)


def test_two_pass_empty_latent():
    """An empty latent (C = 0): the one-call encode writes each pass's flush
    blocks, the same bytes as the separate calls, and the one-call decode
    returns no symbols without a launch error."""
    codec = _codec()
    shape, Sa, Sn = (0, 4, 4), 160, 160
    dp = torch.zeros((3, 3, 0), dtype=torch.float32, device="cuda")
    dy = torch.zeros(0, dtype=torch.int32, device="cuda")
    (wa, oa), (wn, on) = codec.ckbd_encode(dp, dy, shape, Sa, Sn)
    (wa2, oa2), (wn2, on2) = codec.ckbd_encode_steps(dp, dy, shape, Sa, Sn)
    assert wa.numel() == 64 * (Sa // 32) and wn.numel() == 64 * (Sn // 32)
    np.testing.assert_array_equal(host_u16(wa), host_u16(wa2))
    np.testing.assert_array_equal(host_u16(wn), host_u16(wn2))
    np.testing.assert_array_equal(oa.cpu().numpy(), oa2.cpu().numpy())
    np.testing.assert_array_equal(on.cpu().numpy(), on2.cpu().numpy())
    y = codec.ckbd_decode(dp, (wa, oa), (wn, on), shape, Sa, Sn)
    assert y.numel() == 0
