"""Checkerboard two-pass coding on the GPU against the oracle: the split of
parameters and symbols into anchors and non-anchors, the merge back, the
stand-in context (bit-exact, fp32 and bf16 hyperprior parameters), the two
streams of the two-pass encode (byte-identical) and the two-pass decode."""
import ctypes

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
