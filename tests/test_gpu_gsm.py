"""The Gaussian single model coder with pre-built tables (Sec. II-C) on the
GPU against the oracle: the tables blob (levels, rows, decoder buckets), the
per-symbol intervals, byte-identical streams (equal to the oracle's K = 1
coder on (1, 0, level) and to the table-free GPU coder on the same
parameters), exact decoding, escapes, custom level sets, bf16 scales, the
Phi variants and the error paths."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, host_u16, host_u32, need_gpu

pytestmark = pytest.mark.gpu

ROWS_OFF, BKT_OFF, BLOB = 512, 66048, 198144


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


def _scales(sig: np.ndarray, bf16: bool = False):
    """Device scales and the fp32 values the GPU sees."""
    if bf16:
        bits = synth.to_bf16_bits(sig)
        return (torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16).contiguous(),
                synth.bf16_bits_to_f32(bits))
    return torch.from_numpy(np.ascontiguousarray(sig, np.float32)).cuda(), np.ascontiguousarray(sig, np.float32)


def _expected_blob(lv: np.ndarray) -> tuple:
    """Rows and buckets derived from the oracle's level tables."""
    lvp, _ = oracle.gsm_params(lv, lv)
    rows = oracle.table(lvp).astype(np.int64)                      # [L, 512]
    bk = np.zeros((lv.size, 258, 2), np.uint32)
    for l in range(lv.size):
        J = np.searchsorted(rows[l, :511], 256 * np.arange(257), side="right") - 1
        bk[l, :257, 0] = J | (rows[l, J] << 16)
        bk[l, :257, 1] = rows[l, J + 1]
    return rows.astype(np.uint16), bk


def _parse(blob: torch.Tensor, L: int):
    b = blob.cpu().numpy()
    assert b.size == BLOB
    hdr_L = int(b[:4].view(np.int32)[0])
    lv = b[16:16 + 4 * 64].view(np.float32)
    rows = b[ROWS_OFF:BKT_OFF].view(np.uint16).reshape(64, 512)[:L]
    bk = b[BKT_OFF:].view(np.uint32).reshape(64, 258, 2)[:L]
    return hdr_L, lv, rows, bk


def test_default_levels_match_oracle():
    codec = _codec()
    np.testing.assert_array_equal(codec.gsm_default_levels().view(np.uint32), oracle.gsm_levels().view(np.uint32))


@pytest.mark.parametrize("levels", [None, [0.5], [0.05, 0.2, 3.0, 700.0], np.geomspace(0.3, 40.0, 17)])
def test_tables_blob_matches_oracle(levels):
    codec = _codec()
    lv = oracle.gsm_levels() if levels is None else np.asarray(levels, np.float32)
    blob = codec.gsm_build(levels)
    L, lvb, rows, bk = _parse(blob, lv.size)
    assert L == lv.size
    np.testing.assert_array_equal(lvb[:L], lv)
    assert np.all(lvb[L:] == 0)
    rows_o, bk_o = _expected_blob(lv)
    np.testing.assert_array_equal(rows, rows_o)
    np.testing.assert_array_equal(bk, bk_o)


@pytest.mark.parametrize("S,bf16,esc,shape", [(32, False, 0.0, (4, 13, 17)), (64, True, 0.02, (8, 16, 16)),
                                                (1024, False, 0.01, (16, 32, 48)), (96, False, 0.0, (1, 1, 5))])
def test_streams_and_decode_match_oracle(S, bf16, esc, shape):
    codec = _codec()
    lat = synth.make_gsm_latent(*shape, seed=800 + S, escape_stress=esc, sigma_max=300.0)
    q = lat.symbols.copy()
    if q.size > 40:
        q[3], q[7], q[11] = np.iinfo(np.int32).min, np.iinfo(np.int32).max, -256
    ds, sig_o = _scales(lat.scales, bf16)
    dq = dev_i32(q)
    blob = codec.gsm_build()
    po, _ = oracle.gsm_params(sig_o)
    np.testing.assert_array_equal(host_u32(codec.gsm_freqs(ds, dq, blob)), oracle.freqs(po, q))
    words, off = codec.gsm_encode(ds, dq, S, blob)
    words_o, off_o = oracle.encode(po, q, S)
    np.testing.assert_array_equal(host_u16(words), words_o)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    # the table-free coder on the same K = 1 parameters writes the same stream
    w2, off2 = codec.encode(dev_params(po), dq, S)
    assert torch.equal(w2, words) and torch.equal(off2, off)
    out = codec.gsm_decode(ds, words, off, S, blob).cpu().numpy()
    np.testing.assert_array_equal(out, q)


@pytest.mark.parametrize("levels", [[0.5], [0.05, 0.2, 3.0, 700.0], np.geomspace(0.3, 40.0, 17)])
def test_custom_levels_round_trip(levels):
    codec = _codec()
    lv = np.asarray(levels, np.float32)
    lat = synth.make_gsm_latent(8, 16, 24, seed=820 + lv.size, escape_stress=0.01, sigma_max=100.0)
    ds, sig_o = _scales(lat.scales)
    dq = dev_i32(lat.symbols)
    blob = codec.gsm_build(lv)
    po, _ = oracle.gsm_params(sig_o, lv)
    words, off = codec.gsm_encode(ds, dq, 128, blob)
    words_o, off_o = oracle.encode(po, lat.symbols, 128)
    np.testing.assert_array_equal(host_u16(words), words_o)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    np.testing.assert_array_equal(codec.gsm_decode(ds, words, off, 128, blob).cpu().numpy(), lat.symbols)


@pytest.mark.parametrize("v", [oracle.PHI_LOGISTIC, oracle.PHI_POLYA])
def test_phi_variant_tables(v):
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    h = codec.handle()
    lat = synth.make_gsm_latent(8, 16, 16, seed=830 + v, escape_stress=0.01)
    ds, sig_o = _scales(lat.scales)
    dq = dev_i32(lat.symbols)
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_PHI, v))
    try:
        blob = codec.gsm_build()
    finally:
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_PHI, _abi.FGMM_PHI_AS))
    po, _ = oracle.gsm_params(sig_o)
    with oracle.approximation(v):
        words_o, off_o = oracle.encode(po, lat.symbols, 64)
    words, off = codec.gsm_encode(ds, dq, 64, blob)
    np.testing.assert_array_equal(host_u16(words), words_o)
    np.testing.assert_array_equal(codec.gsm_decode(ds, words, off, 64, blob).cpu().numpy(), lat.symbols)


def test_full_size_latent_round_trip_and_sampled_intervals():
    """The 320 x 64 x 96 latent the throughput numbers use, at the stream
    counts of the benchmark: exact round trip, intervals checked against the
    oracle on a sample."""
    codec = _codec()
    lat = synth.make_gsm_latent(320, 64, 96, seed=1003)
    ds, sig_o = _scales(lat.scales)
    dq = dev_i32(lat.symbols)
    blob = codec.gsm_build()
    idx = np.random.default_rng(5).choice(lat.N, 20000, replace=False)
    po, _ = oracle.gsm_params(sig_o[idx])
    np.testing.assert_array_equal(host_u32(codec.gsm_freqs(ds, dq, blob))[idx], oracle.freqs(po, lat.symbols[idx]))
    # 262144 streams: 8192 segments, more than one warp per segment slot of
    # the grid, so decoder warps loop over segments
    for S in (1024, 8192, 65536, 262144):
        words, off = codec.gsm_encode(ds, dq, S, blob)
        np.testing.assert_array_equal(codec.gsm_decode(ds, words, off, S, blob).cpu().numpy(), lat.symbols)


def test_empty_latent():
    codec = _codec()
    blob = codec.gsm_build()
    ds = torch.empty(0, dtype=torch.float32, device="cuda")
    dq = torch.empty(0, dtype=torch.int32, device="cuda")
    words, off = codec.gsm_encode(ds, dq, 64, blob)
    assert words.numel() == 128 and off.cpu().tolist() == [0, 64, 128]
    assert codec.gsm_decode(ds, words, off, 64, blob).numel() == 0


def test_errors_are_reported():
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    from paper_2509_18815_gb300._abi import (FGMM_ERR_BAD_PARAMS, FGMM_ERR_CORRUPT, FGMM_ERR_INVALID_ARG,
                                             FgmmError)
    h = codec.handle()
    for lv in ([], [1.0, 1.0], [2.0, 1.0], [0.0, 1.0], [float("nan")], list(np.geomspace(0.2, 9.0, 65))):
        with pytest.raises(FgmmError) as e:
            codec.gsm_build(lv)
        assert e.value.status == FGMM_ERR_INVALID_ARG
    blob = codec.gsm_build()
    # misaligned tables pointer
    lvd = codec.gsm_default_levels()
    st = _abi.fgmm_gsm_build(h.ptr, lvd.ctypes.data_as(ctypes.c_void_p), 64, ctypes.c_void_p(blob.data_ptr() + 8),
                             None)
    assert st == FGMM_ERR_INVALID_ARG
    lat = synth.make_gsm_latent(2, 16, 16, seed=840)
    dq = dev_i32(lat.symbols)
    for v in (0.0, -1.0, float("nan"), float("inf")):
        sig = lat.scales.copy()
        sig[37] = v
        with pytest.raises(FgmmError) as e:
            codec.gsm_encode(_scales(sig)[0], dq, 32, blob)
        assert e.value.status == FGMM_ERR_BAD_PARAMS
    ds = _scales(lat.scales)[0]
    words, off = codec.gsm_encode(ds, dq, 64, blob)
    bad = words.clone()
    bad[int(off[1].item()) - 64] ^= 0x1234
    with pytest.raises(FgmmError) as e:
        codec.gsm_decode(ds, bad, off, 64, blob)
    assert e.value.status == FGMM_ERR_CORRUPT
    with pytest.raises(FgmmError) as e:
        codec.gsm_decode(ds, words[:-5], off, 64, blob)
    assert e.value.status == FGMM_ERR_CORRUPT
    junk = torch.randint(-32768, 32767, words.shape, dtype=torch.int16, device="cuda")
    with pytest.raises(FgmmError) as e:
        codec.gsm_decode(ds, junk, off, 64, blob)
    assert e.value.status == FGMM_ERR_CORRUPT
    # the binding refuses a blob that is too small or on the host, and host symbols
    with pytest.raises(ValueError):
        codec.gsm_decode(ds, words, off, 64, blob[:1000])
    with pytest.raises(ValueError):
        codec.gsm_encode(ds, dq, 64, blob.cpu())
    with pytest.raises(ValueError):
        codec.gsm_encode(ds, dq.cpu(), 64, blob)
    # a blob that was never built decodes garbage but stays in bounds
    raw = torch.randint(0, 255, (BLOB,), dtype=torch.uint8, device="cuda")
    try:
        codec.gsm_decode(ds, words, off, 64, raw)
    except FgmmError as e:
        assert e.status in (FGMM_ERR_CORRUPT, FGMM_ERR_BAD_PARAMS)
    np.testing.assert_array_equal(codec.gsm_decode(ds, words, off, 64, blob).cpu().numpy(), lat.symbols)
