"""The byte container of one coded latent: a round trip of the oracle's
streams through it decodes to the same symbols, and every malformed
container is refused (never read past its end). A GPU test carries GPU
streams through it."""
import numpy as np
import pytest

import oracle
from paper_2509_18815_gb300 import container, synth


def _coded(seed=3, S=64):
    lat = synth.make_latent(4, 8, 16, 3, seed=seed, escape_stress=0.02)
    words, offsets = oracle.encode(lat.params, lat.symbols, S)
    return lat, words, offsets, S


def test_round_trip_decodes_the_same_symbols():
    lat, words, offsets, S = _coded()
    blob = container.pack(words, offsets, S, lat.N, 3)
    assert len(blob) == 36 + 4 * (S // 32) + 2 * words.size
    c = container.unpack(blob)
    assert (c["S"], c["N"], c["K"], c["coder"]) == (S, lat.N, 3, container.CODER_GMM)
    assert (c["phi"], c["dtype"], c["levels"]) == (container.PHI_AS, container.DTYPE_F32, 0)
    container.expect(c, container.PHI_AS, container.DTYPE_F32)
    np.testing.assert_array_equal(c["words"], words)
    np.testing.assert_array_equal(c["offsets"], offsets)
    out, st = oracle.decode(lat.params, c["words"], c["offsets"], c["S"])
    assert st == oracle.OK
    np.testing.assert_array_equal(out, lat.symbols)


def test_gsm_kind_and_empty_latent():
    words, offsets = oracle.encode(np.zeros((3, 1, 0), np.float32), np.zeros(0, np.int32), 32)
    lv = oracle.gsm_levels()
    c = container.unpack(container.pack(words, offsets, 32, 0, 1, coder=container.CODER_GSM, levels=lv))
    assert c["coder"] == container.CODER_GSM and c["N"] == 0 and c["words"].size == 64
    assert c["levels"] == 64 and c["levels_digest"] == container.levels_digest(lv)
    container.expect(c, container.PHI_AS, container.DTYPE_F32, levels=lv)
    other = lv.copy()
    other[7] = np.nextafter(other[7], np.float32(1e9))
    for bad in (None, lv[:63], other):
        with pytest.raises(ValueError):
            container.expect(c, container.PHI_AS, container.DTYPE_F32, levels=bad)
    with pytest.raises(ValueError):
        container.pack(words, offsets, 32, 0, 1, coder=container.CODER_GSM)          # GSM without levels
    with pytest.raises(ValueError):
        container.pack(words, offsets, 32, 0, 1, levels=lv)                          # levels on the mixture coder


def test_logistic_stream_records_its_approximation():
    """A stream coded with the logistic approximation round-trips through
    the container with that approximation recorded; a decoder set to A&S is
    refused before it decodes, and the recorded approximation decodes it."""
    lat = synth.make_latent(4, 8, 16, 3, seed=8)
    with oracle.approximation(oracle.PHI_LOGISTIC):
        words, offsets = oracle.encode(lat.params, lat.symbols, 64)
    blob = container.pack(words, offsets, 64, lat.N, 3, phi=container.PHI_LOGISTIC, dtype=container.DTYPE_BF16)
    c = container.unpack(blob)
    assert (c["phi"], c["dtype"]) == (container.PHI_LOGISTIC, container.DTYPE_BF16)
    with pytest.raises(ValueError):
        container.expect(c, container.PHI_AS, container.DTYPE_BF16)
    with pytest.raises(ValueError):
        container.expect(c, container.PHI_LOGISTIC, container.DTYPE_F32)
    container.expect(c, container.PHI_LOGISTIC, container.DTYPE_BF16)
    with oracle.approximation(c["phi"]):
        out, st = oracle.decode(lat.params, c["words"], c["offsets"], c["S"])
    assert st == oracle.OK
    np.testing.assert_array_equal(out, lat.symbols)
    for field, value in ((21, 3), (22, 2), (23, 5)):   # unknown phi, dtype; levels on the mixture coder
        b = bytearray(blob)
        b[field] = value
        with pytest.raises(ValueError):
            container.unpack(bytes(b))


def test_malformed_containers_are_refused():
    lat, words, offsets, S = _coded()
    blob = container.pack(words, offsets, S, lat.N, 3)
    bad = [blob[:10], blob[:40], blob[:-2], blob + b"\0\0", b"XGMM" + blob[4:],
           blob[:4] + b"\x01\x00" + blob[6:]]
    # a segment length below the 64 words of its final states
    b = bytearray(blob)
    b[36:40] = (10).to_bytes(4, "little")
    bad.append(bytes(b))
    # S not matching the segment count
    b = bytearray(blob)
    b[16:20] = (S + 32).to_bytes(4, "little")
    bad.append(bytes(b))
    for x in bad:
        with pytest.raises(ValueError):
            container.unpack(x)
    with pytest.raises(ValueError):
        container.pack(words, offsets[:-1], S, lat.N, 3)
    with pytest.raises(ValueError):
        container.pack(words, offsets, 48, lat.N, 3)
    with pytest.raises(ValueError):
        container.pack(words[:-5], offsets, S, lat.N, 3)


@pytest.mark.gpu
def test_gpu_streams_through_the_container():
    import torch
    from tests.gpu_util import need_gpu
    need_gpu()
    from paper_2509_18815_gb300 import codec
    lat = synth.make_latent(16, 16, 24, 3, seed=5)
    dp = torch.from_numpy(lat.params).cuda()
    ds = torch.from_numpy(lat.symbols).cuda()
    words, offsets = codec.encode(dp, ds, 256)
    c = container.unpack(container.pack(words, offsets, 256, lat.N, 3))
    w = torch.from_numpy(c["words"].view(np.int16).copy()).cuda()
    o = torch.from_numpy(c["offsets"]).cuda()
    assert torch.equal(codec.decode(dp, w, o, c["S"]), ds)
    # S chosen by the autotuner on encode and read from the offsets on decode
    words, offsets = codec.encode(dp, ds)
    assert (offsets.numel() - 1) * 32 == codec.autotune([lat.N])[0]
    assert torch.equal(codec.decode(dp, words, offsets), ds)
