"""Pins for the oracle's interleaved rANS coder (Sec. II-B, Eq. 3; decode by
binary search, Sec. III-A).

Independent checks: decode(encode(x)) == x with the decoder ending in the
initial state; a single symbol from the initial state equals Eq. 3
evaluated with Python integers; the code length matches the information
content sum(-log2(freq / 2^16)); segments are independent (a segment of an
S=64 coding equals the S=32 coding of the sub-latent that it holds); damage
is reported as CORRUPT.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_18815_gb300 import synth

M = 1 << 16
L = 1 << 16


def _roundtrip(lat_params, syms, S):
    words, offsets = oracle.encode(lat_params, syms, S)
    assert offsets[0] == 0 and offsets[-1] == words.size
    assert np.all(np.diff(offsets) >= 64)
    out, st = oracle.decode(lat_params, words, offsets, S)
    assert st == oracle.OK
    np.testing.assert_array_equal(out, syms)
    return words, offsets


@pytest.mark.parametrize("N", [0, 1, 31, 32, 33, 63, 64, 65, 1000, 4097])
@pytest.mark.parametrize("S", [32, 64, 1024])
def test_roundtrip_sizes(N, S):
    lat = synth.make_latent(1, 1, max(N, 1), 3, seed=N * 7 + S)
    p = lat.params[:, :, :N]
    s = lat.symbols[:N]
    _roundtrip(np.ascontiguousarray(p), np.ascontiguousarray(s), S)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_roundtrip_escapes(K):
    lat = synth.make_latent(2, 16, 16, K, seed=40 + K, escape_stress=0.05)
    s = lat.symbols.copy()
    s[:4] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, -256, 256]
    sf = oracle.freqs(lat.params, s)
    assert ((sf & 0xFFFF) + (sf >> 16) == M).sum() > 20
    _roundtrip(lat.params, s, 64)


def test_roundtrip_extreme_params():
    lat = synth.make_latent(1, 32, 32, 3, seed=9)
    p = lat.params.copy()
    p[2, :, ::7] = 0.11          # scale floor
    p[2, 0, 1::7] = 1e6          # huge scale
    p[1, 1, 2::7] = 1e4          # mean far outside the alphabet
    p[0, :, 3::7] = 0.0          # all weights zero
    p[0, 0, 4::7] = 1.0          # weights summing above 1
    s = lat.symbols.copy()
    _roundtrip(p, s, 96)


def test_single_symbol_is_eq3():
    """N=1, S=32: lane 0 codes one symbol from x = 2^16 with no
    renormalisation when freq >= 2, so its flushed state is Eq. 3:
    C(s, x) = M floor(x / l_s) + b_s + (x mod l_s)."""
    lat = synth.make_latent(1, 1, 64, 3, seed=11)
    for n in range(64):
        p = np.ascontiguousarray(lat.params[:, :, n:n + 1])
        s = lat.symbols[n:n + 1].copy()
        sf = int(oracle.freqs(p, s)[0])
        b, l = sf & 0xFFFF, sf >> 16
        if l < 2:
            continue
        words, _ = oracle.encode(p, s, 32)
        assert words.size == 64
        x = int(words[0]) | (int(words[1]) << 16)
        assert x == M * (L // l) + b + (L % l)
        for lane in range(1, 32):   # idle lanes flush the initial state
            assert (int(words[2 * lane]) | (int(words[2 * lane + 1]) << 16)) == L


def test_code_length_matches_information():
    lat = synth.make_latent(8, 16, 16, 3, seed=21)
    S = 64
    words, offsets = _roundtrip(lat.params, lat.symbols, S)
    sf = oracle.freqs(lat.params, lat.symbols)
    info = float(np.sum(16.0 - np.log2((sf >> 16).astype(np.float64))))
    # each stream ends with a 32-bit state holding < 32 bits of information,
    # and starts from 2^16 (16 bits that are not payload)
    payload_bits = 16.0 * (words.size - 64 * (S // 32))
    flushed = 0.0
    for g in range(S // 32):
        blk = words[offsets[g + 1] - 64:offsets[g + 1]].astype(np.int64)
        xs = blk[0::2] | (blk[1::2] << 16)
        flushed += float(np.sum(np.log2(xs) - 16.0))
    total = payload_bits + flushed
    assert abs(total - info) <= 1e-3 * info + 2.0 * S, (total, info)


def test_segments_are_independent():
    lat = synth.make_latent(4, 16, 16, 3, seed=31)
    N = lat.N
    w64, o64 = oracle.encode(lat.params, lat.symbols, 64)
    for g in range(2):
        idx = np.array([n for n in range(N) if (n % 64) // 32 == g])
        sub_p = np.ascontiguousarray(lat.params[:, :, idx])
        sub_s = np.ascontiguousarray(lat.symbols[idx])
        w32, o32 = oracle.encode(sub_p, sub_s, 32)
        np.testing.assert_array_equal(w32, w64[o64[g]:o64[g + 1]])


def test_damage_is_reported():
    lat = synth.make_latent(2, 16, 16, 3, seed=51)
    words, offsets = oracle.encode(lat.params, lat.symbols, 32)
    bad = words.copy()
    bad[-64] ^= 0x5A5A                       # lane 0 final state
    _, st = oracle.decode(lat.params, bad, offsets, 32)
    assert st == oracle.CORRUPT
    _, st = oracle.decode(lat.params, words[:-10], np.array([0, words.size - 10]), 32)
    assert st == oracle.CORRUPT
    o2 = offsets.copy()
    o2[0] = 5                                # segment shorter than it should be
    _, st = oracle.decode(lat.params, words, o2, 32)
    assert st == oracle.CORRUPT


def test_rate_close_to_entropy_bound():
    lat = synth.make_latent(16, 16, 16, 3, seed=61)
    words, _ = oracle.encode(lat.params, lat.symbols, 32)
    ideal, coded, _, _ = oracle.rate_audit(lat.params, lat.symbols)
    bits = 16.0 * words.size
    assert bits >= coded - 1e-6 * coded
    assert bits <= coded + 32 * 32 + 0.01 * coded
    assert math.isfinite(ideal)


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_oracle_equals_single_thread(threads):
    """The oracle's segment-parallel entry points (used to time it on all
    host cores) give the single-thread words, offsets, symbols and status,
    also with escapes, a ragged last step and a damaged segment."""
    lat = synth.make_latent(8, 16, 17, 3, seed=91, escape_stress=0.01)
    for S in (32, 96, 256):
        w1, o1 = oracle.encode(lat.params, lat.symbols, S)
        wt, ot = oracle.encode(lat.params, lat.symbols, S, threads=threads)
        np.testing.assert_array_equal(w1, wt)
        np.testing.assert_array_equal(o1, ot)
        d1, s1 = oracle.decode(lat.params, w1, o1, S)
        dt, st = oracle.decode(lat.params, w1, o1, S, threads=threads)
        assert s1 == st == oracle.OK
        np.testing.assert_array_equal(d1, dt)
        bad = w1.copy()
        bad[int(o1[1]) - 70] ^= 0x5A5A
        _, sb1 = oracle.decode(lat.params, bad, o1, S)
        _, sbt = oracle.decode(lat.params, bad, o1, S, threads=threads)
        assert sb1 == sbt == oracle.CORRUPT
