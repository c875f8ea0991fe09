"""Pins of the oracle's checkerboard two-pass coding (the context model of
the paper's codecs, Sec. IV-A): the anchor set (h + w even) and its listing
against numpy's mask indexing, split/merge as inverse maps, the fixed
stand-in context against closed forms and a float64 restatement, and the
two-pass round trip."""
import numpy as np
import pytest

import oracle
from paper_2509_18815_gb300 import synth

SHAPES = [(1, 1, 1), (2, 1, 5), (3, 4, 1), (2, 5, 7), (4, 6, 8), (1, 7, 7)]


def _mask(shape):
    C, H, W = shape
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.broadcast_to(((hh + ww) & 1) == 0, (C, H, W)).reshape(-1)


@pytest.mark.parametrize("shape", SHAPES)
def test_split_lists_anchors_in_raster_order(shape):
    C, H, W = shape
    lat = synth.make_latent(*shape, 2, seed=11)
    m = _mask(shape)
    na, nn = oracle.ckbd_counts(shape)
    assert na == int(m.sum()) == C * -(-(H * W) // 2) and nn == m.size - na
    pa, ya, pn, yn = oracle.ckbd_split(lat.params, lat.symbols, shape)
    np.testing.assert_array_equal(ya, lat.symbols[m])
    np.testing.assert_array_equal(yn, lat.symbols[~m])
    np.testing.assert_array_equal(pa, lat.params[:, :, m])
    np.testing.assert_array_equal(pn, lat.params[:, :, ~m])
    np.testing.assert_array_equal(oracle.ckbd_merge(ya, yn, shape), lat.symbols)
    only_a = oracle.ckbd_merge(ya, None, shape)
    np.testing.assert_array_equal(only_a[m], ya)
    assert np.all(only_a[~m] == 0)


def test_context_closed_forms():
    """Constant anchors a and constant parameters: a non-anchor with cnt
    in-bounds neighbours gets mu' = mu + cnt (a - mu) / 8, sigma' = 0.75
    sigma, weights kept (values chosen so every operation is exact)."""
    shape = (2, 5, 6)
    C, H, W = shape
    N = C * H * W
    params = np.empty((3, 2, N), np.float32)
    params[0] = [[0.25], [0.75]]
    params[1] = [[1.5], [-3.0]]
    params[2] = [[2.0], [0.5]]
    y = np.full(N, 7, np.int32)
    pn = oracle.ckbd_context(params, y, shape)
    m = _mask(shape)
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    cnt = ((hh > 0).astype(int) + (hh < H - 1) + (ww > 0) + (ww < W - 1))
    cnt = np.broadcast_to(cnt, shape).reshape(-1)[~m]
    for k, (wk, mu, sg) in enumerate([(0.25, 1.5, 2.0), (0.75, -3.0, 0.5)]):
        assert np.all(pn[0, k] == wk)
        np.testing.assert_array_equal(pn[1, k], (mu + cnt * (7 - mu) / 8.0).astype(np.float32))
        assert np.all(pn[2, k] == np.float32(sg * 0.75))


def test_context_reads_exactly_the_four_neighbours():
    shape = (2, 6, 7)
    C, H, W = shape
    N = C * H * W
    params = np.zeros((3, 1, N), np.float32)
    params[0] = 1.0
    params[2] = 1.0
    m = _mask(shape)
    base = oracle.ckbd_context(params, np.zeros(N, np.int32), shape)
    idx_non = np.flatnonzero(~m)
    for (c, h, w) in [(0, 0, 0), (1, 2, 4), (0, 5, 5), (1, 3, 1), (1, 0, 6)]:
        n = (c * H + h) * W + w
        assert m[n]
        y = np.zeros(N, np.int32)
        y[n] = 16
        pn = oracle.ckbd_context(params, y, shape)
        changed = set(idx_non[pn[1, 0] != base[1, 0]].tolist())
        want = {((c * H + h2) * W + w2) for h2, w2 in [(h - 1, w), (h + 1, w), (h, w - 1), (h, w + 1)]
                if 0 <= h2 < H and 0 <= w2 < W}
        assert changed == want
        assert np.all(pn[1, 0][np.isin(idx_non, list(want))] == 2.0)   # 16 / 8


def test_context_matches_float64_restatement():
    shape = (4, 9, 11)
    lat = synth.make_ckbd_latent(*shape, 3, seed=21)
    lat.symbols[::97] = 100000     # large neighbours (escapes) too
    pn = oracle.ckbd_context(lat.params, lat.symbols, shape).astype(np.float64)
    C, H, W = shape
    y = lat.symbols.astype(np.float64).reshape(C, H, W)
    pad = np.pad(y, ((0, 0), (1, 1), (1, 1)))
    ctx = (pad[:, :-2, 1:-1] + pad[:, 2:, 1:-1] + pad[:, 1:-1, :-2] + pad[:, 1:-1, 2:]).reshape(-1)
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    cnt = np.broadcast_to((hh > 0).astype(int) + (hh < H - 1) + (ww > 0) + (ww < W - 1), shape).reshape(-1)
    m = ~_mask(shape)
    mu = lat.params[1].astype(np.float64)
    want = mu + (ctx[None] - cnt[None] * mu) / 8.0
    np.testing.assert_allclose(pn[1], want[:, m], rtol=1e-6, atol=1e-5)
    np.testing.assert_array_equal(pn[2], (lat.params[2] * np.float32(0.75))[:, m])
    np.testing.assert_array_equal(pn[0], lat.params[0][:, m])


@pytest.mark.parametrize("shape,S", [((4, 16, 16), 32), ((3, 9, 13), 64), ((1, 1, 1), 32)])
def test_two_pass_round_trip(shape, S):
    lat = synth.make_ckbd_latent(*shape, 3, seed=31)
    first, second = oracle.ckbd_encode(lat.params, lat.symbols, shape, S, S)
    y, st = oracle.ckbd_decode(lat.params, first, second, shape, S, S)
    assert st == oracle.OK
    np.testing.assert_array_equal(y, lat.symbols)


def test_context_lowers_the_second_pass_rate():
    """On latents whose non-anchors follow their neighbours, the context's
    parameters code them in fewer bits than the hyperprior's."""
    shape = (8, 16, 16)
    lat = synth.make_ckbd_latent(*shape, 3, seed=41)
    _, _, pn_h, yn = oracle.ckbd_split(lat.params, lat.symbols, shape)
    pn = oracle.ckbd_context(lat.params, lat.symbols, shape)
    _, bits_h, _, _ = oracle.rate_audit(pn_h, yn)
    _, bits_c, _, _ = oracle.rate_audit(pn, yn)
    assert bits_c < 0.8 * bits_h
