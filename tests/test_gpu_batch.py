"""Batched coding: many latents of uneven sizes in one persistent launch per
direction, replayed from CUDA graphs, with autotuned stream counts.

Each latent's slice of the batch stream must equal the single-latent coder's
stream for that latent and S (and the oracle's, for sampled latents), and
decoding the batch must return every symbol."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, host_u16, need_gpu, oracle_params

pytestmark = pytest.mark.gpu


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


def test_autotune_rule():
    codec = _codec()
    Ns = [49152, 294912, 1966080, 100, 0]
    S = codec.autotune(Ns, max_overhead=0.01, bits_per_symbol=3.5)
    t_min = int(np.ceil(32 / (0.01 * 3.5)))
    for n, s in zip(Ns, S):
        assert s % 32 == 0 and s >= 32
        # at least t_min symbols per stream (up to the rounding of S to 32)
        assert s <= max(32, -(-(-(-n // t_min)) // 32) * 32)
    # a looser budget never gives fewer streams
    S2 = codec.autotune(Ns, max_overhead=0.05, bits_per_symbol=3.5)
    assert all(b >= a for a, b in zip(S, S2))


@pytest.mark.parametrize("use_graph", [False, True])
def test_small_mixed_batch_matches_single_latent_coder(use_graph):
    codec = _codec()
    specs = [(16, 8, 8, 3, False, 0.0, 64), (4, 12, 20, 4, True, 0.01, 32), (1, 1, 1, 1, False, 0.0, 32),
             (32, 16, 16, 2, False, 0.002, 256), (8, 8, 12, 3, True, 0.0, 96)]
    lats = [synth.make_latent(C, H, W, K, seed=800 + i, escape_stress=e) for i, (C, H, W, K, _, e, _) in enumerate(specs)]
    params = [dev_params(l.params, s[4]) for l, s in zip(lats, specs)]
    syms = [dev_i32(l.symbols) for l in lats]
    S = [s[6] for s in specs]
    b = codec.Batch(params, syms, S=S)
    if use_graph:
        b.capture()
    for rep in range(2):
        b.encode()
        b.decode()
        for i, l in enumerate(lats):
            w, o = b.latent_stream(i)
            w1, o1 = codec.encode(params[i], syms[i], S[i])
            np.testing.assert_array_equal(o.cpu().numpy(), o1.cpu().numpy())
            np.testing.assert_array_equal(host_u16(w), host_u16(w1))
            np.testing.assert_array_equal(b.decoded[i].cpu().numpy(), l.symbols)
            if rep == 0:
                wc, oc = oracle.encode(oracle_params(l.params, specs[i][4]), l.symbols, S[i])
                np.testing.assert_array_equal(host_u16(w), wc)
    b.close()


def test_batch_of_64_uneven_latents_graph_autotuned():
    """64 latents, H and W uniform over multiples of 4 in [8, 128], C in
    {192, 320}, K = 3 (about 75M symbols): autotuned S, one persistent launch
    per direction replayed from CUDA graphs; every symbol decodes, the
    smallest latents match the oracle's streams, sampled latents match the
    single-latent coder."""
    codec = _codec()
    shapes = synth.batch_shapes(64, seed=1004)
    lats = [synth.make_latent(C, H, W, 3, seed=1004 + i) for i, (C, H, W) in enumerate(shapes)]
    params = [dev_params(l.params) for l in lats]
    syms = [dev_i32(l.symbols) for l in lats]
    total = sum(l.N for l in lats)
    assert 50e6 < total < 110e6
    b = codec.Batch(params, syms)   # S from the autotuner
    b.capture()
    b.encode()
    b.decode()
    for i, l in enumerate(lats):
        assert torch.equal(b.decoded[i], syms[i]), i
    order = np.argsort([l.N for l in lats])
    for i in order[:2]:
        w, o = b.latent_stream(int(i))
        wc, oc = oracle.encode(lats[i].params, lats[i].symbols, b.S[i])
        np.testing.assert_array_equal(o.cpu().numpy(), oc)
        np.testing.assert_array_equal(host_u16(w), wc)
    for i in [int(order[-1]), int(order[len(order) // 2])]:
        w, o = b.latent_stream(i)
        w1, o1 = codec.encode(params[i], syms[i], b.S[i])
        np.testing.assert_array_equal(host_u16(w), host_u16(w1))
    # replay: the same stream again
    first = b.words[: int(b.total.item())].clone()
    b.encode()
    assert torch.equal(first, b.words[: int(b.total.item())])
    b.close()


def test_batch_reports_corruption():
    codec = _codec()
    from paper_2509_18815_gb300._abi import FGMM_ERR_CORRUPT, FgmmError
    lats = [synth.make_latent(4, 8, 8, 3, seed=850 + i) for i in range(3)]
    b = codec.Batch([dev_params(l.params) for l in lats], [dev_i32(l.symbols) for l in lats], S=[32, 64, 32])
    b.encode()
    n = int(b.total.item())
    b.words[n - 64] ^= 0x0F0F
    with pytest.raises(FgmmError) as e:
        b.decode()
    assert e.value.status == FGMM_ERR_CORRUPT
    b.close()
