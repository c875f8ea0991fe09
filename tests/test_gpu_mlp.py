"""Learned decode proposal on the GPU, checked against the FP64 oracle
(oracle/mlp.py) and against plain decoding.

- training triples: slots equal the oracle's interval draw bit for bit,
  features and targets match the FP64 features within FP32 rounding;
- loss and gradient of the GPU training kernels match the FP64 oracle;
- training is deterministic: a checkpoint/resume run equals a straight run;
- BF16 mma inference matches the oracle forward evaluated with the same
  BF16 rounding of weights and layer inputs;
- proposal-bracketed decoding returns exactly the encoded symbols for any
  weights (trained, random, zero, adversarial);
- a trained network makes decoding cheaper than plain binary search
  (fewer CDF evaluations per symbol, high hit rate) on large-scale latents.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, need_gpu

pytestmark = pytest.mark.gpu


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


def _bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return synth.bf16_bits_to_f32(synth.to_bf16_bits(a)).reshape(a.shape).astype(np.float64)


def _data(codec, lat, seed):
    rng = np.random.default_rng(seed)
    u = rng.random(lat.N).astype(np.float32)
    X, t, sl = codec.mlp_data(dev_params(lat.params), dev_i32(lat.symbols), torch.from_numpy(u).cuda(),
                              with_slots=True)
    return u, X, t, sl


def test_training_triples_match_oracle():
    codec = _codec()
    lat = synth.make_latent(8, 16, 16, 3, seed=900, sigma_max=64.0, escape_stress=0.002)
    u, X, t, sl = _data(codec, lat, 1)
    sf = oracle.freqs(lat.params, lat.symbols)
    st = (sf & 0xFFFF).astype(np.int64)
    fr = (sf >> 16).astype(np.int64)
    off = np.floor(u * fr.astype(np.float32)).astype(np.int64)
    slots = st + np.minimum(fr - 1, off)
    np.testing.assert_array_equal(sl.cpu().numpy(), slots)
    xo, m0, s0, to = mlp.features(lat.params, slots, lat.symbols)
    np.testing.assert_allclose(X.cpu().numpy(), xo, rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(t.cpu().numpy(), to, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("act", [mlp.ACT_PL, mlp.ACT_SIGMOID])
def test_loss_and_gradient_match_oracle(act):
    codec = _codec()
    lat = synth.make_latent(4, 16, 16, 3, seed=901, sigma_max=64.0)
    _, X, t, _ = _data(codec, lat, 2)
    rng = np.random.default_rng(3)
    theta = (mlp.init_params(5) + rng.normal(0, 0.05, mlp.N_PARAMS)).astype(np.float32)
    codec.set_mlp_act(act)
    try:
        loss, g = codec.mlp_loss_grad(X, t, torch.from_numpy(theta).cuda())
    finally:
        codec.set_mlp_act(mlp.ACT_PL)
    lo, go = mlp.loss_and_grad(theta.astype(np.float64), X.cpu().numpy().astype(np.float64),
                               t.cpu().numpy().astype(np.float64), act)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    g = g.cpu().numpy().astype(np.float64)
    scale = np.abs(go).max()
    assert np.abs(g - go).max() <= 1e-4 * scale
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    assert cos > 1 - 1e-8


def test_training_is_deterministic_and_resumes_exactly():
    codec = _codec()
    lat = synth.make_latent(16, 16, 16, 3, seed=902, sigma_max=64.0)
    _, X, t, _ = _data(codec, lat, 4)
    theta0 = mlp.init_params(6)
    a = codec.MlpTrainer(theta0)
    tr_a = a.train(X, t, steps=40, batch=512, lr=3e-3).cpu().numpy()
    b = codec.MlpTrainer(theta0)
    tr_b1 = b.train(X, t, steps=20, batch=512, lr=3e-3).cpu().numpy()
    ckpt = b.state_dict()
    c = codec.MlpTrainer(np.zeros(mlp.N_PARAMS))
    c.load_state_dict(ckpt)
    tr_c = c.train(X, t, steps=20, batch=512, lr=3e-3).cpu().numpy()
    np.testing.assert_array_equal(np.concatenate([tr_b1, tr_c]), tr_a)
    assert torch.equal(c.theta, a.theta)
    assert tr_a[-1] < tr_a[0]


@pytest.mark.parametrize("act", [mlp.ACT_PL, mlp.ACT_SIGMOID])
def test_bf16_inference_matches_oracle_with_bf16_rounding(act):
    codec = _codec()
    lat = synth.make_latent(4, 8, 8, 3, seed=903, sigma_max=64.0)
    _, X, _, _ = _data(codec, lat, 5)
    rng = np.random.default_rng(7)
    theta = (mlp.init_params(8) + rng.normal(0, 0.1, mlp.N_PARAMS)).astype(np.float32)
    codec.set_mlp_act(act)
    try:
        y = codec.mlp_forward(X, codec.mlp_pack(torch.from_numpy(theta).cuda())).cpu().numpy()
    finally:
        codec.set_mlp_act(mlp.ACT_PL)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(theta.astype(np.float64))
    x = _bf16(X.cpu().numpy())
    h1 = _bf16(mlp.act(x @ _bf16(W1) + b1, act))
    h2 = mlp.act(h1 @ _bf16(W2) + b2, act)
    yo = h2 @ w3 + b3
    np.testing.assert_allclose(y, yo, rtol=2e-3, atol=2e-3 * (1 + np.abs(yo).max()))


@pytest.mark.parametrize("kind", ["random", "zero", "huge_bias", "trained_short"])
def test_proposal_decode_is_exact_for_any_weights(kind):
    codec = _codec()
    lat = synth.make_latent(8, 32, 32, 3, seed=904, sigma_max=64.0, escape_stress=0.003)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    if kind == "random":
        theta = np.random.default_rng(9).normal(0, 1, mlp.N_PARAMS)
    elif kind == "zero":
        theta = np.zeros(mlp.N_PARAMS)
    elif kind == "huge_bias":
        theta = np.zeros(mlp.N_PARAMS)
        theta[-1] = 1e6     # every guess far above the window
    else:
        _, X, t, _ = _data(codec, lat, 6)
        tr = codec.MlpTrainer(mlp.init_params(10))
        tr.train(X, t, steps=50, batch=1024, lr=3e-3)
        theta = tr.theta.cpu().numpy()
    P = codec.mlp_pack(torch.as_tensor(theta, dtype=torch.float32).cuda())
    for S in (32, 256):
        words, off = codec.encode(dp, ds, S)
        out = codec.decode_proposal(dp, words, off, S, P).cpu().numpy()
        np.testing.assert_array_equal(out, lat.symbols)


def test_analytic_proposal_decodes_exactly_and_saves_evaluations():
    """The analytic proposal (packed network absent: logistic inverse on the
    dominant component) decodes exactly, also with escapes, and needs fewer
    CDF evaluations per symbol than plain binary search on latents with
    scales up to 64."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    lat = synth.make_latent(16, 32, 32, 3, seed=906, sigma_max=64.0, escape_stress=0.003)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    for S in (32, 256):
        words, off = codec.encode(dp, ds, S)
        np.testing.assert_array_equal(codec.decode_proposal(dp, words, off, S, None).cpu().numpy(), lat.symbols)
    h = codec.handle()
    codec.stats_enable(True)
    codec.stats_read(with_hits=True)
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 1))
    try:
        codec.decode(dp, words, off, 256)
    finally:
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 0))
    ev_plain, n_plain, _ = codec.stats_read(with_hits=True)
    codec.decode_proposal(dp, words, off, 256, None)
    ev_an, n_an, hits = codec.stats_read(with_hits=True)
    codec.stats_enable(False)
    assert n_plain == n_an == lat.N
    print(f"plain {ev_plain / n_plain:.3f} evals/sym; analytic {ev_an / n_an:.3f} evals/sym, "
          f"hit rate {hits / n_an:.3f}")
    assert ev_an < ev_plain


def test_proposal_reports_corruption():
    codec = _codec()
    from paper_2509_18815_gb300._abi import FGMM_ERR_CORRUPT, FgmmError
    lat = synth.make_latent(4, 16, 16, 3, seed=905)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    words, off = codec.encode(dp, ds, 64)
    P = codec.mlp_pack(torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda"))
    junk = torch.randint(-32768, 32767, words.shape, dtype=torch.int16, device="cuda")
    with pytest.raises(FgmmError) as e:
        codec.decode_proposal(dp, junk, off, 64, P)
    assert e.value.status == FGMM_ERR_CORRUPT


def test_trained_proposal_beats_plain_binary_search():
    """Train on 2^21 triples drawn from large-scale (sigma up to 64) latents,
    then decode a held-out 320 x 64 x 96 latent of the same distribution:
    symbols exact, fewer CDF evaluations per symbol than binary search."""
    codec = _codec()
    from paper_2509_18815_gb300 import _abi
    train = synth.make_latent(32, 256, 256, 3, seed=1005, sigma_max=64.0)
    _, X, t, _ = _data(codec, train, 11)
    tr = codec.MlpTrainer(mlp.init_params(12))
    for steps, lr in [(2000, 3e-3), (1000, 1e-3), (1000, 3e-4)]:
        tr.train(X, t, steps=steps, batch=8192, lr=lr)
    P = tr.packed()
    test = synth.make_latent(320, 64, 96, 3, seed=1105, sigma_max=64.0)
    dp, ds = dev_params(test.params), dev_i32(test.symbols)
    S = 2048
    words, off = codec.encode(dp, ds, S)
    h = codec.handle()
    codec.stats_enable(True)
    codec.stats_read(with_hits=True)
    h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 1))
    try:
        out_plain = codec.decode(dp, words, off, S).cpu().numpy()
    finally:
        h.check(_abi.fgmm_set_option(h.ptr, _abi.FGMM_OPT_DECODE_LANES, 0))
    ev_plain, n_plain, _ = codec.stats_read(with_hits=True)
    out_prop = codec.decode_proposal(dp, words, off, S, P).cpu().numpy()
    ev_prop, n_prop, hits = codec.stats_read(with_hits=True)
    codec.stats_enable(False)
    np.testing.assert_array_equal(out_plain, test.symbols)
    np.testing.assert_array_equal(out_prop, test.symbols)
    assert n_plain == n_prop == test.N
    print(f"plain {ev_plain / n_plain:.3f} evals/sym; proposal {ev_prop / n_prop:.3f} evals/sym, "
          f"hit rate {hits / n_prop:.3f}")
    assert ev_prop / n_prop < 0.6 * (ev_plain / n_plain)
    assert hits / n_prop > 0.3


@pytest.mark.parametrize("act", [mlp.ACT_PL, mlp.ACT_SIGMOID])
def test_batched_proposal_decode_is_exact(act):
    """One persistent launch decodes a batch of uneven K = 3 latents (scales
    up to 64, escapes) with the network proposal (trained briefly, either
    activation) and with the analytic proposal: every symbol equals the
    encoded one, and the plain batch decode of the same plan agrees."""
    codec = _codec()
    shapes = [(8, 12, 20), (4, 32, 32), (16, 8, 8), (2, 4, 4)]
    lats = [synth.make_latent(C, H, W, 3, seed=920 + i, sigma_max=64.0, escape_stress=0.002)
            for i, (C, H, W) in enumerate(shapes)]
    params = [dev_params(l.params) for l in lats]
    syms = [dev_i32(l.symbols) for l in lats]
    codec.set_mlp_act(act)
    try:
        _, X, t, _ = _data(codec, lats[1], 12)
        tr = codec.MlpTrainer(mlp.init_params(13))
        tr.train(X, t, steps=60, batch=1024, lr=3e-3)
        P = tr.packed()
        b = codec.Batch(params, syms, S=[64, 96, 32, 32])
        b.encode()
        for packed in (P, None):
            for d in b.decoded:
                d.fill_(12345)
            b.decode_proposal(packed)
            for i in range(len(lats)):
                assert torch.equal(b.decoded[i], syms[i]), (act, packed is None, i)
        for d in b.decoded:
            d.fill_(-7)
        b.decode()
        assert all(torch.equal(b.decoded[i], syms[i]) for i in range(len(lats)))
    finally:
        codec.set_mlp_act(mlp.ACT_PL)
