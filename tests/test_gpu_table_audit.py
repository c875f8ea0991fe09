"""Table-based comparison coder and FP64 rate audit on the GPU.

Table coder (Sec. II-C, Eqs. 4-5): its table equals the oracle's table built
by direct evaluation at every alphabet point (bit-exact), its stream is
byte-identical to the table-free coder's, and it decodes exactly.
Rate audit (Sec. V "no approximation"): the GPU's FP64 sums agree with the
oracle's FP64 sums (different erfc/log2 implementations: relative 1e-9),
coded bits and escape counts agree, and the overhead is within budget.
"""
import numpy as np
import pytest

import oracle
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, host_u16, need_gpu, oracle_params

pytestmark = pytest.mark.gpu


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


@pytest.mark.parametrize("K,bf16,esc", [(3, False, 0.0), (4, True, 0.01), (1, False, 0.02), (2, True, 0.0)])
def test_table_matches_oracle_table(K, bf16, esc):
    codec = _codec()
    lat = synth.make_latent(4, 16, 16, K, seed=600 + K, escape_stress=esc, sigma_max=64.0)
    p = lat.params.copy()
    p[2, :, ::9] = 0.11
    p[1, 0, 1::9] = 250.0
    p[1, 0, 2::9] = -1e4
    tab_g = host_u16(codec.table_build(dev_params(p, bf16)))
    tab_c = oracle.table(oracle_params(p, bf16))
    np.testing.assert_array_equal(tab_g, tab_c)


@pytest.mark.parametrize("S", [32, 1024])
def test_table_stream_identical_to_table_free(S):
    codec = _codec()
    lat = synth.make_latent(192, 16, 16, 3, seed=1001, escape_stress=0.001)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    w_free, o_free = codec.encode(dp, ds, S)
    w_tab, o_tab = codec.table_encode(dp, ds, S)
    np.testing.assert_array_equal(o_tab.cpu().numpy(), o_free.cpu().numpy())
    np.testing.assert_array_equal(host_u16(w_tab), host_u16(w_free))
    out = codec.table_decode(dp, w_free, o_free, S).cpu().numpy()
    np.testing.assert_array_equal(out, lat.symbols)


def test_table_coder_bench_latent():
    codec = _codec()
    lat = synth.make_latent(192, 32, 48, 3, seed=1002)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    w_free, o_free = codec.encode(dp, ds, 1024)
    w_tab, o_tab = codec.table_encode(dp, ds, 1024)
    np.testing.assert_array_equal(host_u16(w_tab), host_u16(w_free))
    np.testing.assert_array_equal(codec.table_decode(dp, w_tab, o_tab, 1024).cpu().numpy(), lat.symbols)


def test_table_decode_reports_corruption():
    codec = _codec()
    import torch
    from paper_2509_18815_gb300._abi import FGMM_ERR_CORRUPT, FgmmError
    lat = synth.make_latent(4, 16, 16, 3, seed=605)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    words, off = codec.encode(dp, ds, 64)
    junk = torch.randint(-32768, 32767, words.shape, dtype=torch.int16, device="cuda")
    with pytest.raises(FgmmError) as e:
        codec.table_decode(dp, junk, off, 64)
    assert e.value.status == FGMM_ERR_CORRUPT


@pytest.mark.parametrize("C,H,W,K,bf16,smax,esc", [
    (192, 16, 16, 3, False, 16.0, 0.0),
    (32, 32, 32, 4, True, 16.0, 0.0),
    (16, 16, 16, 3, False, 64.0, 0.005),
    (16, 16, 16, 1, False, 16.0, 0.0),
])
def test_rate_audit_matches_oracle(C, H, W, K, bf16, smax, esc):
    codec = _codec()
    lat = synth.make_latent(C, H, W, K, seed=700 + K, sigma_max=smax, escape_stress=esc)
    g = codec.rate_audit(dev_params(lat.params, bf16), dev_i32(lat.symbols))
    c = oracle.rate_audit(oracle_params(lat.params, bf16), lat.symbols)
    assert abs(g[0] - c[0]) <= 1e-9 * abs(c[0])
    assert abs(g[1] - c[1]) <= 1e-9 * abs(c[1])
    assert abs(g[2] - c[2]) <= 1e-12
    assert g[3] == c[3]
    if esc == 0.0:
        assert 0.0 < g[1] / g[0] - 1.0 <= 1e-3


def test_rate_audit_workload_320x64x96():
    """Full 1,966,080-symbol latents, K = 3 and 4, fp32 and bf16 parameters:
    overhead within 0.1% and CDF error within the Phi-hat bound."""
    codec = _codec()
    for K in (3, 4):
        lat = synth.make_latent(320, 64, 96, K, seed=1003)
        ds = dev_i32(lat.symbols)
        for bf16 in (False, True):
            ideal, coded, maxerr, nesc = codec.rate_audit(dev_params(lat.params, bf16), ds)
            assert 0.0 < coded / ideal - 1.0 <= 1e-3
            assert maxerr <= 4e-7
            assert nesc == 0
