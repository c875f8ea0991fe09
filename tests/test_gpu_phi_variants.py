"""The logistic and Polya approximations (Sec. III-B; Sec. V, Table II) on
the GPU equal the oracle's bit for bit: Phi-hat on every point of the 2^-22
grid in [-12, 12] and off the grid, the quantised intervals, the encoded
streams, exact decoding (on the lane decoder the plan then picks), and the
FP64 rate audit. Paths that take A&S only refuse the option."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2509_18815_gb300 import synth
from tests.gpu_util import dev_i32, dev_params, host_u16, host_u32, need_gpu, oracle_params

pytestmark = pytest.mark.gpu

ZMAX_I = 12 << 22
VARIANTS = [oracle.PHI_LOGISTIC, oracle.PHI_POLYA]


def _codec():
    need_gpu()
    from paper_2509_18815_gb300 import codec
    return codec


class _phi:
    """Handle option FGMM_OPT_PHI inside the block, A&S afterwards."""

    def __init__(self, v):
        self.v = v

    def __enter__(self):
        from paper_2509_18815_gb300 import _abi, codec
        self.h = codec.handle()
        self.h.check(_abi.fgmm_set_option(self.h.ptr, _abi.FGMM_OPT_PHI, self.v))
        return self

    def __exit__(self, *exc):
        from paper_2509_18815_gb300 import _abi
        self.h.check(_abi.fgmm_set_option(self.h.ptr, _abi.FGMM_OPT_PHI, _abi.FGMM_PHI_AS))


@pytest.mark.parametrize("v", VARIANTS)
def test_phi_grid_bit_exact_whole_grid(v):
    codec = _codec()
    chunk = 1 << 24
    z_of = lambda i, n: (np.arange(i, i + n, dtype=np.int64).astype(np.float32) * np.float32(2.0 ** -22))
    with _phi(v):
        i = -ZMAX_I
        while i <= ZMAX_I:
            n = min(chunk, ZMAX_I - i + 1)
            g = codec.phi_grid(i, n).cpu().numpy()
            c = oracle.phi_v(z_of(i, n), v)
            assert np.array_equal(g.view(np.uint32), c.view(np.uint32)), i
            assert np.all(np.diff(g) >= 0)
            i += n


@pytest.mark.parametrize("v", VARIANTS)
def test_phi_off_grid_bit_exact(v):
    codec = _codec()
    rng = np.random.default_rng(14 + v)
    z = np.concatenate([
        rng.uniform(-13, 13, 1_000_000), rng.normal(0, 1e-3, 100_000),
        np.array([0.0, -0.0, 12.0, -12.0, 1e30, -1e30, np.inf, -np.inf, 1e-45, -1e-45, 2 ** -23, -(2 ** -23)]),
    ]).astype(np.float32)
    with _phi(v):
        g = codec.phi(torch.from_numpy(z).cuda()).cpu().numpy()
    assert np.array_equal(g.view(np.uint32), oracle.phi_v(z, v).view(np.uint32))


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("K,bf16,esc,S", [(3, False, 0.01, 64), (4, True, 0.0, 256), (1, False, 0.02, 32)])
def test_intervals_streams_and_decode_match_oracle(v, K, bf16, esc, S):
    codec = _codec()
    lat = synth.make_latent(8, 16, 24, K, seed=700 + K + 10 * v, escape_stress=esc, sigma_max=32.0)
    dp, ds = dev_params(lat.params, bf16), dev_i32(lat.symbols)
    po = oracle_params(lat.params, bf16)
    with oracle.approximation(v):
        sf_o = oracle.freqs(po, lat.symbols)
        words_o, off_o = oracle.encode(po, lat.symbols, S)
    with _phi(v):
        assert codec.decode_plan(S)["kernel"] == "fgmm_dec_kernel"
        sf_g = host_u32(codec.freqs(dp, ds))
        words, off = codec.encode(dp, ds, S)
        out = codec.decode(dp, words, off, S).cpu().numpy()
    np.testing.assert_array_equal(sf_g, sf_o)
    np.testing.assert_array_equal(host_u16(words), words_o)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    np.testing.assert_array_equal(out, lat.symbols)
    # the A&S stream differs
    words_as, _ = codec.encode(dp, ds, S)
    assert not np.array_equal(host_u16(words_as), words_o)


@pytest.mark.parametrize("v", VARIANTS)
def test_rate_audit_matches_oracle(v):
    codec = _codec()
    lat = synth.make_latent(8, 32, 32, 3, seed=720 + v)
    with oracle.approximation(v):
        ideal_o, coded_o, err_o, nesc_o = oracle.rate_audit(lat.params, lat.symbols)
    with _phi(v):
        ideal, coded, err, nesc = codec.rate_audit(dev_params(lat.params), dev_i32(lat.symbols))
    assert abs(ideal - ideal_o) <= 1e-9 * ideal_o
    assert abs(coded - coded_o) <= 1e-9 * coded_o
    assert abs(err - err_o) <= 1e-9 and nesc == nesc_o
    assert coded / ideal - 1.0 < 0.005


def test_a_and_s_only_paths_refuse_the_option():
    codec = _codec()
    from paper_2509_18815_gb300._abi import FGMM_ERR_INVALID_ARG, FgmmError
    lat = synth.make_latent(2, 8, 8, 3, seed=730)
    dp, ds = dev_params(lat.params), dev_i32(lat.symbols)
    with _phi(oracle.PHI_LOGISTIC):
        for fn in (lambda: codec.table_build(dp),
                   lambda: codec.Batch([dp], [ds]),
                   lambda: codec.mlp_data(dp, ds, torch.rand(lat.N, device="cuda"))):
            with pytest.raises(FgmmError) as e:
                fn()
            assert e.value.status == FGMM_ERR_INVALID_ARG
