"""Pins of the oracle's Gaussian single model with pre-built tables (the
scheme of Sec. II-C behind the paper's GSM anchor): 64 scale levels spaced
evenly in log between 0.11 and 256, each scale coded with the smallest level
at or above it, symbols shifted by the rounded mean, and the coding itself
the K = 1 table-free coder on those parameters."""
import numpy as np
import pytest

import oracle
from paper_2509_18815_gb300 import synth


def _gsm_latent(C, H, W, seed, smax=16.0):
    lat = synth.make_latent(C, H, W, 1, seed=seed, sigma_max=smax)
    return lat.params, lat.symbols


def test_levels_are_log_even_from_0_11_to_256():
    lv = oracle.gsm_levels().astype(np.float64)
    assert lv.shape == (64,)
    assert lv[0] == np.float32(0.11) and lv[-1] == 256.0
    assert np.all(np.diff(lv) > 0)
    ratio = (256.0 / 0.11) ** (1.0 / 63.0)
    np.testing.assert_allclose(lv[1:] / lv[:-1], ratio, rtol=2e-7)


def test_level_is_the_smallest_at_or_above_the_scale():
    lv = oracle.gsm_levels()
    rng = np.random.default_rng(1)
    sig = np.concatenate([np.exp(rng.uniform(np.log(0.01), np.log(1000.0), 20000)), lv, np.nextafter(lv, 0),
                          np.nextafter(lv, np.inf), [1e-30, 1e30]]).astype(np.float32)
    N = sig.size
    params = np.zeros((3, 1, N), np.float32)
    params[0] = 1.0
    params[2, 0] = sig
    _, _, li = oracle.gsm_transform(params, np.zeros(N, np.int32))
    want = np.minimum(np.searchsorted(lv, sig, side="left"), 63)
    np.testing.assert_array_equal(li, want)


def test_residual_shift_is_invertible_mod_2_32():
    rng = np.random.default_rng(2)
    N = 10000
    params = np.zeros((3, 1, N), np.float32)
    params[1, 0] = np.concatenate([rng.normal(0, 3, N - 6), [2.5, -2.5, 3.5, 1e9, -1e9, 0.49999997]])
    params[2, 0] = 1.0
    y = rng.integers(-2**31, 2**31, N, dtype=np.int64).astype(np.int32)
    y[:100] = np.iinfo(np.int32).min
    y[100:200] = np.iinfo(np.int32).max
    po, r, _ = oracle.gsm_transform(params, y)
    m = np.rint(np.clip(params[1, 0], -2.0**24, 2.0**24)).astype(np.int64)
    assert m[-6] == 2 and m[-5] == -2 and m[-4] == 4   # half to even
    np.testing.assert_array_equal(((r.astype(np.int64) + m) & 0xffffffff).astype(np.uint32).view(np.int32), y)
    assert np.all(po[0] == 1.0) and np.all(po[1] == 0.0)


def test_bad_parameters_are_refused():
    params = np.ones((3, 1, 4), np.float32)
    for bad in ((1, np.nan), (2, 0.0), (2, -1.0), (2, np.inf)):
        p = params.copy()
        p[bad[0], 0, 2] = bad[1]
        with pytest.raises(ValueError):
            oracle.gsm_transform(p, np.zeros(4, np.int32))


def test_gsm_round_trip_and_tables():
    params, y = _gsm_latent(4, 16, 16, seed=401)
    y[::37] = 10_000   # escapes
    po, r, li = oracle.gsm_transform(params, y)
    for S in (32, 128):
        words, off = oracle.encode(po, r, S)
        out, st = oracle.decode(po, words, off, S)
        assert st == oracle.OK
        np.testing.assert_array_equal(out, r)
    # only 64 distinct tables occur: the table of a symbol is the table of its level
    lv = oracle.gsm_levels()
    lvp = np.zeros((3, 1, 64), np.float32)
    lvp[0] = 1.0
    lvp[2, 0] = lv
    tabs = oracle.table(lvp)
    np.testing.assert_array_equal(oracle.table(po), tabs[li])


def test_gsm_costs_rate_against_the_exact_model():
    """Quantising sigma to 64 levels and dropping the mean's fractional part
    costs rate that the table-free K = 1 coder does not pay."""
    params, y = _gsm_latent(16, 16, 16, seed=402)
    ideal, coded, _, _ = oracle.rate_audit(params, y)
    po, r, _ = oracle.gsm_transform(params, y)
    _, coded_gsm, _, _ = oracle.rate_audit(po, r)
    assert coded / ideal - 1.0 < 1e-3
    assert coded_gsm / ideal - 1.0 > 5 * (coded / ideal - 1.0)
