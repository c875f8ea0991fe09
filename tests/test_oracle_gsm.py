"""Pins of the oracle's Gaussian single model with pre-built tables (the
scheme of Sec. II-C behind the paper's GSM anchor): the quantiser's
mean-shifted residual q is coded with N(0, sigma), sigma quantised to one of
64 levels spaced evenly in log between 0.11 and 256 (the smallest level at
or above it), and the coding itself is the K = 1 table-free coder on those
parameters."""
import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from paper_2509_18815_gb300 import synth


def test_levels_are_log_even_from_0_11_to_256():
    lv = oracle.gsm_levels().astype(np.float64)
    assert lv.shape == (64,)
    assert lv[0] == np.float32(0.11) and lv[-1] == 256.0
    assert np.all(np.diff(lv) > 0)
    ratio = (256.0 / 0.11) ** (1.0 / 63.0)
    np.testing.assert_allclose(lv[1:] / lv[:-1], ratio, rtol=2e-7)


def _sig_cases(lv, rng):
    return np.concatenate([np.exp(rng.uniform(np.log(0.01), np.log(1000.0), 20000)), lv, np.nextafter(lv, 0),
                           np.nextafter(lv, np.inf), [1e-30, 1e30, np.finfo(np.float32).max]]).astype(np.float32)


@pytest.mark.parametrize("levels", [None, [0.5], [0.05, 0.2, 3.0], np.geomspace(0.3, 40.0, 17)])
def test_level_is_the_smallest_at_or_above_the_scale(levels):
    lv = oracle.gsm_levels() if levels is None else np.asarray(levels, np.float32)
    sig = _sig_cases(lv, np.random.default_rng(1))
    po, li = oracle.gsm_params(sig, levels)
    # brute force: first level >= sigma among the first L - 1, else the last
    want = np.array([next((i for i in range(lv.size - 1) if s <= lv[i]), lv.size - 1) for s in sig[:3000]])
    np.testing.assert_array_equal(li[:3000], want)
    np.testing.assert_array_equal(li, np.minimum(np.searchsorted(lv, sig, side="left"), lv.size - 1))
    assert np.all(po[0] == 1.0) and np.all(po[1] == 0.0)
    np.testing.assert_array_equal(po[2, 0], lv[li])


def test_bad_scales_are_refused():
    for bad in (np.nan, 0.0, -1.0, np.inf, -np.inf):
        with pytest.raises(ValueError):
            oracle.gsm_params(np.array([1.0, 2.0, bad, 3.0], np.float32))


def test_level_tables_are_discretised_zero_mean_gaussians():
    """Each level's table is the quantised CDF of N(0, level): within the
    window its frequencies follow the exact discretised Gaussian (scipy's
    ndtr) to the quantisation step, symmetric about 0, every frequency >= 1,
    and symbols outside the window escape."""
    lv = oracle.gsm_levels()
    po, _ = oracle.gsm_params(lv)
    tab = oracle.table(po).astype(np.int64)
    lo, hi = oracle.window(po)
    assert np.all(lo == -hi)
    for i, s in enumerate(lv):
        row = tab[i, lo[i] + 255: hi[i] + 257]          # Q(lo) .. Q(hi + 1)
        freq = np.diff(row)
        assert row[0] == 0 and np.all(freq >= 1) and 65536 - row[-1] >= 1
        # Q(j) = (j - lo) + floor(T' F(j - 1/2)) for lo < j <= hi + 1: the
        # lower tail falls to the first symbol, the upper to the escape slot
        j = np.arange(lo[i] + 1, hi[i] + 2)
        sp = max(float(s), 0.11)
        T = 65536 - (hi[i] - lo[i] + 1) - 1
        d = row[1:] - (j - lo[i]) - T * ndtr((j - 0.5) / sp)
        assert np.all(d <= 1e-6 * T) and np.all(d > -1.0 - 1e-6 * T)
        assert np.abs(freq[1:-1] - freq[-2:0:-1]).max() <= 1     # mirror symmetry up to flooring


def test_gsm_round_trip_and_tables():
    lat = synth.make_gsm_latent(4, 16, 16, seed=401, escape_stress=0.02)
    po, li = oracle.gsm_params(lat.scales)
    for S in (32, 128):
        words, off = oracle.encode(po, lat.symbols, S)
        out, st = oracle.decode(po, words, off, S)
        assert st == oracle.OK
        np.testing.assert_array_equal(out, lat.symbols)
    # only 64 distinct rows occur: a symbol's row is its level's row
    lvp, _ = oracle.gsm_params(oracle.gsm_levels())
    np.testing.assert_array_equal(oracle.table(po), oracle.table(lvp)[li])


def test_gsm_costs_a_little_rate_against_the_exact_scale():
    """Rounding sigma up to the next of 64 levels (ratio 1.131) costs a
    little rate against coding with the exact sigma, never much."""
    lat = synth.make_gsm_latent(16, 16, 16, seed=402)
    exact = np.stack([np.ones_like(lat.scales), np.zeros_like(lat.scales), lat.scales])[:, None, :]
    ideal, coded, _, _ = oracle.rate_audit(exact, lat.symbols)
    po, _ = oracle.gsm_params(lat.scales)
    _, coded_gsm, _, _ = oracle.rate_audit(po, lat.symbols)
    assert coded / ideal - 1.0 < 1e-3
    assert 2 * (coded / ideal - 1.0) < coded_gsm / ideal - 1.0 < 0.02
