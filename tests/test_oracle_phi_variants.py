"""Pins of the oracle's logistic and Polya approximations of Phi (Sec. III-B),
the comparison of Sec. V, Table II. Each is pinned to facts outside its own
code: its known maximum error against the exact normal CDF (scipy's ndtr),
exact values at 0, the mirror symmetry, monotonicity over the whole grid, and
the coding invariants (frequencies >= 1 summing to 2^16, exact round trips)
when the coder uses it."""
import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from paper_2509_18815_gb300 import synth

GRID = 12 * 2**22   # the clamp |z| <= 12 on the grid 2^-22


@pytest.mark.parametrize("v", [oracle.PHI_LOGISTIC, oracle.PHI_POLYA])
def test_monotone_on_the_whole_grid(v):
    viol, *_ = oracle.phi_v_grid_sweep(-GRID, GRID, 0, v)
    assert viol == 0


def test_logistic_error_bound_against_phi():
    # the 1.702 logistic is known to stay within 0.0095 of Phi; its largest
    # error is near |z| = 0.57
    _, _, _, err, zmax = oracle.phi_v_grid_sweep(-GRID, GRID, 97, oracle.PHI_LOGISTIC)
    assert 0.0094 < err < 0.0095
    assert 0.5 < abs(zmax) < 0.65
    z = np.linspace(-8, 8, 200001).astype(np.float32)
    assert np.abs(oracle.phi_v(z, oracle.PHI_LOGISTIC) - ndtr(z.astype(np.float64))).max() < 0.0095


def test_polya_error_bound_against_phi():
    # Polya's form with 2/pi stays within about 0.0032 of Phi (largest near
    # |z| = 1.65); the form printed without 2/pi would be off by 0.057
    _, _, _, err, zmax = oracle.phi_v_grid_sweep(-GRID, GRID, 97, oracle.PHI_POLYA)
    assert 0.0031 < err < 0.0032
    assert 1.55 < abs(zmax) < 1.75
    z = np.linspace(-8, 8, 200001).astype(np.float32)
    assert np.abs(oracle.phi_v(z, oracle.PHI_POLYA) - ndtr(z.astype(np.float64))).max() < 0.0032


@pytest.mark.parametrize("v", [oracle.PHI_LOGISTIC, oracle.PHI_POLYA])
def test_half_at_zero_and_mirror_symmetry(v):
    assert oracle.phi_v(np.array([0.0, -0.0], np.float32), v).tolist() == [0.5, 0.5]
    z = np.random.default_rng(5).normal(0, 3, 100000).astype(np.float32)
    s = oracle.phi_v(z, v).astype(np.float64) + oracle.phi_v(-z, v).astype(np.float64)
    assert np.abs(s - 1.0).max() <= 2**-24
    # saturation beyond the clamp
    hi = oracle.phi_v(np.array([12.0, 50.0, 1e30], np.float32), v)
    assert np.all(hi == hi[0]) and hi[0] == 1.0


@pytest.mark.parametrize("v", [oracle.PHI_AS, oracle.PHI_LOGISTIC, oracle.PHI_POLYA])
def test_coding_invariants_and_round_trip(v):
    lat = synth.make_latent(4, 8, 8, 3, seed=300 + v, escape_stress=0.02)
    with oracle.approximation(v):
        tab = oracle.table(lat.params).astype(np.int64)
        lo, hi = oracle.window(lat.params)
        for n in range(lat.N):
            row = tab[n, lo[n] + 255: hi[n] + 257]           # Q(lo) .. Q(hi+1)
            assert row[0] == 0
            assert np.all(np.diff(row) >= 1)                  # every symbol freq >= 1
            assert 65536 - row[-1] >= 1                       # escape slot freq >= 1
        sf = oracle.freqs(lat.params, lat.symbols)
        assert np.all((sf >> 16) >= 1)
        for S in (32, 64):
            words, off = oracle.encode(lat.params, lat.symbols, S)
            out, st = oracle.decode(lat.params, words, off, S)
            assert st == oracle.OK
            np.testing.assert_array_equal(out, lat.symbols)


def test_approximations_change_the_code_and_the_rate():
    """On Gaussian-mixture data the coded rate follows each approximation's
    accuracy: A&S (error < 7.5e-8) within 0.1% of the FP64 ideal, Polya
    (0.003) and logistic (0.0095) above it; the FP64 ideal itself does not
    depend on the approximation."""
    lat = synth.make_latent(16, 16, 16, 3, seed=310)
    res = {}
    for v in (oracle.PHI_AS, oracle.PHI_LOGISTIC, oracle.PHI_POLYA):
        with oracle.approximation(v):
            ideal, coded, maxerr, _ = oracle.rate_audit(lat.params, lat.symbols)
            res[v] = (ideal, coded / ideal - 1.0, maxerr, oracle.freqs(lat.params, lat.symbols))
    assert res[0][0] == res[1][0] == res[2][0]
    assert res[0][1] < 1e-3
    assert res[oracle.PHI_POLYA][1] > res[0][1] and res[oracle.PHI_LOGISTIC][1] > res[0][1]
    assert res[oracle.PHI_LOGISTIC][2] > 5e-3 > res[oracle.PHI_POLYA][2] > 1e-3 > res[0][2]
    assert not np.array_equal(res[0][3], res[1][3]) and not np.array_equal(res[0][3], res[2][3])
