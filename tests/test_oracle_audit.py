"""Pins for the oracle's FP64 rate audit (exact mixture, Sec. II-A Eq. 2;
"no approximation" reference of Sec. V).

Independent checks: the K=1 mass equals a difference of scipy normal CDFs;
masses over all integers sum to the weight total; sampled symbols occur with
the audited probabilities (Monte Carlo); the mean ideal cost of sampled
symbols matches the model entropy; overhead on a synthetic latent meets the
0.1% budget and the CDF error stays within the Phi-hat bound.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from paper_2509_18815_gb300 import synth


def _one(w, mu, sg):
    K = len(w)
    p = np.empty((3, K, 1), np.float32)
    p[0, :, 0], p[1, :, 0], p[2, :, 0] = w, mu, sg
    return p


@pytest.mark.parametrize("mu,sg", [(0.0, 1.0), (0.3, 0.11), (-7.2, 3.5), (40.0, 16.0), (2.0, 0.05)])
def test_k1_mass_is_normal_difference(mu, sg):
    p = _one([1.0], [mu], [sg])
    sp = max(float(np.float32(sg)), float(np.float32(0.11)))
    m = float(np.float32(mu))
    for s in range(int(m) - 40, int(m) + 41):
        ref = ndtr((s + 0.5 - m) / sp) - ndtr((s - 0.5 - m) / sp)
        got = oracle.p64(p, 0, s)
        assert abs(got - ref) <= 1e-15 + 1e-12 * ref


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_masses_sum_to_weight_total(seed):
    lat = synth.make_latent(1, 1, 4, 3, seed=seed)
    for n in range(4):
        wsum = float(lat.params[0, :, n].astype(np.float64).sum())
        tot = sum(oracle.p64(lat.params, n, s) for s in range(-300, 301))
        assert abs(tot - wsum) <= 1e-12


def test_monte_carlo_frequencies():
    """Symbols drawn by rounding mixture samples occur with probability
    p64(s) (the interval [s-1/2, s+1/2) reading of Eq. 1)."""
    w, mu, sg = [0.5, 0.3, 0.2], [0.4, -3.0, 5.0], [0.8, 2.0, 0.3]
    p = _one(w, mu, sg)
    rng = np.random.default_rng(99)
    n = 2_000_000
    comp = rng.choice(3, n, p=np.array(w) / sum(w))
    y = np.rint(np.array(mu)[comp] + np.array(sg)[comp] * rng.standard_normal(n)).astype(int)
    vals, counts = np.unique(y, return_counts=True)
    for v, c in zip(vals.tolist(), counts.tolist()):
        pv = oracle.p64(p, 0, v)
        sd = math.sqrt(n * pv * (1 - pv)) + 1.0
        assert abs(c - n * pv) <= 5 * sd, (v, c, n * pv)


def test_ideal_bits_match_entropy():
    w, mu, sg = [0.6, 0.4], [0.0, 3.3], [1.5, 0.6]
    p = _one(w, mu, sg)
    probs = np.array([oracle.p64(p, 0, s) for s in range(-60, 61)])
    probs = probs[probs > 0]
    H = float(-(probs * np.log2(probs)).sum())
    rng = np.random.default_rng(5)
    n = 200_000
    comp = rng.choice(2, n, p=w)
    y = np.rint(np.array(mu)[comp] + np.array(sg)[comp] * rng.standard_normal(n)).astype(np.int32)
    pp = np.repeat(p, n, axis=2)
    ideal, coded, _, nesc = oracle.rate_audit(pp, y)
    assert nesc == 0
    assert abs(ideal / n - H) <= 0.01
    assert coded >= ideal


def test_overhead_budget_on_synthetic_latent():
    lat = synth.make_latent(192, 16, 16, 3, seed=1001)
    ideal, coded, maxerr, nesc = oracle.rate_audit(lat.params, lat.symbols)
    over = coded / ideal - 1.0
    assert 0.0 < over <= 1e-3, over
    assert maxerr <= 4e-7
    assert nesc == 0
