"""Pins for the oracle's quantised mixture CDF (Sec. III-A with the window and
escape rule of this coder).

Independent checks: the frequencies of every value of the alphabet, each
computed on its own, sum to 2^16 with all >= 1; the table built by direct
evaluation at every alphabet point agrees with the on-the-fly intervals;
and each frequency matches 1 + T' * P(s), with P(s) the FP64 mixture mass of
[s - 1/2, s + 1/2) computed here with scipy's ndtr (Sec. II-A, Eq. 2, and the
interval form of Eq. 1 / Eq. 5).
"""
import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from paper_2509_18815_gb300 import synth

M = 1 << 16


def _mix_cases():
    """Adversarial and typical single-symbol mixtures: (w, mu, sigma)."""
    cases = [
        ([1.0], [0.0], [1.0]),
        ([1.0], [0.3], [0.11]),                 # scale at the floor
        ([1.0], [0.3], [0.01]),                 # below the floor
        ([0.5, 0.5], [-3.0, 4.0], [0.5, 2.0]),
        ([0.2, 0.3, 0.5], [-100.0, 0.0, 100.0], [1.0, 16.0, 3.0]),
        ([0.0, 1.0, 0.0], [1e4, 2.0, -1e4], [1.0, 1.0, 1.0]),   # zero weights far away
        ([1.0], [1000.0], [1.0]),               # mean outside the alphabet
        ([1.0], [-1e30], [1.0]),
        ([0.25, 0.25, 0.25, 0.25], [0.0, 0.1, 0.2, 0.3], [64.0, 1e3, 1e6, 0.2]),  # huge scales
        ([1.0], [254.6], [0.3]),                # window at the clamp
        ([0.7, 0.3], [0.0, 0.0], [0.11, 40.0]),
        ([0.6, 0.6], [0.0, 1.0], [1.0, 1.0]),   # weights summing above 1
        ([0.0, 0.0], [0.0, 1.0], [1.0, 1.0]),   # all weights 0
    ]
    return cases


def _all_values_latent(w, mu, sg, lo=-300, hi=300):
    vals = np.arange(lo, hi + 1, dtype=np.int32)
    N = vals.size
    K = len(w)
    p = np.empty((3, K, N), np.float32)
    for k in range(K):
        p[0, k, :] = w[k]
        p[1, k, :] = mu[k]
        p[2, k, :] = sg[k]
    return p, vals


@pytest.mark.parametrize("case", range(len(_mix_cases())))
def test_freqs_partition_the_range(case):
    w, mu, sg = _mix_cases()[case]
    p, vals = _all_values_latent(w, mu, sg)
    sf = oracle.freqs(p, vals)
    st = (sf & 0xFFFF).astype(np.int64)
    fr = (sf >> 16).astype(np.int64)
    lo, hi = oracle.window(p[:, :, :1])
    lo, hi = int(lo[0]), int(hi[0])
    assert -255 <= lo <= hi <= 255
    inw = (vals >= lo) & (vals <= hi)
    esc = ~inw
    assert np.all(fr >= 1)
    # every escape gets the same interval [Q(hi+1), 2^16)
    assert np.all(st[esc] + fr[esc] == M)
    assert len(set(st[esc].tolist())) == 1
    # in-window intervals tile [0, Q(hi+1)) in order, then the escape slot
    s_in, f_in = st[inw], fr[inw]
    assert s_in[0] == 0
    assert np.all(s_in[1:] == s_in[:-1] + f_in[:-1])
    assert s_in[-1] + f_in[-1] == st[esc][0]
    assert int(f_in.sum()) + int(fr[esc][0]) == M
    assert np.all(s_in + f_in < M)   # escape detection rule: start+freq == 2^16 only for escapes


@pytest.mark.parametrize("case", range(len(_mix_cases())))
def test_table_equals_on_the_fly(case):
    w, mu, sg = _mix_cases()[case]
    p, vals = _all_values_latent(w, mu, sg)
    tab = oracle.table(p[:, :, :1])[0].astype(np.int64)    # [512] over j in [-255, 256]
    sf = oracle.freqs(p, vals)
    st = (sf & 0xFFFF).astype(np.int64)
    fr = (sf >> 16).astype(np.int64)
    lo, hi = oracle.window(p[:, :, :1])
    lo, hi = int(lo[0]), int(hi[0])
    for i, s in enumerate(vals.tolist()):
        if lo <= s <= hi:
            assert st[i] == tab[s + 255]
            assert st[i] + fr[i] == tab[s + 256]
        else:
            assert st[i] == tab[hi + 1 + 255]
    assert np.all(np.diff(tab) >= 0)
    assert np.all(tab[: lo + 255 + 1] == 0)


def _fp64_mass(w, mu, sg, a, b):
    out = 0.0
    for wk, mk, sk in zip(w, mu, sg):
        sp = max(float(np.float32(sk)), float(np.float32(0.11)))
        out += float(np.float32(wk)) * (ndtr((b - float(np.float32(mk))) / sp) - ndtr((a - float(np.float32(mk))) / sp))
    return out


@pytest.mark.parametrize("case", range(len(_mix_cases())))
def test_freq_matches_fp64_mass(case):
    """freq(s) = 1 + floor(T' F(s+1/2)) - floor(T' F(s-1/2)) should be within
    1 (the two floors) + T' * 2 * (max CDF error) of 1 + T' P(s)."""
    w, mu, sg = _mix_cases()[case]
    p, vals = _all_values_latent(w, mu, sg)
    sf = oracle.freqs(p, vals)
    fr = (sf >> 16).astype(np.int64)
    lo, hi = oracle.window(p[:, :, :1])
    lo, hi = int(lo[0]), int(hi[0])
    Tp = M - (hi - lo + 1) - 1
    wsum = sum(float(np.float32(x)) for x in w)
    tol = 1.0 + Tp * 2 * 4e-7 * max(1.0, wsum)
    for i, s in enumerate(vals.tolist()):
        if not (lo <= s <= hi):
            continue
        a = -np.inf if s == lo else s - 0.5
        P = _fp64_mass(w, mu, sg, a, s + 0.5)
        if wsum > 1.0:
            continue   # min(F, 1) saturates: only the partition test applies
        assert abs(fr[i] - 1 - Tp * P) <= tol, (s, fr[i], 1 + Tp * P)


def test_freqs_on_synthetic_latent_match_mass():
    lat = synth.make_latent(4, 8, 8, 3, seed=77)
    sf = oracle.freqs(lat.params, lat.symbols)
    fr = (sf >> 16).astype(np.int64)
    lo, hi = oracle.window(lat.params)
    for n in range(lat.N):
        s = int(lat.symbols[n])
        w, mu, sg = lat.params[0, :, n], lat.params[1, :, n], lat.params[2, :, n]
        assert lo[n] <= s <= hi[n]
        Tp = M - (hi[n] - lo[n] + 1) - 1
        a = -np.inf if s == lo[n] else s - 0.5
        P = _fp64_mass(w, mu, sg, a, s + 0.5)
        assert abs(fr[n] - 1 - Tp * P) <= 1.0 + Tp * 8e-7


def test_window_rule():
    lat = synth.make_latent(2, 8, 8, 4, seed=5)
    lo, hi = oracle.window(lat.params)
    sp = np.maximum(lat.params[2], np.float32(0.11)).astype(np.float64)
    mu = lat.params[1].astype(np.float64)
    elo = np.clip(np.floor((mu - 8 * sp).min(axis=0)), -255, 255)
    ehi = np.clip(np.ceil((mu + 8 * sp).max(axis=0)), -255, 255)
    # fmaf in FP32 vs exact FP64: equal except when mu -/+ 8 sigma' sits within
    # one FP32 rounding of an integer
    assert np.mean(lo == elo) > 0.999 and np.mean(hi == ehi) > 0.999
    assert np.all(np.abs(lo - elo) <= 1) and np.all(np.abs(hi - ehi) <= 1)


def test_bad_params_rejected():
    p, vals = _all_values_latent([1.0], [0.0], [1.0], -2, 2)
    for (c, v) in [(0, -0.1), (0, np.nan), (1, np.inf), (2, 0.0), (2, -1.0), (2, np.nan)]:
        q = p.copy()
        q[c, 0, 2] = v
        with pytest.raises(ValueError):
            oracle.freqs(q, vals)
