"""Pins for the oracle's FP32 exp and Phi-hat (A&S 26.2.17, Sec. III-B Eq. 8).

Checked against things the oracle does not compute itself: FP64 exp and
erfc from libm/scipy, the paper's stated A&S error bound (Sec. V), the
symmetry Phi(-z) = 1 - Phi(z), and monotonicity on the whole input grid.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

import oracle
from tests.golden import paper

GRID = 2.0 ** -22          # z is rounded to this grid before evaluation
ZMAX_I = 12 << 22          # grid index of z = 12


def _ulp32(x):
    x = np.abs(np.asarray(x, dtype=np.float32))
    return np.spacing(x).astype(np.float64)


def test_exp_against_fp64():
    rng = np.random.default_rng(1)
    a = np.concatenate([
        rng.uniform(-72.0, 0.0, 400_000).astype(np.float32),
        np.float32(-np.arange(0, 73)),                        # exact integers
        np.float32(-(np.arange(0, 104) + 0.5) * math.log(2)),  # range-reduction edges
        np.array([0.0, -1e-30, -1e-7, -0.34657359, -0.34657360], np.float32),
    ])
    e = oracle.exp(a)
    ref = np.exp(a.astype(np.float64))
    err_ulp = np.abs(e.astype(np.float64) - ref) / _ulp32(ref)
    assert err_ulp.max() <= 2.0, err_ulp.max()
    assert e[a == 0][0] == 1.0


def test_phi_monotone_on_whole_grid():
    """Exhaustive: every grid point in [-12, 12] (2 * 12 * 2^22 + 1 values)."""
    viol, _, _ = oracle.phi_grid_sweep(-ZMAX_I, ZMAX_I, 0)
    assert viol == 0


def _phi_tol():
    # paper's A&S bound + FP32 evaluation (4 ulp of values < 1) + half a grid
    # step at the steepest point of Phi (density 1/sqrt(2 pi))
    return paper.constants()["as_max_error"] + 4 * 2.0 ** -24 + 0.5 * GRID / math.sqrt(2 * math.pi)


def test_phi_error_bound_grid_sample():
    viol, maxerr, _ = oracle.phi_grid_sweep(-ZMAX_I, ZMAX_I, 37)
    assert viol == 0
    assert maxerr <= _phi_tol(), maxerr


def test_phi_error_bound_off_grid():
    rng = np.random.default_rng(2)
    z = np.concatenate([rng.uniform(-13, 13, 300_000), rng.normal(0, 1e-3, 50_000),
                        rng.uniform(-1, 1, 50_000)]).astype(np.float32)
    v = oracle.phi(z).astype(np.float64)
    ref = ndtr(z.astype(np.float64))
    assert np.abs(v - ref).max() <= _phi_tol()


def test_phi_symmetry_and_special_values():
    rng = np.random.default_rng(3)
    z = rng.uniform(-12, 12, 200_000).astype(np.float32)
    s = oracle.phi(z).astype(np.float64) + oracle.phi(-z).astype(np.float64)
    assert np.abs(s - 1.0).max() <= 2.0 ** -24
    assert oracle.phi(np.float32([0.0]))[0] == 0.5
    assert oracle.phi(np.float32([-0.0]))[0] == 0.5
    assert oracle.phi(np.float32([12.0, 50.0, np.inf]))[0] == 1.0
    lo = oracle.phi(np.float32([-12.0, -50.0, -np.inf]))
    assert np.all(lo > 0) and np.all(lo < 1e-30) and lo[0] == lo[1] == lo[2]


@pytest.mark.parametrize("z", [0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0])
def test_phi_textbook_points(z):
    # Phi at textbook points, FP64 reference via erfc
    ref = 0.5 * math.erfc(-z / math.sqrt(2))
    assert abs(float(oracle.phi(np.float32([z]))[0]) - ref) <= _phi_tol()
    assert abs(float(oracle.phi(np.float32([-z]))[0]) - (1 - ref)) <= _phi_tol()
