"""Seeded synthetic latents for the Gaussian-mixture coder.

This module only draws inputs. It holds none of the coder's arithmetic (no
CDF, no quantisation, no rANS), so both the CUDA path and the CPU oracle can
be fed from it without sharing any of the method.

A latent of shape C x H x W has N = C*H*W symbols, indexed channel-major
(n = c*H*W + h*W + w). Its mixture parameters are planar, shape [3, K, N]:
row 0 the weights w_k, row 1 the means mu_k, row 2 the scales sigma_k, the
layout of the per-symbol parameters theta = (w, mu, sigma) of a GMM entropy
model (Sec. II-A, Eq. 2).

Distributions (the synthetic stand-in for a learned codec's hyperprior,
which needs trained weights and images that are not available):
  logits ~ N(0, 1) -> softmax over K -> w
  mu     ~ N(0, 3)
  sigma  = exp(U[ln 0.11, ln sigma_max])   (0.11 is the lowest scale level of
           the CompressAI scale table the paper describes in Sec. II-B)
  symbol = round-half-even(mu_c + sigma_c * N(0, 1)), c ~ Categorical(w)
No clipping: values outside the coder's window are legal (escape path).

The Gaussian single model's coder receives the quantiser's mean-shifted
residual and the scale only (Sec. II-C); its inputs (make_gsm_latent) are
  sigma  = exp(U[ln 0.11, ln sigma_max])
  q      = round-half-even(sigma * N(0, 1))   (= round(y - mu), y ~ N(mu, sigma))

Checkerboard latents (make_ckbd_latent) have the hyperprior parameters
above for every position; anchors (h + w even) are drawn from them, and
each non-anchor from the mixture whose means move toward its 4-neighbour
anchors and whose scales narrow, the way a context model's output does:
  mu'_k = mu_k + (sum of neighbours - cnt mu_k) / 8,  sigma'_k = 0.75 sigma_k
(computed here in float64, only to draw the symbols).
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

SIGMA_MIN = 0.11


@dataclass
class Latent:
    params: np.ndarray      # float32 [3, K, N] (w, mu, sigma)
    symbols: np.ndarray     # int32 [N]
    shape: tuple            # (C, H, W)
    seed: int

    @property
    def N(self) -> int:
        return int(self.symbols.shape[0])

    @property
    def K(self) -> int:
        return int(self.params.shape[1])


def make_latent(C: int, H: int, W: int, K: int, seed: int,
                sigma_max: float = 16.0, escape_stress: float = 0.0) -> Latent:
    """Draw one latent with the distributions listed in the module docstring.

    escape_stress > 0 replaces that fraction of symbols by values far outside
    any window (and outside [-255, 255]), to exercise the escape path.
    """
    rng = np.random.default_rng(seed)
    N = C * H * W
    logits = rng.standard_normal((K, N))
    logits -= logits.max(axis=0, keepdims=True)
    e = np.exp(logits)
    w = (e / e.sum(axis=0, keepdims=True)).astype(np.float32)
    mu = rng.normal(0.0, 3.0, (K, N)).astype(np.float32)
    sigma = np.exp(rng.uniform(math.log(SIGMA_MIN), math.log(sigma_max), (K, N))).astype(np.float32)
    # component choice by inverse-CDF sampling of the categorical weights
    u = rng.random(N)
    cw = np.cumsum(w.astype(np.float64), axis=0)
    comp = (u[None, :] > cw).sum(axis=0)
    comp = np.minimum(comp, K - 1)
    idx = np.arange(N)
    y = mu[comp, idx].astype(np.float64) + sigma[comp, idx].astype(np.float64) * rng.standard_normal(N)
    y = np.clip(np.rint(y), -2.0**31, 2.0**31 - 1)
    sym = y.astype(np.int64).astype(np.int32)
    if escape_stress > 0.0 and N > 0:
        m = rng.random(N) < escape_stress
        nsel = int(m.sum())
        big = rng.integers(-2**31, 2**31 - 1, nsel, dtype=np.int64, endpoint=True)
        near = rng.integers(256, 4000, nsel) * rng.choice([-1, 1], nsel)
        pick = rng.random(nsel) < 0.5
        sym[m] = np.where(pick, big, near).astype(np.int32)
    params = np.stack([w, mu, sigma], axis=0)
    return Latent(params=np.ascontiguousarray(params), symbols=sym, shape=(C, H, W), seed=seed)


@dataclass
class GsmLatent:
    scales: np.ndarray      # float32 [N]
    symbols: np.ndarray     # int32 [N], the mean-shifted residuals q
    shape: tuple
    seed: int

    @property
    def N(self) -> int:
        return int(self.symbols.shape[0])


def make_gsm_latent(C: int, H: int, W: int, seed: int, sigma_max: float = 16.0,
                    escape_stress: float = 0.0) -> GsmLatent:
    """Inputs of the Gaussian single model's coder: scales and residuals
    (module docstring). escape_stress as in make_latent."""
    rng = np.random.default_rng(seed)
    N = C * H * W
    sigma = np.exp(rng.uniform(math.log(SIGMA_MIN), math.log(sigma_max), N)).astype(np.float32)
    q = np.rint(sigma.astype(np.float64) * rng.standard_normal(N)).astype(np.int64).astype(np.int32)
    if escape_stress > 0.0 and N > 0:
        m = rng.random(N) < escape_stress
        nsel = int(m.sum())
        big = rng.integers(-2**31, 2**31 - 1, nsel, dtype=np.int64, endpoint=True)
        near = rng.integers(256, 4000, nsel) * rng.choice([-1, 1], nsel)
        pick = rng.random(nsel) < 0.5
        q[m] = np.where(pick, big, near).astype(np.int32)
    return GsmLatent(scales=sigma, symbols=q, shape=(C, H, W), seed=seed)


def _draw_mixture(rng, w, mu, sigma):
    K, N = w.shape
    u = rng.random(N)
    cw = np.cumsum(w.astype(np.float64), axis=0)
    comp = np.minimum((u[None, :] > cw).sum(axis=0), K - 1)
    idx = np.arange(N)
    y = mu[comp, idx].astype(np.float64) + sigma[comp, idx].astype(np.float64) * rng.standard_normal(N)
    return np.clip(np.rint(y), -2.0**31, 2.0**31 - 1).astype(np.int64).astype(np.int32)


def make_ckbd_latent(C: int, H: int, W: int, K: int, seed: int, sigma_max: float = 16.0) -> Latent:
    """Hyperprior parameters for all C*H*W positions and symbols whose
    non-anchors depend on their anchor neighbours (module docstring)."""
    lat = make_latent(C, H, W, K, seed, sigma_max)
    rng = np.random.default_rng(seed + 7919)
    w, mu, sigma = (lat.params[i].astype(np.float64) for i in range(3))
    y = lat.symbols.astype(np.int64).reshape(C, H, W)
    hh, ww = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    non = ((hh + ww) & 1) == 1
    pad = np.pad(y, ((0, 0), (1, 1), (1, 1)))
    ctx = pad[:, :-2, 1:-1] + pad[:, 2:, 1:-1] + pad[:, 1:-1, :-2] + pad[:, 1:-1, 2:]
    cnt = ((hh > 0).astype(np.int64) + (hh < H - 1) + (ww > 0) + (ww < W - 1))[None].repeat(C, 0)
    sel = np.broadcast_to(non, (C, H, W)).reshape(-1)
    mu2 = mu + (ctx.reshape(-1)[None, :] - cnt.reshape(-1)[None, :] * mu) / 8.0
    yn = _draw_mixture(rng, w[:, sel], mu2[:, sel], 0.75 * sigma[:, sel])
    sym = lat.symbols.copy()
    sym[sel] = yn
    return Latent(params=lat.params, symbols=sym, shape=(C, H, W), seed=seed)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """fp32 -> bf16 bit patterns, round to nearest even (inputs are finite)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    """bf16 bit patterns -> the fp32 values they denote (exact)."""
    return (b.astype(np.uint32) << 16).view(np.float32)


def batch_shapes(n_latents: int, seed: int):
    """Shapes for the uneven batch: H, W uniform over multiples of 4 in
    [8, 128], C uniform over {192, 320}."""
    rng = np.random.default_rng(seed)
    Hs = rng.integers(2, 33, n_latents) * 4
    Ws = rng.integers(2, 33, n_latents) * 4
    Cs = rng.choice([192, 320], n_latents)
    return [(int(c), int(h), int(w)) for c, h, w in zip(Cs, Hs, Ws)]


# Workloads with their sizes (seed = 1000 + workload number).
WORKLOADS = {
    "latent_192x16x16_k3": dict(C=192, H=16, W=16, K=3, S=32, seed=1001),
    "latent_192x32x48_k3": dict(C=192, H=32, W=48, K=3, S=1024, seed=1002),
    "latent_320x64x96_k3": dict(C=320, H=64, W=96, K=3, S=None, seed=1003),
    "latent_320x64x96_k4": dict(C=320, H=64, W=96, K=4, S=None, seed=1003),
}
