"""FP64 oracle of the learned decode proposal (test infrastructure only).

The proposal is a small MLP that maps a symbol's mixture parameters and its
rANS slot to a guess of the symbol; the decoder checks the guess against the
exact quantised CDF and finishes with a bracketed search, so the guess only
affects speed. The paper has no learned part; the network shape (10 inputs,
64, 64, 1 output, GELU) is fixed by the coder's specification. This module
writes the feature map, the forward pass and its gradient out in plain numpy
FP64, one layer at a time, so that the GPU kernels can be checked against it.

Definitions (K = 3):
  sigma'_k = max(sigma_k, 0.11); components sorted by mean (stable);
  m0 = sum_k w_k mu_k;  s0 = sqrt(max(sum_k w_k (sigma'_k^2 + (mu_k - m0)^2), 1e-4));
  u  = (slot + 1/2) / 2^16;
  x  = [w_(1), w_(2), w_(3), (mu_(k) - m0)/s0 (k=1..3), log(sigma'_(k)/s0) (k=1..3), u - 1/2];
  target t = (s - m0)/s0 clipped to [-8, 8];  guess g = round(m0 + s0 * y).
  act(z) (kind ACT_PL, the default) = z * clamp(1/2 + c z, 0, 1), c = 1.702/4:
  GELU x Phi(x) with Phi replaced by its tangent line at 0 as given by the
  logistic form of Eq. 9, clamped to [0, 1] (a piecewise-linear GELU; no
  exp); or (kind ACT_SIGMOID) z / (1 + exp(-1.702 z)): GELU with Phi replaced
  by the logistic form of Eq. 9 itself.
  h1 = act(x W1 + b1), h2 = act(h1 W2 + b2), y = h2 . w3 + b3;
  loss = mean((y - t)^2).
Parameter vector (fp32 on the GPU): W1[10][64], b1[64], W2[64][64], b2[64],
w3[64], b3[1] -- 4929 values.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 10, 64
N_PARAMS = N_IN * N_HID + N_HID + N_HID * N_HID + N_HID + N_HID + 1
ACT_C = 1.702 / 4.0
ACT_PL, ACT_SIGMOID = 0, 1
SIG_A = 1.702
SIGMA_MIN = float(np.float32(0.11))
TARGET_CLIP = 8.0


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    o = 0
    W1 = theta[o:o + N_IN * N_HID].reshape(N_IN, N_HID); o += N_IN * N_HID
    b1 = theta[o:o + N_HID]; o += N_HID
    W2 = theta[o:o + N_HID * N_HID].reshape(N_HID, N_HID); o += N_HID * N_HID
    b2 = theta[o:o + N_HID]; o += N_HID
    w3 = theta[o:o + N_HID]; o += N_HID
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """Uniform fan-in initialisation, seeded."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (N_IN, N_HID)) * np.sqrt(3.0 / N_IN)
    W2 = rng.uniform(-1, 1, (N_HID, N_HID)) * np.sqrt(3.0 / N_HID)
    w3 = rng.uniform(-1, 1, N_HID) * np.sqrt(3.0 / N_HID)
    return pack(W1, np.zeros(N_HID), W2, np.zeros(N_HID), w3, 0.0)


def features(params, slots, symbols=None):
    """params: [3, 3, N] (w, mu, sigma); slots: [N] ints in [0, 2^16).
    Returns (x [N, 10], m0 [N], s0 [N], target [N] or None)."""
    p = np.asarray(params, dtype=np.float64)
    w, mu, sg = p[0], p[1], np.maximum(p[2], SIGMA_MIN)
    order = np.argsort(mu, axis=0, kind="stable")
    w = np.take_along_axis(w, order, 0)
    mu = np.take_along_axis(mu, order, 0)
    sg = np.take_along_axis(sg, order, 0)
    m0 = (w * mu).sum(0)
    s0 = np.sqrt(np.maximum((w * (sg ** 2 + (mu - m0) ** 2)).sum(0), 1e-4))
    u = (np.asarray(slots, dtype=np.float64) + 0.5) / 65536.0
    x = np.concatenate([w, (mu - m0) / s0, np.log(sg / s0), (u - 0.5)[None, :]], axis=0).T
    t = None
    if symbols is not None:
        t = np.clip((np.asarray(symbols, dtype=np.float64) - m0) / s0, -TARGET_CLIP, TARGET_CLIP)
    return x, m0, s0, t


def _sigmoid(v):
    return 0.5 * (1.0 + np.tanh(0.5 * v))   # 1 / (1 + exp(-v)) without overflow


def act(z, kind=ACT_PL):
    if kind == ACT_SIGMOID:
        return z * _sigmoid(SIG_A * z)
    return z * np.clip(0.5 + ACT_C * z, 0.0, 1.0)


def act_grad(z, kind=ACT_PL):
    if kind == ACT_SIGMOID:
        sg = _sigmoid(SIG_A * z)
        return sg + SIG_A * z * sg * (1.0 - sg)
    r = 0.5 + ACT_C * z
    inside = (r > 0.0) & (r < 1.0)
    return np.clip(r, 0.0, 1.0) + np.where(inside, ACT_C * z, 0.0)


def forward(theta, x, kind=ACT_PL):
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    z1 = x @ W1 + b1
    h1 = act(z1, kind)
    z2 = h1 @ W2 + b2
    h2 = act(z2, kind)
    y = h2 @ w3 + b3
    return y, (z1, h1, z2, h2)


def loss_and_grad(theta, x, t, kind=ACT_PL):
    """Mean squared error and its gradient with respect to theta (by hand,
    layer by layer)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    B = x.shape[0]
    y, (z1, h1, z2, h2) = forward(theta, x, kind)
    r = y - t
    loss = float((r * r).mean())
    dy = 2.0 * r / B
    dw3 = h2.T @ dy
    db3 = dy.sum()
    d2 = np.outer(dy, w3) * act_grad(z2, kind)
    dW2 = h1.T @ d2
    db2 = d2.sum(0)
    d1 = (d2 @ W2.T) * act_grad(z1, kind)
    dW1 = x.T @ d1
    db1 = d1.sum(0)
    return loss, pack(dW1, db1, dW2, db2, dw3, db3)


def guess(theta, params, slots, kind=ACT_PL):
    """Integer guesses from the network (FP64 evaluation)."""
    x, m0, s0, _ = features(params, slots)
    y, _ = forward(theta, x, kind)
    return np.rint(m0 + s0 * y)
