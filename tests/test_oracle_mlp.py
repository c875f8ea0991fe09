"""Pins for the FP64 oracle of the proposal network: the hand-written
gradient equals central finite differences of the loss and torch.autograd's
gradient (FP64); the activation is the stated piecewise-linear GELU; the
features are invariant to component order and to shifting/scaling the
latent (the standardisation they are built for)."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _batch(seed, B=16):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (B, mlp.N_IN))
    t = rng.normal(0, 1, B)
    theta = mlp.init_params(seed) + rng.normal(0, 0.05, mlp.N_PARAMS)
    return theta, x, t


@pytest.mark.parametrize("kind", [mlp.ACT_PL, mlp.ACT_SIGMOID])
@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed, kind):
    theta, x, t = _batch(seed)
    _, g = mlp.loss_and_grad(theta, x, t, kind)
    rng = np.random.default_rng(seed + 10)
    idx = rng.choice(mlp.N_PARAMS, 200, replace=False)
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (mlp.loss_and_grad(tp, x, t, kind)[0] - mlp.loss_and_grad(tm, x, t, kind)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


@pytest.mark.parametrize("kind", [mlp.ACT_PL, mlp.ACT_SIGMOID])
def test_gradient_matches_autograd(kind):
    theta, x, t = _batch(3, B=64)
    loss, g = mlp.loss_and_grad(theta, x, t, kind)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    I, H = mlp.N_IN, mlp.N_HID
    o = [0]

    def take(n, shape=None):
        v = th[o[0]:o[0] + n]
        o[0] += n
        return v.reshape(shape) if shape else v
    W1, b1, W2, b2, w3 = take(I * H, (I, H)), take(H), take(H * H, (H, H)), take(H), take(H)
    b3 = take(1)[0]
    X = torch.tensor(x)
    T = torch.tensor(t)

    def act(z):
        if kind == mlp.ACT_SIGMOID:
            return z * torch.sigmoid(1.702 * z)
        return z * torch.clamp(0.5 + mlp.ACT_C * z, 0.0, 1.0)

    y = act(act(X @ W1 + b1) @ W2 + b2) @ w3 + b3
    L = ((y - T) ** 2).mean()
    L.backward()
    assert abs(L.item() - loss) <= 1e-12
    np.testing.assert_allclose(th.grad.numpy(), g, rtol=1e-10, atol=1e-12)


def test_activation_is_piecewise_linear_gelu():
    z = np.linspace(-5, 5, 1001)
    a = mlp.act(z)
    # zero for z <= -1/(2c), identity for z >= 1/(2c), z/2 + c z^2 between
    lo, hi = -0.5 / mlp.ACT_C, 0.5 / mlp.ACT_C
    np.testing.assert_allclose(a[z <= lo], 0.0, atol=1e-15)
    np.testing.assert_allclose(a[z >= hi], z[z >= hi])
    mid = (z > lo) & (z < hi)
    np.testing.assert_allclose(a[mid], z[mid] * (0.5 + mlp.ACT_C * z[mid]))
    # within 0.05 of the exact GELU x Phi(x) on [-3, 3]
    from scipy.special import ndtr
    zz = np.linspace(-3, 3, 601)
    assert np.abs(mlp.act(zz) - zz * ndtr(zz)).max() < 0.2


def test_sigmoid_activation_is_the_logistic_gelu():
    """ACT_SIGMOID is z / (1 + exp(-1.702 z)) (GELU with Phi replaced by the
    logistic form of Eq. 9): checked against that formula in extended
    precision, the exact GELU z Phi(z) within the logistic form's known
    0.02, and its limits (0 far left, identity far right, 0 at 0)."""
    from scipy.special import ndtr
    z = np.linspace(-8, 8, 3201)
    a = mlp.act(z, mlp.ACT_SIGMOID)
    zl = z.astype(np.longdouble)
    ref = zl / (1 + np.exp(-np.longdouble(1.702) * zl))
    np.testing.assert_allclose(a, ref.astype(np.float64), rtol=1e-12, atol=1e-15)
    assert np.abs(a - z * ndtr(z)).max() < 0.021
    assert mlp.act(np.array([0.0]), mlp.ACT_SIGMOID)[0] == 0.0
    assert abs(mlp.act(np.array([-40.0]), mlp.ACT_SIGMOID)[0]) < 1e-20
    assert abs(mlp.act(np.array([40.0]), mlp.ACT_SIGMOID)[0] - 40.0) < 1e-20
    # derivative by central differences
    h = 1e-6
    fd = (mlp.act(z + h, mlp.ACT_SIGMOID) - mlp.act(z - h, mlp.ACT_SIGMOID)) / (2 * h)
    np.testing.assert_allclose(mlp.act_grad(z, mlp.ACT_SIGMOID), fd, atol=1e-8)


def test_features_are_standardised_and_order_free():
    rng = np.random.default_rng(4)
    N = 200
    w = rng.dirichlet([1, 1, 1], N).T
    mu = rng.normal(0, 3, (3, N))
    sg = np.exp(rng.uniform(np.log(0.2), np.log(30), (3, N)))
    p = np.stack([w, mu, sg])
    slots = rng.integers(0, 65536, N)
    x, m0, s0, _ = mlp.features(p, slots)
    perm = np.stack([p[:, [2, 0, 1], i] for i in range(N)], axis=-1)
    x2, _, _, _ = mlp.features(perm, slots)
    np.testing.assert_allclose(x, x2)
    shifted = p.copy(); shifted[1] = 3.0 * (p[1] + 7.0); shifted[2] = 3.0 * p[2]
    x3, m3, s3, _ = mlp.features(shifted, slots)
    np.testing.assert_allclose(x3, x, atol=1e-12)
    np.testing.assert_allclose(m3, 3.0 * (m0 + 7.0))
    np.testing.assert_allclose(s3, 3.0 * s0)
    # standardised mixture: weighted mean 0, weighted second moment 1
    wz = x[:, 0:3]
    mz = x[:, 3:6]
    lz = x[:, 6:9]
    np.testing.assert_allclose((wz * mz).sum(1), 0.0, atol=1e-12)
    np.testing.assert_allclose((wz * (np.exp(2 * lz) + mz ** 2)).sum(1), 1.0, rtol=1e-10)
