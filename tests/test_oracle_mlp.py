"""Pins for the FP64 selector-MLP oracle: central finite differences, PyTorch
autograd on the same network, bfloat16 rounding against torch's conversion, and a
hand-computed forward pass."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(0, scale, s) for k, s in mlp.SHAPES.items()}


def _data(seed, n=64):
    rng = np.random.default_rng(seed + 100)
    X = rng.normal(2.0, 3.0, (n, 8))
    y = rng.integers(0, 3, n)
    s = rng.uniform(0.5, 2.0, n)
    mu = X.mean(axis=0)
    sd = X.std(axis=0) + 0.1
    return X, y, s, mu, sd


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_finite_differences(seed):
    P = _params(seed)
    X, y, s, mu, sd = _data(seed)
    L, g = mlp.backward(P, X, y, s, mu, sd)
    h = 1e-6
    rng = np.random.default_rng(seed + 7)
    for k in mlp.ORDER:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(P, X, mu, sd)[0], y, s)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(P, X, mu, sd)[0], y, s)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_backward_matches_torch_autograd():
    P = _params(3)
    X, y, s, mu, sd = _data(3, n=200)
    L, g = mlp.backward(P, X, y, s, mu, sd)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in P.items()}
    xn = (torch.tensor(X) - torch.tensor(mu)) / torch.tensor(sd)
    h1 = torch.relu(xn @ tp["W1"].T + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"].T + tp["b2"])
    z = h2 @ tp["W3"].T + tp["b3"]
    ce = torch.nn.functional.cross_entropy(z, torch.tensor(y), reduction="none")
    st = torch.tensor(s)
    tl = (st * ce).sum() / st.sum()
    tl.backward()
    assert abs(tl.item() - L) < 1e-12
    for k in mlp.ORDER:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-13)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 3.0,
                        1.00390625, 1.01171875, -2.5]]).astype(np.float32)
    want = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), want)


def test_forward_hand_computed():
    """One-hot style weights: h1 = relu(xn), h2 = relu(h1), z = first three of h2."""
    P = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    P["W1"][:8, :8] = np.eye(8)
    P["W2"][:32, :32] = np.eye(32)
    P["W3"][:, :3] = np.eye(3)
    P["b3"][:] = [0.5, 0.0, -0.5]
    X = np.array([[1.0, -2.0, 3.0, 0, 0, 0, 0, 0]])
    z, _ = mlp.forward(P, X, np.zeros(8), np.ones(8))
    np.testing.assert_array_equal(z[0], [1.5, 0.0, 2.5])
    assert mlp.predict(P, X, np.zeros(8), np.ones(8)).tolist() == [2]
