"""Pins of the FP64 network reference: central finite differences and torch autograd
for the exact network, torch's own BF16 conversion for the rounding function."""
import numpy as np
import torch

from oracle import mlp


def _case(seed=0, B=8):
    rng = np.random.default_rng(seed)
    P = rng.normal(scale=0.2, size=mlp.NPARAM)
    X = rng.uniform(0, 1, size=(B, 48))
    t = rng.uniform(0, 1, size=B)
    return P, X, t


def test_bf16_matches_torch():
    x = np.random.default_rng(1).normal(size=10000) * 10.0 ** np.random.default_rng(2).integers(-8, 8, 10000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)


def test_gradients_match_finite_differences():
    P, X, t = _case()
    loss, g = mlp.gradients(P, X, t, rounding=False)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(12288, 20), 12288 + rng.choice(256, 10), 12544 + rng.choice(65536, 30),
                          78080 + rng.choice(256, 10), 78336 + rng.choice(256, 10), [78592]])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        num = (mlp.gradients(Pp, X, t, False)[0] - mlp.gradients(Pm, X, t, False)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_gradients_match_torch_autograd():
    P, X, t = _case(4, 16)
    loss, g = mlp.gradients(P, X, t, rounding=False)
    p = {k: torch.tensor(v, requires_grad=True) for k, v in mlp.unpack(P).items()}
    Xt, tt = torch.tensor(X), torch.tensor(t)
    h1 = torch.relu(Xt @ p["W1"].T + p["b1"])
    h2 = torch.relu(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["w3"] + p["b3"][0]
    L = torch.mean((y - tt) ** 2)
    L.backward()
    ref = np.concatenate([p[k].grad.numpy().ravel() for k, _ in mlp.SIZES])
    assert abs(L.item() - loss) < 1e-12
    np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-13)


def test_adam_first_step_moves_by_lr():
    P, X, t = _case()
    _, g = mlp.gradients(P, X, t, rounding=False)
    P2, m, v = mlp.adam(P, np.zeros_like(P), np.zeros_like(P), g, 1, 1e-3)
    nz = np.abs(g) > 1e-4  # |step| = lr |g| / (|g| + eps)
    np.testing.assert_allclose(np.abs(P2 - P)[nz], 1e-3, rtol=1e-3)
