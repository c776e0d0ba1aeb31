"""Pins of the FP64 numpy MLP used to check the GPU training kernels:
central finite differences of the loss (without the BF16 roundings, where
the loss is smooth) against the analytic backward pass, a hand-computed
forward pass, and the BF16 rounding helper against torch's bfloat16
conversion (a library)."""
import numpy as np
import pytest

from oracle import mlp as M


def _batch(n=64, seed=1):
    rng = np.random.default_rng(seed)
    r = rng.uniform(1e-5, 1 - 1e-5, n)
    g = np.exp(rng.uniform(np.log(10), np.log(1e4), n))
    w = np.exp(rng.uniform(-3, 19, n))
    t = rng.uniform(-6.0, 2.5, n)       # ln x of the spectrum's bulk
    return r, g, w, t


def test_backward_matches_finite_differences():
    p = M.glorot(3)
    r, g, w, t = _batch()
    _, grad = M.loss_and_grad(p, r, g, w, t, rounding=False)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.arange(M.OFF_W1, M.OFF_B1), 6),
                          rng.choice(np.arange(M.OFF_B1, M.OFF_W2), 4),
                          rng.choice(np.arange(M.OFF_W2, M.OFF_B2), 10),
                          rng.choice(np.arange(M.OFF_B2, M.OFF_W3), 4),
                          rng.choice(np.arange(M.OFF_W3, M.OFF_B3), 4), [M.OFF_B3]])
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        lp, _ = M.loss_and_grad(pp, r, g, w, t, rounding=False)
        lm, _ = M.loss_and_grad(pm, r, g, w, t, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).normal(0, 10, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)


def test_f16_rounding_matches_torch_and_bf16_values_are_exact_halves():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(3).normal(0, 3, 10000)
    ref = torch.tensor(x, dtype=torch.float64).to(torch.float16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.f16(x), ref)
    # the weights' BF16 values (8 significant bits) are exact in f16 down to
    # 2^-17 in magnitude, so the f16 products use exactly the BF16 weights
    rng = np.random.default_rng(4)
    w = M.bf16(rng.choice([-1.0, 1.0], 10000) * 2.0 ** -rng.uniform(0.0, 20.0, 10000))
    big = np.abs(w) >= 2.0 ** -17
    assert big.sum() > 5000
    np.testing.assert_array_equal(M.f16(w[big]), w[big])


def test_features_definition():
    f = M.features(np.array([0.5, 1 / (1 + np.e ** 8)]), np.array([316.2, 1e6]),
                   np.array([np.exp(8.2), 1e-30]))
    assert f[0] == pytest.approx([0.0, 0.0, 0.0], abs=1e-4)
    assert f[1] == pytest.approx([-1.0, 1.0, -1.0], abs=1e-12)


def test_forward_matches_torch_layers():
    """The forward pass (without the roundings) against torch's own SiLU and
    matrix products in float64, on a net whose W2 shifts units (output unit
    j reads h1[j-1]): a transposed W2, a dropped bias or another activation
    changes the output."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    p = M.glorot(21)
    W2 = np.zeros((M.H, M.H))
    W2[np.arange(1, M.H), np.arange(0, M.H - 1)] = rng.uniform(0.5, 1.5, M.H - 1)
    p[M.OFF_W2:M.OFF_B2] = W2.ravel()
    p[M.OFF_B1:M.OFF_W2] = np.where(np.arange(M.H) < 16, 1.5, -2.0)
    r, g, w, _ = _batch(n=32, seed=5)
    f = M.features(r, g, w)
    o, _ = M.forward(p, f, rounding=False)
    t = torch.tensor
    W1 = t(p[M.OFF_W1:M.OFF_B1].reshape(M.H, 3))
    lin1 = t(f) @ W1.T + t(p[M.OFF_B1:M.OFF_W2])
    h1 = torch.nn.functional.silu(lin1)
    h2 = torch.nn.functional.silu(h1 @ t(W2).T + t(p[M.OFF_B2:M.OFF_W3]))
    ref = (h2 @ t(p[M.OFF_W3:M.OFF_B3]) + p[M.OFF_B3]).numpy()
    np.testing.assert_allclose(o, ref, rtol=1e-13, atol=1e-13)
    # the transposed shift gives a different output
    bad = p.copy()
    bad[M.OFF_W2:M.OFF_B2] = W2.T.ravel()
    assert np.max(np.abs(M.forward(bad, f, rounding=False)[0] - o)) > 1e-3
