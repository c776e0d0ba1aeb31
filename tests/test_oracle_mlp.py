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


def test_forward_closed_form():
    """W1 = 0, b1 = 1.5 on units 0..15 and -2 elsewhere: h1 = relu(b1);
    W2 shifts (output unit j reads h1[j-1]), b2 = -0.25: h2[j] = 1.25 for
    j = 1..16, else relu(-0.25) = 0; W3 = 1, b3 = 0.125: o = 16 * 1.25 +
    0.125 = 20.125 (every value exact in BF16 and f16).  A transposed W2
    gives 15 live units, a smooth activation a different value."""
    p = np.zeros(M.NUM_PARAMS)
    b1 = np.where(np.arange(M.H) < 16, 1.5, -2.0)
    p[M.OFF_B1:M.OFF_W2] = b1
    W2 = np.zeros((M.H, M.H))
    W2[np.arange(1, M.H), np.arange(0, M.H - 1)] = 1.0
    p[M.OFF_W2:M.OFF_B2] = W2.ravel()
    p[M.OFF_B2:M.OFF_W3] = -0.25
    p[M.OFF_W3:M.OFF_B3] = 1.0
    p[M.OFF_B3] = 0.125
    f = M.features(np.array([0.3, 0.9]), np.array([50.0, 2e3]), np.array([1.0, 1e6]))
    for rounding in (True, False):
        o, _ = M.forward(p, f, rounding)
        np.testing.assert_array_equal(o, [20.125, 20.125])
    # the prior carries the output: ln x = o + prior(r)
    r = np.array([0.3])
    assert M.ln_x(p, r, np.array([50.0]), np.array([1.0]))[0] == pytest.approx(
        20.125 + np.log(-np.log1p(-0.3)) + 2 * 0.7 * np.log(0.3), rel=1e-15)
