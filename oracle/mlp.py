"""FP64 numpy restatement of the learned inverse-CDF sampler (TEST INFRASTRUCTURE).

The network maps (r, gamma, omega_c dt) to ln x with G(x) = r, G the
photon-number CDF of the synchrotron spectrum (Eqs. (7)-(8) of
arXiv:1409.5574).  Model definition (as documented with the C ABI):

  features  f0 = logit(r) / 8
            f1 = clip((ln gamma - 5.7565) / 3.4539, -1, 1)
            f2 = clip((ln(omega_c dt) - 8.2) / 11.6, -1, 1)
  layer 1   z1 = W1 f + b1,  h1 = f16(silu(z1))         (W1 in BF16)
  layer 2   z2 = W2 h1 + b2, h2 = f16(silu(z2))         (W2 in BF16)
  layer 3   o  = W3 h2 + b3                             (W3 in BF16)
  output    ln x = prior(r) + o,  prior(r) = ln(-ln(1 - r)) + 2 (1 - r) ln r
  loss      mean over samples of w (o - (ln x_target - prior(r)))^2,
            w = (1 + x_target) / 1.308 (energy weighting, mean 1)

Parameter vector: W1[64][3], b1[64], W2[64][64], b2[64], W3[64], b3 (4481).
Everything here is FP64 except the roundings the definition names (weights
to BF16, activations to IEEE half; W2 and W3 enter the f16 products as the
half-precision images of their BF16 values, identical for |w| >= 2^-17);
gradients treat the roundings as identity (straight-through).  Only tests
import this module.
"""
from __future__ import annotations

import numpy as np

H = 64
OFF_W1, OFF_B1 = 0, 192
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NUM_PARAMS = OFF_B3 + 1


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via float32 bits."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def f16(x):
    """Round to the nearest IEEE half (ties to even)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(H, 3), p[OFF_B1:OFF_W2],
            p[OFF_W2:OFF_B2].reshape(H, H), p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3],
            p[OFF_B3])


def features(r, gamma, wdt):
    r = np.asarray(r, dtype=np.float64)
    f0 = (np.log(r) - np.log1p(-r)) / 8.0
    f1 = np.clip((np.log(gamma) - 5.7565) / 3.4539, -1.0, 1.0)
    f2 = np.clip((np.log(wdt) - 8.2) / 11.6, -1.0, 1.0)
    return np.stack([f0, f1, f2], 1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s + z * s * (1.0 - s)


def forward(p, f, rounding=True):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    ident = lambda v: np.asarray(v, dtype=np.float64)  # noqa: E731
    rw = bf16 if rounding else ident
    rh = f16 if rounding else ident
    W1r, W2r, W3r = rw(W1), rh(rw(W2)), rh(rw(W3))
    z1 = f @ W1r.T + b1
    h1 = rh(silu(z1))
    z2 = h1 @ W2r.T + b2
    h2 = rh(silu(z2))
    o = h2 @ W3r + b3
    return o, (f, z1, h1, z2, h2, W1r, W2r, W3r)


def prior(r):
    r = np.asarray(r, dtype=np.float64)
    return np.log(-np.log1p(-r)) + 2.0 * (1.0 - r) * np.log(r)


def ln_x(p, r, gamma, wdt, rounding=True):
    o, _ = forward(p, features(r, gamma, wdt), rounding)
    return o + prior(r)


def loss_and_grad(p, r, gamma, wdt, lnx_target, rounding=True):
    f = features(r, gamma, wdt)
    o, (f, z1, h1, z2, h2, W1r, W2r, W3r) = forward(p, f, rounding)
    t = np.asarray(lnx_target, dtype=np.float64) - prior(r)
    n = o.size
    diff = o - t
    wgt = (1.0 + np.exp(np.asarray(lnx_target, dtype=np.float64))) / 1.308
    loss = np.mean(wgt * diff * diff)
    do = 2.0 * wgt * diff / n
    g = np.zeros(NUM_PARAMS)
    g[OFF_W3:OFF_B3] = h2.T @ do
    g[OFF_B3] = do.sum()
    d2 = np.outer(do, W3r) * silu_grad(z2)
    g[OFF_W2:OFF_B2] = (d2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = d2.sum(0)
    d1 = (d2 @ W2r) * silu_grad(z1)
    g[OFF_W1:OFF_B1] = (d1.T @ f).ravel()
    g[OFF_B1:OFF_W2] = d1.sum(0)
    return loss, g


def glorot(seed=0):
    rng = np.random.default_rng(seed)
    p = np.zeros(NUM_PARAMS)
    p[OFF_W1:OFF_B1] = rng.uniform(-1, 1, 3 * H) * np.sqrt(6 / (3 + H))
    p[OFF_W2:OFF_B2] = rng.uniform(-1, 1, H * H) * np.sqrt(6 / (2 * H))
    p[OFF_W3:OFF_B3] = rng.uniform(-1, 1, H) * np.sqrt(6 / (H + 1))
    p[OFF_B1:OFF_W2] = rng.normal(0, 0.1, H)
    p[OFF_B2:OFF_W3] = rng.normal(0, 0.1, H)
    p[OFF_B3] = -0.1
    return p
