"""FP64 reference of the surrogate MLP: 5 -> 128 -> 128 -> 128 -> 4, GELU.

TEST INFRASTRUCTURE ONLY: only tests/ may import it.  Plain numpy, written to
be checked by eye: forward, back-propagation, mean-squared-error loss and
the Adam update (Kingma & Ba 2015).  Shares nothing with the CUDA kernels.

Parameter layout (one flat vector, the same order the library documents):
  for each layer l = 1..4 with fan-in n_in and fan-out n_out:
    W_l (n_out x n_in, row-major), then b_l (n_out)
"""
from __future__ import annotations

import math

import numpy as np

SIZES = (5, 128, 128, 128, 4)


def param_count(sizes=SIZES) -> int:
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unpack(theta: np.ndarray, sizes=SIZES):
    """[(W, b)] views of a flat parameter vector."""
    out, p = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    return out


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    """x * Phi(x), Phi the standard normal CDF (exact erf form)."""
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    cdf = 0.5 * (1.0 + _erf(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def forward(theta, x, sizes=SIZES):
    """Returns y and the cache of pre-activations / activations."""
    layers = unpack(np.asarray(theta, np.float64), sizes)
    a = np.asarray(x, np.float64)
    acts, pres = [a], []
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        pres.append(z)
        a = gelu(z) if l < len(layers) - 1 else z       # linear output layer
        acts.append(a)
    return a, (acts, pres)


def mse(y, t):
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def loss_and_grad(theta, x, t, sizes=SIZES):
    """MSE over all outputs and samples and its gradient w.r.t. theta."""
    theta = np.asarray(theta, np.float64)
    y, (acts, pres) = forward(theta, x, sizes)
    n = y.size
    dy = 2.0 * (y - np.asarray(t, np.float64)) / n
    layers = unpack(theta, sizes)
    grads = []
    delta = dy
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = delta.T @ acts[l]
        gb = delta.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            delta = (delta @ W) * gelu_grad(pres[l - 1])
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return mse(y, t), flat


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (bias-corrected moments)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x):
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as
    FP64 -- the weights the mixed-precision forward actually uses."""
    f = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> np.uint64(16)) & np.uint64(1)
    r = (f + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
