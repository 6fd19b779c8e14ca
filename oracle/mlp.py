"""Learned nonlinear reconstructor (FP64): a multilayer perceptron from slopes
to modal coefficients, trained on simulator-generated pairs.

Not in the paper (its reconstructor is the linear Modalrec, App. A, Tab. 4);
the learned reconstructor, its sizes (2400 -> 1024 -> 1024 -> 500 and
14000 -> 2048 -> 2048 -> 4000), BF16 weights with FP32 accumulation, batch
256 and Adam are this library's learned-reconstructor configuration (the
learned8m workload and the ELT-scale network).
Readings:

* layers y = W x + b, GELU with the exact error function between layers:
      gelu(z) = z Phi(z),  Phi(z) = (1 + erf(z / sqrt 2)) / 2,
      gelu'(z) = Phi(z) + z phi(z),  phi(z) = exp(-z^2 / 2) / sqrt(2 pi);
* loss = mean over the batch and the outputs of (y - t)^2;
* initialisation W, b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), drawn by synth;
* Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
        w -= lr sqrt(1 - b2^t) / (1 - b1^t) * m / (sqrt(v) + eps),
  lr 1e-3, b1 0.9, b2 0.999, eps 1e-8, no weight decay.
"""
import math

import numpy as np
from scipy.special import erf

import synth

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) * INV_SQRT_2PI


def init_params(sizes, seed):
    """[(W (out, in), b (out,)), ...] for consecutive sizes [n_in, h1, ..., n_out]."""
    params = []
    for l in range(len(sizes) - 1):
        fan_in, fan_out = sizes[l], sizes[l + 1]
        bound = 1.0 / math.sqrt(fan_in)
        W = synth.uniform_draws(seed * 100 + 2 * l, (fan_out, fan_in), -bound, bound)
        b = synth.uniform_draws(seed * 100 + 2 * l + 1, (fan_out,), -bound, bound)
        params.append((W, b))
    return params


def forward(params, X):
    """X (B, n_in) -> Y (B, n_out); cache of pre-activations and activations."""
    acts = [np.asarray(X, dtype=np.float64)]
    zs = []
    h = acts[0]
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        if l < len(params) - 1:
            h = gelu(z)
            acts.append(h)
        else:
            h = z
    return h, (zs, acts)


def mse(Y, T):
    d = np.asarray(Y, np.float64) - np.asarray(T, np.float64)
    return float(np.mean(d * d))


def backward(params, cache, Y, T):
    """Gradients [(dW, db), ...] of the MSE loss."""
    zs, acts = cache
    B, n_out = Y.shape
    d = 2.0 * (Y - T) / (B * n_out)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * gelu_grad(zs[l - 1])
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads):
        self.t += 1
        lr_t = self.lr * math.sqrt(1 - self.b2 ** self.t) / (1 - self.b1 ** self.t)
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for k, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[l][k] + (1 - self.b1) * g
                v = self.b2 * self.v[l][k] + (1 - self.b2) * g * g
                self.m[l] = tuple(m if kk == k else self.m[l][kk] for kk in range(2))
                self.v[l] = tuple(v if kk == k else self.v[l][kk] for kk in range(2))
                new.append(p - lr_t * m / (np.sqrt(v) + self.eps))
            out.append((new[0], new[1]))
        return out
