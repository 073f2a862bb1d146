"""FP64 reference of the learned field surrogate (numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's driving field is the elastic energy density plus the dislocation
energy E_rho = 1/2 rho G b^2 of each material point (Sec. 3, Eq. (4)), produced
by the Monte Carlo crystal plasticity of Sec. 2.  The surrogate replaces that
producer by a small multilayer perceptron evaluated once per grain:

    x (11) -> GELU(W1 x + b1) (64) -> GELU(W2 . + b2) (64)
           -> GELU(W3 . + b3) (64) -> W4 . + b4 (2)

with GELU(z) = z/2 (1 + erf(z / sqrt 2)) (exact erf).  The 11 inputs are four
cubic invariants of the grain's loading axis d = R^T e_x (|d| sorted
decreasingly and d1^2 d2^2 + d2^2 d3^2 + d3^2 d1^2; ``oracle.surrogate``), the
six components of the population-average sample-frame stress of the load
step and the average accumulated slip, each divided by a fixed scale; the two
outputs are (w, E_rho), each divided by a fixed scale.  Training minimises the mean squared error
L = 1/(2B) sum_b sum_o (y_bo - t_bo)^2 with Adam (Kingma & Ba, 2015):
m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
theta <- theta - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Weights are stored [out, in] (W_l maps layer l-1 to layer l).
Parity pins: central finite differences and torch.autograd in float64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

LAYERS = (11, 64, 64, 64, 2)
SQRT2 = math.sqrt(2.0)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X):
    """params = [W1, b1, W2, b2, W3, b3, W4, b4]; X [B, 11] -> (Y [B, 2], cache)."""
    a = np.asarray(X, dtype=np.float64)
    cache = [a]
    n_layers = len(params) // 2
    for l in range(n_layers):
        W, b = params[2 * l], params[2 * l + 1]
        z = a @ W.T + b
        if l < n_layers - 1:
            cache.append(z)
            a = gelu(z)
            cache.append(a)
        else:
            a = z
    return a, cache


def loss(Y, T):
    d = Y - T
    return float(np.sum(d * d) / (2.0 * Y.shape[0]))


def backward(params, cache, Y, T):
    """Gradients of L = 1/(2B) sum (Y - T)^2 with respect to every parameter."""
    B = Y.shape[0]
    n_layers = len(params) // 2
    grads = [None] * len(params)
    dz = (Y - T) / B                                   # dL/dY
    for l in range(n_layers - 1, -1, -1):
        a_prev = cache[0] if l == 0 else cache[2 * l]  # input of layer l
        grads[2 * l] = dz.T @ a_prev
        grads[2 * l + 1] = dz.sum(axis=0)
        if l > 0:
            da = dz @ params[2 * l]
            z_prev = cache[2 * l - 1]
            dz = da * gelu_grad(z_prev)
    return grads


def loss_and_grads(params, X, T):
    Y, cache = forward(params, X)
    return loss(Y, T), backward(params, cache, Y, T)


def adam_step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1.0 - b1) * g
        vv = b2 * vv + (1.0 - b2) * g * g
        mh = mm / (1.0 - b1 ** t)
        vh = vv / (1.0 - b2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
