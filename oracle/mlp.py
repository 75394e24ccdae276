"""FP64 oracle of the learned column closure's multilayer perceptron.

ORACLE / TEST INFRASTRUCTURE (see ocn_oracle.h): used only by the tests, the
smoke check and the benchmark's CPU baseline; the CUDA library never imports it.

The network (a learned closure of the kind the paper motivates in Sec. 3.2.3 and
its outlook: a parameterisation calibrated on LES): x (32 features) -> 128 ->
128 -> 128 -> 16 outputs, GELU after every hidden layer,
    z_l = h_{l-1} W_l^T + b_l,   h_l = gelu(z_l),   y = h_3 W_4^T + b_4,
gelu(z) = z Phi(z) with Phi the standard normal CDF (the exact, erf form).
Loss: L = (1 / 2M) sum_m sum_j mask_j (y_mj - t_mj)^2 (only the masked outputs
count).  Gradients by the chain rule written out layer by layer (plain
definitions); Adam as in Kingma & Ba (2015) with bias correction.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = (32, 128, 128, 128, 16)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _erf(x):
    from scipy.special import erf
    return erf(x)


def forward(params, X):
    """params: list of (W_l [n_out, n_in], b_l [n_out]); returns (y, cache of (h_{l-1}, z_l))."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if l < L - 1 else z
    return h, cache


def loss(y, t, mask):
    M = y.shape[0]
    return 0.5 * float(((y - t) ** 2 * mask).sum()) / M


def backward(params, cache, y, t, mask):
    """Gradients of loss() with respect to every W_l and b_l."""
    M = y.shape[0]
    dz = (y - t) * mask / M                      # dL/dy; the last layer is linear
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        h_prev, z = cache[l]
        W, _ = params[l]
        grads[l] = (dz.T @ h_prev, dz.sum(axis=0))
        if l > 0:
            dh = dz @ W
            dz = dh * gelu_prime(cache[l - 1][1])
    return grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state: dict with 't' and lists 'm', 'v' (created if empty)."""
    if not state:
        state["t"] = 0
        state["m"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state["v"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    state["t"] += 1
    t = state["t"]
    out = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for i, (p, g) in enumerate(((W, gW), (b, gb))):
            m = beta1 * state["m"][l][i] + (1 - beta1) * g
            v = beta2 * state["v"][l][i] + (1 - beta2) * g * g
            state["m"][l] = tuple(m if j == i else x for j, x in enumerate(state["m"][l]))
            state["v"][l] = tuple(v if j == i else x for j, x in enumerate(state["v"][l]))
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append((new[0], new[1]))
    return out


def closure_fluxes(params, X, mu, sigma, scale, shape):
    """The learned column closure's face fluxes from raw features X [(Nz+1)*Ny*Nx][NF]:
    y = forward((X - mu) / sigma), F_q = scale_q * y_q for q = b, ubar, vbar, reshaped to
    [3][Nz+1][Ny][Nx]; the wall faces carry no flux."""
    Xn = (np.asarray(X, np.float64) - mu) / sigma
    y, _ = forward(params, Xn)
    Nz1, Ny, Nx = shape
    F = np.stack([scale[q] * y[:, q].reshape(Nz1, Ny, Nx) for q in range(3)])
    F[:, 0] = 0.0
    F[:, -1] = 0.0
    return F


def closure_diffusivities(params, X, mu, sigma, scale, shape):
    """The learned column closure in diffusivity form: K_q = max(0, scale_q * y_q) for q = 0
    (tracers), 1 (momentum) at every w-face, [3][Nz+1][Ny][Nx] (K[2] = 0, walls 0)."""
    K = np.maximum(closure_fluxes(params, X, mu, sigma, scale, shape), 0.0)
    K[2] = 0.0
    return K
