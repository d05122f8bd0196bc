"""CPU FP64 reference of the seed network (TEST INFRASTRUCTURE ONLY).

The step's learned part is a multilayer perceptron that maps a cell's state, fields
and step length to its state at the end of the step.  Its prediction seeds the
implicit solve, and the solve then runs to convergence.  This module states that
network in plain numpy float64: the forward pass, the mean-squared-error loss and the
analytic backward pass.  The CUDA training kernels are checked against it; it shares
no code with them.

Layout (the same conventions as the library's blob):
    inputs   x[B, 13]  (already normalised)
    layer l  h_l = silu(h_{l-1} W_l^T + b_l),  W_1: [64, 13], W_2, W_3: [64, 64]
    output   o = h_3 W_4^T + b_4,  W_4: [3, 64]
    loss     L = sum_b sum_j w_j (o_bj - y_bj)^2 / B
silu(z) = z / (1 + exp(-z)).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 13, 64, 3
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unflatten(theta):
    """Splits a flat parameter vector into [W1, b1, W2, b2, W3, b3, W4, b4]."""
    theta = np.asarray(theta, dtype=np.float64)
    out, k = [], 0
    for s in SHAPES:
        m = int(np.prod(s))
        out.append(theta[k:k + m].reshape(s))
        k += m
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x):
    """Returns the outputs o[B, 3] and the pre-activations [z1, z2, z3] and activations
    [x, h1, h2, h3] needed by the backward pass."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    z3 = h2 @ W3.T + b3
    h3 = silu(z3)
    o = h3 @ W4.T + b4
    return o, (z1, z2, z3), (x, h1, h2, h3)


def forward_bf16_inputs(theta, x):
    """Outputs o[B, 3] with every layer's inputs rounded to BF16 first (the normalised
    features and each hidden activation), the rounding of an inference on BF16 tensor
    cores; sums in FP64."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta)
    h = bf16_round(np.asarray(x, dtype=np.float64))
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        h = bf16_round(silu(h @ W.T + b))
    return h @ W4.T + b4


def loss(theta, x, y, w=(1.0, 1.0, 1.0)):
    o, _, _ = forward(theta, x)
    d = o - np.asarray(y, dtype=np.float64)
    return float(np.sum(np.asarray(w) * d * d) / x.shape[0])


def grad(theta, x, y, w=(1.0, 1.0, 1.0)):
    """Analytic gradient of loss() with respect to the flat parameter vector, by the
    chain rule applied layer by layer from the output back to the input."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta)
    o, (z1, z2, z3), (x0, h1, h2, h3) = forward(theta, x)
    B = x0.shape[0]
    g_o = 2.0 * np.asarray(w) * (o - np.asarray(y, dtype=np.float64)) / B   # dL/do
    gW4 = g_o.T @ h3
    gb4 = g_o.sum(axis=0)
    g_z3 = (g_o @ W4) * silu_grad(z3)
    gW3 = g_z3.T @ h2
    gb3 = g_z3.sum(axis=0)
    g_z2 = (g_z3 @ W3) * silu_grad(z2)
    gW2 = g_z2.T @ h1
    gb2 = g_z2.sum(axis=0)
    g_z1 = (g_z2 @ W2) * silu_grad(z1)
    gW1 = g_z1.T @ x0
    gb1 = g_z1.sum(axis=0)
    return flatten([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


def bf16_round(a):
    """Rounds float64 values to the nearest bfloat16 (ties to even), returned as float64:
    bfloat16 keeps the top 16 bits of the IEEE float32 pattern."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
