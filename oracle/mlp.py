"""MLP lens-surrogate oracle (TEST INFRASTRUCTURE ONLY; see the package docstring).

A learned stand-in for back-tracking through the galactic field (the paper's
Sect. 4 forward- and back-tracking, used to build lenses): it maps an arrival
direction at Earth and the log rigidity to the direction at the galaxy
border.  Readings (the paper has no learned component; the architecture is
fixed by the workload description): inputs (n_x, n_y, n_z, (log10 R - 19)),
hidden layers of width 256 with ReLU, a linear output of 3 normalised to a
unit vector, loss mean(1 - cos angle) = mean(1 - y_hat . t), Adam with
bias correction.  Plain numpy binary64; matrix products are library
primitives.  Parameters are packed as [W1, b1, W2, b2, ...] with W_l of shape
(n_out, n_in) (row-major), the layout the GPU library uses.

Pins: central finite differences of the loss against the backward pass, and
an explicit-loop forward on a tiny network.

bf16 mode (``bf16=True`` in forward / backward): the same network with the
values rounded to bfloat16 at the points where the GPU stores them in that
format, everything else binary64: the hidden-to-hidden weights; every
hidden activation h_l = bf16(ReLU(z_l)) (z_l from the rounded inputs, the
thin first layer from the binary32 inputs and weights); the output layer
reads the rounded last activation; in the backward pass every hidden
backward signal dz_l = bf16((dz_{l+1} W_{l+1}) masked by h_l > 0), and
dy = dL/dy of the output layer stays unrounded.  The weight and bias
gradients are the binary64 products and sums of those rounded values.  The
rounding itself (round to nearest even, through binary32 like the GPU's
binary32 accumulators) is pinned by its own test.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(n_in=4, hidden=256, n_hidden=4, n_out=3):
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def n_params(shapes):
    return sum(o * i + o for o, i in shapes)


def unpack(flat, shapes):
    Ws, bs, k = [], [], 0
    for o, i in shapes:
        Ws.append(flat[k:k + o * i].reshape(o, i))
        k += o * i
        bs.append(flat[k:k + o])
        k += o
    return Ws, bs


def pack(Ws, bs):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])


def bf16_round(a):
    """Round binary64 values to the nearest bfloat16 (ties to even), as
    binary64 (through binary32, which is exact for the bfloat16 grid)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weights(flat, shapes):
    """The parameters with the hidden-to-hidden weights rounded to bf16 (the
    first and the output layer's weights and every bias unrounded)."""
    Ws, bs = unpack(np.array(flat, dtype=np.float64), shapes)
    for l in range(1, len(shapes) - 1):
        Ws[l] = bf16_round(Ws[l])
    return pack(Ws, bs)


def forward(flat, shapes, x, bf16=False):
    """Returns (y_hat [n, 3] unit vectors, cache).  bf16: see the module
    docstring (the caller passes bf16_weights(flat) to round the weights)."""
    Ws, bs = unpack(flat, shapes)
    hs, zs = [x], []
    h = x
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ W.T + b
        zs.append(z)
        h = np.maximum(z, 0.0) if l < len(Ws) - 1 else z
        if bf16 and l < len(Ws) - 1:
            h = bf16_round(h)
        hs.append(h)
    y = hs[-1]
    norm = np.linalg.norm(y, axis=1, keepdims=True)
    return y / norm, dict(hs=hs, zs=zs, norm=norm)


def loss(y_hat, t):
    return float(np.mean(1.0 - np.sum(y_hat * t, axis=1)))


def backward(flat, shapes, cache, t, bf16=False):
    """Gradient of mean(1 - y_hat . t) with respect to the packed parameters.
    bf16: the hidden backward signals rounded (see the module docstring)."""
    Ws, bs = unpack(flat, shapes)
    hs, zs, norm = cache["hs"], cache["zs"], cache["norm"]
    n = len(t)
    y = hs[-1]
    y_hat = y / norm
    # d(1 - y_hat.t)/dy = -(t - (y_hat.t) y_hat) / |y|
    dy = -(t - np.sum(y_hat * t, axis=1, keepdims=True) * y_hat) / norm / n
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    dz = dy
    for l in range(len(Ws) - 1, -1, -1):
        dWs[l] = dz.T @ hs[l]
        dbs[l] = dz.sum(axis=0)
        if l > 0:
            dh = dz @ Ws[l]
            dz = dh * (zs[l - 1] > 0.0)
            if bf16:
                dz = bf16_round(dz)
    return pack(dWs, dbs)


def adam(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; returns new
    (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def angle_deg(a, b):
    c = np.clip(np.sum(a * b, axis=1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1)),
                -1.0, 1.0)
    return np.degrees(np.arccos(c))


def inputs(dirs, rigidity_V):
    """Network inputs from arrival directions and rigidities [V]."""
    return np.concatenate([dirs, (np.log10(rigidity_V) - 19.0)[:, None]], axis=1)
