"""FP64 oracle of the proposal network (TEST INFRASTRUCTURE ONLY).

MLP 62 -> 256 -> 256 -> 256 -> 48, GELU(z) = z Phi(z), mean-squared-error loss
over all outputs, its gradient by backpropagation, and one AdamW step.  With
`mirror=True` the values are rounded to BF16 (round-to-nearest-even) exactly
where the tensor-core kernels keep BF16 (inputs, weights, hidden activations,
the output-side gradients fed to the next GEMM) and everything else is FP64,
so a parity test measures only accumulation-order differences.  Parameter
layout: W1 [256][62], b1, W2 [256][256], b2, W3, b3, W4 [48][256], b4.
The network is a proposal distribution for the knots, which the paper leaves
to future work (arXiv 2409.10469, Sec. V-B).
"""
from __future__ import annotations

import math

import numpy as np

SIZES = [(256, 62), (256, 256), (256, 256), (48, 256)]


def n_params():
    return sum(o * i + o for o, i in SIZES)


def unpack(p):
    p = np.asarray(p, np.float64)
    out, o = [], 0
    for (no, ni) in SIZES:
        W = p[o:o + no * ni].reshape(no, ni)
        o += no * ni
        b = p[o:o + no]
        o += no
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def bf16(x):
    """Round to BF16 (nearest, ties to even) and return as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    u = ((u + r) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def forward(p, X, mirror=True):
    """Returns (Y, cache): Y = W4 h3 + b4 with h_l = GELU(W_l h_{l-1} + b_l)."""
    r = bf16 if mirror else (lambda a: np.asarray(a, np.float64))
    layers = unpack(p)
    h = r(X)
    cache = {"h": [h], "z": []}
    for li, (W, b) in enumerate(layers):
        z = h @ r(W).T + b
        cache["z"].append(z)
        if li < len(layers) - 1:
            h = r(gelu(z))
            cache["h"].append(h)
    return z, cache


def loss_grad(p, X, T, mirror=True):
    """MSE loss mean over B x 48 and its gradient with respect to p."""
    r = bf16 if mirror else (lambda a: np.asarray(a, np.float64))
    layers = unpack(p)
    Y, c = forward(p, X, mirror)
    n = Y.size
    d = Y - np.asarray(T, np.float64)
    loss = float(np.sum(d * d) / n)
    dz = 2.0 * d / n
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        dzr = r(dz)
        dW = dzr.T @ c["h"][li]
        db = dz.sum(0)
        grads[li] = (dW, db)
        if li == 0:
            break
        dh = dzr @ r(W)
        dz = dh * gelu_grad(c["z"][li - 1])
    return loss, pack(grads)


def adamw(p, g, m1, m2, step, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    c1, c2 = 1 - b1 ** step, 1 - b2 ** step
    p = p - lr * ((m1 / c1) / (np.sqrt(m2 / c2) + eps) + wd * p)
    return p, m1, m2


def init_params(seed=0):
    """He-style uniform init (an input choice)."""
    rng = np.random.default_rng(seed)
    layers = []
    for no, ni in SIZES:
        lim = math.sqrt(6.0 / (ni + no))
        layers.append((rng.uniform(-lim, lim, (no, ni)), np.zeros(no)))
    return pack(layers).astype(np.float32)
