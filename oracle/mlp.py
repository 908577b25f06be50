"""FP64 CPU oracle of the learned-warm-start network (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import it; it shares no code with the CUDA path.

Network: z_l = a_l W_l^T + b_l; hidden layers a_{l+1} = GELU(z_l) with
GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2; linear output y = z_{L-1};
loss mean((y - t)^2) over all entries; Adam (Kingma & Ba 2015).  With
``bf16=True`` the values the GPU rounds to BF16 before a GEMM (inputs,
hidden activations, weights, back-propagated dz) are rounded here too
(round to nearest even from float32), and everything else is float64.

Parameter packing: for each layer W_l [out][in] then b_l [out].
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def bf16(v):
    """Round to BF16 (nearest even) through float32, returned as float64."""
    f = np.asarray(v, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    rounded = ((bits + np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1)))
               >> np.uint64(16)) << np.uint64(16)
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(params, widths):
    Ws, bs, o = [], [], 0
    for l in range(len(widths) - 1):
        nin, nout = widths[l], widths[l + 1]
        Ws.append(np.asarray(params[o:o + nin * nout], dtype=np.float64).reshape(nout, nin))
        o += nin * nout
        bs.append(np.asarray(params[o:o + nout], dtype=np.float64))
        o += nout
    return Ws, bs


def pack(Ws, bs):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)])


def forward(params, widths, x, bf16_ops=True):
    """Returns (y, cache) with cache = (activations a_l, pre-activations z_l)."""
    r = bf16 if bf16_ops else (lambda v: np.asarray(v, dtype=np.float64))
    Ws, bs = unpack(params, widths)
    a = [r(x)]
    zs = []
    L = len(Ws)
    for l in range(L):
        z = a[l] @ r(Ws[l]).T + bs[l]
        zs.append(z)
        if l < L - 1:
            a.append(r(gelu(z)))
    return zs[-1], (a, zs)


def loss_and_grads(params, widths, x, t, bf16_ops=True):
    """MSE loss and its gradient w.r.t. the packed parameters (backprop)."""
    r = bf16 if bf16_ops else (lambda v: np.asarray(v, dtype=np.float64))
    Ws, bs = unpack(params, widths)
    y, (a, zs) = forward(params, widths, x, bf16_ops)
    n = y.size
    loss = float(np.mean((y - t) ** 2))
    dz = 2.0 * (y - t) / n
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        gb[l] = dz.sum(axis=0)
        gW[l] = r(dz).T @ a[l]
        if l > 0:
            da = r(dz) @ r(Ws[l])
            dz = da * gelu_grad(zs[l - 1])
    return loss, pack(gW, gb)


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v
