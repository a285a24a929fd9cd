"""Reference 3x3 convolutional correction network (forward, backward, loss,
Adam) for the learned-correction form.  This network is not in the paper; it is
the reference the GPU kernels are checked against.

Test infrastructure only (see oracle/__init__.py).

Network: four 3x3 correlation layers on an NHWC grid with zero padding,
channels 3 -> 32 -> 32 -> 32 -> 2, ReLU after the first three layers:
    Y[b,y,x,co] = sum_{dy,dx,ci} W[co, dy+1, dx+1, ci] X[b, y+dy, x+dx, ci] + bias[co].
Loss per sample: ||Y4 - T||^2 / ||T||^2, averaged over the batch.
With bf16=True every layer input (network input and hidden activations) and
every weight is rounded to bfloat16 (round to nearest even) before use, as the
GPU kernels store them; accumulation stays exact (float64).

Pins (tests/test_oracle_cnn.py): single-channel layer = scipy.signal.correlate2d,
gradients = central finite differences, Adam step = its closed form on a
quadratic.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (3, 32, 32, 32, 2)


def bf16_round(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def param_shapes():
    out = []
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        out.append(((co, 3, 3, ci), (co,)))
    return out


def num_params() -> int:
    return sum(int(np.prod(w)) + int(np.prod(b)) for w, b in param_shapes())


def unflatten(theta):
    """Flat parameter vector (layer by layer: W then bias) -> list of (W, b)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, k = [], 0
    for ws, bs in param_shapes():
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((theta[k:k + nw].reshape(ws), theta[k + nw:k + nw + nb].reshape(bs)))
        k += nw + nb
    return out


def flatten(params):
    return np.concatenate([np.concatenate([w.reshape(-1), b.reshape(-1)]) for w, b in params])


def conv3x3(X, W, b):
    """X: (B, H, W, Ci); W: (Co, 3, 3, Ci); b: (Co,) -> (B, H, W, Co)."""
    Bn, H, Wd, Ci = X.shape
    Xp = np.zeros((Bn, H + 2, Wd + 2, Ci))
    Xp[:, 1:-1, 1:-1, :] = X
    Y = np.zeros((Bn, H, Wd, W.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            Y += np.einsum('bhwc,oc->bhwo', Xp[:, dy:dy + H, dx:dx + Wd, :], W[:, dy, dx, :])
    return Y


def conv3x3_backward(X, W, dY):
    """Gradients of conv3x3 w.r.t. X, W and b for upstream gradient dY."""
    Bn, H, Wd, Ci = X.shape
    Xp = np.zeros((Bn, H + 2, Wd + 2, Ci))
    Xp[:, 1:-1, 1:-1, :] = X
    dW = np.zeros_like(W)
    dXp = np.zeros_like(Xp)
    for dy in range(3):
        for dx in range(3):
            dW[:, dy, dx, :] = np.einsum('bhwo,bhwc->oc', dY, Xp[:, dy:dy + H, dx:dx + Wd, :])
            dXp[:, dy:dy + H, dx:dx + Wd, :] += np.einsum('bhwo,oc->bhwc', dY, W[:, dy, dx, :])
    db = dY.sum(axis=(0, 1, 2))
    return dXp[:, 1:-1, 1:-1, :], dW, db


def forward(params, X, bf16=False):
    """Returns the output and the list of layer inputs (for backward)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    acts = []
    h = rnd(X)
    for l, (W, b) in enumerate(params):
        acts.append(h)
        y = conv3x3(h, rnd(W), b)
        if l < 3:
            h = rnd(np.maximum(y, 0.0))
        else:
            h = y
    return h, acts


def loss_and_grad(params, X, T, bf16=False):
    """Mean over samples of ||Y - T||^2 / ||T||^2, and its gradient (list of (dW, db))."""
    rnd = bf16_round if bf16 else (lambda a: a)
    Y, acts = forward(params, X, bf16)
    Bn = X.shape[0]
    num = ((Y - T) ** 2).sum(axis=(1, 2, 3))
    den = (T ** 2).sum(axis=(1, 2, 3))
    loss = float(np.mean(num / den))
    dY = 2.0 * (Y - T) / (den[:, None, None, None] * Bn)
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, b = params[l]
        if bf16:
            dY = bf16_round(dY)
        dX, dW, db = conv3x3_backward(acts[l], rnd(W), dY)
        grads[l] = (dW, db)
        if l > 0:
            dY = dX * (acts[l] > 0)
    return loss, grads


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on flat arrays; t is the 1-based step count."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
