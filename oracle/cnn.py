"""Learned initial guess for the 2D Sternheimer solves: a 4-layer periodic CNN (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The shifted Sternheimer solves of Alg. 3 (Q(H - s)Q x = Q b on the 2D grid, Eq. eqncompressU)
start their Krylov iteration from an initial guess x0.  The solves are refined to the same
tolerance whatever x0 is, so x0 changes iteration counts, not results.  This module defines the
network that proposes x0 and what training it needs, in plain FP64 numpy:

* fields are arrays (C, ny, nx) with x fastest (grid index ix + nx iy);
* one layer: z_o = b_o + sum_c W_oc (*) a_c with the 3 x 3 periodic cross-correlation
  (W (*) a)[i, j] = sum_{p, q in {-1, 0, 1}} W[p + 1, q + 1] a[(i + p) mod ny, (j + q) mod nx],
  then tanh on layers 1-3; channels 2 -> 32 -> 32 -> 32 -> 1;
* inputs: channel 0 = r / rms(r) (right-hand side or residual), channel 1 = V_eff - s (the
  shifted potential); output x0 = rms(r) net(r / rms(r), V_eff - s), so x0 is homogeneous of
  degree one in r (r = 0 gives x0 = 0);
* training loss on solved systems: mean over samples of ||x0 - x*||^2 / ||x*||^2, x* the
  solution;
* the device keeps FP32 master weights and convolves with bfloat16 copies: ``to_bf16`` rounds
  the same way, and ``forward(..., bf16=True)`` evaluates the network on the rounded weights
  (biases stay FP32 on the device);
* Adam (Kingma and Ba, 2015: first and second moment estimates with bias correction) updates
  the FP64 master weights.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 32, 32, 1)


def to_bf16(x):
    """The device's weight rounding: to FP32 (its master copy), then to the nearest bfloat16
    (8 exponent bits, 7 stored mantissa bits; ties to even) by rounding away the low 16 bits of
    the FP32 pattern.  Finite inputs only."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(a, W, b):
    """z[o] = b[o] + sum_c sum_{p,q} W[o, c, p+1, q+1] a[c, (i+p) mod ny, (j+q) mod nx]."""
    O = W.shape[0]
    z = np.broadcast_to(np.asarray(b, dtype=np.float64)[:, None, None], (O,) + a.shape[1:]).copy()
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            shifted = np.roll(a, shift=(-p, -q), axis=(1, 2))  # shifted[c, i, j] = a[c, i+p, j+q]
            z += np.einsum("oc,cij->oij", W[:, :, p + 1, q + 1], shifted)
    return z


def conv3x3_backward(a, W, g):
    """Gradients of sum(g * conv3x3(a, W, b)) with respect to a, W and b."""
    dW = np.empty_like(W)
    da = np.zeros_like(a)
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            shifted = np.roll(a, shift=(-p, -q), axis=(1, 2))
            dW[:, :, p + 1, q + 1] = np.einsum("oij,cij->oc", g, shifted)
            # z[o, i, j] gets W a[c, i+p, j+q]: a[c, k, l] receives g[o, k-p, l-q]
            da += np.einsum("oc,oij->cij", W[:, :, p + 1, q + 1], np.roll(g, shift=(p, q), axis=(1, 2)))
    db = g.sum(axis=(1, 2))
    return da, dW, db


def rms(r):
    return float(np.sqrt(np.mean(np.asarray(r, dtype=np.float64) ** 2)))


def forward(params, r, vs, bf16=False, return_cache=False):
    """x0 for one right-hand side.  params: [(W1, b1), ..., (W4, b4)]; r, vs: (ny, nx)."""
    s = rms(r)
    if s == 0.0:
        out = np.zeros_like(np.asarray(r, dtype=np.float64))
        return (out, None) if return_cache else out
    a = np.stack([np.asarray(r, dtype=np.float64) / s, np.asarray(vs, dtype=np.float64)])
    acts = [a]
    n = len(params)
    for l, (W, b) in enumerate(params):
        z = conv3x3(a, to_bf16(W) if bf16 else W, b)
        a = np.tanh(z) if l < n - 1 else z
        acts.append(a)
    out = s * a[0]
    if return_cache:
        return out, (s, acts)
    return out


def backward(params, cache, g_out):
    """Gradients of sum(g_out * x0) with respect to every (W, b) (FP64 weights)."""
    s, acts = cache
    n = len(params)
    g = (s * g_out)[None]
    grads = [None] * n
    for l in range(n - 1, -1, -1):
        W, _ = params[l]
        if l < n - 1:
            g = g * (1.0 - acts[l + 1] ** 2)  # tanh' = 1 - tanh^2
        da, dW, db = conv3x3_backward(acts[l], W, g)
        grads[l] = (dW, db)
        g = da
    return grads


def loss_and_grads(params, samples):
    """Mean relative squared error over samples [(r, vs, x_star), ...] and its gradients."""
    total = 0.0
    acc = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    m = len(samples)
    for r, vs, xs in samples:
        x0, cache = forward(params, r, vs, return_cache=True)
        nrm = float(np.sum(xs ** 2))
        d = x0 - xs
        total += float(np.sum(d ** 2)) / nrm / m
        if cache is None:
            continue
        gr = backward(params, cache, 2.0 * d / nrm / m)
        for k, (dW, db) in enumerate(gr):
            acc[k] = (acc[k][0] + dW, acc[k][1] + db)
    return total, acc


class Adam:
    """Adam on a list of arrays: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr mhat / (sqrt(vhat) + eps), mhat = m / (1-b1^t), vhat = v / (1-b2^t)."""

    def __init__(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.t = 0
        self.m = None
        self.v = None

    def step(self, theta, grads):
        if self.m is None:
            self.m = [np.zeros_like(x) for x in theta]
            self.v = [np.zeros_like(x) for x in theta]
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for i, (x, g) in enumerate(zip(theta, grads)):
            self.m[i] = self.b1 * self.m[i] + (1.0 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1.0 - self.b2) * g * g
            out.append(x - self.lr * (self.m[i] / c1) / (np.sqrt(self.v[i] / c2) + self.eps))
        return out


def flatten(params):
    return [x for Wb in params for x in Wb]


def unflatten(flat):
    return [(flat[2 * i], flat[2 * i + 1]) for i in range(len(flat) // 2)]
