"""Seeded weights of the learned initial guess (4-layer periodic CNN, channels 2 -> 32 -> 32 ->
32 -> 1, 3 x 3 kernels) in the packed order of the library: W1 (32,2,3,3), b1, W2 (32,32,3,3), b2,
W3 (32,32,3,3), b3, W4 (1,32,3,3), b4, each row-major, as FP32.

Weights are drawn as Gaussians with standard deviation gain / sqrt(9 c_in) and biases with
standard deviation 0.1 (a variance-preserving start for tanh layers); nothing here evaluates the
network."""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 32, 32, 1)


def pack(params) -> np.ndarray:
    """[(W, b), ...] -> one FP32 vector in the library's order."""
    return np.concatenate([np.concatenate([np.asarray(W).ravel(), np.asarray(b).ravel()]) for W, b in params]) \
        .astype(np.float32)


def unpack(w) -> list:
    """FP32 vector -> [(W, b), ...] as FP64 arrays holding the FP32 values."""
    w = np.asarray(w, dtype=np.float32).astype(np.float64)
    out, k = [], 0
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        W = w[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = w[k:k + co]
        k += co
        out.append((W.copy(), b.copy()))
    if k != w.size:
        raise ValueError(f"expected {k} weights, got {w.size}")
    return out


def init_weights(seed: int, gain: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(10_000 + seed)
    params = [(rng.standard_normal((co, ci, 3, 3)) * gain / np.sqrt(9 * ci), 0.1 * rng.standard_normal(co))
              for ci, co in zip(CHANNELS[:-1], CHANNELS[1:])]
    return pack(params)
