"""Shared set-up of the GPU parity tests: seeded systems, their ground states, the oracle model and
a library context built from the same inputs."""
import functools

import numpy as np

import acp_workloads as W


@functools.lru_cache(maxsize=None)
def system(name):
    if name == "c1":
        s = W.config(1)
    elif name == "c2":
        s = W.config(2)
    elif name.startswith("small"):
        # small<atoms>_<grid>_<seed>
        a, n, seed = (int(x) for x in name[5:].split("_"))
        s = W.small_chain(a, n, seed)
    else:
        raise KeyError(name)
    gs = W.ground_state(s)
    return s, gs


def model(name):
    from oracle.model import Model1D
    s, gs = system(name)
    return Model1D(s, gs)


def context(name, **opts):
    import torch

    import paper_1605_08021_gb300 as P
    s, gs = system(name)
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), dtype=torch.float64, device="cuda")
    o = P.options(occ=float(s.occ), **opts)
    ctx = P.Context(s.n[0], s.L[0], s.kappa, s.scale, V, psi, gs.eps[: gs.n_orb], o)
    return ctx


def to_gpu(X):
    """(N, m) numpy block -> (m, N) CUDA tensor."""
    import torch
    return torch.tensor(np.ascontiguousarray(np.asarray(X).T), dtype=torch.float64, device="cuda")


def to_np(T):
    return T.detach().cpu().numpy().T


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
