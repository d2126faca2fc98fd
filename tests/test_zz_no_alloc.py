"""The projector entry point that allocates no device memory (acp_project_noalloc) gives the same
Y = Q X as the context's projector (acp_project), on two calls in a row that share its fixed
scratch array, and rejects sizes beyond that array.

It is called through the C ABI directly, with the orbitals, inputs and outputs in caller-owned
device memory.  The bar is the one of the FP64 projector tests: equal up to rounding, 1e-12.
"""
import ctypes

import numpy as np
import pytest

from gpu_systems import context, model, rel, to_gpu, to_np

pytestmark = pytest.mark.gpu

MAX_ELEMS = 1 << 20  # n_orb * ncol capacity of the fixed scratch array


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("name", ["small6_240_1", "c1"])
def test_project_noalloc_matches_project(name):
    import torch

    import paper_1605_08021_gb300 as P
    lib = P.load()
    m = model(name)
    ctx = context(name)
    psi = to_gpu(m.psi)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(17)
    for ncol in (37, 5):  # two calls in a row; the second reuses the scratch the first left behind
        X = to_gpu(rng.standard_normal((m.N, ncol)))
        Y = torch.empty_like(X)
        st = lib.acp_project_noalloc(_ptr(psi), m.N, m.n_orb, m.h, _ptr(X), ncol, _ptr(Y), stream)
        assert st == 0
        torch.cuda.synchronize()
        assert rel(to_np(Y), to_np(ctx.project(X))) < 1e-12


def test_project_noalloc_in_place_and_limits():
    import torch

    import paper_1605_08021_gb300 as P
    lib = P.load()
    name = "c1"
    m = model(name)
    ctx = context(name)
    psi = to_gpu(m.psi)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    X = to_gpu(np.random.default_rng(18).standard_normal((m.N, 9)))
    ref = to_np(ctx.project(X))
    assert lib.acp_project_noalloc(_ptr(psi), m.N, m.n_orb, m.h, _ptr(X), 9, _ptr(X), stream) == 0
    torch.cuda.synchronize()
    assert rel(to_np(X), ref) < 1e-12
    # beyond the scratch array: a clear argument error, nothing enqueued
    too_many = MAX_ELEMS // m.n_orb + 1
    assert lib.acp_project_noalloc(_ptr(psi), m.N, m.n_orb, m.h, _ptr(X), too_many, _ptr(X), stream) == 1
    assert lib.acp_project_noalloc(None, m.N, m.n_orb, m.h, _ptr(X), 9, _ptr(X), stream) == 1
    assert lib.acp_project_noalloc(_ptr(psi), m.N, m.n_orb, m.h, _ptr(X), 0, _ptr(X), stream) == 0
