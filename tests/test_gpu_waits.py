"""Failure detection on the GPU without a fault: the bounded mbarrier waits of the tensor-core
projector GEMM run out on a barrier that nothing completes (its TMA loads are withheld), the kernel
frees its tensor memory and reports through the device status word, and the host returns
ACP_E_TIMEOUT with the context still usable.  Every wait is bounded, so the call ends by itself."""
import time

import numpy as np
import pytest

from gpu_systems import context, model, rel, to_gpu, to_np

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_stays_usable():
    m = model("small4_160_0")
    ctx = context("small4_160_0", precision=1)
    rng = np.random.default_rng(30)
    X = rng.standard_normal((m.N, 9))
    ref = m.project(X)
    assert rel(to_np(ctx.project_mixed(to_gpu(X))), ref) < 1e-6
    for wait_s in (0.05, 0.02):
        t0 = time.perf_counter()
        assert ctx.selftest_wait_timeout(wait_s) == "ACP_E_TIMEOUT"
        dt = time.perf_counter() - t0
        assert dt < 2.0, dt
        assert "timed out" in ctx.lib.acp_last_error(ctx.ptr).decode()
        # the status word was cleared and the tensor memory freed: the projector works again
        assert rel(to_np(ctx.project_mixed(to_gpu(X))), ref) < 1e-6
    assert ctx.selftest_wait_timeout(0.0) == "ACP_E_ARG"
    assert ctx.selftest_wait_timeout(2.0) == "ACP_E_ARG"
