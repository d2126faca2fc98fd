"""The learned initial guess of the 2D Sternheimer solves (4-layer periodic CNN, bfloat16 weights,
FP32 activations and accumulation) against the oracle's network (``oracle/cnn.py``) evaluated in
FP64 on the same bfloat16-rounded weights.

Bar for the network output: the device rounds its inputs to FP32 (relative 6e-8), accumulates
each of its 32-channel layers over 288 products in FP32 (~sqrt(288) x 6e-8 ~ 1e-6 relative per
layer) and evaluates tanh in FP32; over four layers of unit gain that stays below 2e-5 relative.
Solves started from the guess refine to the same tolerance as solves started from zero, so the
solutions agree to the Krylov bar of the other 2D tests (1e-8).

Grids: 32 x 32 (two full tiles of 16 per axis), 30 x 30 and 36 x 36 (ragged last tiles), and
40 x 24 (nx != ny, ragged in both directions).
"""
import numpy as np
import pytest

import acp_workloads as W
from gpu_systems import context, model, rel, to_gpu, to_np

pytestmark = pytest.mark.gpu

SYSTEMS = ["lat2x2_32_0", "lat2x2_30_1", "latz3x2_36_2", "rect2x2_40x24_0"]


@pytest.mark.parametrize("name", SYSTEMS)
def test_cnn_apply_matches_oracle(name):
    from oracle import cnn as C
    m = model(name)
    ctx = context(name)
    w = W.learned.init_weights(1)
    ctx.cnn_set_weights(w)
    params = W.learned.unpack(w)
    rng = np.random.default_rng(30)
    R = rng.standard_normal((m.N, 4))
    R[:, 2] = 0.0
    shifts = m.eps[rng.integers(0, m.n_orb, 4)]
    X0 = to_np(ctx.cnn_apply(to_gpu(R), shifts))
    for j in range(4):
        ref = C.forward(params, R[:, j].reshape(m.ny, m.nx), (m.V - shifts[j]).reshape(m.ny, m.nx),
                        bf16=True).reshape(-1)
        if j == 2:
            assert not np.any(X0[:, j])
        else:
            assert rel(X0[:, j], ref) < 2e-5, j


def test_learned_start_gives_the_same_solution():
    from oracle.chi0 import sternheimer_operator
    from oracle.minres import minres
    name = "lat2x2_30_1"
    m = model(name)
    rng = np.random.default_rng(31)
    Bm = rng.standard_normal((m.N, 5))
    shifts = m.eps[rng.integers(0, m.n_orb, 5)]
    ctx = context(name, stern_tol=1e-12, precision=1, learned=1)
    ctx.cnn_set_weights(W.learned.init_weights(2, gain=0.5))
    X1, st1 = ctx.sternheimer_solve(to_gpu(Bm), shifts)
    X0, st0 = context(name, stern_tol=1e-12, precision=1).sternheimer_solve(to_gpu(Bm), shifts)
    assert st1["rhs_solved"] == 5 and st0["rhs_solved"] == 5
    A = sternheimer_operator(m)
    QB = m.project(Bm)
    Xo = minres(A, QB, shifts, tol=1e-13)
    assert rel(to_np(X1), Xo) < 1e-8
    assert rel(to_np(X1), to_np(X0)) < 1e-8


def test_learned_form_argument_errors():
    import torch

    import paper_1605_08021_gb300 as P
    name = "lat2x2_32_0"
    m = model(name)
    B = torch.zeros((2, m.N), dtype=torch.float64, device="cuda")
    B[0, 3] = 1.0
    # learned start without weights: the solve refuses instead of starting from zero
    ctx = context(name, precision=1, learned=1)
    with pytest.raises(P.AcpError) as e:
        ctx.sternheimer_solve(B, m.eps[:2])
    assert e.value.name == "ACP_E_ARG"
    with pytest.raises(P.AcpError) as e:
        ctx.cnn_set_weights(np.zeros(100, dtype=np.float32))
    assert e.value.name == "ACP_E_ARG"
    # the network is defined on 2D grids only
    ctx1 = context("small4_160_0")
    with pytest.raises(P.AcpError) as e:
        ctx1.cnn_set_weights(W.learned.init_weights(0))
    assert e.value.name == "ACP_E_ARG"


def test_training_step_matches_oracle():
    """One training step on the context's own grid: the loss and its gradient against the
    oracle's backward pass (FP64 on the same FP32 master weights; the device runs the forward and
    data-gradient passes in FP32 and sums weight gradients in FP64: 1e-5 on the loss, 1e-4 on the
    gradient); the Adam update against the oracle's Adam fed the device gradient (FP32 update
    arithmetic, 1e-6 absolute); the inference copies follow the new weights; and repeated steps
    lower the loss."""
    from oracle import cnn as C
    name = "rect2x2_40x24_0"
    m = model(name)
    ctx = context(name)
    w = W.learned.init_weights(3)
    ctx.cnn_set_weights(w)
    rng = np.random.default_rng(32)
    S = 3
    R = rng.standard_normal((m.N, S))
    R[:, 1] = 0.0
    shifts = m.eps[rng.integers(0, m.n_orb, S)]
    Xs = rng.standard_normal((m.N, S))
    VS = m.V[:, None] - shifts[None, :]
    grid = (m.nx, m.ny)
    loss, g = ctx.cnn_train_step(grid, to_gpu(R), to_gpu(VS), to_gpu(Xs), lr=1e-3, return_grad=True)
    params = W.learned.unpack(w)
    samples = [(R[:, s].reshape(m.ny, m.nx), (m.V - shifts[s]).reshape(m.ny, m.nx), Xs[:, s].reshape(m.ny, m.nx))
               for s in range(S)]
    Lo, go = C.loss_and_grads(params, samples)
    assert abs(loss - Lo) <= 1e-5 * Lo
    g_ref = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in go])
    assert rel(g.astype(np.float64), g_ref) < 1e-4
    w1 = ctx.cnn_get_weights()
    ref = C.Adam(lr=1e-3).step([w.astype(np.float64)], [g.astype(np.float64)])[0]
    assert np.abs(w1 - ref).max() < 1e-6
    # the bfloat16 inference copies are rebuilt from the new master weights
    X0 = to_np(ctx.cnn_apply(to_gpu(R[:, :1]), shifts[:1]))[:, 0]
    x_ref = C.forward(W.learned.unpack(w1), R[:, 0].reshape(m.ny, m.nx), (m.V - shifts[0]).reshape(m.ny, m.nx),
                      bf16=True).reshape(-1)
    assert rel(X0, x_ref) < 2e-5
    losses = [ctx.cnn_train_step(grid, to_gpu(R), to_gpu(VS), to_gpu(Xs), lr=1e-3) for _ in range(20)]
    assert losses[-1] < loss


def test_training_on_another_grid():
    """A batch on a grid other than the context's (7 x 5 here: every point's neighbourhood wraps)
    trains the same weights; loss and gradient as in the oracle."""
    from oracle import cnn as C
    ctx = context("lat2x2_32_0")
    w = W.learned.init_weights(4)
    ctx.cnn_set_weights(w)
    rng = np.random.default_rng(33)
    nx, ny, S = 7, 5, 2
    R = rng.standard_normal((nx * ny, S))
    VS = rng.standard_normal((nx * ny, S))
    Xs = rng.standard_normal((nx * ny, S))
    loss, g = ctx.cnn_train_step((nx, ny), to_gpu(R), to_gpu(VS), to_gpu(Xs), lr=0.0, return_grad=True)
    samples = [(R[:, s].reshape(ny, nx), VS[:, s].reshape(ny, nx), Xs[:, s].reshape(ny, nx)) for s in range(S)]
    Lo, go = C.loss_and_grads(W.learned.unpack(w), samples)
    assert abs(loss - Lo) <= 1e-5 * Lo
    assert rel(g.astype(np.float64), np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in go])) < 1e-4
    assert np.array_equal(ctx.cnn_get_weights(), w)  # lr = 0 leaves the weights as they were


def test_trained_guess_cuts_krylov_steps():
    """The network trained on this library's own solutions (paper_1605_08021_gb300/weights, 200
    seeded lattices; the run's record is cnn_x0.json beside the weights) starts the solves of a
    lattice held out of training closer to the solution: fewer Lanczos steps than from zero, to the
    same stern_tol (1e-8) checked as a true FP64 residual of the oracle's operator, and the same
    solutions."""
    import os

    import torch

    import paper_1605_08021_gb300 as P
    from oracle.chi0 import sternheimer_operator
    from oracle.model import Model2D
    from paper_1605_08021_gb300.train_cnn import _context, _samples
    wdir = os.path.join(os.path.dirname(P.__file__), "weights")
    w = np.load(os.path.join(wdir, "cnn_x0.npy"))
    s = W.training_lattices(1, first=203)[0]  # systems 200-207 were held out of the training run
    gs = W.ground_state(s, tol=1e-8)
    rng = np.random.default_rng(7)
    R, _, X0, shifts, st0 = _samples(P, s, gs, 32, rng, 1e-8)
    ctx = _context(P, s, gs, stern_tol=1e-8, learned=1)
    ctx.cnn_set_weights(w)
    X1, st1 = ctx.sternheimer_solve(R, shifts)
    torch.cuda.synchronize()
    assert st0["rhs_solved"] == 32 and st1["rhs_solved"] == 32
    assert st1["lanczos_steps"] <= 0.97 * st0["lanczos_steps"], (st1["lanczos_steps"], st0["lanczos_steps"])
    m = Model2D(s, gs)
    A = sternheimer_operator(m)
    Rn, X0n, X1n = to_np(R), to_np(X0), to_np(X1)
    for X in (X0n, X1n):
        res = np.linalg.norm(A(X, shifts) - Rn, axis=0) / np.linalg.norm(Rn, axis=0)
        assert res.max() < 2e-8
    assert rel(X1n, X0n) < 1e-6
