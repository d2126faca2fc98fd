"""Mixed precision against the FP64 oracle: FP32 Krylov vectors and FFTs, the projector Q on the
tensor cores (3xTF32 tcgen05 GEMMs with FP32 accumulation), and FP64 iterative refinement.

* The tensor-core projector alone: FP32 inputs carry a relative rounding of 6e-8 and the FP32
  accumulation over K <= 5120 terms adds at most ~1e-6 relative, so Y = Q X must match the FP64
  projection to 2e-6 and leave occupied components below 1e-6 of the input.
* Solves and pipelines: refinement drives the FP64 residual to the requested tolerance, so the
  bars are those of the FP64 path (Krylov solutions: residual tolerance times the condition
  number).
"""
import os

import numpy as np
import pytest

import acp_workloads as W
from gpu_systems import context, model, rel, system, to_gpu, to_np

pytestmark = pytest.mark.gpu

MIXED = 1


@pytest.mark.parametrize("name", ["small3_96_2", "small6_240_1", "c1", "c2"])
def test_project_mixed(name):
    m = model(name)
    ctx = context(name)
    rng = np.random.default_rng(11)
    for ncol in (1, 7, 130, 300):
        X = rng.standard_normal((m.N, ncol))
        Y = to_np(ctx.project_mixed(to_gpu(X)))
        assert rel(Y, m.project(X)) < 2e-6
        assert np.abs(m.psi.T @ Y * m.h).max() < 1e-6 * np.abs(X).max()


def test_project_mixed_orbital_products():
    """Products psi_i * g (the right-hand sides of Alg. 1) lie mostly in the occupied space, so the
    projection cancels ~3 digits; the result still stays within FP32 of the FP64 one."""
    name = "c1"
    m = model(name)
    ctx = context(name)
    G, _ = m.perturbations()
    P = (m.psi[:, :, None] * G[:, None, :]).reshape(m.N, -1)
    Y = to_np(ctx.project_mixed(to_gpu(P)))
    err = np.linalg.norm(Y - m.project(P), axis=0) / np.linalg.norm(P, axis=0)
    assert err.max() < 2e-6


@pytest.mark.parametrize("name", ["small3_96_2", "small6_240_1", "c1"])
def test_sternheimer_mixed(name):
    from oracle.chi0 import sternheimer_operator
    from oracle.minres import minres
    m = model(name)
    ctx = context(name, stern_tol=1e-12, precision=MIXED)
    rng = np.random.default_rng(3)
    Bm = rng.standard_normal((m.N, 5))
    shifts = m.eps[rng.integers(0, m.n_orb, 5)]
    ctx.profile(True)
    X, st = ctx.sternheimer_solve(to_gpu(Bm), shifts)
    tc = ctx.profile_get("tc_gemm")
    ctx.profile(False)
    assert tc["launches"] > 0
    X = to_np(X)
    A = sternheimer_operator(m)
    QB = m.project(Bm)
    res = np.linalg.norm(A(X, shifts) - QB, axis=0) / np.linalg.norm(QB, axis=0)
    assert res.max() < 1e-10
    Xo = minres(A, QB, shifts, tol=1e-13)
    assert rel(X, Xo) < 1e-8
    assert st["rhs_solved"] == 5


@pytest.mark.parametrize("name", ["small4_160_0", "c1"])
def test_chi0_plain_mixed(name):
    from oracle.chi0 import chi0_matrix_sos
    m = model(name)
    G, _ = m.perturbations()
    ctx = context(name, method=0, stern_tol=1e-12, precision=MIXED)
    U, st = ctx.apply_chi0(to_gpu(G))
    assert rel(to_np(U), chi0_matrix_sos(m) @ G * m.h) < 1e-9
    assert st["rhs_solved"] == m.n_orb * G.shape[1]


@pytest.mark.parametrize("name", ["small4_160_0", "small6_240_1"])
def test_chi0_acp_mixed(name):
    from oracle import acp as A
    m = model(name)
    G, _ = m.perturbations()
    om = W.srft_sketch(G.shape[1], 4, 0)
    ctx = context(name, method=1, sketch=om, id_tol=1e-9, n_cheb=16, stern_tol=1e-12, precision=MIXED)
    U, st = ctx.apply_chi0(to_gpu(G))
    ref = A.chi0_acp_apply(m, G, om, 1e-9, 16, tol=1e-13)
    assert rel(to_np(U), ref) < 1e-8
    assert st["rhs_solved"] == st["n_mu"] * 16


def test_dynamical_matrix_c1_mixed():
    """Config 1 plain DFPT with mixed-precision solves: D within 1e-8 of the oracle's exact D."""
    import torch
    from oracle import dmat as Dm
    from oracle.chi0 import chi0_matrix_sos
    from oracle.dyson import dyson_dense
    s, gs = system("c1")
    m = model("c1")
    G, _ = m.perturbations()
    D_ref, _ = Dm.dynamical_matrix(m, dyson_dense(m, G, chi0_matrix_sos(m)))
    ctx = context("c1", method=0, stern_tol=1e-13, dyson_tol=1e-13, dyson_maxit=80, precision=MIXED)
    rho = torch.tensor(gs.rho, dtype=torch.float64, device="cuda")
    D, st = ctx.dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
    assert rel(D, D_ref) < 1e-8
    w = ctx.phonons(D)
    w_ref, _ = Dm.phonons(D_ref)
    assert np.abs(w - w_ref).max() <= 1e-5 * np.abs(w_ref).max()


def test_c2_acp_mixed_matches_fp64():
    """Config 2, ACP: the mixed-precision form gives the FP64 form's D (same compression, same
    shifts; only the arithmetic of the solves differs, recovered to the same tolerance)."""
    import torch
    s, gs = system("c2")
    om = W.srft_sketch(s.n_pert, 8, 2)
    rho = torch.tensor(gs.rho, dtype=torch.float64, device="cuda")
    kw = dict(method=1, sketch=om, id_tol=1e-9, n_cheb=20, dyson_tol=1e-9, dyson_maxit=20, stern_tol=1e-11)
    D64, st64 = context("c2", **kw).dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
    D32, st32 = context("c2", precision=MIXED, **kw).dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
    assert abs(st32["n_mu"] - st64["n_mu"]) <= 0.02 * st64["n_mu"]
    assert rel(D32, D64) < 1e-6
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_exact_dmat.npz"))
    from oracle import dmat as DM
    assert rel(D32, ref["D"]) < 1e-5
    assert DM.phonon_error(D32, ref["D"], s.n_atoms, 1)[1] < 1e-5
