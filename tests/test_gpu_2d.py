"""The 2D model on the GPU (multi-pass 2D FFTs in FP64 and FP32, 2D perturbations, the spectral
ion-ion Hessian, D in 2D) against the oracle's Model2D, element by element.

Systems: 2 x 2 lattices of mixed charges on 32 x 32 (radix 4, 2) and 30 x 30 (radices 2, 3, 5)
grids, and a 3 x 2 lattice of Z = 2 atoms (occupation 2) in a rectangular box (hx != hy).  Bars as in 1D: spectral stages and
perturbations to rounding (1e-12, 1e-11), Krylov solutions to the residual tolerance times the
condition number (1e-9), D of the FP64 and mixed forms within 1e-8 of the oracle's exact D.
"""
import numpy as np
import pytest

import acp_workloads as W
from gpu_systems import context, model, rel, system, to_gpu, to_np

pytestmark = pytest.mark.gpu

SYSTEMS = ["lat2x2_32_0", "lat2x2_30_1", "latz3x2_36_2"]


@pytest.mark.parametrize("name", SYSTEMS)
@pytest.mark.parametrize("passes", [0, 1])
def test_hamiltonian_and_kernel_2d(name, passes):
    """Both transforms: one column pair per CTA in shared memory (passes = 0 on these grids) and
    the row / column passes through device memory (passes = 1)."""
    m = model(name)
    ctx = context(name, fft2d_passes=passes)
    rng = np.random.default_rng(0)
    for ncol in (1, 5, 8):
        X = rng.standard_normal((m.N, ncol))
        sh = rng.standard_normal(ncol)
        assert rel(to_np(ctx.hamiltonian_apply(to_gpu(X), sh)), m.apply_H(X, sh)) < 1e-12
    X = rng.standard_normal((m.N, 3))
    assert rel(to_np(ctx.kernel_apply(to_gpu(X))), m.apply_K(X)) < 1e-12
    assert rel(to_np(ctx.kernel_apply(to_gpu(X), inverse=True)), m.apply_Kinv(X)) < 1e-12


@pytest.mark.parametrize("name", SYSTEMS)
def test_perturbations_2d(name):
    s, gs = system(name)
    m = model(name)
    ctx = context(name)
    G, B, D2 = (to_np(t) for t in ctx.perturbations(s.R, s.Z, s.sigma))
    Go, Bo = m.perturbations()
    assert rel(G, Go) < 1e-11
    assert rel(B, Bo) < 1e-11
    blk = m.second_derivative_blocks()
    ref = np.stack([blk[:, :, 0, 0], blk[:, :, 0, 1], blk[:, :, 1, 1]], axis=2).reshape(m.N, -1)
    assert rel(D2, ref) < 1e-11


@pytest.mark.parametrize("precision,passes", [(0, 0), (1, 0), (1, 1)])
def test_sternheimer_2d(precision, passes):
    from oracle.chi0 import sternheimer_operator
    from oracle.minres import minres
    name = "lat2x2_30_1"
    m = model(name)
    ctx = context(name, stern_tol=1e-12, precision=precision, fft2d_passes=passes)
    rng = np.random.default_rng(3)
    Bm = rng.standard_normal((m.N, 5))
    shifts = m.eps[rng.integers(0, m.n_orb, 5)]
    X, st = ctx.sternheimer_solve(to_gpu(Bm), shifts)
    A = sternheimer_operator(m)
    QB = m.project(Bm)
    Xo = minres(A, QB, shifts, tol=1e-13)
    assert rel(to_np(X), Xo) < 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_chi0_2d(precision):
    from oracle import acp as A
    from oracle.chi0 import chi0_matrix_sos
    name = "lat2x2_32_0"
    m = model(name)
    G, _ = m.perturbations()
    ctx = context(name, method=0, stern_tol=1e-12, precision=precision)
    U, st = ctx.apply_chi0(to_gpu(G))
    assert rel(to_np(U), chi0_matrix_sos(m) @ G * m.h) < 1e-9
    om = W.srft_sketch(G.shape[1], 4, 0)
    ctx = context(name, method=1, sketch=om, id_tol=1e-9, n_cheb=16, stern_tol=1e-12, precision=precision)
    U, st = ctx.apply_chi0(to_gpu(G))
    ref = A.chi0_acp_apply(m, G, om, 1e-9, 16, tol=1e-13)
    assert rel(to_np(U), ref) < 1e-8


@pytest.mark.parametrize("name,precision", [("lat2x2_32_0", 0), ("latz3x2_36_2", 0), ("lat2x2_32_0", 1)])
def test_dynamical_matrix_2d(name, precision):
    import torch
    from oracle import dmat as Dm
    from oracle.chi0 import chi0_matrix_sos
    from oracle.dyson import dyson_dense
    s, gs = system(name)
    m = model(name)
    G, _ = m.perturbations()
    D_ref, _ = Dm.dynamical_matrix(m, dyson_dense(m, G, chi0_matrix_sos(m)))
    # the mixed form's refinement bottoms out near 4e-13 on these grids (FP32 projection residue)
    tol = 1e-13 if precision == 0 else 1e-12
    ctx = context(name, method=0, stern_tol=tol, dyson_tol=tol, dyson_maxit=80, precision=precision)
    rho = torch.tensor(gs.rho, dtype=torch.float64, device="cuda")
    D, st = ctx.dynamical_matrix(s.R, s.Z, s.sigma, rho)
    assert D.shape == (2 * s.n_atoms, 2 * s.n_atoms)
    assert rel(D, D_ref) < 1e-8
    w = ctx.phonons(D)
    w_ref, _ = Dm.phonons(D_ref)
    assert np.abs(w - w_ref).max() <= 1e-5 * np.abs(w_ref).max()
