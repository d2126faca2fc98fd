"""Stage parity of the CUDA path against the CPU oracle (FP64, element by element).

Sizes cover several GEMM/FFT tiles and ragged tails: grids 96 (2^5 3), 160 (2^5 5), 240 (2^4 3 5)
and 320 (4^3 5); orbital counts 5, 8 and 11; odd column counts exercise the packed pair of the
spectral kernel with a missing partner.  Tolerances: spectral and GEMM stages are exact up to
rounding (1e-12 relative); Krylov solutions follow from residual tolerances times the
condition number (<= 3e3 here), so 1e-9.
"""
import numpy as np
import pytest

from gpu_systems import context, model, rel, system, to_gpu, to_np

pytestmark = pytest.mark.gpu

SYSTEMS = ["small3_96_2", "small4_160_0", "small6_240_1", "c1"]


@pytest.fixture(scope="module", params=SYSTEMS)
def sysname(request):
    return request.param


def test_hamiltonian_apply(sysname):
    m = model(sysname)
    ctx = context(sysname)
    rng = np.random.default_rng(0)
    for ncol in (1, 7, 16):
        X = rng.standard_normal((m.N, ncol))
        sh = rng.standard_normal(ncol)
        Y = to_np(ctx.hamiltonian_apply(to_gpu(X), sh))
        assert rel(Y, m.apply_H(X, sh)) < 1e-12
        Y0 = to_np(ctx.hamiltonian_apply(to_gpu(X)))
        assert rel(Y0, m.apply_H(X)) < 1e-12


def test_kernel_apply(sysname):
    m = model(sysname)
    ctx = context(sysname)
    X = np.random.default_rng(1).standard_normal((m.N, 5))
    assert rel(to_np(ctx.kernel_apply(to_gpu(X))), m.apply_K(X)) < 1e-12
    assert rel(to_np(ctx.kernel_apply(to_gpu(X), inverse=True)), m.apply_Kinv(X)) < 1e-12


def test_project(sysname):
    m = model(sysname)
    ctx = context(sysname)
    X = np.random.default_rng(2).standard_normal((m.N, 9))
    Y = to_np(ctx.project(to_gpu(X)))
    assert rel(Y, m.project(X)) < 1e-12
    assert np.abs(m.psi.T @ Y * m.h).max() < 1e-12 * np.abs(X).max()


def test_perturbations(sysname):
    s, gs = system(sysname)
    m = model(sysname)
    ctx = context(sysname)
    G, B, D2 = (to_np(t) for t in ctx.perturbations(s.R[:, 0], s.Z, s.sigma))
    Go, Bo = m.perturbations()
    assert rel(G, Go) < 1e-11
    assert rel(B, Bo) < 1e-11
    assert rel(D2, m.second_derivatives()) < 1e-11


def test_sternheimer_solve(sysname):
    from oracle.chi0 import sternheimer_operator
    from oracle.minres import minres
    m = model(sysname)
    ctx = context(sysname, stern_tol=1e-13)
    rng = np.random.default_rng(3)
    Bm = rng.standard_normal((m.N, 5))
    shifts = m.eps[rng.integers(0, m.n_orb, 5)]
    X, st = ctx.sternheimer_solve(to_gpu(Bm), shifts)
    X = to_np(X)
    A = sternheimer_operator(m)
    QB = m.project(Bm)
    res = np.linalg.norm(A(X, shifts) - QB, axis=0) / np.linalg.norm(QB, axis=0)
    assert res.max() < 1e-11
    Xo = minres(A, QB, shifts, tol=1e-13)
    assert rel(X, Xo) < 1e-9
    assert st["rhs_solved"] == 5


def test_compress_matches_oracle(sysname):
    import acp_workloads as W
    from oracle import acp as A
    m = model(sysname)
    G, _ = m.perturbations()
    om = W.srft_sketch(G.shape[1], 4, 0)
    for eps in (1e-3, 1e-8):
        ctx = context(sysname, sketch=om, id_tol=eps)
        k, piv, Xi, rd = ctx.compress(to_gpu(G))
        ref = A.interpolative_decomposition(m, G, om, eps)
        assert k == ref.pivots.size
        assert np.array_equal(piv, ref.pivots)
        assert np.allclose(rd, ref.Rdiag[:k], rtol=1e-10)
        # Xi = R11^{-1} R12: forward error <= cond(R11) n u with cond(R11) <= 1/eps
        assert rel(to_np(Xi), ref.Xi) < 10 * k * 1.1e-16 / eps


def test_phonon_eigensolver():
    ctx = context("small4_160_0")
    rng = np.random.default_rng(4)
    for n in (1, 8, 37, 128):
        A = rng.standard_normal((n, n))
        D = A + A.T
        w, V = ctx.phonons(D, modes=True)
        lam = np.linalg.eigvalsh(D)
        assert np.allclose(np.sign(w) * w ** 2, lam, atol=1e-12 * np.abs(lam).max())
        assert np.allclose(D @ V, V * (np.sign(w) * w ** 2), atol=1e-10 * np.abs(lam).max())
