"""Pipeline parity of the CUDA path against the CPU oracle: chi0 G (Alg. 1 and Alg. 3), chi G
(GMRES and Alg. 4), the dynamical matrix and the phonon frequencies, plus error handling.

The dynamical matrix of these chains is a cancellation of terms ~3e4 times larger than D itself,
so the FP64 bar (1e-8 relative Frobenius on D) needs Sternheimer and Dyson tolerances of 1e-13.
"""
import numpy as np
import pytest

import acp_workloads as W
from gpu_systems import context, model, rel, system, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sos():
    from oracle.chi0 import chi0_matrix_sos
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = chi0_matrix_sos(model(name))
        return cache[name]
    return get


@pytest.mark.parametrize("name", ["small4_160_0", "small6_240_1", "c1"])
def test_chi0_plain(name, sos):
    m = model(name)
    G, _ = m.perturbations()
    ctx = context(name, method=0, stern_tol=1e-13)
    U, st = ctx.apply_chi0(to_gpu(G))
    assert rel(to_np(U), sos(name) @ G * m.h) < 1e-10
    assert st["rhs_solved"] == m.n_orb * G.shape[1]


@pytest.mark.parametrize("name", ["small4_160_0", "small6_240_1"])
def test_chi0_acp(name):
    from oracle import acp as A
    m = model(name)
    G, _ = m.perturbations()
    om = W.srft_sketch(G.shape[1], 4, 0)
    for eps, nc in ((1e-4, 8), (1e-9, 16)):
        ctx = context(name, method=1, sketch=om, id_tol=eps, n_cheb=nc, stern_tol=1e-13)
        U, st = ctx.apply_chi0(to_gpu(G))
        ref = A.chi0_acp_apply(m, G, om, eps, nc, tol=1e-13)
        assert rel(to_np(U), ref) < 1e-9
        assert st["rhs_solved"] == st["n_mu"] * nc


@pytest.mark.parametrize("name", ["small4_160_0", "c1"])
def test_dyson_plain(name, sos):
    from oracle.dyson import dyson_dense
    m = model(name)
    G, _ = m.perturbations()
    ctx = context(name, method=0, stern_tol=1e-13, dyson_tol=1e-13, dyson_maxit=80)
    U, st = ctx.dyson_solve(to_gpu(G))
    assert rel(to_np(U), dyson_dense(m, G, sos(name))) < 1e-10


def test_dyson_acp_matches_oracle_alg4():
    from oracle import acp as A
    name = "small4_160_0"
    m = model(name)
    G, _ = m.perturbations()
    om = W.srft_sketch(G.shape[1], 4, 0)
    ctx = context(name, method=1, sketch=om, id_tol=1e-9, n_cheb=16, stern_tol=1e-13, dyson_tol=1e-12,
                  dyson_maxit=5)
    U, st = ctx.dyson_solve(to_gpu(G), allow_noconv=True)
    Uo, it = A.chi_acp(m, G, om, 1e-9, 16, delta=1e-12, maxit=5, tol=1e-13)
    assert st["outer_iters"] == it
    assert rel(to_np(U), Uo) < 1e-7


def test_dynamical_matrix_c1_fp64(sos):
    """Config 1: plain DFPT FP64 on the GPU matches the oracle D to 1e-8 (relative Frobenius)."""
    from oracle import dmat as Dm
    from oracle.dyson import dyson_dense
    import torch
    s, gs = system("c1")
    m = model("c1")
    G, _ = m.perturbations()
    D_ref, _ = Dm.dynamical_matrix(m, dyson_dense(m, G, sos("c1")))
    ctx = context("c1", method=0, stern_tol=1e-13, dyson_tol=1e-13, dyson_maxit=80)
    rho = torch.tensor(gs.rho, dtype=torch.float64, device="cuda")
    D, st = ctx.dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
    assert rel(D, D_ref) < 1e-8
    w = ctx.phonons(D)
    w_ref, _ = Dm.phonons(D_ref)
    assert np.abs(w - w_ref).max() <= 1e-5 * np.abs(w_ref).max()


def test_error_statuses():
    import torch
    import paper_1605_08021_gb300 as P
    name = "small4_160_0"
    s, gs = system(name)
    m = model(name)
    G, _ = m.perturbations()
    om = W.srft_sketch(G.shape[1], 4, 0)
    # G = 0: the pivoted QR has rank 0
    ctx = context(name, method=1, sketch=om)
    with pytest.raises(P.AcpError) as e:
        ctx.apply_chi0(torch.zeros((4, m.N), dtype=torch.float64, device="cuda"))
    assert e.value.name == "ACP_E_RANK"
    # NaN in the right-hand side
    ctx = context(name, method=0)
    Gn = G.copy()
    Gn[3, 1] = np.nan
    with pytest.raises(P.AcpError) as e:
        ctx.apply_chi0(to_gpu(Gn))
    assert e.value.name == "ACP_E_NUMERIC"
    # iteration cap
    ctx = context(name, method=0, stern_maxit=2)
    with pytest.raises(P.AcpError) as e:
        ctx.apply_chi0(to_gpu(G))
    assert e.value.name == "ACP_E_NOCONV"
    # eigenvalues not ascending
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), device="cuda")
    with pytest.raises(P.AcpError) as e:
        P.Context(m.N, m.L, s.kappa, s.scale, V, psi, gs.eps[: gs.n_orb][::-1].copy())
    assert e.value.name == "ACP_E_GAP"
    # unsupported grid size (7 is not a radix)
    with pytest.raises(P.AcpError) as e:
        P.Context(7 * 16, m.L, s.kappa, s.scale, torch.zeros(112, dtype=torch.float64, device="cuda"),
                  torch.zeros((2, 112), dtype=torch.float64, device="cuda"), np.array([0.0, 1.0]))
    assert e.value.name == "ACP_E_ARG"
    # empty input is a no-op
    ctx = context(name, method=0)
    U, _ = ctx.apply_chi0(torch.zeros((0, m.N), dtype=torch.float64, device="cuda"))
    assert U.shape == (0, m.N)


def test_deadline_returns_timeout_status():
    """deadline_s is checked on the host between launches (every 16 MINRES steps here): a call that
    overruns it returns ACP_E_TIMEOUT with its kernels finished, and the context stays usable."""
    import paper_1605_08021_gb300 as P
    name = "small4_160_0"
    m = model(name)
    G, _ = m.perturbations()
    ctx = context(name, method=0, deadline_s=1e-9)
    with pytest.raises(P.AcpError) as e:
        ctx.apply_chi0(to_gpu(G[:, :2]))
    assert e.value.name == "ACP_E_TIMEOUT"
    Y = to_np(ctx.hamiltonian_apply(to_gpu(G[:, :2])))
    assert rel(Y, m.apply_H(G[:, :2])) < 1e-12


def test_multishift_storage_variants_agree():
    """The stored-basis multi-shift solver and the per-shift-vector solver give the same chi0~ G."""
    name = "small6_240_1"
    m = model(name)
    G, _ = m.perturbations()
    om = W.srft_sketch(G.shape[1], 4, 0)
    kw = dict(method=1, sketch=om, id_tol=1e-9, n_cheb=16, stern_tol=1e-13)
    Ub, sb = context(name, ms_variant=1, **kw).apply_chi0(to_gpu(G))
    Uv, sv = context(name, ms_variant=2, **kw).apply_chi0(to_gpu(G))
    assert rel(to_np(Ub), to_np(Uv)) < 1e-11
    assert sb["rhs_solved"] == sv["rhs_solved"]


def test_contexts_of_different_grids_coexist():
    """The shared-memory limit of the spectral kernels is process-wide: a context on a small grid
    created after one on a large grid must not lower it below what the large grid needs."""
    m = model("c2")
    big = context("c2")
    small = context("small3_96_2")
    X = np.random.default_rng(7).standard_normal((m.N, 3))
    assert rel(to_np(big.hamiltonian_apply(to_gpu(X))), m.apply_H(X)) < 1e-12
    del small
