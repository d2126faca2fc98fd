"""1D grids beyond the 512-thread FFT plan: the spectral kernels run one transform per CTA of up to
1024 threads with five radix-2 butterflies per thread (every 2^a 3^b 5^c grid up to 10240 points;
36 of the 64 batched chains need it).

Systems: chains of the batched configuration (atoms every 10 bohr, Z in {1, 2}, occupation 1)
with ground states from the cached potentials:
* c4_35: 106 atoms, N = 4320 = 2^5 3^3 5 (the smallest such grid, a radix-2 stage of 2160
  butterflies: 448 threads);
* c4_20: 122 atoms, N = 5000 = 2^3 5^4 (512 threads);
* c4_15: 252 atoms, N = 10125 = 3^4 5^3 (odd, 1024 threads).

Bars as in the smaller stage tests: spectral operators and perturbations are exact up to rounding
(1e-12, 1e-11 relative); Krylov solutions follow from the residual tolerance times the condition
number (1e-9 FP64, 1e-8 mixed); the batched form reproduces single contexts to 1e-9 (same
arithmetic on another stream) and the mixed D the FP64 D to 1e-6 (same options; the Alg. 4
recompressions see iterates that differ at the Sternheimer tolerance, and with ~1000 pivots a near
tie may pick another pivot, which moves D by the compression error, id_tol = 1e-10 times the
cancellation in D); sampled columns of the batched D of c4_35 match the oracle's exact D
(tests/golden/c4_35_exact_dcols.npz, written by tests/golden/make_dcols_reference.py from the
oracle only) within the ACP error budget.
"""
import os

import numpy as np
import pytest

import acp_workloads as W
from gpu_systems import context, model, rel, system, to_gpu, to_np

pytestmark = pytest.mark.gpu

WIDE = ["c4_35", "c4_20", "c4_15"]


@pytest.mark.parametrize("name", WIDE)
def test_grid_needs_the_wide_plan(name):
    s, _ = system(name)
    n = s.n[0]
    # the narrow plan fits at most 512 threads x (4, 4, 3, 2) butterflies of radix (2, 3, 4, 5)
    m, rad = n, []
    for r, b in ((4, 3), (2, 4), (3, 4), (5, 2)):
        while m % r == 0:
            rad.append((r, b))
            m //= r
    assert m == 1
    assert max(-(-(n // r) // b) for r, b in rad) > 512


@pytest.mark.parametrize("name", WIDE)
def test_spectral_operators_wide(name):
    m = model(name)
    ctx = context(name)
    rng = np.random.default_rng(20)
    for ncol in (1, 7):
        X = rng.standard_normal((m.N, ncol))
        sh = rng.standard_normal(ncol)
        assert rel(to_np(ctx.hamiltonian_apply(to_gpu(X), sh)), m.apply_H(X, sh)) < 1e-12
        assert rel(to_np(ctx.kernel_apply(to_gpu(X))), m.apply_K(X)) < 1e-12
        assert rel(to_np(ctx.kernel_apply(to_gpu(X), inverse=True)), m.apply_Kinv(X)) < 1e-12


@pytest.mark.parametrize("name", WIDE)
def test_perturbations_wide(name):
    s, _ = system(name)
    m = model(name)
    G, B, D2 = (to_np(t) for t in context(name).perturbations(s.R[:, 0], s.Z, s.sigma))
    Go, Bo = m.perturbations()
    assert rel(G, Go) < 1e-11
    assert rel(B, Bo) < 1e-11
    assert rel(D2, m.second_derivatives()) < 1e-11


@pytest.mark.parametrize("name,precision", [("c4_35", 0), ("c4_35", 1), ("c4_15", 0), ("c4_15", 1)])
def test_sternheimer_wide(name, precision):
    from oracle.chi0 import sternheimer_operator
    from oracle.minres import minres
    m = model(name)
    ctx = context(name, stern_tol=1e-13 if precision == 0 else 1e-12, precision=precision)
    rng = np.random.default_rng(21)
    Bm = rng.standard_normal((m.N, 5))
    shifts = m.eps[rng.integers(0, m.n_orb, 5)]
    X, st = ctx.sternheimer_solve(to_gpu(Bm), shifts)
    X = to_np(X)
    A = sternheimer_operator(m)
    QB = m.project(Bm)
    res = np.linalg.norm(A(X, shifts) - QB, axis=0) / np.linalg.norm(QB, axis=0)
    assert res.max() < (1e-11 if precision == 0 else 1e-10)
    Xo = minres(A, QB, shifts, tol=1e-13)
    assert rel(X, Xo) < (1e-9 if precision == 0 else 1e-8)
    assert st["rhs_solved"] == 5


def test_dynamical_matrix_wide_batched_single_and_fp64():
    import torch

    import paper_1605_08021_gb300 as P
    names = ["c4_35", "c4_20"]
    kw = dict(method=1, id_tol=1e-10, n_cheb=24, dyson_tol=1e-11, dyson_maxit=30, stern_tol=1e-12)
    sysgs = [system(n) for n in names]
    sketches = [W.srft_sketch(s.n_pert, 4, 0) for s, _ in sysgs]
    rhos = [torch.tensor(gs.rho, dtype=torch.float64, device="cuda") for _, gs in sysgs]
    atoms = [(s.R[:, 0], s.Z, s.sigma) for s, _ in sysgs]
    streams = [torch.cuda.Stream() for _ in names]
    ctxs = []
    for n, om, st in zip(names, sketches, streams):
        ctxs.append(context(n, stream=st, sketch=om, precision=1, use_graphs=1, **kw))
    torch.cuda.synchronize()
    Ds, stats, status = P.batch_dynamical_matrix(ctxs, atoms, rhos, n_workers=2)
    torch.cuda.synchronize()
    assert status == ["ACP_OK"] * len(names), [c.lib.acp_last_error(c.ptr).decode() for c in ctxs]
    for n, om, (s, gs), D, rho in zip(names, sketches, sysgs, Ds, rhos):
        D1, _ = context(n, sketch=om, precision=1, **kw).dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
        assert rel(D, D1) < 1e-9
    s, gs = sysgs[0]
    D64, _ = context(names[0], sketch=sketches[0], precision=0, **kw).dynamical_matrix(s.R[:, 0], s.Z, s.sigma,
                                                                                      rhos[0])
    assert rel(Ds[0], D64) < 1e-6
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_35_exact_dcols.npz"))
    assert str(ref["key"]) == s.key()
    cols = ref["cols"]
    err = rel(Ds[0][:, cols], ref["D_cols"])
    print(f"c4_35 sampled columns of D: relative error {err:.3e}")
    assert err < 1e-6
