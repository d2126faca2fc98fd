"""Full-size checks on configuration 2 (1D chain, 128 atoms, N = 5120, 192 orbitals, 128
perturbations), in the launch configuration bench.py times.

* Plain path: sampled columns of U = chi G (GMRES per column is independent, so a column
  sample is an exact sub-problem) against the oracle's sum-over-states chi0 + GMRES.
* ACP: the dynamical matrix against the oracle's exact D (tests/golden/c2_exact_dmat.npz,
  written by tests/golden/make_c2_reference.py from the oracle only), within the 1e-5 relative
  phonon-frequency bar.  ACP is an approximation: its error budget is the Chebyshev
  interpolation error rho^-N_c with rho = a + sqrt(a^2 - 1), a = 1 + 2 gap / (eps_N - eps_1)
  (Sec. 3.1), amplified by the ~3e4-fold cancellation in D, plus the compression threshold.
* Properties that hold at any size: the interpolation property Xi(r_mu, :) = I of the
  full-size compression and N_mu between 3 and 8 times N_e (Table 2 reports 4-6 N_e).
"""
import os

import numpy as np
import pytest

import acp_workloads as W
from gpu_systems import context, model, rel, system, to_gpu, to_np

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_exact_dmat.npz")
SAMPLE = [0, 63, 127]


@pytest.fixture(scope="module")
def c2():
    s, gs = system("c2")
    return s, gs, model("c2")


def test_c2_plain_sampled_columns(c2):
    from oracle import chi0 as C
    from oracle.dyson import gmres_columns
    s, gs, m = c2
    G, _ = m.perturbations()
    Gs = G[:, SAMPLE]
    ctx = context("c2", method=0, stern_tol=1e-12, dyson_tol=1e-12, dyson_maxit=80)
    U, st = ctx.dyson_solve(to_gpu(Gs))
    spec = C.full_spectrum(m)

    def chi0(X):
        return C.chi0_apply_sos(m, X, spec)
    Uo, _ = gmres_columns(lambda V: V - chi0(m.apply_K(V)), chi0(Gs), tol=1e-13, maxit=120)
    assert rel(to_np(U), Uo) < 1e-9


def test_c2_compression_properties(c2):
    s, gs, m = c2
    G, _ = m.perturbations()
    om = W.srft_sketch(s.n_pert, 8, 2)
    ctx = context("c2", method=1, sketch=om, id_tol=1e-8)
    k, piv, Xi, rd = ctx.compress(to_gpu(G), cap=3072)
    Xi = to_np(Xi)
    assert np.array_equal(Xi[piv, :], np.eye(k))
    assert 3 * m.n_orb <= k <= 8 * m.n_orb
    # |R_mm| non-increasing up to the rounding of the downdated norms, and above the threshold
    assert np.all(rd[1:] <= rd[:-1] * (1 + 1e-8))
    assert rd[-1] >= 1e-8 * rd[0]


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="exact reference not generated")
@pytest.mark.parametrize("eps,nc,delta,precision,bound", [(1e-9, 20, 1e-8, 1, 1e-5), (1e-10, 24, 1e-11, 0, 1e-7)])
def test_c2_acp_dynamical_matrix_vs_exact(c2, eps, nc, delta, precision, bound):
    """The accelerated forms meet the 1e-5 relative phonon-frequency bar (frequencies with the
    acoustic sum rule imposed by projection, the reading Table 2 fixes; oracle.dmat.phonon_error)
    and D the same bound, at the benchmark's settings (mixed, N_c = 20) and at tighter FP64
    settings.  The error follows the Chebyshev interpolation budget rho^-N_c of Sec. 3.1 (rho =
    2.71 at this band and gap), amplified by the ~3e4-fold cancellation in D: measured D errors are
    5.7e-5 at N_c = 16 (the configuration's count, which misses the bar), 5.9e-7 at 20, 1.6e-8 at
    24."""
    import torch

    from oracle import dmat as DM
    s, gs, m = c2
    ref = np.load(GOLDEN)
    om = W.srft_sketch(s.n_pert, 8, 2)
    ctx = context("c2", method=1, sketch=om, id_tol=eps, n_cheb=nc, dyson_tol=delta, dyson_maxit=25,
                  precision=precision, stern_tol=1e-11)
    rho = torch.tensor(gs.rho, dtype=torch.float64, device="cuda")
    D, st = ctx.dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
    # interpolation error budget of Sec. 3.1 for this band and gap
    a = 1 + 2 * gs.gap / (gs.eps[gs.n_orb - 1] - gs.eps[0])
    rho_c = a + np.sqrt(a * a - 1)
    assert rho_c ** -nc < 1e-7
    _, err = DM.phonon_error(D, ref["D"], s.n_atoms, 1)
    assert err < bound
    assert rel(D, ref["D"]) < bound
    # the library's own eigensolver agrees with the oracle's on the same D
    w = ctx.phonons(D)
    assert np.abs(w - DM.phonons(D)[0]).max() <= 1e-10 * np.abs(w).max()
