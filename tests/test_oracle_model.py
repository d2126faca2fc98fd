"""Pins of the model layer (oracle O1) and of the ground-state input generator.

Each test fixes a convention against something outside the code under test: numbers the
paper prints, closed forms, brute-force sums or finite differences.
"""
import json
import os

import numpy as np
import pytest

import acp_workloads as W
from oracle.model import Model1D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "paper_1d_model.json")))["cases"])
def test_paper_worked_example(case):
    """Sec. 4.1: gap and density range of the 60-atom chain pin kernel, sign and occupation."""
    sysm = W.paper_chain(60, case["eps0"])
    gs = W.ground_state(sysm, use_cache=False, tol=1e-10)
    assert abs(gs.gap - case["gap"]) < 0.6e-4
    assert abs(gs.rho.min() - case["rho_min"]) < 0.6e-4
    assert abs(gs.rho.max() - case["rho_max"]) < 0.6e-4
    # charge neutrality and orbital normalisation
    h = sysm.h[0]
    assert abs(gs.rho.sum() * h - sysm.n_elec) < 1e-10
    assert np.allclose(gs.psi.T @ gs.psi * h, np.eye(gs.n_orb), atol=1e-12)


def _tiny_model(n_atoms=3, n=96, spacing=4.0, disp=0.2):
    rng = np.random.default_rng(3)
    s = W.chain_1d("tiny", n_atoms, spacing, rng.integers(1, 3, n_atoms).astype(float), 0.6, 0.05, 0.7, n,
                   occ=1, displacement=disp, rng=rng)
    return s, Model1D(s)


def test_kernel_symbol_matches_real_space_yukawa():
    """Khat = 4 pi s/(k^2 + kappa^2) is the Fourier transform of 2 pi s exp(-kappa|x|)/kappa (Eq. yukawa)."""
    s, m = _tiny_model(n=2048)
    x = np.arange(m.N) * m.h
    # brute-force periodic image sum of the real-space kernel
    Kx = sum(2 * np.pi * s.scale / s.kappa * np.exp(-s.kappa * np.abs(x + n * m.L)) for n in range(-400, 401))
    assert np.allclose(m._kper(x), Kx, rtol=1e-12)
    coeff = np.real(np.fft.fft(Kx)) * m.h
    low = np.abs(m.k) < 0.05 * np.abs(m.k).max()
    assert np.allclose(coeff[low], m.khat[low], rtol=3e-3)
    # the ODE -K'' + kappa^2 K = 4 pi s delta in Fourier form, and K'' = kappa^2 K away from 0
    assert np.allclose(m.khat * (m.k ** 2 + s.kappa ** 2), 4 * np.pi * s.scale)
    xx = np.linspace(0.3, m.L - 0.3, 7)
    d = 1e-3
    fd2 = (m._kper(xx + d) - 2 * m._kper(xx) + m._kper(xx - d)) / d ** 2
    assert np.allclose(m._kper(xx, 2), fd2, rtol=1e-5)
    fd1 = (m._kper(xx + d) - m._kper(xx - d)) / (2 * d)
    assert np.allclose(m._kper(xx, 1), fd1, rtol=1e-6)


def test_pseudocharge_normalisation():
    """int m_I = -Z_I (Eq. pseudocharge) and m_I is the Gaussian of Sec. 4.1."""
    s, m = _tiny_model(n=256)
    mm = m.pseudocharge()
    assert abs(mm.sum() * m.h + s.Z.sum()) < 1e-12
    x = np.arange(m.N) * m.h
    ref = sum(-s.Z[I] / np.sqrt(2 * np.pi * s.sigma[I] ** 2)
              * sum(np.exp(-(x - s.R[I, 0] + n * m.L) ** 2 / (2 * s.sigma[I] ** 2)) for n in (-1, 0, 1))
              for I in range(s.n_atoms))
    assert np.allclose(mm, ref, atol=1e-12)


def test_perturbations_are_position_derivatives():
    """g_I = dV_ion/dR_I, B = dm/dR_I = K^-1 G and d2V = dg/dR_I, against central differences."""
    s, m = _tiny_model()
    G, B = m.perturbations()
    D2 = m.second_derivatives()
    d = 1e-4
    for I in range(s.n_atoms):
        Rp, Rm = s.R.copy(), s.R.copy()
        Rp[I, 0] += d
        Rm[I, 0] -= d
        mp = Model1D(W.System(**{**s.__dict__, "R": Rp}))
        mn = Model1D(W.System(**{**s.__dict__, "R": Rm}))
        fdV = (mp.V_ion() - mn.V_ion()) / (2 * d)
        fdm = (mp.pseudocharge() - mn.pseudocharge()) / (2 * d)
        fdg = (mp.perturbations()[0][:, I] - mn.perturbations()[0][:, I]) / (2 * d)
        assert np.allclose(G[:, I], fdV, atol=1e-7 * np.abs(G[:, I]).max())
        assert np.allclose(B[:, I], fdm, atol=1e-7 * np.abs(B[:, I]).max())
        assert np.allclose(D2[:, I], fdg, atol=1e-6 * np.abs(D2[:, I]).max())
    assert np.allclose(m.apply_K(B), G, atol=1e-10 * np.abs(G).max())


def test_ion_energy_derivatives():
    """Closed-form image sums for E_II and its gradient/Hessian against finite differences."""
    s, m = _tiny_model()
    d = 1e-4
    g = m.ion_gradient()
    Hm = m.ion_hessian()
    for I in range(s.n_atoms):
        Rp, Rm = s.R.copy(), s.R.copy()
        Rp[I, 0] += d
        Rm[I, 0] -= d
        mp = Model1D(W.System(**{**s.__dict__, "R": Rp}))
        mn = Model1D(W.System(**{**s.__dict__, "R": Rm}))
        assert abs((mp.ion_energy() - mn.ion_energy()) / (2 * d) - g[I]) < 1e-6 * max(1, abs(g[I]))
        assert np.allclose((mp.ion_gradient() - mn.ion_gradient()) / (2 * d), Hm[:, I], atol=1e-5)
    # translation invariance of the pair energy
    assert np.allclose(Hm.sum(axis=1), 0, atol=1e-10)


def test_srft_sketch_shape_and_scale():
    om = W.srft_sketch(16, 4, 0)
    assert om.shape == (16, 8)
    # each complex column has unit norm once split into real and imaginary parts
    nrm = om[:, 0::2] ** 2 + om[:, 1::2] ** 2
    assert np.allclose(nrm.sum(axis=0), 1.0)
