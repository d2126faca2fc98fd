"""Pins of the oracle's chi0 (Alg. 1, Eq. AdlerWiser) and MINRES."""
import numpy as np
import pytest

import acp_workloads as W
from oracle import chi0 as C
from oracle.minres import minres
from oracle.model import Model1D


@pytest.fixture(scope="module")
def small():
    s = W.small_chain(4, 160, 0)
    gs = W.ground_state(s, use_cache=False)
    return s, gs, Model1D(s, gs)


def test_minres_against_dense_solve():
    """Brute force: MINRES on random symmetric shifted systems equals numpy.linalg.solve."""
    rng = np.random.default_rng(0)
    n = 60
    A = rng.standard_normal((n, n))
    A = A + A.T
    lam = np.linalg.eigvalsh(A)
    shifts = np.array([lam[0] - 1.0, 0.37, lam[-1] + 2.0, 0.5 * (lam[10] + lam[11])])
    Bm = rng.standard_normal((n, 4))
    X = minres(lambda V, s: A @ V - s * V, Bm, shifts, tol=1e-13, maxit=2000)
    for j in range(4):
        ref = np.linalg.solve(A - shifts[j] * np.eye(n), Bm[:, j])
        assert np.linalg.norm(X[:, j] - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("args", [(4, 160, 0), (6, 240, 1)])
def test_sternheimer_equals_sum_over_states(args):
    """Eq. Sternheimer is exact in the discrete basis: Alg. 1 equals Eq. AdlerWiser.

    At tol 1e-13 some solves need well over a hundred iterations; without re-projecting each
    Lanczos vector the occupied-space rounding grows geometrically and spoils the result."""
    s = W.small_chain(*args)
    m = Model1D(s, W.ground_state(s, use_cache=False))
    G, _ = m.perturbations()
    U1 = C.chi0_apply(m, G, tol=1e-13)
    Us = C.chi0_matrix_sos(m) @ G * m.h
    assert np.linalg.norm(U1 - Us) <= 1e-12 * np.linalg.norm(Us)


def test_chi0_symmetric_nsd_charge_conserving(small):
    s, gs, m = small
    rng = np.random.default_rng(1)
    X = rng.standard_normal((m.N, 6))
    CX = C.chi0_apply(m, X)
    Mq = X.T @ CX * m.h
    assert np.allclose(Mq, Mq.T, atol=1e-10 * np.abs(Mq).max())
    assert np.linalg.eigvalsh(0.5 * (Mq + Mq.T)).max() <= 1e-10 * np.abs(Mq).max()
    assert np.abs(CX.sum(axis=0) * m.h).max() <= 1e-10 * np.abs(CX).max()


class _FreeGS:
    pass


@pytest.mark.parametrize("occ", [1, 2])
def test_free_electron_lindhard(occ):
    """V_eff = 0 with closed shells: chi0 is diagonal in planewaves with the Lindhard sum.

    chi0 e^{iqx} = chihat(q) e^{iqx},
    chihat(q) = (f/L) sum_{k occ} [1(k+q unocc)/(eps_k - eps_{k+q}) + 1(k-q unocc)/(eps_k - eps_{k-q})].
    """
    N, L, nmax = 64, 20.0, 2
    s = W.chain_1d("free", 1, L, 1.0, 0.5, 0.1, 1.0, N, occ=1)
    m = Model1D(s)
    x = np.arange(N) * m.h
    cols, eps = [np.full(N, 1 / np.sqrt(L))], [0.0]
    for n in range(1, nmax + 1):
        kk = 2 * np.pi * n / L
        cols += [np.sqrt(2 / L) * np.cos(kk * x), np.sqrt(2 / L) * np.sin(kk * x)]
        eps += [0.5 * kk ** 2] * 2
    gs = _FreeGS()
    gs.V = np.zeros(N)
    gs.psi = np.array(cols).T
    gs.eps = np.array(eps)
    gs.n_orb = len(eps)
    gs.rho = occ * np.sum(gs.psi ** 2, axis=1)
    m = Model1D(s, gs)
    m.f = occ
    occn = set(range(-nmax, nmax + 1))
    for nq in (1, 3, 5):
        q = 2 * np.pi * nq / L
        chi = 0.0
        for n in occn:
            ek = 0.5 * (2 * np.pi * n / L) ** 2
            for sgn in (1, -1):
                if n + sgn * nq not in occn:
                    chi += 1.0 / (ek - 0.5 * (2 * np.pi * (n + sgn * nq) / L) ** 2)
        chi *= occ / L
        g = np.stack([np.cos(q * x), np.sin(q * x)], axis=1)
        U = C.chi0_apply(m, g)
        assert np.allclose(U, chi * g, atol=1e-10 * abs(chi))


@pytest.mark.parametrize("args", [(4, 160, 0), (6, 240, 1)])
def test_sos_columnwise_equals_dense_sum(args):
    """Eq. AdlerWiser summed column by column (the form that writes the stored exact D of the
    128-atom chain) equals the dense sum over states on two small chains, element by element."""
    s = W.small_chain(*args)
    m = Model1D(s, W.ground_state(s, use_cache=False))
    G, _ = m.perturbations()
    spec = C.full_spectrum(m)
    Ua = C.chi0_apply_sos(m, G, spectrum=spec)
    Ud = C.chi0_matrix_sos(m, spectrum=spec) @ G * m.h
    assert np.abs(Ua - Ud).max() <= 1e-13 * np.abs(Ud).max()


@pytest.mark.parametrize("occ", [1, 2])
def test_sos_columnwise_free_electron_lindhard(occ):
    """The column-by-column Adler-Wiser sum reproduces the free-electron Lindhard closed form:
    chi0 e^{iqx} = chihat(q) e^{iqx} with
    chihat(q) = (f/L) sum_{k occ} sum_{+-} 1(k+-q unocc) / (eps_k - eps_{k+-q}).
    A wrong sign of the energy denominator, a dropped quadrature weight h or a dropped
    occupation factor each fails this (chihat < 0 and its scale are fixed)."""
    N, L, nmax = 64, 20.0, 2
    s = W.chain_1d("free", 1, L, 1.0, 0.5, 0.1, 1.0, N, occ=1)
    m = Model1D(s)
    x = np.arange(N) * m.h
    gs = _FreeGS()
    gs.V = np.zeros(N)
    # occupied planewaves |n| <= nmax as real cos/sin pairs, normalised with weight h
    cols, eps = [np.full(N, 1 / np.sqrt(L))], [0.0]
    for n in range(1, nmax + 1):
        kk = 2 * np.pi * n / L
        cols += [np.sqrt(2 / L) * np.cos(kk * x), np.sqrt(2 / L) * np.sin(kk * x)]
        eps += [0.5 * kk ** 2] * 2
    gs.psi = np.array(cols).T
    gs.eps = np.array(eps)
    gs.n_orb = len(eps)
    gs.rho = occ * np.sum(gs.psi ** 2, axis=1)
    m = Model1D(s, gs)
    m.f = occ
    # the spectrum of H = -1/2 d^2/dx^2 on the grid: occupied block first, as full_spectrum orders it
    w, Phi = C.full_spectrum(m)
    assert np.allclose(w[:gs.n_orb], np.sort(eps), atol=1e-12)
    occn = set(range(-nmax, nmax + 1))
    for nq in (1, 3, 5):
        q = 2 * np.pi * nq / L
        chi = 0.0
        for n in occn:
            ek = 0.5 * (2 * np.pi * n / L) ** 2
            for sgn in (1, -1):
                if n + sgn * nq not in occn:
                    chi += 1.0 / (ek - 0.5 * (2 * np.pi * (n + sgn * nq) / L) ** 2)
        chi *= occ / L
        g = np.stack([np.cos(q * x), np.sin(q * x)], axis=1)
        U = C.chi0_apply_sos(m, g, spectrum=(w, Phi))
        assert chi < 0
        assert np.allclose(U, chi * g, atol=1e-10 * abs(chi))
