"""Pins of the oracle's Dyson solve and dynamical matrix (Eq. dyson, Eq. SecDeriv)."""
import os

import numpy as np
import pytest

import acp_workloads as W
from oracle import chi0 as C
from oracle import dmat as Dm
from oracle import dyson as Dy
from oracle.model import Model1D


@pytest.fixture(scope="module")
def small():
    s = W.small_chain(4, 160, 0)
    gs = W.ground_state(s, use_cache=False)
    m = Model1D(s, gs)
    Cm = C.chi0_matrix_sos(m)
    return s, gs, m, Cm


def test_gmres_equals_dense_dyson(small):
    s, gs, m, Cm = small
    G, _ = m.perturbations()
    Ud = Dy.dyson_dense(m, G, Cm)
    Ug, k = Dy.dyson_gmres(m, G, chi0=lambda X: Cm @ X * m.h, tol=1e-13)
    assert np.linalg.norm(Ug - Ud) <= 1e-10 * np.linalg.norm(Ud)


def test_chi_symmetric_nsd_and_weak_coupling_limit(small):
    """chi = (I - chi0 K)^-1 chi0 is symmetric negative semidefinite; K -> 0 gives chi = chi0."""
    s, gs, m, Cm = small
    rng = np.random.default_rng(2)
    X = rng.standard_normal((m.N, 5))
    U = Dy.dyson_dense(m, X, Cm)
    Mq = X.T @ U * m.h
    assert np.allclose(Mq, Mq.T, atol=1e-9 * np.abs(Mq).max())
    assert np.linalg.eigvalsh(0.5 * (Mq + Mq.T)).max() <= 1e-9 * np.abs(Mq).max()
    m0 = Model1D(s, gs)
    m0.khat = m0.khat * 1e-14
    U0 = Dy.dyson_dense(m0, X, Cm)
    assert np.allclose(U0, Cm @ X * m.h, atol=1e-9 * np.abs(U0).max())


def test_dynamical_matrix_symmetry_and_acoustic_sum_rule(small):
    s, gs, m, Cm = small
    G, _ = m.perturbations()
    D, asym = Dm.dynamical_matrix(m, Dy.dyson_dense(m, G, Cm))
    assert asym < 1e-8
    assert np.abs(D.sum(axis=1)).max() <= 1e-6 * np.linalg.norm(D)


def _bonded(R=None):
    rng = np.random.default_rng(11)
    s = W.chain_1d("bonded", 4, 3.0, 1.0, 0.5, 0.1, 1.0, 96, occ=1, displacement=0.15, rng=rng)
    if R is not None:
        s = W.System(**{**s.__dict__, "R": R})
    return s


def _forces(R, V_start=None):
    s = _bonded(R)
    gs = W.ground_state(s, use_cache=False, tol=1e-14, maxit=300, V_start=V_start)
    return Model1D(s, gs).forces(), gs


def test_dynamical_matrix_equals_frozen_phonon_differences():
    """D from DFPT equals central differences of Hellmann-Feynman forces (Sec. 1, Eq. force)."""
    s = _bonded()
    gs = W.ground_state(s, use_cache=False, tol=1e-14, maxit=300)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    D, _ = Dm.dynamical_matrix(m, Dy.dyson_dense(m, G))
    Dfd = np.zeros_like(D)
    for J in range(s.n_atoms):
        cols = []
        for d in (2e-3, 1e-3):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[J, 0] += d
            Rm[J, 0] -= d
            Fp, _ = _forces(Rp, gs.V)
            Fm, _ = _forces(Rm, gs.V)
            cols.append(-(Fp - Fm) / (2 * d))
        Dfd[:, J] = (4 * cols[1] - cols[0]) / 3.0
    assert np.linalg.norm(D - Dfd) <= 1e-6 * np.linalg.norm(D)


def test_phonon_dos_normalisation_moments_and_counting():
    """Eq. phononspec with the Gaussian delta of Sec. 4.1: rho_D integrates to 1 (the 1 / d N_A
    normalisation), its mean is the mean frequency and its variance the frequencies' variance plus
    sigma^2; each mode is scipy's normal density; as sigma -> 0 the integral of rho_D up to a point
    between two frequencies counts the fraction of modes below it."""
    from scipy import integrate, stats
    rng = np.random.default_rng(7)
    om = np.sort(np.concatenate([[0.0, 0.0], rng.uniform(0.05, 0.9, 14)]))
    sig = 0.01
    lo, hi = om.min() - 40 * sig, om.max() + 40 * sig
    pts = list(om)
    f = lambda x: Dm.phonon_dos(om, x, sig)[0]  # noqa: E731
    mass = integrate.quad(f, lo, hi, points=pts, limit=500)[0]
    mean = integrate.quad(lambda x: x * f(x), lo, hi, points=pts, limit=500)[0]
    var = integrate.quad(lambda x: (x - mean) ** 2 * f(x), lo, hi, points=pts, limit=500)[0]
    assert abs(mass - 1.0) < 1e-9
    assert abs(mean - om.mean()) < 1e-9
    assert abs(var - (om.var() + sig ** 2)) < 1e-9
    w = np.linspace(-0.1, 1.0, 301)
    ref = stats.norm.pdf(w[:, None], loc=om[None, :], scale=sig).mean(axis=1)
    assert np.allclose(Dm.phonon_dos(om, w, sig), ref, rtol=1e-13, atol=1e-300)
    gaps = np.diff(om)
    j = int(np.argmax(gaps))
    cut = 0.5 * (om[j] + om[j + 1])
    xs = np.arange(-0.05, cut, 1e-5)  # sigma / 10: the trapezoid rule is exact to rounding here
    below = np.trapezoid(Dm.phonon_dos(om, xs, 1e-4), xs)
    assert abs(below - (j + 1) / om.size) < 1e-9


@pytest.mark.parametrize("kind", ["1d", "2d"])
def test_sampled_exact_columns_equal_full_dynamical_matrix(kind):
    """The sampled-column form that writes the stored exact columns of D (GMRES on the Dyson
    equation with the sum-over-states chi0, Eq. SecDeriv assembled per column) equals the columns
    of the dense route (dense Dyson solve, full D), on a chain and on a 2D lattice."""
    import importlib.util
    from oracle import chi0 as C
    from oracle import dmat as DM
    from oracle import dyson as Dy
    from oracle.model import Model1D, Model2D
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_dcols_reference.py")
    spec_ = importlib.util.spec_from_file_location("make_dcols_reference", path)
    mk = importlib.util.module_from_spec(spec_)
    spec_.loader.exec_module(mk)
    if kind == "1d":
        s = W.small_chain(4, 160, 0)
        m = Model1D(s, W.ground_state(s, use_cache=False))
        cols = [0, 3]
    else:
        s = W.small_lattice(2, 2, 24, 0)
        m = Model2D(s, W.ground_state(s, use_cache=False))
        cols = [0, 3, 6]
    G, _ = m.perturbations()
    D, _ = DM.dynamical_matrix(m, Dy.dyson_dense(m, G))
    Dc, _, res = mk.exact_columns(m, cols, C.full_spectrum(m))
    assert res < 1e-12
    assert np.abs(Dc - D[:, cols]).max() <= 1e-9 * np.abs(D).max()
