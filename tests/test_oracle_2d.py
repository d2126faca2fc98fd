"""Pins of the oracle's 2D model (the 2D lattices of Sec. 4 with the 2D forms of Eq. yukawa and
Eq. pseudocharge) against closed forms, finite differences and the sum over states.

* Yukawa kernel: for two charges smeared into Gaussians of width sigma, the spectral sum of
  Khat = 4 pi s / (|k|^2 + kappa^2) equals exp(sigma^2 kappa^2) times the image sum of
  2 s K0(kappa d) for the point charges (write 1/(k^2 + kappa^2) as the heat-kernel integral
  over t; the Gaussians shift it by sigma^2; the part t < sigma^2 is ~exp(-d^2 / 4 sigma^2),
  here e^-69): pins the normalisation of K0 against the Fourier symbol and the periodic images.
* pseudocharges integrate to -Z and sample the Gaussian;
* g, B and the second derivatives of V_I are central differences of V_I and m_I in R_I;
* the ion-ion gradient and Hessian are central differences of E_II;
* Alg. 1 equals the Adler-Wiser sum over states of a full eigendecomposition;
* D is symmetric, obeys the acoustic sum rule in both directions, and equals central differences
  of the Hellmann-Feynman forces (frozen phonons, SCF per geometry).
"""
import numpy as np
import pytest

import acp_workloads as W
from oracle import chi0 as C
from oracle import dmat as Dm
from oracle import dyson as Dy
from oracle.model import Model2D


@pytest.fixture(scope="module")
def lat():
    s = W.small_lattice(2, 2, 32, 0)
    gs = W.ground_state(s, use_cache=False, tol=1e-12)
    return s, gs, Model2D(s, gs)


def test_yukawa_image_sum_matches_spectral_gaussians():
    s = W.lattice_2d("pair", 2, 1, 20.0, 1.0, 1.2, 0.05, 0.7, 96, occ=1)   # 40 x 20 box, atoms 20 apart
    s = W.System(**{**s.__dict__, "n": (160, 80)})
    m = Model2D(s)
    d = s.R[0] - s.R[1]
    e_point = s.Z[0] * s.Z[1] * m._image_sum(d[0], d[1], 0)
    c0, c1 = m._atom_coeffs(0), m._atom_coeffs(1)
    area = m.Lx * m.Ly
    e_gauss = float(np.real(np.sum(m.khat * c0 * np.conj(c1))) / area)
    assert abs(e_gauss - np.exp((s.sigma[0] * s.kappa) ** 2) * e_point) <= 1e-9 * abs(e_point)


def test_pseudocharge_normalisation_and_shape(lat):
    s, gs, m = lat
    mI = m._from_coeffs(m._atom_coeffs(0))
    assert abs(mI.sum() * m.h + s.Z[0]) < 1e-12
    ys, xs = np.meshgrid(np.arange(m.ny) * m.hy, np.arange(m.nx) * m.hx, indexing="ij")
    ref = np.zeros_like(xs)
    for nx in (-1, 0, 1):
        for ny in (-1, 0, 1):
            r2 = (xs - s.R[0, 0] + nx * m.Lx) ** 2 + (ys - s.R[0, 1] + ny * m.Ly) ** 2
            ref += -s.Z[0] * np.exp(-0.5 * r2 / s.sigma[0] ** 2) / (2 * np.pi * s.sigma[0] ** 2)
    assert np.abs(mI - ref.reshape(-1)).max() < 1e-9 * np.abs(ref).max()


def test_perturbations_are_position_derivatives(lat):
    s, gs, m = lat
    G, B = m.perturbations()
    D2 = m.second_derivative_blocks()
    d = 1e-4
    for I in (0, 2):
        for a in (0, 1):
            Rp, Rm = s.R[I].copy(), s.R[I].copy()
            Rp[a] += d
            Rm[a] -= d
            Vp = m._from_coeffs(m.khat * m._atom_coeffs(I, Rp))
            Vm = m._from_coeffs(m.khat * m._atom_coeffs(I, Rm))
            mp = m._from_coeffs(m._atom_coeffs(I, Rp))
            mm = m._from_coeffs(m._atom_coeffs(I, Rm))
            gfd = (Vp - Vm) / (2 * d)
            assert np.abs(G[:, 2 * I + a] - gfd).max() < 1e-6 * np.abs(gfd).max()
            assert np.abs(B[:, 2 * I + a] - (mp - mm) / (2 * d)).max() < 1e-6 * np.abs(B[:, 2 * I + a]).max()
            # second derivatives: central difference of g_{I,b} in R_{I,a}
            for b in (0, 1):
                kb = (m.kx_odd, m.ky_odd)[b]
                gp = m._from_coeffs(m.khat * (-1j * kb) * m._atom_coeffs(I, Rp))
                gm = m._from_coeffs(m.khat * (-1j * kb) * m._atom_coeffs(I, Rm))
                fd = (gp - gm) / (2 * d)
                assert np.abs(D2[:, I, a, b] - fd).max() < 1e-5 * np.abs(fd).max()


def test_ion_energy_derivatives():
    s = W.lattice_2d("ions", 2, 2, 9.0, [1.0, 2.0, 2.0, 1.0], 1.2, 0.05, 0.8, 32, occ=1,
                     displacement=0.4, rng=np.random.default_rng(4))
    m = Model2D(s, images=40)
    g = m.ion_gradient()
    Hm = m.ion_hessian()
    d = 1e-4

    def at(R):
        return Model2D(W.System(**{**s.__dict__, "R": R}), images=40)
    for I in range(s.n_atoms):
        for a in (0, 1):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[I, a] += d
            Rm[I, a] -= d
            mp, mm = at(Rp), at(Rm)
            assert abs((mp.ion_energy() - mm.ion_energy()) / (2 * d) - g[2 * I + a]) < 1e-7 * np.abs(g).max()
            col = (mp.ion_gradient() - mm.ion_gradient()) / (2 * d)
            assert np.abs(col - Hm[:, 2 * I + a]).max() < 1e-6 * np.abs(Hm).max()


def test_sternheimer_equals_sum_over_states(lat):
    s, gs, m = lat
    G, _ = m.perturbations()
    U = C.chi0_apply(m, G[:, :3], tol=1e-13)
    ref = C.chi0_matrix_sos(m) @ G[:, :3] * m.h
    assert np.linalg.norm(U - ref) <= 1e-10 * np.linalg.norm(ref)


def test_dynamical_matrix_symmetry_and_acoustic_sum_rule(lat):
    s, gs, m = lat
    G, _ = m.perturbations()
    D, asym = Dm.dynamical_matrix(m, Dy.dyson_dense(m, G))
    assert asym < 1e-8
    nA = s.n_atoms
    for a in (0, 1):
        for b in (0, 1):
            # sum over J of D_{Ia,Jb} vanishes for every I (rigid translation along b)
            rows = D[a::2, :][:, b::2].sum(axis=1)
            assert np.abs(rows).max() <= 1e-6 * np.linalg.norm(D)
    assert D.shape == (2 * nA, 2 * nA)


def _pair(R=None):
    s = W.lattice_2d("pair2d", 2, 1, 6.0, [1.0, 2.0], 1.0, 0.1, 1.0, 32, occ=1, displacement=0.2,
                     rng=np.random.default_rng(5))
    if R is not None:
        s = W.System(**{**s.__dict__, "R": R})
    return s


def _forces(R):
    s = _pair(R)
    gs = W.ground_state(s, use_cache=False, tol=1e-13, maxit=300)
    return Model2D(s, gs, images=40).forces()


@pytest.mark.slow
def test_dynamical_matrix_equals_frozen_phonon_differences():
    s = _pair()
    gs = W.ground_state(s, use_cache=False, tol=1e-13, maxit=300)
    m = Model2D(s, gs, images=40)
    G, _ = m.perturbations()
    D, _ = Dm.dynamical_matrix(m, Dy.dyson_dense(m, G))
    Dfd = np.zeros_like(D)
    d = 1e-3
    for J in range(s.n_atoms):
        for b in (0, 1):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[J, b] += d
            Rm[J, b] -= d
            Dfd[:, 2 * J + b] = -(_forces(Rp) - _forces(Rm)) / (2 * d)
    assert np.linalg.norm(D - Dfd) <= 1e-5 * np.linalg.norm(D)


class _FreeGS:
    pass


@pytest.mark.parametrize("occ", [1, 2])
def test_free_electron_lindhard_2d(occ):
    """V_eff = 0 in a rectangular box with the five lowest planewaves occupied (k = 0, +-k_x1,
    +-k_y1): Alg. 1 acting on e^{iq.r} gives chihat(q) e^{iq.r} with the 2D Lindhard sum
    chihat(q) = (f/A) sum_{k occ} sum_{+-} 1(k +- q unocc) / (eps_k - eps_{k+-q}),
    the free-electron response written out in planewaves (A = Lx Ly)."""
    from oracle import chi0 as C
    nx, ny, Lx, Ly = 24, 20, 12.0, 10.0
    s = W.lattice_2d("free2d", 1, 1, 1.0, 1.0, 0.5, 0.1, 1.0, 8, 1)
    s = W.System(**{**s.__dict__, "n": (nx, ny), "L": (Lx, Ly)})
    A = Lx * Ly
    ys, xs = np.meshgrid(np.arange(ny) * Ly / ny, np.arange(nx) * Lx / nx, indexing="ij")
    xs, ys = xs.reshape(-1), ys.reshape(-1)   # index ix + nx iy
    occn = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]

    def kvec(n):
        return 2 * np.pi * n[0] / Lx, 2 * np.pi * n[1] / Ly

    def energy(n):
        kx, ky = kvec(n)
        return 0.5 * (kx * kx + ky * ky)

    cols, eps = [np.full(nx * ny, 1 / np.sqrt(A))], [0.0]
    for n in [(1, 0), (0, 1)]:
        kx, ky = kvec(n)
        ph = kx * xs + ky * ys
        cols += [np.sqrt(2 / A) * np.cos(ph), np.sqrt(2 / A) * np.sin(ph)]
        eps += [energy(n)] * 2
    order = np.argsort(eps, kind="stable")
    gs = _FreeGS()
    gs.V = np.zeros(nx * ny)
    gs.psi = np.array(cols).T[:, order]
    gs.eps = np.array(eps)[order]
    gs.n_orb = len(eps)
    gs.rho = occ * np.sum(gs.psi ** 2, axis=1)
    m = Model2D(s, gs)
    m.f = occ
    assert np.allclose(gs.psi.T @ gs.psi * m.h, np.eye(5), atol=1e-12)
    occset = set(occn)
    for q in [(1, 0), (1, 1), (2, -1), (0, 3)]:
        chi = 0.0
        for n in occn:
            for sgn in (1, -1):
                nq = (n[0] + sgn * q[0], n[1] + sgn * q[1])
                if nq not in occset:
                    chi += 1.0 / (energy(n) - energy(nq))
        chi *= occ / A
        qx, qy = kvec(q)
        g = np.stack([np.cos(qx * xs + qy * ys), np.sin(qx * xs + qy * ys)], axis=1)
        U = C.chi0_apply(m, g)
        assert np.allclose(U, chi * g, atol=1e-10 * abs(chi)), q
