"""Dynamical matrix and phonon frequencies (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. SecDeriv: d^2E/dR_I dR_J = int g_I (chi g_J) + delta_IJ int rho d^2V_I/dR_I^2 + d^2E_II/dR_I dR_J,
with chi g_J = U_J from the Dyson equation (Eq. chiterm).  D_IJ = that / sqrt(M_I M_J) and
D u_k = omega_k^2 u_k (Sec. 2.2).  Frequencies of negative eigenvalues are reported as
-sqrt(|lambda|).  Eq. phononspec: the phonon spectrum rho_D(w) = (1 / d N_A) sum_k delta(w - omega_k),
with the Gaussian regularised delta of Sec. 4.1.
"""
from __future__ import annotations

import numpy as np


def dynamical_matrix(model, U, symmetrize=True):
    G, _ = model.perturbations()
    Hm = (G.T @ U) * model.h
    if model.sys.dim == 1:
        D2 = model.second_derivatives()
        Hm = Hm + np.diag(D2.T @ model.rho * model.h)
    else:
        # delta_IJ int rho d^2 V_I / dR_Ia dR_Ib: one d x d block per atom
        blk = np.einsum("r,rIab->Iab", model.rho, model.second_derivative_blocks()) * model.h
        d = model.sys.dim
        for I in range(model.sys.n_atoms):
            Hm[d * I:d * I + d, d * I:d * I + d] += blk[I]
    Hm = Hm + model.ion_hessian()
    mass = np.repeat(model.sys.mass, model.sys.dim)
    D = Hm / np.sqrt(np.outer(mass, mass))
    asym = np.linalg.norm(D - D.T) / max(np.linalg.norm(D), 1e-300)
    if symmetrize:
        D = 0.5 * (D + D.T)
    return D, float(asym)


def phonons(D):
    lam, modes = np.linalg.eigh(0.5 * (D + D.T))
    return np.sign(lam) * np.sqrt(np.abs(lam)), modes


def translation_projector(n_atoms, dim):
    """P = I - T T^T, T the d orthonormal rigid translations (column a: 1/sqrt(N_A) on every
    perturbation index d I + a).  An exact D annihilates T (the acoustic sum rule
    sum_J D_{Ia,Jb} = 0, from the invariance of E_tot under a rigid shift), so P D P = D for it."""
    n = n_atoms * dim
    T = np.zeros((n, dim))
    for a in range(dim):
        T[a::dim, a] = 1.0 / np.sqrt(n_atoms)
    return np.eye(n) - T @ T.T


def phonon_error(D, D_ref, n_atoms, dim):
    """The L-infinity phonon-frequency error of Table 2, read as the frequencies of P D P (the acoustic
    sum rule imposed by projecting out the rigid translations, on both sides), omega = sign(lambda)
    sqrt(|lambda|), eigenvalues in ascending order.  Returns (absolute, relative to max |omega_ref|).

    Without the projection the d translation modes (omega_ref = 0) turn an error dlambda of a
    compressed D into |domega| = sqrt(|dlambda|); Table 2's ACP errors (2.7e-6 at eps = 1e-5) are
    far below that square root and match this reading."""
    P = translation_projector(n_atoms, dim)
    w, _ = phonons(P @ D @ P)
    wr, _ = phonons(P @ D_ref @ P)
    e = float(np.abs(w - wr).max())
    return e, e / max(float(np.abs(wr).max()), 1e-300)


def phonon_dos(omega, w, sigma):
    """Eq. phononspec with delta_sigma(x) = exp(-x^2 / (2 sigma^2)) / sqrt(2 pi sigma^2) (Sec. 4.1):
    rho(w_j) = (1 / n) sum_k delta_sigma(w_j - omega_k), n = d N_A = len(omega)."""
    omega = np.asarray(omega, dtype=np.float64)
    w = np.atleast_1d(np.asarray(w, dtype=np.float64))
    rho = np.zeros(w.size)
    for wk in omega:
        rho += np.exp(-((w - wk) ** 2) / (2.0 * sigma ** 2)) / np.sqrt(2.0 * np.pi * sigma ** 2)
    return rho / omega.size
