"""O1: the periodic 1D reduced Hartree-Fock model on a planewave grid (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (Sec. 2.2 notation; Sec. 4.1 Eq. 1DHamil, Eq. yukawa; Eq. pseudocharge):
  * grid x_alpha = alpha h, alpha = 0..N-1, box [0, L), h = L / N; integrals are sums times h;
  * wavenumbers k_n = 2 pi n / L, n in [-N/2, N/2).  Multipliers that are odd in k (first
    derivatives) are zeroed at the Nyquist index so that real functions stay real;
  * Yukawa kernel K(x) = 2 pi s exp(-kappa |x|) / kappa, Fourier symbol
    Khat(k) = 4 pi s / (k^2 + kappa^2) (s = 1/eps0), applied as a periodic convolution;
  * pseudocharge m_I(x) = -Z_I exp(-(x - R_I)^2 / 2 sigma^2) / sqrt(2 pi sigma^2), whose
    Fourier coefficient int m_I e^{-ikx} dx is -Z_I exp(-sigma^2 k^2 / 2) exp(-i k R_I);
  * V_I = K * m_I (Eq. pseudocharge); g_I = dV_I(x - R_I)/dR_I (Sec. 2.2 below Eq. chi);
    B = K^-1 G = d m_I(x - R_I)/dR_I (change of variables below Eq. dyson2);
  * ion-ion energy E_II = 1/2 sum_{I != J} Z_I Z_J K(R_I - R_J) summed over periodic images
    (Sec. 4.1 states E_II uses the Yukawa K), with the closed form
    sum_n exp(-kappa |x + nL|) = cosh(kappa (x - L/2)) / sinh(kappa L / 2), 0 <= x < L.
"""
from __future__ import annotations

import numpy as np


class Model1D:
    """Model on a 1D grid built from a System and its ground state (V_eff, Psi, eps, rho)."""

    def __init__(self, sysm, gs=None):
        if sysm.dim != 1:
            raise NotImplementedError("oracle model is 1D")
        self.sys = sysm
        self.N = sysm.n[0]
        self.L = sysm.L[0]
        self.h = self.L / self.N
        n = np.fft.fftfreq(self.N, d=1.0 / self.N)
        self.k = 2.0 * np.pi * n / self.L
        self.k_odd = self.k.copy()
        if self.N % 2 == 0:
            self.k_odd[self.N // 2] = 0.0
        self.khat = 4.0 * np.pi * sysm.scale / (self.k ** 2 + sysm.kappa ** 2)
        self.f = sysm.occ
        if gs is not None:
            self.V = np.asarray(gs.V, dtype=np.float64)
            self.psi = np.asarray(gs.psi, dtype=np.float64)
            self.eps = np.asarray(gs.eps[: gs.n_orb], dtype=np.float64)
            self.rho = np.asarray(gs.rho, dtype=np.float64)
            self.n_orb = gs.n_orb

    # ---- operators on blocks of grid functions (columns) ---------------------------------
    def _spectral(self, X, mult):
        X = np.asarray(X, dtype=np.float64)
        return np.real(np.fft.ifft(mult[:, None] * np.fft.fft(X, axis=0), axis=0)) if X.ndim == 2 else \
            np.real(np.fft.ifft(mult * np.fft.fft(X)))

    def apply_T(self, X):
        """Kinetic term -1/2 d^2/dx^2 (Eq. Hamil), spectral."""
        return self._spectral(X, 0.5 * self.k ** 2)

    def apply_H(self, X, shift=0.0):
        """(H - shift) X with H = -1/2 Laplacian + V_eff; shift may be a scalar or per column."""
        X = np.asarray(X, dtype=np.float64)
        Y = self.apply_T(X)
        if X.ndim == 2:
            return Y + self.V[:, None] * X - np.asarray(shift) * X
        return Y + self.V * X - shift * X

    def apply_K(self, X):
        """v_hxc = K (no exchange-correlation kernel): periodic convolution with the Yukawa kernel."""
        return self._spectral(X, self.khat)

    def apply_Kinv(self, X):
        return self._spectral(X, 1.0 / self.khat)

    def project(self, X):
        """Q X with Q = I - sum_i psi_i psi_i^T h (projector onto the unoccupied space)."""
        X = np.asarray(X, dtype=np.float64)
        return X - self.psi @ (self.psi.T @ X * self.h)

    # ---- atom-dependent functions -------------------------------------------------------
    def _atom_coeffs(self, I):
        s = self.sys
        return -s.Z[I] * np.exp(-0.5 * (s.sigma[I] * self.k) ** 2) * np.exp(-1j * self.k * s.R[I, 0])

    def _from_coeffs(self, c):
        return np.real(np.fft.ifft(c)) / self.h

    def pseudocharge(self):
        return sum(self._from_coeffs(self._atom_coeffs(I)) for I in range(self.sys.n_atoms))

    def V_ion(self):
        return sum(self._from_coeffs(self.khat * self._atom_coeffs(I)) for I in range(self.sys.n_atoms))

    def perturbations(self):
        """G (N x N_p) with g_I = dV_I/dR_I, and B = K^-1 G = dm_I/dR_I, spectrally."""
        nA = self.sys.n_atoms
        G = np.empty((self.N, nA))
        B = np.empty((self.N, nA))
        for I in range(nA):
            c = -1j * self.k_odd * self._atom_coeffs(I)
            B[:, I] = self._from_coeffs(c)
            G[:, I] = self._from_coeffs(self.khat * c)
        return G, B

    def second_derivatives(self):
        """d^2 V_I(x - R_I)/dR_I^2 per atom (N x N_A): multiplier (-ik)^2 = -k^2."""
        nA = self.sys.n_atoms
        D2 = np.empty((self.N, nA))
        for I in range(nA):
            D2[:, I] = self._from_coeffs(-(self.k ** 2) * self.khat * self._atom_coeffs(I))
        return D2

    # ---- ion-ion interaction ------------------------------------------------------------
    def _kper(self, x, deriv=0):
        s = self.sys
        kap, L = s.kappa, self.L
        x = np.mod(x, L)
        pref = 2.0 * np.pi * s.scale / kap / np.sinh(0.5 * kap * L)
        if deriv == 0:
            return pref * np.cosh(kap * (x - 0.5 * L))
        if deriv == 1:
            return pref * kap * np.sinh(kap * (x - 0.5 * L))
        return pref * kap ** 2 * np.cosh(kap * (x - 0.5 * L))

    def ion_energy(self):
        s = self.sys
        e = 0.0
        for I in range(s.n_atoms):
            for J in range(s.n_atoms):
                if I != J:
                    e += 0.5 * s.Z[I] * s.Z[J] * self._kper(s.R[I, 0] - s.R[J, 0])
        return e

    def ion_gradient(self):
        s = self.sys
        g = np.zeros(s.n_atoms)
        for I in range(s.n_atoms):
            for J in range(s.n_atoms):
                if I != J:
                    g[I] += s.Z[I] * s.Z[J] * self._kper(s.R[I, 0] - s.R[J, 0], 1)
        return g

    def ion_hessian(self):
        s = self.sys
        nA = s.n_atoms
        Hm = np.zeros((nA, nA))
        for I in range(nA):
            for J in range(nA):
                if I != J:
                    v = s.Z[I] * s.Z[J] * self._kper(s.R[I, 0] - s.R[J, 0], 2)
                    Hm[I, J] = -v
                    Hm[I, I] += v
        return Hm

    def forces(self, rho=None):
        """Hellmann-Feynman forces (Eq. force): F_I = -int g_I rho - dE_II/dR_I."""
        rho = self.rho if rho is None else rho
        G, _ = self.perturbations()
        return -(G.T @ rho) * self.h - self.ion_gradient()
