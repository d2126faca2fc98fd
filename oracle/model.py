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


class Model2D:
    """The same model on a periodic 2D grid (Sec. 4 uses 2D lattices of atoms; the kernel and the
    pseudocharges are the 2D forms of Eq. yukawa and Eq. pseudocharge).

    Conventions: grid (x_i, y_j) = (i hx, j hy), grid functions flattened with x fastest (index
    i + nx j); the quadrature weight h = hx hy multiplies every integral; wavevectors
    k = (2 pi n / Lx, 2 pi m / Ly); first-derivative factors drop the Nyquist index of their axis;
    Khat(k) = 4 pi s / (|k|^2 + kappa^2), whose periodic real-space form is the image sum of
    2 s K0(kappa r); m_I(r) = -Z_I exp(-|r - R_I|^2 / 2 sigma^2) / (2 pi sigma^2), Fourier
    coefficient -Z_I exp(-sigma^2 |k|^2 / 2) exp(-i k.R_I).  Perturbation columns are ordered
    p = 2 I + a (a = 0: x, 1: y), the index of D_{Ia,Jb}.  The image sums of E_II run over
    |n| <= images per axis (default: enough shells for exp(-kappa r) < exp(-40)).
    """

    def __init__(self, sysm, gs=None, images=None):
        if sysm.dim != 2:
            raise ValueError("Model2D needs a 2D system")
        # images of the periodic E_II sum: K0(kappa r) ~ exp(-kappa r), so shells out to
        # r = 40 / kappa leave less than exp(-40) of the sum
        if images is None:
            images = max(2, int(np.ceil(40.0 / (sysm.kappa * min(sysm.L)))))
        self.sys = sysm
        self.nx, self.ny = sysm.n
        self.Lx, self.Ly = sysm.L
        self.N = self.nx * self.ny
        self.hx, self.hy = self.Lx / self.nx, self.Ly / self.ny
        self.h = self.hx * self.hy
        kx1 = 2.0 * np.pi * np.fft.fftfreq(self.nx, d=1.0 / self.nx) / self.Lx
        ky1 = 2.0 * np.pi * np.fft.fftfreq(self.ny, d=1.0 / self.ny) / self.Ly
        kxo, kyo = kx1.copy(), ky1.copy()
        if self.nx % 2 == 0:
            kxo[self.nx // 2] = 0.0
        if self.ny % 2 == 0:
            kyo[self.ny // 2] = 0.0
        # 2D arrays indexed [j, i] (y, x); flattened C-order gives x fastest
        self.kx, self.ky = np.meshgrid(kx1, ky1)
        self.kx_odd, self.ky_odd = np.meshgrid(kxo, kyo)
        self.k2 = self.kx ** 2 + self.ky ** 2
        self.khat = 4.0 * np.pi * sysm.scale / (self.k2 + sysm.kappa ** 2)
        self.f = sysm.occ
        self.images = images
        if gs is not None:
            self.V = np.asarray(gs.V, dtype=np.float64)
            self.psi = np.asarray(gs.psi, dtype=np.float64)
            self.eps = np.asarray(gs.eps[: gs.n_orb], dtype=np.float64)
            self.rho = np.asarray(gs.rho, dtype=np.float64)
            self.n_orb = gs.n_orb

    # ---- operators on blocks of grid functions (columns of length N) ---------------------
    def _spectral(self, X, mult):
        X = np.asarray(X, dtype=np.float64)
        one = X.ndim == 1
        Xb = X.reshape(self.ny, self.nx, -1)
        Y = np.real(np.fft.ifft2(mult[:, :, None] * np.fft.fft2(Xb, axes=(0, 1)), axes=(0, 1)))
        Y = Y.reshape(self.N, -1)
        return Y[:, 0] if one else Y

    def apply_T(self, X):
        return self._spectral(X, 0.5 * self.k2)

    def apply_H(self, X, shift=0.0):
        X = np.asarray(X, dtype=np.float64)
        Y = self.apply_T(X)
        if X.ndim == 2:
            return Y + self.V[:, None] * X - np.asarray(shift) * X
        return Y + self.V * X - shift * X

    def apply_K(self, X):
        return self._spectral(X, self.khat)

    def apply_Kinv(self, X):
        return self._spectral(X, 1.0 / self.khat)

    def project(self, X):
        X = np.asarray(X, dtype=np.float64)
        return X - self.psi @ (self.psi.T @ X * self.h)

    def dense_H(self):
        """H = -1/2 Laplacian + V as a dense N x N matrix (kinetic term: Kronecker sum of the 1D
        spectral second-derivative circulants)."""
        def circ(n, L):
            k = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / L
            t = np.real(np.fft.ifft(0.5 * k ** 2))
            idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n
            return t[idx]
        Tx, Ty = circ(self.nx, self.Lx), circ(self.ny, self.Ly)
        T = np.kron(np.eye(self.ny), Tx) + np.kron(Ty, np.eye(self.nx))
        return T + np.diag(self.V)

    # ---- atom-dependent functions -------------------------------------------------------
    def _atom_coeffs(self, I, R=None):
        s = self.sys
        Rx, Ry = (s.R[I] if R is None else R)
        return -s.Z[I] * np.exp(-0.5 * (s.sigma[I] ** 2) * self.k2) * np.exp(-1j * (self.kx * Rx + self.ky * Ry))

    def _from_coeffs(self, c):
        return np.real(np.fft.ifft2(c)).reshape(-1) / self.h

    def pseudocharge(self):
        return sum(self._from_coeffs(self._atom_coeffs(I)) for I in range(self.sys.n_atoms))

    def V_ion(self):
        return sum(self._from_coeffs(self.khat * self._atom_coeffs(I)) for I in range(self.sys.n_atoms))

    def perturbations(self):
        """G (N x 2 N_A): g_{I,a} = dV_I/dR_{I,a}, and B = K^-1 G = dm_I/dR_{I,a}, spectrally."""
        nA = self.sys.n_atoms
        G = np.empty((self.N, 2 * nA))
        B = np.empty((self.N, 2 * nA))
        for I in range(nA):
            c = self._atom_coeffs(I)
            for a, ka in enumerate((self.kx_odd, self.ky_odd)):
                d = -1j * ka * c
                B[:, 2 * I + a] = self._from_coeffs(d)
                G[:, 2 * I + a] = self._from_coeffs(self.khat * d)
        return G, B

    def second_derivative_blocks(self):
        """d^2 V_I / dR_{I,a} dR_{I,b} per atom: (N, N_A, 2, 2).  Multiplier (-i k_a)(-i k_b);
        the diagonal uses -k_a^2 (even, Nyquist kept), the off-diagonal the odd factors."""
        nA = self.sys.n_atoms
        out = np.empty((self.N, nA, 2, 2))
        for I in range(nA):
            c = self.khat * self._atom_coeffs(I)
            out[:, I, 0, 0] = self._from_coeffs(-(self.kx ** 2) * c)
            out[:, I, 1, 1] = self._from_coeffs(-(self.ky ** 2) * c)
            xy = self._from_coeffs(-(self.kx_odd * self.ky_odd) * c)
            out[:, I, 0, 1] = xy
            out[:, I, 1, 0] = xy
        return out

    # ---- ion-ion interaction: point charges, periodic Yukawa kernel 2 s K0(kappa r) ------------
    def _image_sum(self, dx, dy, order):
        """sum over images n of f(r_n), r_n = (dx + nx Lx, dy + ny Ly), for f = 2 s K0(kappa r):
        order 0 the value, 1 the gradient (2,), 2 the Hessian (2, 2)."""
        from scipy.special import k0, k1
        s = self.sys
        kap, pre = s.kappa, 2.0 * s.scale
        n = np.arange(-self.images, self.images + 1)
        X = dx + n[:, None] * self.Lx + 0.0 * n[None, :]
        Y = dy + n[None, :] * self.Ly + 0.0 * n[:, None]
        r = np.hypot(X, Y)
        x = kap * r
        if order == 0:
            return pre * np.sum(k0(x))
        fp = -pre * kap * k1(x)                       # f'(r)
        if order == 1:
            return np.array([np.sum(fp * X / r), np.sum(fp * Y / r)])
        fpp = pre * kap ** 2 * (k0(x) + k1(x) / x)     # f''(r)
        ux, uy = X / r, Y / r
        Hxx = np.sum(fpp * ux * ux + fp / r * (1 - ux * ux))
        Hyy = np.sum(fpp * uy * uy + fp / r * (1 - uy * uy))
        Hxy = np.sum((fpp - fp / r) * ux * uy)
        return np.array([[Hxx, Hxy], [Hxy, Hyy]])

    def ion_energy(self):
        s = self.sys
        e = 0.0
        for I in range(s.n_atoms):
            for J in range(s.n_atoms):
                if I != J:
                    d = s.R[I] - s.R[J]
                    e += 0.5 * s.Z[I] * s.Z[J] * self._image_sum(d[0], d[1], 0)
        return e

    def ion_gradient(self):
        s = self.sys
        g = np.zeros(2 * s.n_atoms)
        for I in range(s.n_atoms):
            for J in range(s.n_atoms):
                if I != J:
                    d = s.R[I] - s.R[J]
                    g[2 * I:2 * I + 2] += s.Z[I] * s.Z[J] * self._image_sum(d[0], d[1], 1)
        return g

    def ion_hessian(self):
        s = self.sys
        nA = s.n_atoms
        Hm = np.zeros((2 * nA, 2 * nA))
        for I in range(nA):
            for J in range(nA):
                if I != J:
                    d = s.R[I] - s.R[J]
                    blk = s.Z[I] * s.Z[J] * self._image_sum(d[0], d[1], 2)
                    Hm[2 * I:2 * I + 2, 2 * J:2 * J + 2] = -blk
                    Hm[2 * I:2 * I + 2, 2 * I:2 * I + 2] += blk
        return Hm

    def forces(self, rho=None):
        """Hellmann-Feynman forces (Eq. force): F = -int g rho - dE_II/dR, (2 N_A,)."""
        rho = self.rho if rho is None else rho
        G, _ = self.perturbations()
        return -(G.T @ rho) * self.h - self.ion_gradient()
