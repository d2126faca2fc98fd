"""Ground state of the periodic reduced Hartree-Fock model (input preparation).

The polarizability method takes the converged effective potential V_eff, the occupied
orbitals Psi and their eigenvalues eps as inputs (Sec. 2.1, Eq. Hamil and Eq. effV, with no
exchange-correlation term as in Sec. 4.1).  This module produces them with an Anderson-mixed
self-consistent field iteration and a dense symmetric eigensolver on the planewave grid.  It
contains none of the linear-response arithmetic.

Discretisation (planewave, uniform grid x_alpha = alpha h):
  * kinetic term: -1/2 d^2/dx^2 acts as multiplication by k^2/2 in Fourier space,
    k = 2 pi n / L with n in [-N/2, N/2);
  * grid functions are normalised so that sum_alpha psi_i psi_j h = delta_ij;
  * V_eff = IFFT[Khat (FFT(rho + m))] with the k = 0 term removed (neutral cell).
"""
from __future__ import annotations

import dataclasses
import os
import time

import numpy as np
import scipy.linalg as sla

from .systems import System

# converged potentials, one file per system key (ACP_GS_CACHE names another directory)
CACHE_DIR = os.environ.get("ACP_GS_CACHE") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "cache")


@dataclasses.dataclass
class GroundState:
    V: np.ndarray        # (N_g,) effective potential the orbitals are eigenvectors for
    psi: np.ndarray      # (N_g, n_orb) occupied orbitals, column-major friendly, sum psi^2 h = 1
    eps: np.ndarray      # (n_orb + n_extra,) lowest eigenvalues (ascending)
    rho: np.ndarray      # (N_g,) f * sum_i psi_i^2
    m: np.ndarray        # (N_g,) total pseudocharge on the grid
    n_orb: int
    scf_residual: float  # ||rho_out - rho_in|| sqrt(h) / N_e at the last iteration
    iterations: int
    seconds: float

    @property
    def gap(self) -> float:
        return float(self.eps[self.n_orb] - self.eps[self.n_orb - 1])

    @property
    def eps_occ(self) -> np.ndarray:
        return self.eps[: self.n_orb]


def _wavenumbers_1d(n: int, L: float) -> np.ndarray:
    return 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / L


def _pseudocharge_1d(sysm: System, k: np.ndarray) -> np.ndarray:
    h = sysm.h[0]
    F = np.zeros(k.shape[0], dtype=np.complex128)
    for RI, ZI, sI in zip(sysm.R[:, 0], sysm.Z, sysm.sigma):
        F += -ZI * np.exp(-0.5 * (sI * k) ** 2) * np.exp(-1j * k * RI)
    return np.real(np.fft.ifft(F)) / h


def _kinetic_dense_1d(n: int, k: np.ndarray) -> np.ndarray:
    t = np.real(np.fft.ifft(0.5 * k ** 2))
    idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n
    return t[idx]


def _lowest(H: np.ndarray, count: int):
    return sla.eigh(H, subset_by_index=[0, count - 1], driver="evr")


def _atom_density_1d(Zv: float, sigma: float, kappa: float, scale: float, occ: int, h: float,
                     cell: float = 40.0):
    """Self-consistent density of one isolated atom in a wide cell, centred at cell/2."""
    from .systems import chain_1d
    n = int(round(cell / h))
    atom = chain_1d("atom", 1, n * h, Zv, sigma, kappa, scale, n, occ)
    gs = scf(atom, tol=1e-8, maxit=200, initial="gaussian", use_cache=False)
    x = np.arange(n) * h - 0.5 * n * h
    return gs.rho, x


def _initial_density_1d(sysm: System, k: np.ndarray, kind: str) -> np.ndarray:
    h = sysm.h[0]
    F = np.zeros(k.shape[0], dtype=np.complex128)
    if kind == "gaussian":
        for RI, ZI in zip(sysm.R[:, 0], sysm.Z):
            F += ZI * np.exp(-0.5 * (1.5 * k) ** 2) * np.exp(-1j * k * RI)
        return np.real(np.fft.ifft(F)) / h
    # superposition of isolated-atom densities, shifted spectrally onto the system grid
    atoms = {}
    for ZI, sI in zip(sysm.Z, sysm.sigma):
        key = (float(ZI), float(sI))
        if key not in atoms:
            rho_a, xa = _atom_density_1d(ZI, sI, sysm.kappa, sysm.scale, sysm.occ, h)
            atoms[key] = (np.exp(-1j * np.outer(k, xa)) @ rho_a) * h
    for RI, ZI, sI in zip(sysm.R[:, 0], sysm.Z, sysm.sigma):
        F += atoms[(float(ZI), float(sI))] * np.exp(-1j * k * RI)
    return np.real(np.fft.ifft(F)) / h


def scf(sysm: System, tol: float = 1e-11, maxit: int = 200, beta: float = 0.3, history: int = 12,
        n_extra: int = 4, initial: str = "atoms", use_cache: bool = True, verbose: bool = False,
        V_start: np.ndarray | None = None) -> GroundState:
    """Anderson-mixed SCF for the 1D model; returns exact eigenpairs of H[V] for the final V."""
    if sysm.dim != 1:
        raise NotImplementedError("only 1D ground states are generated")
    t0 = time.time()
    n, L, h = sysm.n[0], sysm.L[0], sysm.h[0]
    n_orb, f = sysm.n_orb, sysm.occ
    k = _wavenumbers_1d(n, L)
    khat = 4.0 * np.pi * sysm.scale / (k ** 2 + sysm.kappa ** 2)
    m = _pseudocharge_1d(sysm, k)
    T = _kinetic_dense_1d(n, k)

    def potential(rho):
        c = np.fft.fft(rho + m)
        c[0] = 0.0
        return np.real(np.fft.ifft(khat * c))

    def solve(V):
        w, U = _lowest(T + np.diag(V), n_orb + n_extra)
        psi = U[:, :n_orb] / np.sqrt(h)
        return w, psi, f * np.sum(psi ** 2, axis=1)

    cache_file = os.path.join(CACHE_DIR, sysm.key() + ".npy")
    if use_cache and V_start is None and os.path.exists(cache_file):
        V = np.load(cache_file)
        w, psi, rho = solve(V)
        res = np.linalg.norm(potential(rho) - V) / max(np.linalg.norm(V), 1e-300)
        # A loose tolerance (the batched configuration's 1e-4) accepts the cached potential as it
        # is: the potential check above amplifies long-wavelength density changes by
        # Khat(k -> 0) ~ 4 pi s / kappa^2, so it cannot confirm a density residual of 1e-4, and
        # the linear-response path only needs exact eigenpairs of H[V] for the V it is given.
        if res < max(1e-7, 100.0 * tol) or tol >= 1e-5:
            return GroundState(V=V, psi=np.asfortranarray(psi), eps=w, rho=rho, m=m, n_orb=n_orb,
                               scf_residual=float(res), iterations=0, seconds=time.time() - t0)
        V_start = V

    if V_start is not None:
        _, _, rho = solve(V_start)
    else:
        rho = _initial_density_1d(sysm, k, initial)
    X, Rr = [], []
    err = np.inf
    it = 0
    for it in range(maxit):
        V = potential(rho)
        w, psi, rho_out = solve(V)
        res = rho_out - rho
        err = float(np.linalg.norm(res) * np.sqrt(h) / sysm.n_elec)
        if verbose:
            print(f"scf {it:3d} residual {err:.3e} gap {w[n_orb] - w[n_orb - 1]:.6f}", flush=True)
        if err < tol:
            break
        X.append(rho.copy())
        Rr.append(res.copy())
        X, Rr = X[-history:], Rr[-history:]
        if len(X) > 1:
            dR = np.array([Rr[i + 1] - Rr[i] for i in range(len(Rr) - 1)]).T
            dX = np.array([X[i + 1] - X[i] for i in range(len(X) - 1)]).T
            gam = np.linalg.lstsq(dR, res, rcond=1e-12)[0]
            rho = rho - dX @ gam + beta * (res - dR @ gam)
        else:
            rho = rho + beta * res
    gs = GroundState(V=V, psi=np.asfortranarray(psi), eps=w, rho=rho_out, m=m, n_orb=n_orb,
                     scf_residual=err, iterations=it + 1, seconds=time.time() - t0)
    if use_cache and err < tol:
        os.makedirs(CACHE_DIR, exist_ok=True)
        np.save(cache_file, V)
    return gs


def _grid_2d(sysm: System):
    nx, ny = sysm.n
    Lx, Ly = sysm.L
    kx = 2.0 * np.pi * np.fft.fftfreq(nx, d=1.0 / nx) / Lx
    ky = 2.0 * np.pi * np.fft.fftfreq(ny, d=1.0 / ny) / Ly
    KX, KY = np.meshgrid(kx, ky)
    return KX, KY, KX ** 2 + KY ** 2


def _lowest_2d(sysm: System, V: np.ndarray, k2: np.ndarray, count: int, dense_limit: int = 4096):
    """Lowest `count` eigenpairs of H = -1/2 Laplacian + V on the 2D grid (x fastest)."""
    nx, ny = sysm.n
    N = nx * ny
    if N <= dense_limit:
        def circ(n, L):
            k = 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n) / L
            t = np.real(np.fft.ifft(0.5 * k ** 2))
            idx = (np.arange(n)[:, None] - np.arange(n)[None, :]) % n
            return t[idx]
        T = np.kron(np.eye(ny), circ(nx, sysm.L[0])) + np.kron(circ(ny, sysm.L[1]), np.eye(nx))
        return sla.eigh(T + np.diag(V), subset_by_index=[0, count - 1], driver="evr")
    import scipy.sparse.linalg as spla
    half_k2 = 0.5 * k2

    def mv(x):
        X = x.reshape(ny, nx, -1) if x.ndim > 1 else x.reshape(ny, nx)
        if X.ndim == 3:
            Y = np.real(np.fft.ifft2(half_k2[:, :, None] * np.fft.fft2(X, axes=(0, 1)), axes=(0, 1)))
            return Y.reshape(N, -1) + V[:, None] * x.reshape(N, -1)
        return np.real(np.fft.ifft2(half_k2 * np.fft.fft2(X))).reshape(N) + V * x.reshape(N)
    op = spla.LinearOperator((N, N), matvec=mv, matmat=mv, dtype=np.float64)
    w, U = spla.eigsh(op, k=count, which="SA", tol=1e-14, ncv=min(N, 2 * count + 40),
                      v0=np.ones(N) / np.sqrt(N))
    order = np.argsort(w)
    return w[order], U[:, order]


def scf_2d(sysm: System, tol: float = 1e-9, maxit: int = 100, beta: float = 0.3, history: int = 12,
           n_extra: int = 4, use_cache: bool = True, verbose: bool = False) -> GroundState:
    """Anderson-mixed SCF for the 2D model; returns exact eigenpairs of H[V] for the final V.

    Dense eigensolver for small grids, Lanczos (ARPACK, FFT matrix-vector products, tolerance
    1e-14) for large ones."""
    t0 = time.time()
    nx, ny = sysm.n
    N = nx * ny
    dV = sysm.dV
    n_orb, f = sysm.n_orb, sysm.occ
    KX, KY, k2 = _grid_2d(sysm)
    khat = 4.0 * np.pi * sysm.scale / (k2 + sysm.kappa ** 2)
    F = np.zeros((ny, nx), dtype=np.complex128)
    G0 = np.zeros((ny, nx), dtype=np.complex128)
    for (Rx, Ry), ZI, sI in zip(sysm.R, sysm.Z, sysm.sigma):
        ph = np.exp(-1j * (KX * Rx + KY * Ry))
        F += -ZI * np.exp(-0.5 * sI ** 2 * k2) * ph
        G0 += ZI * np.exp(-0.5 * 1.5 ** 2 * k2) * ph
    m = np.real(np.fft.ifft2(F)).reshape(N) / dV

    def potential(rho):
        c = np.fft.fft2((rho + m).reshape(ny, nx))
        c[0, 0] = 0.0
        return np.real(np.fft.ifft2(khat * c)).reshape(N)

    def solve(V):
        w, U = _lowest_2d(sysm, V, k2, n_orb + n_extra)
        psi = U[:, :n_orb] / np.sqrt(dV)
        return w, psi, f * np.sum(psi ** 2, axis=1)

    cache_file = os.path.join(CACHE_DIR, sysm.key() + ".npy")
    if use_cache and os.path.exists(cache_file):
        V = np.load(cache_file)
        w, psi, rho = solve(V)
        res = np.linalg.norm(potential(rho) - V) / max(np.linalg.norm(V), 1e-300)
        if res < max(1e-7, 100.0 * tol):
            return GroundState(V=V, psi=np.asfortranarray(psi), eps=w, rho=rho, m=m, n_orb=n_orb,
                               scf_residual=float(res), iterations=0, seconds=time.time() - t0)
    rho = np.real(np.fft.ifft2(G0)).reshape(N) / dV
    X, Rr = [], []
    err = np.inf
    it = 0
    for it in range(maxit):
        V = potential(rho)
        w, psi, rho_out = solve(V)
        res = rho_out - rho
        err = float(np.linalg.norm(res) * np.sqrt(dV) / sysm.n_elec)
        if verbose:
            print(f"scf2d {it:3d} residual {err:.3e} gap {w[n_orb] - w[n_orb - 1]:.6f}", flush=True)
        if err < tol:
            break
        X.append(rho.copy())
        Rr.append(res.copy())
        X, Rr = X[-history:], Rr[-history:]
        if len(X) > 1:
            dR = np.array([Rr[i + 1] - Rr[i] for i in range(len(Rr) - 1)]).T
            dX = np.array([X[i + 1] - X[i] for i in range(len(X) - 1)]).T
            gam = np.linalg.lstsq(dR, res, rcond=1e-12)[0]
            rho = rho - dX @ gam + beta * (res - dR @ gam)
        else:
            rho = rho + beta * res
    gs = GroundState(V=V, psi=np.asfortranarray(psi), eps=w, rho=rho_out, m=m, n_orb=n_orb,
                     scf_residual=err, iterations=it + 1, seconds=time.time() - t0)
    if use_cache and err < tol:
        os.makedirs(CACHE_DIR, exist_ok=True)
        np.save(cache_file, V)
    return gs


def ground_state(sysm: System, **kw) -> GroundState:
    if sysm.dim == 2:
        kw.pop("initial", None)
        return scf_2d(sysm, **kw)
    return scf(sysm, **kw)
