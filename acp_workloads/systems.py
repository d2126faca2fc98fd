"""Seeded synthetic model systems (atoms, grids, kernel strength) and the random sketch.

This module draws random numbers and lays out geometry; it holds none of the
polarizability / Sternheimer / compression / Dyson / Hessian arithmetic, so the
CPU oracle and the CUDA path can both take their inputs from it.

Model (Sec. 4.1, Eq. 1DHamil and Eq. yukawa): atoms carry Gaussian pseudocharges
m_I(x) = -Z_I / sqrt(2 pi sigma^2) exp(-x^2 / 2 sigma^2) and interact through the
Yukawa kernel, whose Fourier symbol is Khat(k) = 4 pi s / (|k|^2 + kappa^2) with
s = 1/eps0 (times an optional depth scaling).  Atomic units throughout.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

BASE_SEED = 160508021


@dataclasses.dataclass(frozen=True)
class System:
    """One periodic model system.

    dim       : 1 or 2
    n         : grid points per axis (x fastest)
    L         : box lengths per axis (bohr)
    R         : (n_atoms, dim) atom positions in [0, L)
    Z         : (n_atoms,) nuclear charges
    sigma     : (n_atoms,) Gaussian widths of the pseudocharges
    mass      : (n_atoms,) nuclear masses (1 = dynamical matrix is the Hessian)
    kappa     : Yukawa screening parameter
    scale     : prefactor s of Khat = 4 pi s / (k^2 + kappa^2)  (s = 1/eps0)
    occ       : occupation f per orbital (rho = f sum_i psi_i^2)
    name      : label
    """
    name: str
    dim: int
    n: tuple
    L: tuple
    R: np.ndarray
    Z: np.ndarray
    sigma: np.ndarray
    mass: np.ndarray
    kappa: float
    scale: float
    occ: int

    @property
    def n_atoms(self) -> int:
        return int(self.Z.shape[0])

    @property
    def n_grid(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_pert(self) -> int:
        return self.dim * self.n_atoms

    @property
    def n_elec(self) -> int:
        return int(round(float(np.sum(self.Z))))

    @property
    def n_orb(self) -> int:
        ne = self.n_elec
        if ne % self.occ:
            raise ValueError(f"{self.name}: {ne} electrons cannot fill orbitals of occupation {self.occ}")
        return ne // self.occ

    @property
    def h(self) -> tuple:
        return tuple(Li / ni for Li, ni in zip(self.L, self.n))

    @property
    def dV(self) -> float:
        return float(np.prod(self.h))

    def key(self) -> str:
        """Stable identifier of the geometry and parameters (for the ground-state cache)."""
        import hashlib
        m = hashlib.sha256()
        for a in (self.dim, self.n, self.L, self.kappa, self.scale, self.occ):
            m.update(repr(a).encode())
        for arr in (self.R, self.Z, self.sigma):
            m.update(np.ascontiguousarray(arr, dtype=np.float64).tobytes())
        return f"{self.name}-{m.hexdigest()[:12]}"


def _rng(config: int, system: int = 0) -> np.random.Generator:
    return np.random.default_rng(BASE_SEED + 1000 * config + system)


def chain_1d(name, n_atoms, spacing, Z, sigma, kappa, scale, n_grid, occ, displacement=0.0, rng=None,
             mass=1.0) -> System:
    """Periodic 1D chain: atom I sits at (I + 1/2) * spacing plus a uniform displacement."""
    L = n_atoms * spacing
    R = (np.arange(n_atoms) + 0.5) * spacing
    if displacement:
        R = R + rng.uniform(-displacement, displacement, n_atoms)
    Z = np.broadcast_to(np.asarray(Z, dtype=np.float64), (n_atoms,)).copy()
    return System(name=name, dim=1, n=(int(n_grid),), L=(float(L),), R=R.reshape(n_atoms, 1),
                  Z=Z, sigma=np.full(n_atoms, float(sigma)), mass=np.full(n_atoms, float(mass)),
                  kappa=float(kappa), scale=float(scale), occ=int(occ))


def paper_chain(n_atoms=60, eps0=1.0, n_grid=None) -> System:
    """The 1D test system of Sec. 4.1: spacing 2.4, kappa 0.1, Z = 1, sigma 0.3, eps0 = 1 or 10."""
    if n_grid is None:
        n_grid = 10 * n_atoms * 12 // 5  # h = 0.1
    return chain_1d(f"paper1d_na{n_atoms}_eps{eps0:g}", n_atoms, 2.4, 1.0, 0.3, 0.1, 1.0 / eps0,
                    n_grid, occ=1)


def config(index: int) -> System:
    """The benchmark configurations (1-based index, 1D ones; 2D ones are not built).

    1: 8 atoms every 10 bohr (L = 80), Z = 2, sigma = 1, kappa = 0.01, N = 320, occupation 2.
    2: 128 atoms every 10 bohr with uniform +-0.5 displacements, Z uniform in {1, 2}, sigma = 1,
       kappa = 0.01, N = 5120, occupation 1, kernel strength s = 0.5 (the small-gap end of the
       depth-scaling range 0.5-1.0; gap 0.2435).
    """
    if index == 1:
        return chain_1d("chain8_z2", 8, 10.0, 2.0, 1.0, 0.01, 1.0, 320, occ=2)
    if index == 2:
        rng = _rng(2)
        disp = rng.uniform(-0.5, 0.5, 128)
        Z = rng.integers(1, 3, 128).astype(np.float64)
        R = ((np.arange(128) + 0.5) * 10.0 + disp).reshape(128, 1)
        return System(name="chain128_mixed", dim=1, n=(5120,), L=(1280.0,), R=R, Z=Z,
                      sigma=np.ones(128), mass=np.ones(128), kappa=0.01, scale=0.5, occ=1)
    if index == 3:
        # 8 x 8 square lattice, spacing 10 bohr, one vacancy (drawn), Z = 2, sigma = 1.2,
        # kappa = 0.01, grid 160 x 160 (h = 0.5), occupation 2: 63 atoms, 63 orbitals, 126 perturbations
        rng = _rng(3)
        vac = int(rng.integers(0, 64))
        return lattice_2d("lattice8x8_vac", 8, 8, 10.0, 2.0, 1.2, 0.01, 1.0, 160, occ=2, vacancies=(vac,))
    raise ValueError(f"configuration {index} is not available")


def smooth_5(n: int) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5."""
    m = max(int(n), 1)
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def batch_config(index: int = 4, n_sys: int = 64, min_atoms: int = 16, max_atoms: int = 256) -> list:
    """Configuration 4: independent 1D chains of uneven size for the batched form.

    System k draws N_A uniform in [min_atoms, max_atoms], atoms every 10 bohr with uniform
    +-0.5 displacements, Z uniform in {1, 2}, sigma 1, kappa 0.01, kernel strength s uniform in
    [0.3, 1.0] (the depth scaling that spreads the gaps), occupation 1, and the grid N = smallest
    2-3-5-smooth integer >= 40 N_A (h close to 0.25).  Smaller n_sys / max_atoms give the same
    recipe at test sizes."""
    out = []
    for k in range(n_sys):
        rng = _rng(index, k)
        n_atoms = int(rng.integers(min_atoms, max_atoms + 1))
        scale = float(rng.uniform(0.3, 1.0))
        disp = rng.uniform(-0.5, 0.5, n_atoms)
        Z = rng.integers(1, 3, n_atoms).astype(np.float64)
        R = ((np.arange(n_atoms) + 0.5) * 10.0 + disp).reshape(n_atoms, 1)
        n_grid = smooth_5(40 * n_atoms)
        out.append(System(name=f"batch{index}_{k}_na{n_atoms}", dim=1, n=(n_grid,), L=(10.0 * n_atoms,), R=R, Z=Z,
                          sigma=np.ones(n_atoms), mass=np.ones(n_atoms), kappa=0.01, scale=scale, occ=1))
    return out


def lattice_2d(name, nxa, nya, spacing, Z, sigma, kappa, scale, n_grid, occ, vacancies=(), displacement=0.0,
               rng=None, mass=1.0) -> System:
    """Periodic square lattice of nxa x nya sites at ((i + 1/2), (j + 1/2)) * spacing, optional
    vacancies (site indices i + nxa j) and uniform displacements per coordinate; grid n_grid^2."""
    sites = [(i, j) for j in range(nya) for i in range(nxa) if i + nxa * j not in set(vacancies)]
    R = (np.array(sites, dtype=np.float64) + 0.5) * spacing
    if displacement:
        R = R + rng.uniform(-displacement, displacement, R.shape)
    n_atoms = R.shape[0]
    Zv = np.broadcast_to(np.asarray(Z, dtype=np.float64), (n_atoms,)).copy()
    return System(name=name, dim=2, n=(int(n_grid), int(n_grid)), L=(nxa * spacing, nya * spacing), R=R, Z=Zv,
                  sigma=np.full(n_atoms, float(sigma)), mass=np.full(n_atoms, float(mass)), kappa=float(kappa),
                  scale=float(scale), occ=int(occ))


def small_lattice(nxa=2, nya=2, n_grid=32, seed=0, spacing=8.0, occ=1, scale=1.0, mixed=True,
                  displacement=0.3, sigma=1.2) -> System:
    """Small 2D lattices for parity tests (dense eigensolvers and dense chi0 stay cheap)."""
    rng = _rng(91, seed)
    n = nxa * nya
    Z = rng.integers(1, 3, n).astype(np.float64) if mixed else np.full(n, 2.0)
    if occ == 2 and int(Z.sum()) % 2:
        Z[0] = 3.0 - Z[0]
    return lattice_2d(f"lat{nxa}x{nya}_{n_grid}_s{seed}", nxa, nya, spacing, Z, sigma, 0.01, scale, n_grid, occ,
                      displacement=displacement, rng=rng)


def training_lattices(n_sys: int = 200, min_side: int = 3, max_side: int = 5, h: float = 0.5,
                      first: int = 0) -> list:
    """Training systems of the learned initial guess: system k has nxa x nya sites (each uniform
    in [min_side, max_side]) every 10 bohr with uniform +-0.3 displacements and, with probability
    1/2, one random vacancy; Z = 2, sigma 1.2, kappa 0.01, kernel strength 1, occupation 2 (the
    closed-shell recipe of configuration 3, which keeps a gap; Z in {1, 2} alloys at occupation 1
    close it on these lattices), and per axis the smallest 2-3-5-smooth grid with spacing at most
    h."""
    out = []
    for k in range(first, first + n_sys):
        rng = _rng(5, k)
        nxa, nya = (int(v) for v in rng.integers(min_side, max_side + 1, 2))
        vac = (int(rng.integers(0, nxa * nya)),) if rng.random() < 0.5 else ()
        s = lattice_2d(f"train5_{k}_{nxa}x{nya}", nxa, nya, 10.0, 2.0, 1.2, 0.01, 1.0, 8, 2, vacancies=vac,
                       displacement=0.3, rng=rng)
        n = tuple(smooth_5(int(np.ceil(Li / h - 1e-9))) for Li in s.L)
        out.append(System(**{**s.__dict__, "n": n}))
    return out


def mixed_chain(n_atoms: int, n_grid: int, seed: int = 0, scale: float = 0.5) -> System:
    """Config-2 recipe at another size: atoms every 10 bohr with uniform +-0.5 displacements,
    Z uniform in {1, 2}, sigma 1, kappa 0.01, occupation 1 (for mid-size profiling runs)."""
    rng = _rng(50, seed)
    disp = rng.uniform(-0.5, 0.5, n_atoms)
    Z = rng.integers(1, 3, n_atoms).astype(np.float64)
    R = ((np.arange(n_atoms) + 0.5) * 10.0 + disp).reshape(n_atoms, 1)
    return System(name=f"chain{n_atoms}_mixed_s{seed}", dim=1, n=(int(n_grid),), L=(10.0 * n_atoms,), R=R, Z=Z,
                  sigma=np.ones(n_atoms), mass=np.ones(n_atoms), kappa=0.01, scale=scale, occ=1)


def small_chain(n_atoms=4, n_grid=160, seed=0, mixed=True, displacement=0.3, spacing=10.0, occ=1,
                scale=1.0) -> System:
    """Small random chains for parity tests (several tiles and a ragged tail at small sizes)."""
    rng = _rng(90, seed)
    Z = rng.integers(1, 3, n_atoms).astype(np.float64) if mixed else np.full(n_atoms, 2.0)
    if occ == 2 and int(Z.sum()) % 2:
        Z[0] = 3.0 - Z[0]
    sysm = chain_1d(f"small{n_atoms}_{n_grid}_s{seed}", n_atoms, spacing, Z, 1.0, 0.01, scale,
                    n_grid, occ=occ, displacement=displacement, rng=rng)
    return sysm


def srft_sketch(n_cols: int, r: int, seed: int) -> np.ndarray:
    """Real form of the subsampled randomized Fourier transform applied to G (Alg. 2 step 1, Remark).

    Column nu of the SRFT is sum_j exp(-2 pi i j nu / n) eta_j e_j with |eta_j| = 1 random; r
    distinct frequencies nu are drawn.  Its real and imaginary parts give 2r real columns, so the
    returned Omega has shape (n_cols, 2r) (column-major friendly) and G_tilde = G @ Omega.
    """
    rng = np.random.default_rng(BASE_SEED + 7919 * seed + 17)
    u = rng.uniform(0.0, 1.0, n_cols)
    nus = rng.choice(n_cols, size=min(r, n_cols), replace=False)
    j = np.arange(n_cols)
    om = np.empty((n_cols, 2 * len(nus)))
    for t, nu in enumerate(nus):
        ph = 2.0 * np.pi * (u - j * nu / n_cols)
        om[:, 2 * t] = np.cos(ph)
        om[:, 2 * t + 1] = np.sin(ph)
    return om / np.sqrt(n_cols)
