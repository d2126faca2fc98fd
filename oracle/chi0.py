"""chi0 g: Alg. 1 (Sternheimer) and the Adler-Wiser sum over states (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

With occupation f per orbital the density is rho = f sum_i psi_i^2, so the prefactor 2 of
Eq. AdlerWiser (spinless, f = 1) becomes 2f.  Discrete operators act on grid values with the
quadrature weight h: (chi0 g)(r) = sum_r' chi0(r, r') g(r') h, Q = I - sum_i psi_i psi_i^T h.
"""
from __future__ import annotations

import numpy as np

from .minres import minres


def sternheimer_operator(model):
    """A(V, s) = Q (H - s) Q V, the projected shifted Hamiltonian (Eq. Sternheimer)."""
    def apply(V, s):
        QV = model.project(V)
        return model.project(model.apply_H(QV, s))
    return apply


def chi0_apply(model, G, tol=1e-12, maxit=5000, chunk=2048, return_info=False):
    """Alg. 1 for every column g of G.

    For each occupied i: solve Q(eps_i - H)Q zeta_i = Q(psi_i * g) and accumulate
    u += 2 f psi_i * zeta_i.  The solve is done as Q(H - eps_i)Q x = Q(psi_i * g) with
    zeta_i = -x (the projected operator Q(H - eps_i)Q is positive definite on range(Q)).
    Pairs (i, j) use the stacked index i + j * N_e of Sec. 2.2 and are solved in chunks.
    """
    G = np.asarray(G, dtype=np.float64)
    N, nc = G.shape
    no = model.n_orb
    U = np.zeros((N, nc))
    A = sternheimer_operator(model)
    pairs = np.arange(no * nc)
    its = []
    for s0 in range(0, pairs.size, chunk):
        p = pairs[s0:s0 + chunk]
        i = p % no
        j = p // no
        P = model.psi[:, i] * G[:, j]
        R = model.project(P)
        # a right-hand side that Q annihilates (it lies in the occupied space) is zero; its
        # rounding residue must not be solved for
        tiny = np.linalg.norm(R, axis=0) <= 1e-13 * np.linalg.norm(P, axis=0)
        R[:, tiny] = 0.0
        X, info = minres(A, R, model.eps[i], tol=tol, maxit=maxit, return_info=True, keep=model.project)
        its.append(info["iterations"])
        # the outer Q of Eq. Sternheimer: the solution lies in the unoccupied space
        Z = -model.project(X)
        contrib = 2.0 * model.f * model.psi[:, i] * Z
        np.add.at(U.T, j, contrib.T)
    if return_info:
        return U, dict(iterations=np.concatenate(its))
    return U


def full_spectrum(model):
    """All eigenpairs of the grid Hamiltonian (dense), eigenvectors normalised with weight h."""
    if hasattr(model, "dense_H"):
        H = model.dense_H()
    else:
        N = model.N
        t = np.real(np.fft.ifft(0.5 * model.k ** 2))
        idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
        H = t[idx] + np.diag(model.V)
    w, U = np.linalg.eigh(H)
    return w, U / np.sqrt(model.h)


def chi0_matrix_sos(model, spectrum=None):
    """Dense chi0(r, r') from Eq. AdlerWiser with every unoccupied state of the grid Hamiltonian.

    chi0 = 2f sum_{i <= N_e} sum_{a > N_e} (psi_i psi_a)(psi_i psi_a)^T / (eps_i - eps_a);
    the returned matrix C satisfies chi0 g = C @ g * h.
    """
    w, Phi = full_spectrum(model) if spectrum is None else spectrum
    no = model.n_orb
    C = np.zeros((model.N, model.N))
    for i in range(no):
        P = Phi[:, i:i + 1] * Phi[:, no:]
        C += (P / (w[i] - w[no:])) @ P.T
    return 2.0 * model.f * C


def chi0_apply_sos(model, G, spectrum=None):
    """chi0 G from Eq. AdlerWiser without forming the N x N matrix (large grids, few columns).

    For each column g: chi0 g = 2f sum_i psi_i * [sum_{a > N_e} phi_a (phi_a . (psi_i g) h) / (eps_i - eps_a)].
    """
    w, Phi = full_spectrum(model) if spectrum is None else spectrum
    no = model.n_orb
    Pu, wu = Phi[:, no:], w[no:]
    Po, wo = Phi[:, :no], w[:no]
    G = np.asarray(G, dtype=np.float64)
    out = np.zeros_like(G)
    for j in range(G.shape[1]):
        M = Po * G[:, j:j + 1]                      # psi_i * g, (N, N_e)
        T = (Pu.T @ M) * model.h                    # (N_u, N_e)
        T /= (wo[None, :] - wu[:, None])
        out[:, j] = 2.0 * model.f * np.sum(Po * (Pu @ T), axis=1)
    return out
