"""Adaptively compressed polarizability: Alg. 2 (Remark variant), Alg. 3 and Alg. 4 (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Steps, in the paper's order and notation:
  Alg. 2 (step 1 as written, or with the Remark): the SRFT of M, or of G only, G_tilde = G Omega (Omega drawn by
    ``acp_workloads.srft_sketch``; complex columns are split into real and imaginary parts).
    Row alpha of M_tilde is the Kronecker product psi(r_alpha, :) (x) G_tilde(r_alpha, :), with
    the stacked column index i + t * N_e (Sec. 2.2).  Pivoted QR of M_tilde^T (LAPACK geqp3),
    N_mu = #{mu : |R_mu,mu| >= eps |R_11|}, pivots r_mu, and
    Xi^T = R_11^{-1} R_{1:N_mu,:} Pi^{-1}.
  Eq. eqnparam and the Chebyshev nodes of Sec. 3.1 on [eps_1, eps_Ne]; Lagrange weights in
    product form (Eq. LagPoly).
  Eq. eqncompressU: Q(eps_c - H)Q zeta_{c mu} = Q xi_mu, solved by MINRES one pair at a time.
  Eq. eqnW: W_mu = 2f sum_i psi_i * (sum_c zeta_{c mu} L_c(eps_i)) psi_i(r_mu).
  Eq. chi0gcompress2: chi0_tilde G = W Pi^T G = W G(r_mu, :).
  Alg. 4: U_tilde^0 = B = K^{-1} G; repeat {compress with K U_tilde^k; Eq. dyson4} until
    ||U_tilde^k - U_tilde^{k-1}|| < delta ||U_tilde^k||; U = U_tilde - B.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .chi0 import sternheimer_operator
from .minres import minres


def chebyshev_nodes(e1, eN, n_cheb):
    """eps_c = (e1 + eN)/2 + (e1 - eN)/2 cos(pi (c - 1/2) / N_c), c = 1..N_c (Sec. 3.1).

    A degenerate interval (eN - e1 < 1e-10 max(1, |e1|)) collapses to one node at the midpoint.
    """
    if eN - e1 < 1e-10 * max(1.0, abs(e1)):
        return np.array([0.5 * (e1 + eN)])
    c = np.arange(1, n_cheb + 1)
    return 0.5 * (e1 + eN) + 0.5 * (e1 - eN) * np.cos(np.pi * (c - 0.5) / n_cheb)


def lagrange_weights(nodes, x):
    """L_c(x) = prod_{c' != c} (x - eps_c') / (eps_c - eps_c')  (Eq. LagPoly); shape (N_c, len(x))."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    Lw = np.ones((nodes.size, x.size))
    for c in range(nodes.size):
        for cp in range(nodes.size):
            if cp != c:
                Lw[c] *= (x - nodes[cp]) / (nodes[c] - nodes[cp])
    return Lw


@dataclasses.dataclass
class Compression:
    pivots: np.ndarray   # r_mu (grid indices), length N_mu
    Xi: np.ndarray       # N_g x N_mu interpolation vectors
    Rdiag: np.ndarray    # |diag(R)| of the pivoted QR


def sketch_rows(model, Gk, Omega):
    """M_tilde^T (r N_e x N_g): column alpha is psi(r_alpha,:) (x) G_tilde(r_alpha,:) (Remark)."""
    Gt = np.asarray(Gk, dtype=np.float64) @ np.asarray(Omega, dtype=np.float64)
    N = model.N
    M = (model.psi[:, :, None] * Gt[:, None, :])          # (N, N_e, r): index i fastest after reshape
    return np.transpose(M, (0, 2, 1)).reshape(N, -1).T    # rows ordered i + t N_e


def full_sketch_rows(model, Gk, Omega):
    """Alg. 2 step 1 as written (no Remark): M_tilde = M Omega, where column I = i + N_e j of M is
    psi_i * g_j (Eq. MID) and Omega ((N_e N_p) x n_s) holds the real and imaginary parts of the SRFT
    columns over the index I.  Returns M_tilde^T (n_s x N_g)."""
    Gk = np.asarray(Gk, dtype=np.float64)
    M = (model.psi[:, None, :] * Gk[:, :, None]).reshape(model.N, -1)  # (N, N_p, N_e): I = i + N_e j
    return (M @ np.asarray(Omega, dtype=np.float64)).T


def interpolative_decomposition(model, Gk, Omega, eps_tol, max_rank=None, full=False):
    """Alg. 2 steps 2-4 on the sketched matrix: the Remark's (Omega over the N_p columns of G), or
    with ``full`` step 1 as written (Omega over the N_e N_p columns of M)."""
    MT = full_sketch_rows(model, Gk, Omega) if full else sketch_rows(model, Gk, Omega)
    R, piv = sla.qr(MT, mode="r", pivoting=True)
    d = np.abs(np.diag(R))
    n_mu = int(np.sum(d >= eps_tol * d[0]))
    if max_rank is not None:
        n_mu = min(n_mu, max_rank)
    R11 = np.triu(R[:n_mu, :n_mu])
    XiT = np.empty((n_mu, model.N))
    XiT[:, piv] = sla.solve_triangular(R11, R[:n_mu, :])
    return Compression(pivots=piv[:n_mu].copy(), Xi=XiT.T.copy(), Rdiag=d)


def compressed_solves(model, Xi, nodes, tol=1e-12, maxit=5000, chunk=2048, spectrum=None):
    """Eq. eqncompressU: zeta[c][:, mu] solves Q(eps_c - H)Q zeta = Q xi_mu.

    By MINRES, or, when ``spectrum`` = (w, Phi) holds every eigenpair of the grid Hamiltonian
    (``chi0.full_spectrum``, small grids), exactly in that eigenbasis: on range(Q), spanned by the
    unoccupied eigenvectors phi_a, zeta = sum_{a > N_e} phi_a (phi_a . xi_mu h) / (eps_c - eps_a).
    """
    if spectrum is not None:
        w, Phi = spectrum
        Pu, wu = Phi[:, model.n_orb:], w[model.n_orb:]
        T = (Pu.T @ np.asarray(Xi, dtype=np.float64)) * model.h     # (N_u, N_mu)
        return [Pu @ (T / (ec - wu)[:, None]) for ec in nodes]
    A = sternheimer_operator(model)
    RHS = model.project(Xi)
    n_mu = Xi.shape[1]
    Zs = []
    for ec in nodes:
        Z = np.empty_like(RHS)
        for s0 in range(0, n_mu, chunk):
            sl = slice(s0, min(n_mu, s0 + chunk))
            X = minres(A, RHS[:, sl], np.full(sl.stop - sl.start, ec), tol=tol, maxit=maxit, keep=model.project)
            Z[:, sl] = -model.project(X)  # zeta lies in the unoccupied space (Eq. eqncompressU)
        Zs.append(Z)
    return Zs


def build_W(model, zetas, nodes, pivots):
    """Eq. eqnW with the mu index on zeta (Eq. eqncompressU)."""
    Lw = lagrange_weights(nodes, model.eps)                 # (N_c, N_e)
    W = np.zeros((model.N, pivots.size))
    psi_mu = model.psi[pivots, :]                            # (N_mu, N_e)
    for i in range(model.n_orb):
        Zi = sum(zetas[c] * Lw[c, i] for c in range(len(nodes)))
        W += 2.0 * model.f * model.psi[:, i:i + 1] * Zi * psi_mu[:, i][None, :]
    return W


def compressed_chi0(model, Gk, Omega, eps_tol, n_cheb, tol=1e-12, max_rank=None, spectrum=None):
    """Alg. 3: returns (W, pivots, compression) with chi0_tilde = W Pi^T.

    ``max_rank`` caps N_mu; with ``eps_tol = 0`` it fixes N_mu, as Table 1 does (N_mu = l N_e).
    ``spectrum`` selects the exact eigenbasis solves of ``compressed_solves``.
    """
    comp = interpolative_decomposition(model, Gk, Omega, eps_tol, max_rank=max_rank)
    nodes = chebyshev_nodes(model.eps[0], model.eps[-1], n_cheb)
    zetas = compressed_solves(model, comp.Xi, nodes, tol=tol, spectrum=spectrum)
    W = build_W(model, zetas, nodes, comp.pivots)
    return W, comp.pivots, comp


def chi0_acp_apply(model, G, Omega, eps_tol, n_cheb, tol=1e-12):
    """chi0_tilde G = W Pi^T G (Eq. chi0gcompress2) with the compression built from G itself."""
    W, piv, _ = compressed_chi0(model, G, Omega, eps_tol, n_cheb, tol=tol)
    return W @ np.asarray(G)[piv, :]


def chi_acp(model, G, Omega, eps_tol, n_cheb, delta=1e-9, maxit=8, tol=1e-12, history=None,
            max_rank=None, spectrum=None):
    """Alg. 4: U ~ chi G with the adaptively compressed polarizability (``max_rank`` and
    ``spectrum`` as in ``compressed_chi0``)."""
    G = np.asarray(G, dtype=np.float64)
    B = model.apply_Kinv(G)
    Ut = B.copy()
    iters = 0
    for k in range(maxit):
        Gk = model.apply_K(Ut)
        W, piv, _ = compressed_chi0(model, Gk, Omega, eps_tol, n_cheb, tol=tol, max_rank=max_rank,
                                    spectrum=spectrum)
        S = model.apply_K(W)[piv, :]
        X = np.linalg.solve(np.eye(piv.size) - S, G[piv, :])
        Ut_new = B + W @ X
        iters = k + 1
        change = np.linalg.norm(Ut_new - Ut) / max(np.linalg.norm(Ut_new), 1e-300)
        Ut = Ut_new
        if history is not None:
            history.append(dict(U=Ut - B, n_mu=piv.size, change=change))
        if change < delta:
            break
    return Ut - B, iters
