"""u = chi g from the Dyson equation u = chi0 g + chi0 v_hxc u (Eq. dyson) (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

There is no exchange-correlation kernel in the model (Sec. 4.1), so v_hxc = K, the Yukawa
kernel.  Two routes:
  * dense: U = (I - chi0 K)^{-1} chi0 G with the dense chi0 of the sum over states (Eq. chi);
  * GMRES: the linear system (I - chi0 K) u = chi0 g solved per column by GMRES with
    modified Gram-Schmidt Arnoldi; chi0 is applied by any routine (Alg. 1 by default).
"""
from __future__ import annotations

import numpy as np

from .chi0 import chi0_apply, chi0_matrix_sos


def kernel_matrix(model):
    """Dense matrix of the periodic convolution with K acting on grid values."""
    N = model.N
    if model.sys.dim == 2:
        # column j = K applied to the unit vector e_j, spectrally
        return model.apply_K(np.eye(N))
    kc = np.real(np.fft.ifft(model.khat))
    idx = (np.arange(N)[:, None] - np.arange(N)[None, :]) % N
    return kc[idx]


def dyson_dense(model, G, chi0_mat=None):
    """U = (I - chi0 K)^{-1} chi0 G with chi0 from the sum over states."""
    C = chi0_matrix_sos(model) if chi0_mat is None else chi0_mat
    chi0_op = C * model.h
    Kmat = kernel_matrix(model)
    A = np.eye(model.N) - chi0_op @ Kmat
    return np.linalg.solve(A, chi0_op @ np.asarray(G, dtype=np.float64))


def gmres_columns(apply_A, Bm, tol=1e-12, maxit=200):
    """GMRES (no restart) for A x_j = b_j, all columns in lockstep; A acts on (N, m) blocks."""
    Bm = np.asarray(Bm, dtype=np.float64)
    N, m = Bm.shape
    beta = np.linalg.norm(Bm, axis=0)
    X = np.zeros_like(Bm)
    nz = beta > 0
    if not np.any(nz):
        return X, 0
    Vs = [Bm / np.where(nz, beta, 1.0)]
    Hs = np.zeros((maxit + 1, maxit, m))
    cs = np.zeros((maxit, m))
    sn = np.zeros((maxit, m))
    g = np.zeros((maxit + 1, m))
    g[0] = beta
    k_used = 0
    for k in range(maxit):
        w = apply_A(Vs[k])
        for i in range(k + 1):
            hik = np.einsum("ij,ij->j", Vs[i], w)
            Hs[i, k] = hik
            w = w - hik * Vs[i]
        hn = np.linalg.norm(w, axis=0)
        Hs[k + 1, k] = hn
        Vs.append(w / np.where(hn > 0, hn, 1.0))
        for i in range(k):
            t = cs[i] * Hs[i, k] + sn[i] * Hs[i + 1, k]
            Hs[i + 1, k] = -sn[i] * Hs[i, k] + cs[i] * Hs[i + 1, k]
            Hs[i, k] = t
        r = np.hypot(Hs[k, k], Hs[k + 1, k])
        r = np.where(r > 0, r, 1.0)
        cs[k] = Hs[k, k] / r
        sn[k] = Hs[k + 1, k] / r
        Hs[k, k] = r
        Hs[k + 1, k] = 0.0
        g[k + 1] = -sn[k] * g[k]
        g[k] = cs[k] * g[k]
        k_used = k + 1
        if np.all(np.abs(g[k + 1]) <= tol * np.where(nz, beta, 1.0)):
            break
    for j in range(m):
        if not nz[j]:
            continue
        y = np.linalg.solve(np.triu(Hs[:k_used, :k_used, j]), g[:k_used, j])
        X[:, j] = sum(y[i] * Vs[i][:, j] for i in range(k_used))
    return X, k_used


def dyson_gmres(model, G, chi0=None, tol=1e-11, maxit=200, stern_tol=1e-12):
    """Solve (I - chi0 K) U = chi0 G column by column with GMRES."""
    if chi0 is None:
        def chi0(X):
            return chi0_apply(model, X, tol=stern_tol)
    rhs = chi0(np.asarray(G, dtype=np.float64))

    def A(V):
        return V - chi0(model.apply_K(V))
    return gmres_columns(A, rhs, tol=tol, maxit=maxit)
