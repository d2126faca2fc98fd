"""MINRES (Paige and Saunders, 1975) for symmetric shifted systems, vectorised over columns.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.2 (below Eq. Sternheimer) names MINRES as the solver of the Sternheimer equations.
Each column j solves (A - s_j I) x_j = b_j from x_j = 0, where A is symmetric and given as a
function on blocks of columns.  The iteration is the textbook one: a Lanczos three-term
recurrence builds an orthonormal basis v_1, v_2, ... of the Krylov space with tridiagonal
coefficients (alpha_k, beta_k); Givens rotations factor that tridiagonal matrix as it grows and
give the residual norm |phibar| for free; the iterate is updated through direction vectors
w_k = (v_k - eps_k w_{k-2} - delta_k w_{k-1}) / gamma_k.  A column stops when
|phibar| <= tol * ||b||; converged columns are frozen.

``keep`` (optional) maps each new Lanczos vector back into a subspace the operator must not
leave.  For the projected Sternheimer operator Q(H - s)Q the occupied space is its null space:
rounding puts tiny occupied components into every Lanczos vector, and the three-term recurrence
multiplies them by the Lanczos polynomials evaluated at 0, which lies outside the spectrum and
grows geometrically with the iteration count.  Projecting each new vector with Q removes them.
"""
from __future__ import annotations

import numpy as np


def minres(apply_A, B, shifts, tol=1e-12, maxit=5000, return_info=False, keep=None):
    """Solve (A - shifts[j]) X[:, j] = B[:, j] for every column j.

    apply_A(V, s) must return A V - s V column-wise for V of shape (N, m) and s of shape (m,).
    """
    B = np.asarray(B, dtype=np.float64)
    N, m = B.shape
    shifts = np.broadcast_to(np.asarray(shifts, dtype=np.float64), (m,)).copy()
    X = np.zeros_like(B)
    beta1 = np.linalg.norm(B, axis=0)
    active = beta1 > 0.0
    safe = np.where(active, beta1, 1.0)
    V = B / safe
    V_prev = np.zeros_like(B)
    Wd = np.zeros_like(B)       # w_{k-1}
    Wd2 = np.zeros_like(B)      # w_{k-2}
    beta = beta1.copy()         # beta_k coefficient multiplying v_{k-1} in the next step
    beta_prev_used = np.zeros(m)
    cs = -np.ones(m)
    sn = np.zeros(m)
    dbar = np.zeros(m)
    epsln = np.zeros(m)
    phibar = beta1.copy()
    iters = np.zeros(m, dtype=np.int64)
    first = True
    for it in range(maxit):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        v = V[:, idx]
        P = apply_A(v, shifts[idx])
        if not first:
            P -= beta_prev_used[idx] * V_prev[:, idx]
        alpha = np.einsum("ij,ij->j", v, P)
        P -= alpha * v
        if keep is not None:
            P = keep(P)
        beta_next = np.linalg.norm(P, axis=0)
        # Givens QR of the growing tridiagonal matrix
        oldeps = epsln[idx]
        delta = cs[idx] * dbar[idx] + sn[idx] * alpha
        gbar = sn[idx] * dbar[idx] - cs[idx] * alpha
        epsln[idx] = sn[idx] * beta_next
        dbar[idx] = -cs[idx] * beta_next
        gamma = np.maximum(np.hypot(gbar, beta_next), np.finfo(float).tiny)
        c_new = gbar / gamma
        s_new = beta_next / gamma
        phi = c_new * phibar[idx]
        phibar[idx] = s_new * phibar[idx]
        cs[idx] = c_new
        sn[idx] = s_new
        w_new = (v - oldeps * Wd2[:, idx] - delta * Wd[:, idx]) / gamma
        Wd2[:, idx] = Wd[:, idx]
        Wd[:, idx] = w_new
        X[:, idx] += phi * w_new
        iters[idx] += 1
        # next Lanczos vector
        V_prev[:, idx] = v
        beta_prev_used[idx] = beta_next
        V[:, idx] = P / np.where(beta_next > 0, beta_next, 1.0)
        first = False
        done = (np.abs(phibar[idx]) <= tol * beta1[idx]) | (beta_next == 0.0)
        active[idx[done]] = False
    if return_info:
        return X, dict(iterations=iters, residual_estimate=np.abs(phibar) / np.where(beta1 > 0, beta1, 1.0),
                       converged=~active)
    return X
