"""Write exact columns of the dynamical matrix of one system from the CPU oracle only.

chi0 is applied by the Adler-Wiser sum over states (Eq. AdlerWiser) from a full eigendecomposition
of the grid Hamiltonian, U_j = chi g_j by GMRES on the Dyson equation (Eq. dyson) for the sampled
perturbation columns j, and column j of D by Eq. SecDeriv:
  D[:, j] = h G^T U_j + e_j h (d^2 V_j)^T rho  (2D: the d x d block of the atom)  + d^2 E_II[:, j]
(all masses 1).

Usage: python tests/golden/make_dcols_reference.py <system> <col> [<col> ...]
  <system>: c3 (the 63-atom 2D lattice, 160 x 160 grid) or c4_<i> (chain i of the batched
  configuration, ground state from its cached potential).
Output: tests/golden/<system>_exact_dcols.npz with cols, D_cols (N_p x len(cols)), the GMRES
residual and the system key.  c4_35: about a minute; c3: about fifteen minutes on 8 cores.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import acp_workloads as W  # noqa: E402
from oracle import chi0 as C  # noqa: E402
from oracle.dyson import gmres_columns  # noqa: E402
from oracle.model import Model1D, Model2D  # noqa: E402


def load(name):
    if name == "c3":
        s = W.config(3)
        return s, W.ground_state(s)
    if name.startswith("c4_"):
        s = W.batch_config(4)[int(name[3:])]
        return s, W.ground_state(s, tol=1e-4)
    raise KeyError(name)


def exact_columns(m, cols, spec, tol=1e-13):
    G, _ = m.perturbations()
    Gs = G[:, cols]

    def chi0(X):
        return C.chi0_apply_sos(m, X, spec)

    rhs = chi0(Gs)
    U, its = gmres_columns(lambda V: V - chi0(m.apply_K(V)), rhs, tol=tol, maxit=150)
    res = np.linalg.norm(U - chi0(m.apply_K(U)) - rhs) / np.linalg.norm(rhs)
    Dc = (G.T @ U) * m.h
    d = m.sys.dim
    if d == 1:
        D2 = m.second_derivatives()
        for k, j in enumerate(cols):
            Dc[j, k] += D2[:, j] @ m.rho * m.h
    else:
        blk = np.einsum("r,rIab->Iab", m.rho, m.second_derivative_blocks()) * m.h
        for k, j in enumerate(cols):
            I, b = divmod(j, d)
            Dc[d * I:d * I + d, k] += blk[I][:, b]
    Dc += m.ion_hessian()[:, cols]
    return Dc, its, res


def main(argv):
    name, cols = argv[0], [int(c) for c in argv[1:]]
    t0 = time.time()
    s, gs = load(name)
    m = Model2D(s, gs) if s.dim == 2 else Model1D(s, gs)
    spec = C.full_spectrum(m)
    print(f"{name}: N = {m.N}, N_e = {m.n_orb}, spectrum in {time.time() - t0:.0f} s", flush=True)
    Dc, its, res = exact_columns(m, cols, spec)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_exact_dcols.npz")
    np.savez(out, cols=np.array(cols), D_cols=Dc, gmres_iterations=its, residual=res, key=s.key())
    print(f"GMRES iterations {its}, residual {res:.2e}, {time.time() - t0:.0f} s -> {out}")


if __name__ == "__main__":
    main(sys.argv[1:])
