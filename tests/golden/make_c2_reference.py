"""Write the exact dynamical matrix of configuration 2 (1D chain, 128 atoms, N = 5120) from the
CPU oracle only: chi0 by the Adler-Wiser sum over states (Eq. AdlerWiser) from a full
eigendecomposition, U = chi G by GMRES on the Dyson equation (Eq. dyson), D by Eq. SecDeriv.

Usage: python tests/golden/make_c2_reference.py   (about ten minutes on 8 cores)
Output: tests/golden/c2_exact_dmat.npz with D (128 x 128), omega, and the GMRES residual.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import acp_workloads as W  # noqa: E402
from oracle import chi0 as C  # noqa: E402
from oracle import dmat as Dm  # noqa: E402
from oracle.dyson import gmres_columns  # noqa: E402
from oracle.model import Model1D  # noqa: E402


def main():
    t0 = time.time()
    s = W.config(2)
    gs = W.ground_state(s)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    spec = C.full_spectrum(m)

    def chi0(X):
        return C.chi0_apply_sos(m, X, spec)

    rhs = chi0(G)
    U, its = gmres_columns(lambda V: V - chi0(m.apply_K(V)), rhs, tol=1e-13, maxit=150)
    res = np.linalg.norm(U - chi0(m.apply_K(U)) - rhs) / np.linalg.norm(rhs)
    D, asym = Dm.dynamical_matrix(m, U)
    w, _ = Dm.phonons(D)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_exact_dmat.npz")
    np.savez(out, D=D, omega=w, gmres_iterations=its, residual=res, asymmetry=asym, key=s.key())
    print(f"GMRES iterations {its}, residual {res:.2e}, asymmetry {asym:.2e}, {time.time() - t0:.0f} s -> {out}")


if __name__ == "__main__":
    main()
