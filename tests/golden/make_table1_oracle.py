"""Write the oracle's Table 1 (Sec. 4.1) on the semiconducting 60-atom chain (eps0 = 10; the reading
that its N_c = 5 row saturates near 1.7e-3): the relative Frobenius error of U = chi G from Alg. 4
(four iterations, N_mu fixed at l N_e, l = 3..6, N_c = 5, 10, 15, 20; SRFT sketch of 8 complex
columns, seed 0) against the dense Dyson solve.  The compressed Sternheimer equations are solved
exactly in the eigenbasis of the grid Hamiltonian.  Calls only the oracle.

Usage: python tests/golden/make_table1_oracle.py   (about a minute on 8 cores)
Output: tests/golden/table1_oracle.json
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import acp_workloads as W  # noqa: E402
from oracle import acp as A  # noqa: E402
from oracle import chi0 as C  # noqa: E402
from oracle import dyson as Dy  # noqa: E402
from oracle.model import Model1D  # noqa: E402

N_CHEB = (5, 10, 15, 20)
L_FAC = (3, 4, 5, 6)


def table1_cells(cells=None, seed=0):
    """{(N_c, l): relative Frobenius error of U} for the requested cells (all 16 by default)."""
    s = W.paper_chain(60, 10.0)
    gs = W.ground_state(s, use_cache=False, tol=1e-10)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    spec = C.full_spectrum(m)
    U_ref = Dy.dyson_dense(m, G, chi0_mat=C.chi0_matrix_sos(m, spectrum=spec))
    om = W.srft_sketch(G.shape[1], 8, seed)
    out = {}
    for nc, lf in cells or [(a, b) for a in N_CHEB for b in L_FAC]:
        U, _ = A.chi_acp(m, G, om, 0.0, nc, delta=0.0, maxit=4, max_rank=lf * m.n_orb, spectrum=spec)
        out[(nc, lf)] = float(np.linalg.norm(U - U_ref) / np.linalg.norm(U_ref))
    return out


def main():
    cells = table1_cells()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "table1_oracle.json")
    rows = {str(nc): [cells[(nc, lf)] for lf in L_FAC] for nc in N_CHEB}
    with open(out, "w") as f:
        json.dump({"description": "oracle's Alg. 4 on the semiconducting 60-atom chain, seed-0 SRFT sketch of 8 "
                                  "complex columns, four iterations; written by make_table1_oracle.py",
                   "l": list(L_FAC), "rows": rows}, f, indent=1)
    print(rows, "->", out)


if __name__ == "__main__":
    main()
