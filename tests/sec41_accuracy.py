"""Oracle runs of the accuracy figures of Sec. 4.1 (Table 1, Table 2, Fig. adapconv) on the 60-atom
chain of that section.  Not a test: one cell takes minutes on the host (N_c N_mu MINRES solves of
1440 points per Alg. 4 iteration).

For every Alg. 4 iteration it prints N_mu, the relative error of U = chi G against the dense
Dyson solve (Frobenius and spectral norm) and the L-infinity error of the phonon frequencies
(M_I = 1).

  python tests/sec41_accuracy.py --eps0 10 --n-cheb 5 --l 3          # Table 1 cell (fixed N_mu = 3 N_e)
  python tests/sec41_accuracy.py --eps0 1 --n-cheb 20 --id-tol 1e-3  # Table 2 / Fig. adapconv
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import acp_workloads as W  # noqa: E402
from oracle import acp as A  # noqa: E402
from oracle import dmat as DM  # noqa: E402
from oracle import dyson as Dy  # noqa: E402
from oracle.model import Model1D  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--eps0", type=float, default=10.0, help="1: insulating chain, 10: semiconducting chain")
    ap.add_argument("--n-cheb", type=int, default=5)
    ap.add_argument("--l", type=int, default=0, help="fix N_mu = l N_e (Table 1); 0: use --id-tol (Table 2)")
    ap.add_argument("--id-tol", type=float, default=1e-3)
    ap.add_argument("--sketch-r", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--stern-tol", type=float, default=1e-10)
    args = ap.parse_args(argv)

    s = W.paper_chain(60, args.eps0)
    gs = W.ground_state(s, use_cache=False, tol=1e-10)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    U_ref = Dy.dyson_dense(m, G)
    w_ref = DM.phonons(DM.dynamical_matrix(m, U_ref)[0])[0]
    om = W.srft_sketch(G.shape[1], args.sketch_r, args.seed)
    eps_tol, cap = (0.0, args.l * m.n_orb) if args.l > 0 else (args.id_tol, None)
    hist = []
    A.chi_acp(m, G, om, eps_tol, args.n_cheb, delta=0.0, maxit=args.iters, tol=args.stern_tol, history=hist,
              max_rank=cap)
    print(f"chain eps0={args.eps0:g}: N_g={m.N}, N_e={m.n_orb}, N_c={args.n_cheb}, "
          + (f"N_mu={args.l} N_e" if cap else f"eps={args.id_tol:g}"))
    for k, h in enumerate(hist):
        E = h["U"] - U_ref
        w = DM.phonons(DM.dynamical_matrix(m, h["U"])[0])[0]
        print(f"iteration {k + 1}: N_mu {h['n_mu']}, U error {np.linalg.norm(E) / np.linalg.norm(U_ref):.4e} "
              f"(Frobenius) {np.linalg.norm(E, 2) / np.linalg.norm(U_ref, 2):.4e} (spectral), "
              f"omega Linf error {np.abs(w - w_ref).max():.4e}")


if __name__ == "__main__":
    main()
