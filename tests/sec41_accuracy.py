"""Oracle runs of the accuracy figures of Sec. 4.1 (Table 1, Table 2, Fig. adapconv) on the 60-atom
chain of that section.  Not a test: one cell takes minutes on the host (N_c N_mu MINRES solves of
1440 points per Alg. 4 iteration).

For every Alg. 4 iteration it prints N_mu, the relative error of U = chi G against the dense
Dyson solve (Frobenius and spectral norm) and the L-infinity error of the phonon frequencies
(M_I = 1).

  python tests/sec41_accuracy.py --eps0 10 --n-cheb 5 --l 3          # Table 1 cell (fixed N_mu = 3 N_e)
  python tests/sec41_accuracy.py --eps0 1 --n-cheb 20 --id-tol 1e-3  # Table 2 / Fig. adapconv

With --gpu the ACP result comes from the library (acp_dyson_solve, FP64, on cuda:0) instead of the
oracle's Alg. 4, for one cell or, with --table1, all 16 cells of Table 1; the reference U stays the
oracle's dense Dyson solve.  Only the final iterate is printed for each cell.
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
    ap.add_argument("--gpu", action="store_true", help="ACP by the library on cuda:0")
    ap.add_argument("--table1", action="store_true", help="with --gpu: every cell of Table 1")
    args = ap.parse_args(argv)

    s = W.paper_chain(60, args.eps0)
    gs = W.ground_state(s, use_cache=False, tol=1e-10)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    U_ref = Dy.dyson_dense(m, G)
    w_ref = DM.phonons(DM.dynamical_matrix(m, U_ref)[0])[0]
    om = W.srft_sketch(G.shape[1], args.sketch_r, args.seed)
    if args.gpu:
        return run_library(args, s, gs, m, G, U_ref, w_ref, om)
    eps_tol, cap = (0.0, args.l * m.n_orb) if args.l > 0 else (args.id_tol, None)
    hist = []
    A.chi_acp(m, G, om, eps_tol, args.n_cheb, delta=0.0, maxit=args.iters, tol=args.stern_tol, history=hist,
              max_rank=cap)
    print(f"chain eps0={args.eps0:g}: N_g={m.N}, N_e={m.n_orb}, N_c={args.n_cheb}, "
          + (f"N_mu={args.l} N_e" if cap else f"eps={args.id_tol:g}"))
    for k, h in enumerate(hist):
        print(f"iteration {k + 1}: N_mu {h['n_mu']}, " + report(m, h["U"], U_ref, w_ref))


def report(m, U, U_ref, w_ref):
    E = U - U_ref
    w = DM.phonons(DM.dynamical_matrix(m, U)[0])[0]
    return (f"U error {np.linalg.norm(E) / np.linalg.norm(U_ref):.4e} (Frobenius) "
            f"{np.linalg.norm(E, 2) / np.linalg.norm(U_ref, 2):.4e} (spectral), "
            f"omega Linf error {np.abs(w - w_ref).max():.4e}")


def run_library(args, s, gs, m, G, U_ref, w_ref, om):
    import torch

    import paper_1605_08021_gb300 as P
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), dtype=torch.float64, device="cuda")
    Gd = torch.tensor(np.ascontiguousarray(G.T), dtype=torch.float64, device="cuda")
    cells = [(nc, l) for nc in (5, 10, 15, 20) for l in (3, 4, 5, 6)] if args.table1 else [(args.n_cheb, args.l)]
    for nc, l in cells:
        cap = l * m.n_orb if l > 0 else 0
        # dyson_tol must be positive: 1e-300 runs all --iters Alg. 4 iterations
        o = P.options(method=P.ACP_METHOD_ACP, occ=float(s.occ), n_cheb=nc, id_tol=0.0 if cap else args.id_tol,
                      sketch=om, max_rank=cap, stern_tol=args.stern_tol, dyson_tol=1e-300, dyson_maxit=args.iters,
                      precision=P.ACP_PREC_FP64)
        ctx = P.Context(s.n[0], s.L[0], s.kappa, s.scale, V, psi, gs.eps[: gs.n_orb], o)
        U, st = ctx.dyson_solve(Gd, allow_noconv=True)
        torch.cuda.synchronize()
        label = f"N_mu={l} N_e" if cap else f"eps={args.id_tol:g}"
        print(f"library, N_c={nc}, {label}: {st['outer_iters']} Alg. 4 iterations, N_mu {st['n_mu']}, "
              + report(m, U.cpu().numpy().T, U_ref, w_ref), flush=True)
        ctx.close()


if __name__ == "__main__":
    main()
