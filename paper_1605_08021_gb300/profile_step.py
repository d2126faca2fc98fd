"""One dynamical matrix of the 128-atom chain (N = 5120, 192 orbitals, 128 perturbations) at the
benchmark's settings (mixed-precision ACP, N_c = 20, id_tol 1e-9, Alg. 4 delta 1e-8, SRFT r = 8),
for profiler captures of single kernels: the launch sequence is the same on every run, so
`ncu -k <kernel> -s <n> -c <m>` selects the same launches.

Usage: python -m paper_1605_08021_gb300.profile_step
"""
from __future__ import annotations

import numpy as np


def main():
    import torch

    import acp_workloads as W
    import paper_1605_08021_gb300 as P
    s = W.config(2)
    gs = W.ground_state(s)
    om = W.srft_sketch(s.n_pert, 8, 2)
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), dtype=torch.float64, device="cuda")
    rho = torch.tensor(gs.rho, dtype=torch.float64, device="cuda")
    o = P.options(occ=float(s.occ), method=P.ACP_METHOD_ACP, sketch=om, id_tol=1e-9, n_cheb=20, dyson_tol=1e-8,
                  dyson_maxit=20, stern_tol=1e-11, precision=P.ACP_PREC_MIXED)
    ctx = P.Context(s.n[0], s.L[0], s.kappa, s.scale, V, psi, gs.eps[: gs.n_orb], o)
    D, st = ctx.dynamical_matrix(s.R[:, 0], s.Z, s.sigma, rho)
    torch.cuda.synchronize()
    print(st)


if __name__ == "__main__":
    main()
