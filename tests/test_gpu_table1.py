"""Table 1 (Sec. 4.1) through the library: Alg. 4 (acp_dyson_solve, FP64, four iterations, N_mu fixed
at l N_e by the rank cap) on the semiconducting 60-atom chain for all 16 cells N_c = 5..20 x
l = 3..6, against the oracle's Alg. 4 on the same sketch (tests/golden/table1_oracle.json, written
by tests/golden/make_table1_oracle.py from the oracle only) and against the printed table.

Bars: the library and the oracle run the same Alg. 2-4 on the same sketch; their Sternheimer solves
differ at the solve tolerance (1e-10), which moves the error of U by far less than 1% of itself;
against the paper, whose sketch was another draw, every cell within 10x."""
import json
import os

import numpy as np
import pytest

import acp_workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_table1_all_cells():
    import torch

    import paper_1605_08021_gb300 as P
    from oracle import chi0 as C
    from oracle import dyson as Dy
    from oracle.model import Model1D
    s = W.paper_chain(60, 10.0)
    gs = W.ground_state(s, use_cache=False, tol=1e-10)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    U_ref = Dy.dyson_dense(m, G, chi0_mat=C.chi0_matrix_sos(m))
    om = W.srft_sketch(G.shape[1], 8, 0)
    V = torch.tensor(gs.V, dtype=torch.float64, device="cuda")
    psi = torch.tensor(np.ascontiguousarray(gs.psi.T), dtype=torch.float64, device="cuda")
    Gd = torch.tensor(np.ascontiguousarray(G.T), dtype=torch.float64, device="cuda")
    oracle = json.load(open(os.path.join(GOLDEN, "table1_oracle.json")))["rows"]
    paper = json.load(open(os.path.join(GOLDEN, "paper_table1.json")))["rows"]
    got = {}
    for nc in (5, 10, 15, 20):
        for lf in (3, 4, 5, 6):
            # dyson_tol must be positive: 1e-300 runs all four Alg. 4 iterations
            o = P.options(method=P.ACP_METHOD_ACP, occ=float(s.occ), n_cheb=nc, id_tol=0.0, sketch=om,
                          max_rank=lf * m.n_orb, stern_tol=1e-10, dyson_tol=1e-300, dyson_maxit=4,
                          precision=P.ACP_PREC_FP64)
            ctx = P.Context(s.n[0], s.L[0], s.kappa, s.scale, V, psi, gs.eps[: gs.n_orb], o)
            U, st = ctx.dyson_solve(Gd, allow_noconv=True)  # the capped Alg. 4 stops at its iteration cap
            assert st["n_mu"] == lf * m.n_orb
            e = float(np.linalg.norm(U.cpu().numpy().T - U_ref) / np.linalg.norm(U_ref))
            got[(nc, lf)] = e
            ctx.close()
            ref = oracle[str(nc)][lf - 3]
            assert abs(e - ref) <= 0.01 * ref, (nc, lf, e, ref)
            p = paper[str(nc)][lf - 3]
            assert 0.1 * p <= e <= 10 * p, (nc, lf, e, p)
    for nc in (5, 10, 15, 20):
        row = [got[(nc, lf)] for lf in (3, 4, 5, 6)]
        assert all(b <= 1.05 * a for a, b in zip(row, row[1:])), (nc, row)
