"""Pins of the phonon-frequency error reading against Table 2 (Sec. 4.1) and of the oracle's exact
eigenbasis solves of Eq. eqncompressU that make Table 2's cells affordable on the host.

Table 2 (insulating 60-atom chain, N_c = 20): the L-infinity error of the phonon frequencies is
3.6436e-4 at eps = 1e-3 (N_mu = 241) and 2.7380e-6 at eps = 1e-5 (N_mu = 359).  Read as the
frequencies of D itself, the rigid-translation mode (omega_ref = 0) carries |domega| =
sqrt(|dlambda|) ~ 1e-3 at eps = 1e-5, 400 times the printed value; read with the acoustic sum rule
imposed by projecting out the rigid translations (oracle.dmat.phonon_error), the oracle lands on
the printed values within the spread of the random sketch.
"""
import json
import os

import numpy as np
import pytest

import acp_workloads as W
from oracle import acp as A
from oracle import chi0 as C
from oracle import dmat as DM
from oracle import dyson as Dy
from oracle.model import Model1D

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_eigenbasis_solves_equal_minres():
    """Eq. eqncompressU solved in the eigenbasis equals the MINRES solve of the same equation."""
    s = W.small_chain(5, 240, 3)
    m = Model1D(s, W.ground_state(s, use_cache=False))
    rng = np.random.default_rng(4)
    Xi = rng.standard_normal((m.N, 7))
    nodes = A.chebyshev_nodes(m.eps[0], m.eps[m.n_orb - 1], 4)
    Zm = A.compressed_solves(m, Xi, nodes, tol=1e-14)
    Ze = A.compressed_solves(m, Xi, nodes, spectrum=C.full_spectrum(m))
    for a, b in zip(Zm, Ze):
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)
    # and it solves the equation: Q(eps_c - H)Q zeta = Q xi
    Aop = C.sternheimer_operator(m)
    for ec, Z in zip(nodes, Ze):
        r = -Aop(Z, np.full(Z.shape[1], ec)) - m.project(Xi)
        assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(m.project(Xi))


def test_translation_projector_and_sum_rule():
    """P removes exactly the rigid translations, and the exact D obeys the acoustic sum rule, so the
    projection leaves it (and its frequencies) unchanged; a D that breaks the rule is changed."""
    s = W.small_chain(4, 160, 0)
    m = Model1D(s, W.ground_state(s, use_cache=False))
    G, _ = m.perturbations()
    D, _ = DM.dynamical_matrix(m, Dy.dyson_dense(m, G))
    P = DM.translation_projector(s.n_atoms, 1)
    assert np.abs(P @ np.ones(s.n_atoms)).max() < 1e-15
    assert np.allclose(P @ P, P, atol=1e-15)
    assert np.abs(D.sum(axis=1)).max() <= 1e-6 * np.abs(D).max()
    assert DM.phonon_error(D, D, s.n_atoms, 1)[0] == 0.0
    assert np.abs(P @ D @ P - D).max() <= 1e-6 * np.abs(D).max()
    # 2D: two translations, index 2 I + a
    P2 = DM.translation_projector(3, 2)
    T = np.zeros((6, 2))
    T[0::2, 0] = 1.0
    T[1::2, 1] = 1.0
    assert np.abs(P2 @ T).max() < 1e-15 and np.linalg.matrix_rank(P2) == 4
    E = np.zeros_like(D)
    E[0, 0] = 1e-6
    assert DM.phonon_error(D + E, D, s.n_atoms, 1)[0] > 0.0


@pytest.fixture(scope="module")
def chain60():
    s = W.paper_chain(60, 1.0)
    gs = W.ground_state(s, use_cache=False, tol=1e-11)
    m = Model1D(s, gs)
    G, _ = m.perturbations()
    spec = C.full_spectrum(m)
    U = Dy.dyson_dense(m, G, chi0_mat=C.chi0_matrix_sos(m, spectrum=spec))
    D_ref, _ = DM.dynamical_matrix(m, U)
    return s, m, G, spec, D_ref


@pytest.mark.slow
@pytest.mark.parametrize("case", [0, 1])
def test_table2_phonon_errors(chain60, case):
    """Alg. 4 (N_c = 20, SRFT r = 8, four iterations) on the insulating 60-atom chain reproduces
    Table 2's L-infinity phonon errors under the sum-rule reading: the median over three sketches
    within 3x of the printed value, every sketch within 10x; the plain frequencies of D miss the
    eps = 1e-5 value by more than 50x."""
    s, m, G, spec, D_ref = chain60
    cell = json.load(open(os.path.join(GOLDEN, "paper_table2.json")))["cases"][case]
    errs, raw = [], []
    for seed in range(3):
        om = W.srft_sketch(G.shape[1], 8, seed)
        U, _ = A.chi_acp(m, G, om, cell["eps"], 20, delta=0.0, maxit=4, spectrum=spec)
        D, _ = DM.dynamical_matrix(m, U)
        errs.append(DM.phonon_error(D, D_ref, s.n_atoms, 1)[0])
        wr, w = DM.phonons(D_ref)[0], DM.phonons(D)[0]
        raw.append(float(np.abs(w - wr).max()))
    paper = cell["linf_phonon_error"]
    ratio = np.array(errs) / paper
    assert 1 / 3 <= np.median(ratio) <= 3, (errs, paper)
    assert np.all((ratio >= 0.1) & (ratio <= 10)), (errs, paper)
    if cell["eps"] == 1e-5:
        assert min(raw) > 50 * paper, raw


def _table1_module():
    import importlib.util
    path = os.path.join(GOLDEN, "make_table1_oracle.py")
    spec = importlib.util.spec_from_file_location("make_table1_oracle", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.slow
def test_table1_oracle_cells_match_paper_and_stored():
    """Table 1 (Sec. 4.1), semiconducting 60-atom chain: the oracle's Alg. 4 reproduces the printed
    relative errors of U within the spread of the random sketch (10x per cell), keeps the table's
    shape (N_mu = 3 N_e leaves ~2e-2 at every N_c; the N_c = 5 row saturates at the 5-node
    interpolation error above 1e-3; more points and nodes go below 1e-4), and reproduces the stored
    tests/golden/table1_oracle.json that the GPU test compares against."""
    mod = _table1_module()
    cells = [(5, 3), (5, 4), (5, 6), (20, 4), (20, 6)]
    got = mod.table1_cells(cells)
    paper = json.load(open(os.path.join(GOLDEN, "paper_table1.json")))["rows"]
    stored = json.load(open(os.path.join(GOLDEN, "table1_oracle.json")))["rows"]
    for nc, lf in cells:
        e = got[(nc, lf)]
        p = paper[str(nc)][lf - 3]
        assert 0.1 * p <= e <= 10 * p, (nc, lf, e, p)
        assert abs(e - stored[str(nc)][lf - 3]) <= 1e-6 * e, (nc, lf)
    assert got[(5, 3)] > 1e-2 and got[(5, 6)] > 1e-3
    assert abs(got[(5, 4)] - got[(5, 6)]) <= 0.05 * got[(5, 6)]
    assert got[(20, 6)] < 1e-4 < got[(20, 4)]


@pytest.mark.slow
def test_fig_adapconv_convergence(chain60):
    """Fig. adapconv (Sec. 4.1), insulating 60-atom chain, N_c = 20, with the paper's relative L2
    error taken as the spectral norm ||U - U_acp||_2 / ||U||_2: at eps = 1e-3 the first Alg. 4
    iterate is within 15% of the printed 0.0339 and four iterations bring the error below the
    printed 0.0008, at least 100x under the first iterate; at eps = 1e-5 four iterations end at or
    below the printed 'around 1e-5'."""
    s, m, G, spec, D_ref = chain60
    paper = json.load(open(os.path.join(GOLDEN, "paper_fig_adapconv.json")))
    U_ref = Dy.dyson_dense(m, G, chi0_mat=C.chi0_matrix_sos(m, spectrum=spec))
    nref = np.linalg.norm(U_ref, 2)
    for seed in (0, 1):
        om = W.srft_sketch(G.shape[1], 8, seed)
        hist = []
        A.chi_acp(m, G, om, 1e-3, 20, delta=0.0, maxit=4, history=hist, spectrum=spec)
        e = [np.linalg.norm(h["U"] - U_ref, 2) / nref for h in hist]
        p3 = paper["eps_1e-3"]
        assert abs(e[0] / p3["first_iteration"] - 1.0) < 0.15, e
        assert e[-1] < p3["after_four"] and e[-1] < e[0] / 100, e
        hist = []
        A.chi_acp(m, G, om, 1e-5, 20, delta=0.0, maxit=4, history=hist, spectrum=spec)
        e5 = np.linalg.norm(hist[-1]["U"] - U_ref, 2) / nref
        assert e5 <= 2 * paper["eps_1e-5"]["after_four_about"], e5
