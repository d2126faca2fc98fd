"""acp_phonon_dos (Eq. phononspec with the Gaussian delta of Sec. 4.1) against the oracle's
phonon_dos.  The entry point is host code (n * n_w exponentials; no GPU, no context), so these
parity tests run without a GPU.

Bar: both sides evaluate the same sum in FP64 and differ only in rounding order (the library
folds 1/n into the prefactor), so 1e-13 relative to the largest value of the spectrum.
"""
import os

import numpy as np
import pytest

import paper_1605_08021_gb300 as P
from oracle import dmat as Dm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_exact_dmat.npz")


@pytest.fixture(scope="module")
def lib():
    from paper_1605_08021_gb300.build import build
    build()
    return P.load()


def _close(a, b):
    return np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("sigma", [0.01, 0.08])
def test_dos_of_the_128_atom_chain_matches_oracle(lib, sigma):
    """The 128 frequencies of the oracle's exact dynamical matrix of the 128-atom chain (two of
    them acoustic, one slightly negative), on a grid of 2001 points and a ragged one of 7."""
    om = np.load(GOLDEN)["omega"]
    for w in (np.linspace(om.min() - 5 * sigma, om.max() + 5 * sigma, 2001), np.array([-1.0, 0.0, 0.013, 0.5,
                                                                                          om.max(), 3.0, 1e3])):
        assert _close(P.phonon_dos(om, w, sigma), Dm.phonon_dos(om, w, sigma))


def test_dos_edge_cases(lib):
    # one mode: the peak of the Gaussian at its frequency, nothing far away
    rho = P.phonon_dos([0.3], [0.3, 0.3 + 40 * 0.02, -1e300], 0.02)
    assert abs(rho[0] - 1.0 / np.sqrt(2 * np.pi * 0.02 ** 2)) <= 1e-14 * rho[0]
    assert rho[1] == 0.0 and rho[2] == 0.0
    # degenerate frequencies count with their multiplicity
    assert _close(P.phonon_dos([0.2, 0.2, 0.5], [0.2, 0.35], 0.05), Dm.phonon_dos([0.2, 0.2, 0.5], [0.2, 0.35], 0.05))
    # no sample points: nothing to write
    assert P.phonon_dos([0.1, 0.2], [], 0.01).size == 0
    for omega, w, sigma in (([], [0.1], 0.01), ([0.1], [0.1], 0.0), ([0.1], [0.1], -1.0), ([0.1], [0.1], np.nan),
                            ([0.1], [0.1], np.inf), ([np.nan], [0.1], 0.01), ([0.1], [np.inf], 0.01)):
        with pytest.raises(P.AcpError) as e:
            P.phonon_dos(omega, w, sigma)
        assert e.value.name == "ACP_E_ARG"
