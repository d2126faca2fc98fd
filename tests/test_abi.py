"""The C ABI library builds, loads without a GPU and exports every symbol include/acp.h declares;
the ctypes structures have the C layout.  No compute call is made here."""
import ctypes
import os
import subprocess

import pytest

import paper_1605_08021_gb300 as P
from paper_1605_08021_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_08021_gb300.build import build
    build()
    return P.load()


def test_exports_every_declared_symbol(lib):
    syms = P.declared_symbols()
    assert "acp_init" in syms and "acp_apply_chi0" in syms and "acp_phonons" in syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing


def test_status_strings_and_defaults(lib):
    assert lib.acp_status_string(0).decode() == "ok"
    assert "rank" in lib.acp_status_string(7).decode()
    o = B.Options()
    lib.acp_options_default(ctypes.byref(o))
    assert o.method == B.ACP_METHOD_ACP and o.n_cheb == 16 and o.stern_maxit == 5000
    assert abs(o.stern_tol - 1e-11) < 1e-25


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "acp.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(acp_grid), sizeof(acp_kernel),"
        " sizeof(acp_atoms), sizeof(acp_options), sizeof(acp_stats), offsetof(acp_options, sketch),"
        " offsetof(acp_options, project_every), offsetof(acp_stats, asymmetry)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    py = [ctypes.sizeof(B.Grid), ctypes.sizeof(B.Kernel), ctypes.sizeof(B.Atoms), ctypes.sizeof(B.Options),
          ctypes.sizeof(B.Stats), B.Options.sketch.offset, B.Options.project_every.offset, B.Stats.asymmetry.offset]
    assert out == py


def test_null_arguments_are_rejected_without_a_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.acp_init(ctypes.byref(out), None, None, None, None, None, 0, None, None) == 1
    assert lib.acp_apply_chi0(None, None, 0, None, None) == 1
    # the learned initial guess: a null context is refused before any device work
    assert lib.acp_cnn_set_weights(None, None, 0) == 1
    assert lib.acp_cnn_apply(None, None, 1, None, None) == 1
    assert lib.acp_cnn_train_step(None, 8, 8, None, None, None, 1, 0.0, None, None) == 1
    assert lib.acp_cnn_get_weights(None, None) == 1


def _smooth(n):
    for r in (2, 3, 5):
        while n % r == 0:
            n //= r
    return n == 1


def test_grid_support_bounds(lib):
    """Every 2^a 3^b 5^c grid in [8, 10240] is accepted in 1D (the plans that need CTAs of more than
    512 threads take the wide form of the spectral kernels), nothing else is; 2D axes up to 4096."""
    for n in range(1, 10300):
        assert P.grid_supported(n) == (8 <= n <= 10240 and _smooth(n)), n
    assert P.grid_supported((160, 160)) and P.grid_supported((4096, 8))
    assert not P.grid_supported((4320, 8)) and not P.grid_supported((160, 7))
    g = B.Grid()
    g.dim = 3
    assert lib.acp_grid_supported(ctypes.byref(g)) == 1
    assert lib.acp_grid_supported(None) == 1


def test_training_lattices_have_supported_grids_and_closed_shells():
    import acp_workloads as W
    systems = W.training_lattices(208)
    assert len({s.name for s in systems}) == 208
    for s in systems:
        assert P.grid_supported(s.n), s.n
        assert max(s.h) <= 0.5 + 1e-12 and s.n_elec % 2 == 0 and s.n_orb == s.n_elec // 2


def test_benchmark_recipes_match_their_statements(lib):
    """The seeded inputs of configurations 1-4 have the sizes, charges, displacements and
    kernel strengths their recipes state, and every grid is one the library accepts."""
    import numpy as np

    import acp_workloads as W
    c1 = W.config(1)
    assert c1.n == (320,) and c1.L == (80.0,) and c1.occ == 2 and np.all(c1.Z == 2.0)
    assert np.allclose(np.diff(c1.R[:, 0]), 10.0) and c1.n_orb == 8
    c2 = W.config(2)
    site = (np.arange(128) + 0.5) * 10.0
    assert c2.n == (5120,) and c2.occ == 1 and c2.scale == 0.5 and set(np.unique(c2.Z)) == {1.0, 2.0}
    assert np.abs(c2.R[:, 0] - site).max() <= 0.5 and c2.n_orb == int(c2.Z.sum())
    c3 = W.config(3)
    assert c3.n == (160, 160) and c3.R.shape == (63, 2) and c3.occ == 2 and c3.n_orb == 63
    c4 = W.batch_config(4)
    assert len(c4) == 64 and len({s.name for s in c4}) == 64
    for s in c4:
        na = s.R.shape[0]
        assert 16 <= na <= 256 and 0.3 <= s.scale <= 1.0 and s.occ == 1
        assert s.n[0] == W.systems.smooth_5(40 * na) and s.n[0] >= 40 * na
        assert 0.23 < s.h[0] <= 0.25 + 1e-12 and P.grid_supported(s.n), s.name
        assert np.abs(s.R[:, 0] - (np.arange(na) + 0.5) * 10.0).max() <= 0.5
    # seeded: the same recipe gives the same systems
    assert all(np.array_equal(a.R, b.R) and np.array_equal(a.Z, b.Z) for a, b in zip(c4, W.batch_config(4)))
    for P_ in (c1, c2, c3):
        assert P.grid_supported(P_.n)
