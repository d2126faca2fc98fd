"""ctypes binding of libacp (include/acp.h): argument marshalling only.

Blocks of grid functions are torch CUDA tensors of shape (ncol, N), float64, contiguous: row j is
grid function j, which is the column-major N x ncol layout of the C ABI.  Every computation runs
in the library's CUDA kernels; there is no fallback: a missing library raises at import of the
first context.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_double, c_int, c_longlong, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libacp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "acp.h")

ACP_METHOD_PLAIN = 0
ACP_METHOD_ACP = 1
ACP_PREC_FP64 = 0
ACP_PREC_MIXED = 1
ACP_CNN_WEIGHTS = 19393

STATUS = {0: "ACP_OK", 1: "ACP_E_ARG", 2: "ACP_E_CUDA", 3: "ACP_E_OOM", 4: "ACP_E_NOCONV",
          5: "ACP_E_TIMEOUT", 6: "ACP_E_GAP", 7: "ACP_E_RANK", 8: "ACP_E_NUMERIC"}


class AcpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 2), ("L", c_double * 2)]


class Kernel(ctypes.Structure):
    _fields_ = [("kappa", c_double), ("scale", c_double)]


class Atoms(ctypes.Structure):
    _fields_ = [("n_atoms", c_int), ("R", POINTER(c_double)), ("Z", POINTER(c_double)),
                ("sigma", POINTER(c_double)), ("mass", POINTER(c_double))]


class Options(ctypes.Structure):
    _fields_ = [("method", c_int), ("occ", c_double), ("n_cheb", c_int), ("id_tol", c_double),
                ("sketch_cols", c_int), ("sketch", POINTER(c_double)), ("max_rank", c_int),
                ("stern_tol", c_double), ("stern_maxit", c_int), ("dyson_tol", c_double),
                ("dyson_maxit", c_int), ("rhs_batch", c_int), ("deadline_s", c_double),
                ("project_every", c_int), ("ms_variant", c_int), ("precision", c_int),
                ("use_graphs", c_int), ("fft2d_passes", c_int), ("learned", c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_mu", c_int), ("outer_iters", c_int), ("rhs_solved", c_longlong),
                ("lanczos_steps", c_longlong), ("max_iters", c_longlong), ("max_rel_res", c_double),
                ("ms_solve", c_double), ("ms_compress", c_double), ("ms_total", c_double),
                ("asymmetry", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def declared_symbols():
    """Names of the functions declared in include/acp.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(acp_[a-z0-9_]+)\s*\(", text)))


def load():
    """Load libacp.so (built in-tree by ``paper_1605_08021_gb300.build``); raise if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libacp.so is not built ({LIB_PATH}); run python -m paper_1605_08021_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I = c_void_p, POINTER(c_double), c_int
    sig = {
        "acp_options_default": (None, [POINTER(Options)]),
        "acp_grid_supported": (I, [POINTER(Grid)]),
        "acp_init": (I, [POINTER(P), POINTER(Grid), POINTER(Kernel), P, P, D, I, POINTER(Options), P]),
        "acp_set_options": (I, [P, POINTER(Options)]),
        "acp_apply_chi0": (I, [P, P, I, P, POINTER(Stats)]),
        "acp_dyson_solve": (I, [P, P, I, P, POINTER(Stats)]),
        "acp_perturbations": (I, [P, POINTER(Atoms), P, P, P]),
        "acp_dynamical_matrix": (I, [P, POINTER(Atoms), P, D, P, POINTER(Stats)]),
        "acp_phonons": (I, [P, D, I, D, D]),
        "acp_phonon_dos": (I, [D, I, D, I, ctypes.c_double, D]),
        "acp_batch_dynamical_matrix": (I, [POINTER(P), I, POINTER(Atoms), POINTER(P), POINTER(D), POINTER(Stats),
                                           POINTER(c_int), I]),
        "acp_hamiltonian_apply": (I, [P, P, I, D, P]),
        "acp_project": (I, [P, P, I, P]),
        "acp_project_mixed": (I, [P, P, I, P]),
        "acp_project_noalloc": (I, [P, I, I, c_double, P, I, P, P]),
        "acp_kernel_apply": (I, [P, P, I, I, P]),
        "acp_selftest_wait_timeout": (I, [P, c_double]),
        "acp_sternheimer_solve": (I, [P, P, I, D, P, POINTER(Stats)]),
        "acp_compress": (I, [P, P, I, I, POINTER(c_int), POINTER(c_int), P, D]),
        "acp_cnn_set_weights": (I, [P, POINTER(ctypes.c_float), c_longlong]),
        "acp_cnn_apply": (I, [P, P, I, D, P]),
        "acp_cnn_train_step": (I, [P, I, I, P, P, P, I, ctypes.c_float, D, POINTER(ctypes.c_float)]),
        "acp_cnn_get_weights": (I, [P, POINTER(ctypes.c_float)]),
        "acp_update": (I, [P, P, P, D, I]),
        "acp_profile_enable": (I, [P, I]),
        "acp_profile_get": (I, [P, ctypes.c_char_p, D, POINTER(c_longlong), D, D]),
        "acp_launch_count": (c_longlong, [P]),
        "acp_destroy": (None, [P]),
        "acp_last_error": (ctypes.c_char_p, [P]),
        "acp_status_string": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _tptr(t):
    return c_void_p(t.data_ptr())


def _check_block(t, N, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.dim() != 2 or t.shape[1] != N:
        raise ValueError(f"{name} must have shape (ncol, {N}), got {tuple(t.shape)}")


def options(method=ACP_METHOD_ACP, occ=1.0, n_cheb=16, id_tol=1e-5, sketch=None, max_rank=0,
            stern_tol=1e-11, stern_maxit=5000, dyson_tol=1e-10, dyson_maxit=30, rhs_batch=0,
            deadline_s=0.0, project_every=0, ms_variant=0, precision=0, use_graphs=0, fft2d_passes=0, learned=0):
    """Options as a dict (the sketch Omega, if given, is an (n_cols, r) float64 array)."""
    return dict(method=method, occ=occ, n_cheb=n_cheb, id_tol=id_tol, sketch=sketch, max_rank=max_rank,
                stern_tol=stern_tol, stern_maxit=stern_maxit, dyson_tol=dyson_tol, dyson_maxit=dyson_maxit,
                rhs_batch=rhs_batch, deadline_s=deadline_s, project_every=project_every,
                ms_variant=ms_variant, precision=precision, use_graphs=use_graphs,
                fft2d_passes=fft2d_passes, learned=learned)


class Context:
    """One acp_ctx bound to the current torch CUDA stream."""

    def __init__(self, n_grid, L, kappa, scale, V, psi, eps, opts=None, stream=None):
        """n_grid, L: an integer and a length (1D), or (nx, ny) and (Lx, Ly) (2D, x fastest)."""
        import torch
        self.lib = load()
        if isinstance(n_grid, (tuple, list)) and len(n_grid) == 2:
            self.dim = 2
            self.shape = (int(n_grid[0]), int(n_grid[1]))
            self.Ls = (float(L[0]), float(L[1]))
            self.N = self.shape[0] * self.shape[1]
            self.h = (self.Ls[0] / self.shape[0]) * (self.Ls[1] / self.shape[1])
            self.L = self.Ls[0]
        else:
            n1 = int(n_grid[0]) if isinstance(n_grid, (tuple, list)) else int(n_grid)
            L1 = float(L[0]) if isinstance(L, (tuple, list)) else float(L)
            self.dim = 1
            self.shape = (n1, 0)
            self.Ls = (L1, 0.0)
            self.N = n1
            self.L = L1
            self.h = self.L / self.N
        self.n_orb = int(psi.shape[0])
        _check_block(psi, self.N, "psi")
        if not (V.is_cuda and V.dtype == torch.float64 and V.is_contiguous() and V.numel() == self.N):
            raise TypeError("V must be a contiguous float64 CUDA vector of length N")
        self._eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64)[: self.n_orb])
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._opts = None
        self._sketch = None
        o = self._make_options(opts or options())
        g = Grid(self.dim, (c_int * 2)(*self.shape), (c_double * 2)(*self.Ls))
        k = Kernel(float(kappa), float(scale))
        ptr = c_void_p()
        st = self.lib.acp_init(ctypes.byref(ptr), ctypes.byref(g), ctypes.byref(k), _tptr(V), _tptr(psi),
                               _dptr(self._eps), self.n_orb, ctypes.byref(o), c_void_p(self.stream.cuda_stream))
        self.ptr = ptr
        if st != 0:
            msg = self.lib.acp_last_error(ptr).decode() if ptr.value else "acp_init failed"
            if ptr.value:
                self.lib.acp_destroy(ptr)
                self.ptr = c_void_p()
            raise AcpError(st, msg)

    def _make_options(self, d):
        o = Options()
        o.method = int(d["method"])
        o.occ = float(d["occ"])
        o.n_cheb = int(d["n_cheb"])
        o.id_tol = float(d["id_tol"])
        sk = d.get("sketch")
        if sk is not None:
            self._sketch = np.asfortranarray(np.asarray(sk, dtype=np.float64))
            o.sketch_cols = int(self._sketch.shape[1])
            o.sketch = self._sketch.ctypes.data_as(POINTER(c_double))
        else:
            self._sketch = None
            o.sketch_cols = 0
            o.sketch = None
        o.max_rank = int(d["max_rank"])
        o.stern_tol = float(d["stern_tol"])
        o.stern_maxit = int(d["stern_maxit"])
        o.dyson_tol = float(d["dyson_tol"])
        o.dyson_maxit = int(d["dyson_maxit"])
        o.rhs_batch = int(d["rhs_batch"])
        o.deadline_s = float(d["deadline_s"])
        o.project_every = int(d.get("project_every", 0))
        o.ms_variant = int(d.get("ms_variant", 0))
        o.precision = int(d.get("precision", 0))
        o.use_graphs = int(d.get("use_graphs", 0))
        o.fft2d_passes = int(d.get("fft2d_passes", 0))
        o.learned = int(d.get("learned", 0))
        self._opts = o
        return o

    def set_options(self, **kw):
        d = {k: getattr(self._opts, k) for k, _ in Options._fields_ if k not in ("sketch", "sketch_cols")}
        d["sketch"] = self._sketch
        d.update(kw)
        o = self._make_options(d)
        self._call(self.lib.acp_set_options(self.ptr, ctypes.byref(o)))

    def _call(self, st, allow_noconv=False):
        if st == 0 or (allow_noconv and st == 4):
            return st
        raise AcpError(st, self.lib.acp_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            self.lib.acp_destroy(self.ptr)
            self.ptr = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- entry points -----------------------------------------------------------------------
    def update(self, V, psi, eps):
        _check_block(psi, self.N, "psi")
        self._eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64)[: self.n_orb])
        self._call(self.lib.acp_update(self.ptr, _tptr(V), _tptr(psi), _dptr(self._eps), self.n_orb))

    def profile(self, enable=True):
        self._call(self.lib.acp_profile_enable(self.ptr, int(bool(enable))))

    def profile_get(self, kernel):
        ms, fl, by = c_double(0), c_double(0), c_double(0)
        n = c_longlong(0)
        self._call(self.lib.acp_profile_get(self.ptr, kernel.encode(), ctypes.byref(ms), ctypes.byref(n),
                                            ctypes.byref(fl), ctypes.byref(by)))
        return dict(ms=ms.value, launches=n.value, flops=fl.value, bytes=by.value)

    def launch_count(self):
        return int(self.lib.acp_launch_count(self.ptr))

    def _out(self, ncol):
        import torch
        return torch.empty((ncol, self.N), dtype=torch.float64, device="cuda")

    def apply_chi0(self, G, out=None):
        _check_block(G, self.N, "G")
        out = self._out(G.shape[0]) if out is None else out
        st = Stats()
        self._call(self.lib.acp_apply_chi0(self.ptr, _tptr(G), G.shape[0], _tptr(out), ctypes.byref(st)))
        return out, st.as_dict()

    def dyson_solve(self, G, out=None, allow_noconv=False):
        _check_block(G, self.N, "G")
        out = self._out(G.shape[0]) if out is None else out
        st = Stats()
        self._call(self.lib.acp_dyson_solve(self.ptr, _tptr(G), G.shape[0], _tptr(out), ctypes.byref(st)),
                   allow_noconv)
        return out, st.as_dict()

    def _atoms(self, R, Z, sigma, mass=None):
        self._atom_arrays = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())
                             for a in (R, Z, sigma)]
        m = None if mass is None else np.ascontiguousarray(np.asarray(mass, dtype=np.float64).ravel())
        self._atom_arrays.append(m)
        a = Atoms()
        a.n_atoms = int(self._atom_arrays[1].size)
        a.R, a.Z, a.sigma = (_dptr(x) for x in self._atom_arrays[:3])
        a.mass = _dptr(m) if m is not None else None
        return a

    def perturbations(self, R, Z, sigma):
        """G, B: (dim nA, N), row dim I + a; second derivatives: (nA, N) in 1D, (3 nA, N) in 2D
        (rows 3I + {xx, xy, yy})."""
        a = self._atoms(R, Z, sigma)
        nA = a.n_atoms
        G, B = self._out(self.dim * nA), self._out(self.dim * nA)
        D2 = self._out(nA if self.dim == 1 else 3 * nA)
        self._call(self.lib.acp_perturbations(self.ptr, ctypes.byref(a), _tptr(G), _tptr(B), _tptr(D2)))
        return G, B, D2

    def dynamical_matrix(self, R, Z, sigma, rho, mass=None, U=None, allow_noconv=False):
        a = self._atoms(R, Z, sigma, mass)
        D = np.zeros((self.dim * a.n_atoms, self.dim * a.n_atoms))
        st = Stats()
        Up = _tptr(U) if U is not None else c_void_p()
        self._call(self.lib.acp_dynamical_matrix(self.ptr, ctypes.byref(a), _tptr(rho), _dptr(D), Up,
                                                 ctypes.byref(st)), allow_noconv)
        return D, st.as_dict()

    def phonons(self, D, modes=False):
        D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
        n = D.shape[0]
        w = np.zeros(n)
        M = np.zeros((n, n)) if modes else None
        self._call(self.lib.acp_phonons(self.ptr, _dptr(D), n, _dptr(w), _dptr(M) if modes else None))
        return (w, M.T.copy()) if modes else w

    def hamiltonian_apply(self, X, shifts=None):
        _check_block(X, self.N, "X")
        Y = self._out(X.shape[0])
        sh = None if shifts is None else np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
        self._call(self.lib.acp_hamiltonian_apply(self.ptr, _tptr(X), X.shape[0], _dptr(sh) if sh is not None
                                                  else None, _tptr(Y)))
        return Y

    def project(self, X):
        _check_block(X, self.N, "X")
        Y = self._out(X.shape[0])
        self._call(self.lib.acp_project(self.ptr, _tptr(X), X.shape[0], _tptr(Y)))
        return Y

    def project_mixed(self, X):
        _check_block(X, self.N, "X")
        Y = self._out(X.shape[0])
        self._call(self.lib.acp_project_mixed(self.ptr, _tptr(X), X.shape[0], _tptr(Y)))
        return Y

    def kernel_apply(self, X, inverse=False):
        _check_block(X, self.N, "X")
        Y = self._out(X.shape[0])
        self._call(self.lib.acp_kernel_apply(self.ptr, _tptr(X), X.shape[0], -1 if inverse else 1, _tptr(Y)))
        return Y

    def cnn_set_weights(self, w):
        """acp_cnn_set_weights: w is the packed weight vector (ACP_CNN_WEIGHTS values)."""
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32).ravel())
        self._call(self.lib.acp_cnn_set_weights(self.ptr, w.ctypes.data_as(POINTER(ctypes.c_float)), w.size))

    def cnn_apply(self, R, shifts):
        """acp_cnn_apply: learned initial guesses for the columns of R (rows of the tensor)."""
        _check_block(R, self.N, "R")
        X0 = self._out(R.shape[0])
        sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
        if sh.shape != (R.shape[0],):
            raise ValueError("one shift per column")
        self._call(self.lib.acp_cnn_apply(self.ptr, _tptr(R), R.shape[0], _dptr(sh), _tptr(X0)))
        return X0

    def cnn_train_step(self, grid, R, VS, Xstar, lr, return_grad=False):
        """acp_cnn_train_step on a batch living on grid = (nx, ny): the columns of R, VS (= V - s of
        each sample) and Xstar are the rows of the tensors.  Returns the loss before the step (and
        the gradient if asked)."""
        nx, ny = (int(g) for g in grid)
        for t, nm in ((R, "R"), (VS, "VS"), (Xstar, "Xstar")):
            _check_block(t, nx * ny, nm)
        if not (VS.shape == R.shape == Xstar.shape):
            raise ValueError("R, VS and Xstar differ in shape")
        loss = np.zeros(1)
        g = np.zeros(ACP_CNN_WEIGHTS, dtype=np.float32) if return_grad else None
        self._call(self.lib.acp_cnn_train_step(
            self.ptr, nx, ny, _tptr(R), _tptr(VS), _tptr(Xstar), R.shape[0], float(lr), _dptr(loss),
            g.ctypes.data_as(POINTER(ctypes.c_float)) if return_grad else None))
        return (float(loss[0]), g) if return_grad else float(loss[0])

    def cnn_get_weights(self):
        w = np.zeros(ACP_CNN_WEIGHTS, dtype=np.float32)
        self._call(self.lib.acp_cnn_get_weights(self.ptr, w.ctypes.data_as(POINTER(ctypes.c_float))))
        return w

    def sternheimer_solve(self, Bm, shifts, allow_noconv=False):
        _check_block(Bm, self.N, "B")
        X = self._out(Bm.shape[0])
        sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
        st = Stats()
        self._call(self.lib.acp_sternheimer_solve(self.ptr, _tptr(Bm), Bm.shape[0], _dptr(sh), _tptr(X),
                                                  ctypes.byref(st)), allow_noconv)
        return X, st.as_dict()

    def selftest_wait_timeout(self, wait_s):
        """Status name of acp_selftest_wait_timeout (ACP_E_TIMEOUT when the bounded waits work)."""
        return STATUS.get(self.lib.acp_selftest_wait_timeout(self.ptr, float(wait_s)))

    def compress(self, G, cap=None):
        import torch
        _check_block(G, self.N, "G")
        cap = cap or self.N
        n_mu = c_int(0)
        piv = (c_int * cap)()
        rd = np.zeros(cap)
        Xi = torch.empty((cap, self.N), dtype=torch.float64, device="cuda")
        self._call(self.lib.acp_compress(self.ptr, _tptr(G), G.shape[0], cap, ctypes.byref(n_mu), piv,
                                         _tptr(Xi), _dptr(rd)))
        k = n_mu.value
        return k, np.array(piv[:k], dtype=np.int64), Xi[:k], rd[:k]


def grid_supported(n):
    """acp_grid_supported: whether a context accepts a grid of n points (an int or a 1-tuple, 1D) or
    n = (nx, ny) (2D).  Host only."""
    g = Grid()
    if np.ndim(n) == 0 or len(n) == 1:
        g.dim, g.n[0], g.n[1] = 1, int(np.ravel(n)[0]), 1
    else:
        g.dim, g.n[0], g.n[1] = 2, int(n[0]), int(n[1])
    return load().acp_grid_supported(ctypes.byref(g)) == 0


def phonon_dos(omega, w, sigma):
    """acp_phonon_dos: the phonon spectrum of the frequencies omega at the points w with Gaussian
    width sigma.  Host only."""
    om = np.ascontiguousarray(omega, dtype=np.float64).ravel()
    ws_ = np.ascontiguousarray(w, dtype=np.float64).ravel()
    rho = np.empty_like(ws_)
    st = load().acp_phonon_dos(_dptr(om), om.size, _dptr(ws_), ws_.size, float(sigma), _dptr(rho))
    if st != 0:
        raise AcpError(st, "acp_phonon_dos: n >= 1, sigma > 0 and finite inputs are required")
    return rho


def batch_dynamical_matrix(contexts, atoms, rhos, n_workers=0):
    """acp_batch_dynamical_matrix over several contexts (one per system, each on its own stream).

    atoms: one (R, Z, sigma) per system (host arrays); rhos: one float64 CUDA density per system.
    Returns (list of D, list of stats dicts, list of status names).  Raises AcpError only for an
    invalid call; per-system failures are reported in the status list.
    """
    lib = load()
    n = len(contexts)
    keep = []
    ctx_arr = (c_void_p * n)(*[c.ptr.value for c in contexts])
    at = (Atoms * n)()
    Ds = []
    for i, (R, Z, sig) in enumerate(atoms):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel()) for a in (R, Z, sig)]
        keep.append(arrs)
        at[i].n_atoms = int(arrs[1].size)
        at[i].R, at[i].Z, at[i].sigma = (_dptr(x) for x in arrs)
        at[i].mass = None
        nd = contexts[i].dim * arrs[1].size
        Ds.append(np.zeros((nd, nd)))
    rho_arr = (c_void_p * n)(*[r.data_ptr() for r in rhos])
    D_arr = (POINTER(c_double) * n)(*[_dptr(D) for D in Ds])
    st = (Stats * n)()
    status = (c_int * n)()
    rc = lib.acp_batch_dynamical_matrix(ctx_arr, n, at, rho_arr, D_arr, st, status, int(n_workers))
    if rc == 1 and all(x == 0 for x in status):
        raise AcpError(rc, "invalid batch arguments")
    return Ds, [x.as_dict() for x in st], [STATUS.get(x, str(x)) for x in status]

