"""FP64 CPU oracle for the P1 pressure system (Section 3.4, weak problem).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library (only the seeded input generator feeds
both).

The arithmetic lives in ``pressure_oracle.c`` (plain C, FP64, built with
-ffp-contract=off); this module compiles it on first use with gcc and wraps it
with ctypes.  Every function takes and returns vectors in the caller's full
node numbering: Dirichlet nodes are eliminated inside (rows and columns
removed, Section 3.6 homogeneous Dirichlet) and come back as 0.

Parity status: every function here is pinned by ``tests/test_oracle.py``
(closed-form stencils, textbook consistent mass, brute-force quadrature,
symmetry / zero row sums / patch test, SPD checks, direct vs CG solves,
manufactured-solution O(h^2) convergence).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pressure_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = C.POINTER(C.c_int64)
_dp = C.POINTER(C.c_double)


class _Csr(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_free", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", _i64p), ("col", _i64p), ("val", _dp),
                ("free_of_node", _i64p), ("node_of_free", _i64p)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (idempotent)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.orc_element_matrix.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double,
                                           _dp, _dp, _dp, _dp, _dp]
        lib.orc_element_matrix.restype = C.c_int
        lib.orc_assemble.argtypes = [C.c_int, C.c_int64, _dp, C.c_int64, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_uint8), _dp, _dp, C.c_double, C.c_int,
                                     C.POINTER(C.POINTER(_Csr))]
        lib.orc_assemble.restype = C.c_int
        lib.orc_csr_free.argtypes = [C.POINTER(_Csr)]
        lib.orc_csr_free.restype = None
        lib.orc_spmv.argtypes = [C.POINTER(_Csr), _dp, _dp]
        lib.orc_spmv.restype = None
        lib.orc_cg.argtypes = [C.POINTER(_Csr), _dp, _dp, C.c_int, C.c_double, C.c_int64,
                               C.c_int, _dp]
        lib.orc_cg.restype = C.c_int
        lib.orc_cholesky_solve.argtypes = [C.POINTER(_Csr), _dp, _dp]
        lib.orc_cholesky_solve.restype = C.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = C.c_int
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_set_threads.restype = None
        _lib = lib
        return lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def element_matrices(dim, xv, alpha_v, beta, dt2):
    """(A^e, M^e, K^e, |T|, det) of one simplex; xv [(d+1), d]."""
    lib = _load()
    nv = dim + 1
    xv = np.ascontiguousarray(xv, dtype=np.float64).reshape(nv * dim)
    av = np.ascontiguousarray(alpha_v, dtype=np.float64).reshape(nv)
    Ae, Me, Ke = (np.zeros(nv * nv) for _ in range(3))
    vol, det = C.c_double(), C.c_double()
    rc = lib.orc_element_matrix(dim, _p(xv, C.c_double), _p(av, C.c_double), float(beta),
                                float(dt2), _p(Ae, C.c_double), _p(Me, C.c_double),
                                _p(Ke, C.c_double), C.byref(vol), C.byref(det))
    if rc != 0:
        raise ValueError("degenerate element")
    return Ae.reshape(nv, nv), Me.reshape(nv, nv), Ke.reshape(nv, nv), vol.value, det.value


class PressureMatrix:
    """The assembled reduced matrix (free nodes only) of one pressure system."""

    def __init__(self, dim, coords, conn, dirichlet, alpha, beta, dt2, part: int = 0):
        lib = _load()
        self._lib = lib
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
        alpha = np.ascontiguousarray(alpha, dtype=np.float64)
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        out = C.POINTER(_Csr)()
        rc = lib.orc_assemble(int(dim), coords.shape[0], _p(coords, C.c_double), conn.shape[0],
                              _p(conn, C.c_int32), _p(dirichlet, C.c_uint8),
                              _p(alpha, C.c_double), _p(beta, C.c_double), float(dt2),
                              int(part), C.byref(out))
        if rc != 0:
            raise ValueError("oracle assembly failed (%d)" % rc)
        self._h = out
        s = out.contents
        self.n_nodes = int(s.n_nodes)
        self.n_free = int(s.n_free)
        self.nnz = int(s.nnz)
        nf = self.n_free
        self.rowptr = np.ctypeslib.as_array(s.rowptr, shape=(nf + 1,)).copy()
        self.col = np.ctypeslib.as_array(s.col, shape=(max(self.nnz, 1),))[:self.nnz].copy()
        self.val = np.ctypeslib.as_array(s.val, shape=(max(self.nnz, 1),))[:self.nnz].copy()
        self.free_of_node = np.ctypeslib.as_array(s.free_of_node, shape=(self.n_nodes,)).copy()
        self.node_of_free = np.ctypeslib.as_array(s.node_of_free, shape=(max(nf, 1),))[:nf].copy()

    @classmethod
    def from_case(cls, case, part: int = 0, beta=None):
        return cls(case.dim, case.coords, case.conn, case.dirichlet, case.alpha,
                   case.beta if beta is None else beta, case.dt2, part)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            self._lib.orc_csr_free(h)
            self._h = None

    # reduced <-> full
    def restrict(self, v_full):
        return np.ascontiguousarray(np.asarray(v_full, dtype=np.float64)[self.node_of_free])

    def extend(self, v_red):
        out = np.zeros(self.n_nodes)
        out[self.node_of_free] = v_red
        return out

    def dense(self):
        A = np.zeros((self.n_free, self.n_free))
        for r in range(self.n_free):
            A[r, self.col[self.rowptr[r]:self.rowptr[r + 1]]] = self.val[self.rowptr[r]:self.rowptr[r + 1]]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n_free, self.n_free))

    def matvec_reduced(self, x_red):
        x = np.ascontiguousarray(x_red, dtype=np.float64)
        y = np.zeros(self.n_free)
        self._lib.orc_spmv(self._h, _p(x, C.c_double), _p(y, C.c_double))
        return y

    def apply(self, x_full):
        """y = A x with Dirichlet rows and columns removed; y = 0 on Dirichlet nodes."""
        return self.extend(self.matvec_reduced(self.restrict(x_full)))

    def residual(self, b_full, x_full):
        """True relative residual ||b - A x||_2 / ||b||_2 over the free nodes."""
        b = self.restrict(b_full)
        r = b - self.matvec_reduced(self.restrict(x_full))
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(r) / (nb if nb > 0 else 1.0))

    def cg(self, b_full, x0_full=None, precond: int = 1, tol: float = 1e-13,
           max_it: int = 1_000_000, max_restarts: int = 8):
        """Textbook (Jacobi-)CG; returns (x_full, status, iters, true_rel_res)."""
        b = self.restrict(b_full)
        x = self.restrict(np.zeros(self.n_nodes) if x0_full is None else x0_full)
        stats = np.zeros(3)
        st = self._lib.orc_cg(self._h, _p(b, C.c_double), _p(x, C.c_double), int(precond),
                              float(tol), int(max_it), int(max_restarts), _p(stats, C.c_double))
        return self.extend(x), int(st), int(stats[0]), float(stats[1])

    def cholesky_solve(self, b_full):
        b = self.restrict(b_full)
        x = np.zeros(self.n_free)
        st = self._lib.orc_cholesky_solve(self._h, _p(b, C.c_double), _p(x, C.c_double))
        if st != 0:
            raise np.linalg.LinAlgError("matrix is not SPD (Cholesky pivot <= 0)")
        return self.extend(x)
