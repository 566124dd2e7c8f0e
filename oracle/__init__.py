"""STA-FEM oracle: plain serial FP64 CPU assembly (ctypes wrapper over sta_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import this package.  The product path (the CUDA library and
its binding) never imports, links or runs it, and the two share no code.

Functions follow STA-FEM (arXiv 2605.11673): Eq. 8 for the assembled operator, Sec. 3.3 for
the rebuild-equality invariant, Sec. 3.5 for the full_rebuild / local_recompute /
streaming_update policies, Eqs. 1-7 and Algorithm 1 for the graph-Laplacian proxy operator,
Eq. 9 (Sec. 6.2) for the implicit-Euler step with the lumped mass.  See sta_oracle.c for the
element formula and summation order.  Every function is pinned by tests/test_oracle_pins.py
against closed forms, invariants, brute force or finite differences; none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sta_oracle.c"
_LIB = _HERE / "_build" / "liboracle_fem.so"
_lib = None

_i64, _f64, _p = C.c_int64, C.c_double, C.c_void_p


def build(force: bool = False) -> Path:
    """Compile sta_oracle.c with gcc -O2 -ffp-contract=off (no FMA contraction)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        _LIB.parent.mkdir(exist_ok=True)
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def use_library(path=None):
    """Bind the wrapper to another build of sta_oracle.c (None: the default build).  Used by the
    mutation tests, which compile deliberately broken copies and check that the pins fail."""
    global _lib
    _lib = None
    return lib(path)


def lib(path=None):
    global _lib
    if _lib is None:
        if path is None:
            build()
        L = C.CDLL(str(path or _LIB))
        L.orc_element.argtypes = [_p, _f64, _f64, _p]
        L.orc_element.restype = C.c_int
        L.orc_element_btdb.argtypes = [_p, _f64, _f64, _p]
        L.orc_element_btdb.restype = C.c_int
        L.orc_element_all.argtypes = [_p, _i64, _p, _p, _p, _p]
        L.orc_element_all.restype = _i64
        L.orc_pattern_create.argtypes = [_i64, _i64, _p]
        L.orc_pattern_create.restype = _p
        L.orc_pattern_free.argtypes = [_p]
        L.orc_pattern_nnz.argtypes = [_p]
        L.orc_pattern_nnz.restype = _i64
        L.orc_pattern_nrows.argtypes = [_p]
        L.orc_pattern_nrows.restype = _i64
        L.orc_pattern_copy.argtypes = [_p, _p, _p, _p]
        L.orc_rebuild.argtypes = [_p, _p, _p, _f64, _p]
        L.orc_entry.argtypes = [_p, _p, _p, _p, _p, _f64, _i64, _i64]
        L.orc_entry.restype = _f64
        L.orc_validate_edits.argtypes = [_i64, _p, _p, _i64]
        L.orc_validate_edits.restype = _i64
        L.orc_local_recompute.argtypes = [_p, _p, _p, _p, _i64, _f64, _p]
        L.orc_local_recompute.restype = _i64
        L.orc_additive_update.argtypes = [_p, _p, _p, _p, _i64, _p]
        L.orc_additive_update.restype = _i64
        L.orc_element_param_grad.argtypes = [_p, _f64, _f64, _p, _p, _p]
        L.orc_element_param_grad.restype = C.c_int
        L.orc_element_x_grad_cs.argtypes = [_p, _f64, _f64, _p, _p]
        L.orc_element_x_grad_cs.restype = C.c_int
        L.orc_grad_all.argtypes = [_p, _p, _p, _p, _p, _p, _p, _p, _p]
        L.orc_grad_all.restype = C.c_int
        L.orc_fx_exponents.argtypes = [_p, _p, _p]
        L.orc_fx_rebuild.argtypes = [_p, _p, _p, _p, _f64, _p, _p]
        L.orc_fx_update.argtypes = [_p, _p, _p, _p, _p, _i64, _f64, _p, _p]
        L.orc_fx_update.restype = _i64
        L.orc_proxy_nnz.argtypes = [_p]
        L.orc_proxy_nnz.restype = _i64
        L.orc_proxy_pattern.argtypes = [_p, _p, _p]
        L.orc_proxy_pattern.restype = None
        L.orc_proxy_rebuild.argtypes = [_p, _p, _f64, _p, _p, _p]
        L.orc_proxy_rebuild.restype = None
        L.orc_proxy_update.argtypes = [_p, _p, _p, _i64, _f64, _p, _p, _p]
        L.orc_proxy_update.restype = _i64
        L.orc_lumped_mass.argtypes = [_p, _p, _f64, _p, _p]
        L.orc_lumped_mass.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def element(x, E: float, nu: float) -> np.ndarray:
    """12x12 element stiffness of one tetrahedron, x = (4, 3) node positions."""
    x = _c(x, np.float64).reshape(12)
    K = np.zeros(144)
    if lib().orc_element(_ptr(x), float(E), float(nu), _ptr(K)) != 0:
        raise ValueError("non-positive determinant")
    return K.reshape(12, 12)


def element_btdb(x, E: float, nu: float) -> np.ndarray:
    """The same matrix formed literally as V B^T D B (independent cross-check)."""
    x = _c(x, np.float64).reshape(12)
    K = np.zeros(144)
    if lib().orc_element_btdb(_ptr(x), float(E), float(nu), _ptr(K)) != 0:
        raise ValueError("non-positive determinant")
    return K.reshape(12, 12)


def element_all(X, tets, E, nu):
    """(T, 144) element matrices and the count of tetrahedra with det <= 0."""
    X = _c(X, np.float64)
    tets = _c(tets, np.int32)
    E = _c(E, np.float64)
    nu = _c(nu, np.float64)
    T = tets.shape[0]
    Ke = np.zeros((T, 144))
    bad = lib().orc_element_all(_ptr(X), T, _ptr(tets), _ptr(E), _ptr(nu), _ptr(Ke))
    return Ke, int(bad)


def element_param_grad(x, E, nu, G):
    x = _c(x, np.float64).reshape(12)
    G = _c(G, np.float64).reshape(144)
    dE, dnu = C.c_double(), C.c_double()
    if lib().orc_element_param_grad(_ptr(x), float(E), float(nu), _ptr(G), C.byref(dE),
                                    C.byref(dnu)) != 0:
        raise ValueError("non-positive determinant")
    return dE.value, dnu.value


def element_x_grad_cs(x, E, nu, G):
    x = _c(x, np.float64).reshape(12)
    G = _c(G, np.float64).reshape(144)
    dx = np.zeros(12)
    if lib().orc_element_x_grad_cs(_ptr(x), float(E), float(nu), _ptr(G), _ptr(dx)) != 0:
        raise ValueError("non-positive determinant")
    return dx.reshape(4, 3)


class Pattern:
    """Superset CSR pattern + scatter map of one mesh (node ids 0..n-1, tets (T, 4))."""

    def __init__(self, n: int, tets):
        self.tets = _c(tets, np.int32)
        self.n, self.T = int(n), int(self.tets.shape[0])
        h = lib().orc_pattern_create(self.n, self.T, _ptr(self.tets))
        if not h:
            raise ValueError("bad mesh (node id out of range, repeated node, or nnz > int32)")
        self._h = C.c_void_p(h)
        self.nnz = int(lib().orc_pattern_nnz(self._h))
        self.nrows = int(lib().orc_pattern_nrows(self._h))
        self.row_ptr = np.zeros(self.nrows + 1, np.int32)
        self.col = np.zeros(self.nnz, np.int32)
        self.scat = np.zeros((self.T, 144), np.int32)
        lib().orc_pattern_copy(self._h, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.scat))

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.orc_pattern_free(self._h)
            self._h = None

    def rebuild(self, Ke, mask, eps: float = 0.0) -> np.ndarray:
        Ke = _c(Ke, np.float64)
        mask = _c(mask, np.uint8)
        val = np.zeros(self.nnz)
        lib().orc_rebuild(self._h, _ptr(Ke), _ptr(mask), float(eps), _ptr(val))
        return val

    def entry(self, X, E, nu, mask, r: int, c: int, eps: float = 0.0) -> float:
        X = _c(X, np.float64)
        E = _c(E, np.float64)
        nu = _c(nu, np.float64)
        mask = _c(mask, np.uint8)
        return lib().orc_entry(self._h, _ptr(X), _ptr(E), _ptr(nu), _ptr(mask), float(eps),
                               int(r), int(c))

    def local_recompute(self, Ke, mask, edits, val, eps: float = 0.0) -> int:
        """In place on mask and val.  Returns the number of distinct touched entries."""
        edits = _c(edits, np.int32).reshape(-1, 3)
        assert mask.dtype == np.uint8 and mask.flags.c_contiguous
        assert val.dtype == np.float64 and val.flags.c_contiguous
        r = lib().orc_local_recompute(self._h, _ptr(_c(Ke, np.float64)), _ptr(mask),
                                      _ptr(edits), edits.shape[0], float(eps), _ptr(val))
        if r < 0:
            raise ValueError(f"invalid edit at index {-r - 2}")
        return int(r)

    def additive_update(self, Ke, mask, edits, val) -> None:
        edits = _c(edits, np.int32).reshape(-1, 3)
        assert mask.dtype == np.uint8 and val.dtype == np.float64
        r = lib().orc_additive_update(self._h, _ptr(_c(Ke, np.float64)), _ptr(mask),
                                      _ptr(edits), edits.shape[0], _ptr(val))
        if r < 0:
            raise ValueError(f"invalid edit at index {-r - 2}")

    # exact additive streaming in fixed point (see orc_fx_exponents)
    def fx_exponents(self, Ke) -> np.ndarray:
        e = np.zeros(self.nnz, np.int32)
        lib().orc_fx_exponents(self._h, _ptr(_c(Ke, np.float64)), _ptr(e))
        return e

    def fx_rebuild(self, Ke, e, mask, eps: float = 0.0):
        """(S, val): exact integer sums and values over the active set."""
        S = np.zeros(self.nnz, np.int64)
        val = np.zeros(self.nnz)
        lib().orc_fx_rebuild(self._h, _ptr(_c(Ke, np.float64)), _ptr(_c(e, np.int32)),
                             _ptr(_c(mask, np.uint8)), float(eps), _ptr(S), _ptr(val))
        return S, val

    def fx_update(self, Ke, e, mask, edits, S, val, eps: float = 0.0) -> None:
        """In place on mask, S and val (additive, O(|Delta|))."""
        edits = _c(edits, np.int32).reshape(-1, 3)
        assert mask.dtype == np.uint8 and S.dtype == np.int64 and val.dtype == np.float64
        r = lib().orc_fx_update(self._h, _ptr(_c(Ke, np.float64)), _ptr(_c(e, np.int32)),
                                _ptr(mask), _ptr(edits), edits.shape[0], float(eps), _ptr(S),
                                _ptr(val))
        if r < 0:
            raise ValueError(f"invalid edit at index {-r - 2}")

    # graph-Laplacian proxy operator (see orc_proxy_rebuild)
    def proxy_pattern(self):
        """(row_ptr (n + 1), col): the node-level superset pattern."""
        nb = int(lib().orc_proxy_nnz(self._h))
        ptr = np.zeros(self.n + 1, np.int32)
        col = np.zeros(nb, np.int32)
        lib().orc_proxy_pattern(self._h, _ptr(ptr), _ptr(col))
        return ptr, col

    def proxy_rebuild(self, mask, eps: float = 0.0):
        """(mult, deg, val): edge multiplicities at both entries of each edge, node degrees,
        and the values of A = L + eps I on the node-level pattern."""
        nb = int(lib().orc_proxy_nnz(self._h))
        mult = np.zeros(nb, np.int32)
        deg = np.zeros(self.n, np.int32)
        val = np.zeros(nb)
        lib().orc_proxy_rebuild(self._h, _ptr(_c(mask, np.uint8)), float(eps), _ptr(mult),
                                _ptr(deg), _ptr(val))
        return mult, deg, val

    def proxy_update(self, mask, edits, mult, deg, val, eps: float = 0.0) -> int:
        """In place on mask, mult, deg and val.  Returns the distinct entries visited."""
        edits = _c(edits, np.int32).reshape(-1, 3)
        assert mask.dtype == np.uint8 and mult.dtype == np.int32 and deg.dtype == np.int32
        assert val.dtype == np.float64
        r = lib().orc_proxy_update(self._h, _ptr(mask), _ptr(edits), edits.shape[0],
                                   float(eps), _ptr(mult), _ptr(deg), _ptr(val))
        if r < 0:
            raise ValueError(f"invalid edit at index {-r - 2}")
        return int(r)

    def lumped_mass(self, X, rho: float, mask) -> np.ndarray:
        """Nodal lumped mass (n,) of the active set (see orc_lumped_mass)."""
        m = np.zeros(self.n)
        lib().orc_lumped_mass(self._h, _ptr(_c(X, np.float64)), float(rho),
                              _ptr(_c(mask, np.uint8)), _ptr(m))
        return m

    def grad_all(self, X, E, nu, mask, grad_val):
        """Reference gradients (dE, dnu per tet, dX (n, 3)) for upstream dL/dval."""
        X = _c(X, np.float64)
        E = _c(E, np.float64)
        nu = _c(nu, np.float64)
        mask = _c(mask, np.uint8)
        gv = _c(grad_val, np.float64)
        dE = np.zeros(self.T)
        dnu = np.zeros(self.T)
        dX = np.zeros((self.n, 3))
        if lib().orc_grad_all(self._h, _ptr(X), _ptr(E), _ptr(nu), _ptr(mask), _ptr(gv),
                              _ptr(dE), _ptr(dnu), _ptr(dX)) != 0:
            raise ValueError("non-positive determinant")
        return dE, dnu, dX

    def csr(self, val):
        """scipy CSR matrix with this pattern and the given values."""
        import scipy.sparse as sp
        return sp.csr_matrix((val, self.col, self.row_ptr), shape=(self.nrows, self.nrows))


def dyn_free(mass, clamped):
    """DOFs the implicit-Euler step solves for: nodes not clamped and with mass (3 per node)."""
    return np.repeat((~np.asarray(clamped, bool)) & (np.asarray(mass) > 0), 3)


def implicit_euler_step(K, mass, u, v, f, h: float, clamped):
    """One step of Sec. 6.2, Eq. 9:  (M + h^2 K) u1 = M (u + h v) + h^2 f  on the free DOFs
    (dyn_free), by a sparse direct solve (scipy spsolve), v1 = (u1 - u) / h there; a clamped
    DOF stays 0 and a DOF of a node without mass keeps its displacement with velocity 0.
    K: the assembled operator (scipy sparse, 3n x 3n); mass: nodal lumped mass (n,);
    b_i = m_i (u_i + h v_i) + (h h) f_i."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    m3 = np.repeat(np.asarray(mass, np.float64), 3)
    free = dyn_free(mass, clamped)
    idx = np.flatnonzero(free)
    A = (sp.diags(m3) + (h * h) * K.tocsr())[idx][:, idx].tocsc()
    b = m3 * (u + h * v) + (h * h) * f
    u1 = np.where(np.repeat(np.asarray(clamped, bool), 3), 0.0, u).astype(np.float64)
    v1 = np.zeros_like(u1)
    if idx.size:
        u1[idx] = spla.spsolve(A, b[idx])
        v1[idx] = (u1[idx] - u[idx]) / h
    return u1, v1


def validate_edits(T: int, mask, edits) -> int:
    """0, or 1 + index of the first invalid edit."""
    edits = _c(edits, np.int32).reshape(-1, 3)
    return int(lib().orc_validate_edits(int(T), _ptr(_c(mask, np.uint8)), _ptr(edits),
                                        edits.shape[0]))


def solve_free(K, f, free):
    """u with K_ff u_f = f_f (sparse direct solve, scipy spsolve), u = 0 on pinned DOFs."""
    import scipy.sparse.linalg as spla
    idx = np.flatnonzero(free)
    Kff = K.tocsr()[idx][:, idx].tocsc()
    u = np.zeros(K.shape[0])
    u[idx] = spla.spsolve(Kff, f[idx])
    return u


def compliance_grad_val(pattern: Pattern, u, free):
    """dL/dval for L = f^T u with K_ff u_f = f_f: -u_i u_j on entries between free DOFs,
    0 elsewhere (pinned DOFs do not enter L)."""
    rows = np.repeat(np.arange(pattern.nrows), np.diff(pattern.row_ptr))
    cols = pattern.col
    g = -u[rows] * u[cols]
    g[~(free[rows] & free[cols])] = 0.0
    return g
