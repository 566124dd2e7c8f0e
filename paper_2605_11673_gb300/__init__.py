"""Python binding of libsta (STA-FEM exact streaming assembly on one GB300).

Argument marshalling only: every step of the assembly runs in the CUDA library
(``_build/libsta.so``, built by ``paper_2605_11673_gb300.build``).  There is no CPU or
PyTorch fallback: if the library is missing, the first call into the binding raises
ImportError.

The functions ``sta_*`` mirror the C-ABI of include/sta.h one to one; ``Assembler`` is a
small convenience wrapper around them.  PyTorch is used for device memory of user-side
tensors and for streams (``stream`` arguments accept a ``torch.cuda.Stream``, a raw
``cudaStream_t`` integer, or None for the current torch stream).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libsta.so"

STA_OK, STA_EINVAL, STA_ESTATE, STA_ERANGE, STA_ENOMEM, STA_ECUDA = 0, -1, -2, -3, -4, -5
STA_DEACTIVATE, STA_ACTIVATE, STA_SWAP = 0, 1, 2

# Every symbol declared in include/sta.h.
EXPORTED = (
    "sta_default_options", "sta_create", "sta_destroy", "sta_full_rebuild", "sta_apply_edits",
    "sta_last_touched", "sta_refold", "sta_csr", "sta_scatter_map", "sta_sizes", "sta_mask",
    "sta_recompute_elements", "sta_set_params", "sta_element_matrices", "sta_last_error",
    "sta_status_string", "sta_apply_edits_noalloc", "sta_adjoint", "sta_spmv", "sta_set_launch",
    "sta_batch_create", "sta_batch_size", "sta_batch_instance", "sta_batch_apply_edits",
    "sta_graph_enable", "sta_graph_disable", "sta_set_policy", "sta_proxy_create",
    "sta_proxy_state", "sta_dyn_setup", "sta_dyn_step", "sta_dyn_state", "sta_dyn_set_state",
    "sta_dyn_apply", "sta_solve", "sta_outer_grad", "sta_set_rebuild_form", "sta_set_fold_depth",
    "sta_get_rebuild_form",
)
STA_NOALLOC_MAX_EDITED = 32768
STA_POLICY_REFOLD = 0
STA_POLICY_FIXED = 1
STA_REBUILD_AUTO = 0
STA_REBUILD_FUSED = 1
STA_REBUILD_ZERO_FILL = 2


class StaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libsta status {status}: {message}")
        self.status = status


class sta_options(C.Structure):
    _fields_ = [("eps", C.c_double), ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32)]


class sta_edit(C.Structure):
    _fields_ = [("op", C.c_int32), ("tet", C.c_int32), ("tet2", C.c_int32)]


_lib = None
_p, _i64, _int = C.c_void_p, C.c_int64, C.c_int
_P = C.POINTER


def load_library(path: Path | str | None = None):
    """Load libsta.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = Path(path) if path else LIB_PATH
    if not path.exists():
        raise ImportError(f"libsta not built: {path} is missing "
                          "(run `python -m paper_2605_11673_gb300.build`)")
    L = C.CDLL(str(path))
    L.sta_default_options.argtypes = [_P(sta_options)]
    L.sta_default_options.restype = None
    L.sta_create.argtypes = [_p, _i64, _p, _i64, _p, _p, _P(sta_options), _p, _P(_p)]
    L.sta_destroy.argtypes = [_p]
    L.sta_full_rebuild.argtypes = [_p, _p, _int, _p]
    L.sta_apply_edits.argtypes = [_p, _p, _i64, _p]
    L.sta_apply_edits_noalloc.argtypes = [_p, _p, _i64, _p]
    L.sta_last_touched.argtypes = [_p, _P(_i64), _p]
    L.sta_refold.argtypes = [_p, _p]
    L.sta_csr.argtypes = [_p, _P(_p), _P(_p), _P(_p), _P(_i64), _P(_i64)]
    L.sta_scatter_map.argtypes = [_p, _P(_p)]
    L.sta_sizes.argtypes = [_p, _P(_i64), _P(_i64), _P(_i64), _P(_i64)]
    L.sta_mask.argtypes = [_p, _P(_p)]
    L.sta_recompute_elements.argtypes = [_p, _int, _p]
    L.sta_set_params.argtypes = [_p, _p, _p, _p, _int, _p]
    L.sta_element_matrices.argtypes = [_p, _p, _i64, _p, _p]
    L.sta_adjoint.argtypes = [_p, _p, _p, _p, _p, _p]
    L.sta_spmv.argtypes = [_p, _p, _p, _p, _p]
    L.sta_set_launch.argtypes = [_p, C.c_int32, C.c_int32]
    L.sta_set_rebuild_form.argtypes = [_p, C.c_int32]
    L.sta_set_fold_depth.argtypes = [_p, C.c_int32]
    L.sta_get_rebuild_form.argtypes = [_p, _P(C.c_int32)]
    L.sta_batch_create.argtypes = [C.c_int32, _p, _p, _p, _p, _p, _p, _P(sta_options), _p, _P(_p)]
    L.sta_batch_size.argtypes = [_p, _P(C.c_int32)]
    L.sta_batch_instance.argtypes = [_p, C.c_int32, _P(_p), _P(_p), _P(_p), _P(_i64), _P(_i64),
                                     _P(_i64)]
    L.sta_batch_apply_edits.argtypes = [_p, _p, _p, _p]
    L.sta_graph_enable.argtypes = [_p, _i64, _p]
    L.sta_graph_disable.argtypes = [_p, _p]
    L.sta_set_policy.argtypes = [_p, C.c_int32, _p]
    L.sta_proxy_create.argtypes = [_i64, _p, _i64, C.c_double, _p, _P(_p)]
    L.sta_proxy_state.argtypes = [_p, _P(_p), _P(_p)]
    L.sta_dyn_setup.argtypes = [_p, C.c_double, C.c_double, _p, _p, _p]
    L.sta_dyn_step.argtypes = [_p, C.c_double, C.c_int32, _P(C.c_int32), _P(C.c_double), _p]
    L.sta_dyn_state.argtypes = [_p, _P(_p), _P(_p), _P(_p)]
    L.sta_dyn_set_state.argtypes = [_p, _p, _p, _int, _p]
    L.sta_dyn_apply.argtypes = [_p, _p, _p, _p]
    L.sta_solve.argtypes = [_p, _p, _p, _p, C.c_double, C.c_int32, _p, _P(C.c_int32),
                            _P(C.c_double), _p]
    L.sta_outer_grad.argtypes = [_p, _p, _p, _p, _p, _p]
    L.sta_last_error.restype = C.c_char_p
    L.sta_status_string.argtypes = [_int]
    L.sta_status_string.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("sta_default_options", "sta_last_error", "sta_status_string"):
            getattr(L, name).restype = _int
    _lib = L
    return L


def _check(status: int) -> None:
    if status != STA_OK:
        raise StaError(status, load_library().sta_last_error().decode())


_cuda_ok = None
_raw_stream = None


def _stream_handle(stream) -> int:
    """cudaStream_t of `stream` (None: torch's current stream on the current device)."""
    global _cuda_ok, _raw_stream
    if stream is None:
        import torch
        if _cuda_ok is None:
            _cuda_ok = torch.cuda.is_available()
            # the raw handle without building a Stream object each call, where torch has it
            f = getattr(torch._C, "_cuda_getCurrentRawStream", None)
            if _cuda_ok and f is not None:
                _raw_stream = lambda: f(torch._C._cuda_getDevice())  # noqa: E731
        if not _cuda_ok:
            return 0
        if _raw_stream is not None:
            return _raw_stream()
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a) -> int:
    """Address of a non-empty C-contiguous host array's data: through the buffer protocol,
    which costs half of `a.ctypes.data` on the per-frame path; read-only arrays take the
    latter."""
    try:
        return C.addressof(C.c_char.from_buffer(a))
    except TypeError:
        return a.ctypes.data


# The C-ABI takes plain pointers and cannot see the length of what they point to, so the
# binding checks every array it passes against the context's sizes: a wrong length raises
# here instead of reading or writing past the end of a buffer.

_fixed = {}  # handle -> the sizes fixed for the context's lifetime


def _sizes(h: int) -> dict:
    s = _fixed.get(h)
    if s is None:
        k = C.c_int32()
        _check(load_library().sta_batch_size(h, C.byref(k)))
        s = _fixed[h] = dict(sta_sizes(h), k=int(k.value))
    return s


def _host_n(a, dtype, n: int, what: str):
    """Host copy of `a` as n contiguous elements of dtype."""
    a = _host(a, dtype).reshape(-1)
    if a.size != n:
        raise ValueError(f"{what} must have {n} elements, got {a.size}")
    return a


def _dev(t, n: int, what: str, dtypes=None):
    """`t` as a contiguous CUDA tensor of n elements; dtypes: the accepted dtypes (default
    float64), or () for any."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    dtypes = (torch.float64,) if dtypes is None else dtypes
    if dtypes and t.dtype not in dtypes:
        raise TypeError(f"{what} must be one of {dtypes}, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{what} must have {n} elements, got {t.numel()}")
    return t.contiguous()


def _dev_flags(t, n: int, what: str):
    """A CUDA tensor of n flags (any dtype) as contiguous uint8."""
    import torch
    return _dev(t, n, what, ()).to(torch.uint8).contiguous()


class DeviceArray:
    """Zero-copy view of context-owned device memory (``__cuda_array_interface__``)."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self._ptr, self._shape, self._typestr, self._owner = int(ptr), tuple(shape), typestr, owner

    @property
    def __cuda_array_interface__(self):
        return {"shape": self._shape, "typestr": self._typestr, "data": (self._ptr, False),
                "version": 3, "strides": None}

    def torch(self):
        import torch
        return torch.as_tensor(self, device="cuda")


# ----------------------------------------------------------------------------------------
# One-to-one wrappers of the C-ABI
# ----------------------------------------------------------------------------------------

def sta_default_options() -> sta_options:
    o = sta_options()
    load_library().sta_default_options(C.byref(o))
    return o


def sta_create(nodes, tets, young, poisson, opt: sta_options | None = None, stream=None) -> int:
    L = load_library()
    nodes = _host(nodes, np.float64).reshape(-1, 3)
    tets = _host(tets, np.int32).reshape(-1, 4)
    young = _host(young, np.float64).reshape(-1)
    poisson = _host(poisson, np.float64).reshape(-1)
    if young.shape[0] != tets.shape[0] or poisson.shape[0] != tets.shape[0]:
        raise ValueError("young/poisson must have one value per tetrahedron")
    h = _p()
    _check(L.sta_create(nodes.ctypes.data, nodes.shape[0], tets.ctypes.data, tets.shape[0],
                        young.ctypes.data, poisson.ctypes.data,
                        C.byref(opt) if opt is not None else None, _stream_handle(stream),
                        C.byref(h)))
    _fixed.pop(h.value, None)  # a new context may reuse a destroyed one's address
    return h.value


def sta_proxy_create(n_nodes: int, tets, eps: float = 0.0, stream=None) -> int:
    """Context of the graph-Laplacian proxy operator A = L + eps I (see include/sta.h)."""
    L = load_library()
    tets = _host(tets, np.int32).reshape(-1, 4)
    h = _p()
    _check(L.sta_proxy_create(int(n_nodes), tets.ctypes.data, tets.shape[0], float(eps),
                              _stream_handle(stream), C.byref(h)))
    _fixed.pop(h.value, None)  # a new context may reuse a destroyed one's address
    return h.value


def sta_proxy_state(h: int, owner=None):
    """(mult per block, degree per node) as zero-copy DeviceArrays."""
    m, d = _p(), _p()
    _check(load_library().sta_proxy_state(h, C.byref(m), C.byref(d)))
    s = sta_sizes(h)
    return (DeviceArray(m.value or 0, (s["n_blocks"],), "<i4", owner),
            DeviceArray(d.value or 0, (s["n_nodes"],), "<i4", owner))


def sta_dyn_setup(h: int, rho: float, dt: float, f=None, clamped=None, stream=None) -> None:
    """Implicit-Euler loop (include/sta.h): density, time step, load (3n), clamped nodes (n)."""
    s = _sizes(h)
    fp = _host_n(f, np.float64, s["n_rows"], "f") if f is not None else None
    cp = (_host_n(np.asarray(clamped) != 0, np.uint8, s["n_nodes"], "clamped")
          if clamped is not None else None)
    _check(load_library().sta_dyn_setup(h, float(rho), float(dt),
                                        fp.ctypes.data if fp is not None else None,
                                        cp.ctypes.data if cp is not None else None,
                                        _stream_handle(stream)))


def sta_dyn_step(h: int, tol: float = 1e-10, max_iter: int = 1000, stream=None):
    """One step; returns (CG iterations, relative residual)."""
    it, rr = C.c_int32(), C.c_double()
    _check(load_library().sta_dyn_step(h, float(tol), int(max_iter), C.byref(it), C.byref(rr),
                                       _stream_handle(stream)))
    return int(it.value), float(rr.value)


def sta_dyn_apply(h: int, x, stream=None):
    """y = (M + h^2 K) x on the free DOFs (CUDA float64 tensors of 3n)."""
    x = _dev(x, _sizes(h)["n_rows"], "x")
    y = x.new_empty(x.shape)
    _check(load_library().sta_dyn_apply(h, x.data_ptr(), y.data_ptr(), _stream_handle(stream)))
    return y


def sta_solve(h: int, b, free, val=None, tol: float = 1e-12, max_iter: int = 20000, x0=None,
              stream=None):
    """Jacobi-PCG for A_ff x_f = b_f (CUDA tensors: b float64 3n, free bool/uint8 3n);
    returns (x, iterations, relative residual)."""
    import torch
    s = _sizes(h)
    b = _dev(b, s["n_rows"], "b")
    fr = _dev_flags(free, s["n_rows"], "free")
    x = torch.zeros_like(b) if x0 is None else _dev(x0, s["n_rows"], "x0").clone()
    val = _dev(val, s["nnz"], "val") if val is not None else None
    vp = val.data_ptr() if val is not None else None
    it, rr = C.c_int32(), C.c_double()
    _check(load_library().sta_solve(h, vp, b.data_ptr(), fr.data_ptr(), float(tol), int(max_iter),
                                    x.data_ptr(), C.byref(it), C.byref(rr), _stream_handle(stream)))
    return x, int(it.value), float(rr.value)


def sta_outer_grad(h: int, lam, u, free, stream=None):
    """dL/dval = -lam_i u_j on entries between free DOFs (CUDA tensors)."""
    import torch
    s = _sizes(h)
    lam, u = _dev(lam, s["n_rows"], "lam"), _dev(u, s["n_rows"], "u")
    fr = _dev_flags(free, s["n_rows"], "free")
    g = torch.empty(s["nnz"], dtype=torch.float64, device=lam.device)
    _check(load_library().sta_outer_grad(h, lam.data_ptr(), u.data_ptr(), fr.data_ptr(),
                                         g.data_ptr(), _stream_handle(stream)))
    return g


def sta_dyn_state(h: int, owner=None):
    """(u, v, mass) as zero-copy DeviceArrays."""
    u, v, m = _p(), _p(), _p()
    _check(load_library().sta_dyn_state(h, C.byref(u), C.byref(v), C.byref(m)))
    n = sta_sizes(h)["n_nodes"]
    return (DeviceArray(u.value or 0, (3 * n,), "<f8", owner),
            DeviceArray(v.value or 0, (3 * n,), "<f8", owner),
            DeviceArray(m.value or 0, (n,), "<f8", owner))


def sta_dyn_set_state(h: int, u=None, v=None, stream=None) -> None:
    """Overwrite u and/or v from host arrays."""
    n = _sizes(h)["n_rows"]
    up = _host_n(u, np.float64, n, "u") if u is not None else None
    vp = _host_n(v, np.float64, n, "v") if v is not None else None
    _check(load_library().sta_dyn_set_state(h, up.ctypes.data if up is not None else None,
                                            vp.ctypes.data if vp is not None else None, 0,
                                            _stream_handle(stream)))


def sta_destroy(h: int) -> None:
    _fixed.pop(h, None)
    _check(load_library().sta_destroy(h))


def sta_full_rebuild(h: int, mask, stream=None) -> None:
    """mask: numpy/host array (copied by the library) or a CUDA tensor (device path)."""
    import torch
    L = load_library()
    T = _sizes(h)["n_tets"]
    if hasattr(mask, "is_cuda") and mask.is_cuda:
        m = _dev(mask, T, "mask", (torch.uint8, torch.bool))
        _check(L.sta_full_rebuild(h, m.data_ptr(), 1, _stream_handle(stream)))
    else:
        m = _host_n(mask, np.uint8, T, "mask")
        _check(L.sta_full_rebuild(h, m.ctypes.data, 0, _stream_handle(stream)))


def sta_apply_edits(h: int, edits, stream=None) -> None:
    """edits: (m, 3) int32 rows (op, tet, tet2) in host memory."""
    e = _host(edits, np.int32)
    if e.ndim != 2 or e.shape[1] != 3:
        e = e.reshape(-1, 3)
    n = e.shape[0]
    _check(load_library().sta_apply_edits(h, _ptr(e) if n else None, n, _stream_handle(stream)))


def sta_apply_edits_noalloc(h: int, edits, stream=None) -> None:
    """Allocation-free variant of sta_apply_edits (fixed scratch; see include/sta.h)."""
    e = _host(edits, np.int32).reshape(-1, 3)
    _check(load_library().sta_apply_edits_noalloc(h, e.ctypes.data if e.shape[0] else None,
                                                  e.shape[0], _stream_handle(stream)))


def sta_refold(h: int, stream=None) -> None:
    _check(load_library().sta_refold(h, _stream_handle(stream)))


def sta_last_touched(h: int, stream=None) -> int:
    v = _i64()
    _check(load_library().sta_last_touched(h, C.byref(v), _stream_handle(stream)))
    return int(v.value)


def sta_sizes(h: int) -> dict:
    n, T, nb, by = _i64(), _i64(), _i64(), _i64()
    L = load_library()
    _check(L.sta_sizes(h, C.byref(n), C.byref(T), C.byref(nb), C.byref(by)))
    nr, nz = _i64(), _i64()
    _check(L.sta_csr(h, None, None, None, C.byref(nr), C.byref(nz)))
    return {"n_nodes": n.value, "n_tets": T.value, "n_blocks": nb.value, "nnz": nz.value,
            "n_rows": nr.value, "device_bytes": by.value}


def sta_csr(h: int, owner=None):
    """(row_ptr, col, val) as zero-copy DeviceArrays over context memory."""
    rp, cl, vl = _p(), _p(), _p()
    nr, nz = _i64(), _i64()
    _check(load_library().sta_csr(h, C.byref(rp), C.byref(cl), C.byref(vl), C.byref(nr),
                                  C.byref(nz)))
    return (DeviceArray(rp.value or 0, (nr.value + 1,), "<i4", owner),
            DeviceArray(cl.value or 0, (nz.value,), "<i4", owner),
            DeviceArray(vl.value or 0, (nz.value,), "<f8", owner))


def sta_scatter_map(h: int, owner=None):
    p = _p()
    _check(load_library().sta_scatter_map(h, C.byref(p)))
    T = sta_sizes(h)["n_tets"]
    return DeviceArray(p.value or 0, (T, 144), "<i4", owner)


def sta_mask(h: int, owner=None):
    p = _p()
    _check(load_library().sta_mask(h, C.byref(p)))
    T = sta_sizes(h)["n_tets"]
    return DeviceArray(p.value or 0, (T,), "|u1", owner)


def sta_recompute_elements(h: int, active_only: bool = False, stream=None) -> None:
    _check(load_library().sta_recompute_elements(h, 1 if active_only else 0,
                                                 _stream_handle(stream)))


def sta_set_params(h: int, nodes=None, young=None, poisson=None, stream=None) -> None:
    """Host (numpy) arrays, or CUDA tensors (then all given arrays must be on the device)."""
    arrs = [a for a in (nodes, young, poisson) if a is not None]
    on_dev = bool(arrs) and all(hasattr(a, "is_cuda") and a.is_cuda for a in arrs)
    s = _sizes(h)
    keep = []

    def ptr(a, n, what):
        if a is None:
            return None
        a = _dev(a, n, what) if on_dev else _host_n(a, np.float64, n, what)
        keep.append(a)
        return a.data_ptr() if on_dev else a.ctypes.data

    _check(load_library().sta_set_params(h, ptr(nodes, 3 * s["n_nodes"], "nodes"),
                                         ptr(young, s["n_tets"], "young"),
                                         ptr(poisson, s["n_tets"], "poisson"),
                                         1 if on_dev else 0, _stream_handle(stream)))


def sta_element_matrices(h: int, tet_ids, stream=None):
    """Full 12x12 element matrices of the given tetrahedra, as a CUDA tensor (n, 12, 12)."""
    import torch
    ids = torch.as_tensor(tet_ids, dtype=torch.int32, device="cuda").contiguous()
    out = torch.empty((ids.numel(), 12, 12), dtype=torch.float64, device="cuda")
    _check(load_library().sta_element_matrices(h, ids.data_ptr(), ids.numel(), out.data_ptr(),
                                               _stream_handle(stream)))
    return out


def sta_adjoint(h: int, grad_val, stream=None):
    """(dE, dnu, dX) CUDA tensors for dL/dval given as a CUDA float64 tensor of nnz values."""
    import torch
    s = _sizes(h)
    g = _dev(grad_val, s["nnz"], "grad_val")
    dE = torch.empty(s["n_tets"], dtype=torch.float64, device=g.device)
    dnu = torch.empty_like(dE)
    dX = torch.empty((s["n_nodes"], 3), dtype=torch.float64, device=g.device)
    _check(load_library().sta_adjoint(h, g.data_ptr(), dE.data_ptr(), dnu.data_ptr(),
                                      dX.data_ptr(), _stream_handle(stream)))
    return dE, dnu, dX


def sta_spmv(h: int, x, val=None, stream=None):
    """y = A x (CUDA float64 tensors) over the pattern, with `val` or the current values."""
    s = _sizes(h)
    x = _dev(x, s["n_rows"], "x")
    y = x.new_empty(x.shape)
    val = _dev(val, s["nnz"], "val") if val is not None else None
    vp = val.data_ptr() if val is not None else None
    _check(load_library().sta_spmv(h, vp, x.data_ptr(), y.data_ptr(), _stream_handle(stream)))
    return y


def sta_set_launch(h: int, block_threads: int = 0, blocks_per_sm: int = 0) -> None:
    _check(load_library().sta_set_launch(h, int(block_threads), int(blocks_per_sm)))


def sta_set_fold_depth(h: int, operands_in_flight: int = 4) -> None:
    _check(load_library().sta_set_fold_depth(h, int(operands_in_flight)))


def sta_set_rebuild_form(h: int, form: int = STA_REBUILD_AUTO) -> None:
    _check(load_library().sta_set_rebuild_form(h, int(form)))


def sta_get_rebuild_form(h: int) -> int:
    f = C.c_int32(0)
    _check(load_library().sta_get_rebuild_form(h, C.byref(f)))
    return f.value


def sta_graph_enable(h: int, max_edited: int, stream=None) -> None:
    _check(load_library().sta_graph_enable(h, int(max_edited), _stream_handle(stream)))


def sta_set_policy(h: int, policy: int, stream=None) -> None:
    """STA_POLICY_REFOLD (canonical FP64 fold) or STA_POLICY_FIXED (exact fixed-point additive
    update); rebuilds every value under the new policy."""
    _check(load_library().sta_set_policy(h, int(policy), _stream_handle(stream)))


def sta_graph_disable(h: int, stream=None) -> None:
    _check(load_library().sta_graph_disable(h, _stream_handle(stream)))


def sta_batch_create(instances, opt: sta_options | None = None, stream=None) -> int:
    """instances: list of (X (n_i, 3), tets (T_i, 4) local ids, E (T_i,), nu (T_i,))."""
    L = load_library()
    k = len(instances)
    keep = []
    arr = {"X": (C.c_void_p * k)(), "T": (C.c_void_p * k)(), "E": (C.c_void_p * k)(),
           "NU": (C.c_void_p * k)()}
    nn = (C.c_int64 * k)()
    nt = (C.c_int64 * k)()
    for i, (X, tets, E, nu) in enumerate(instances):
        X = _host(X, np.float64).reshape(-1, 3)
        tets = _host(tets, np.int32).reshape(-1, 4)
        E = _host(E, np.float64).reshape(-1)
        nu = _host(nu, np.float64).reshape(-1)
        keep += [X, tets, E, nu]
        nn[i], nt[i] = X.shape[0], tets.shape[0]
        arr["X"][i], arr["T"][i] = X.ctypes.data, tets.ctypes.data
        arr["E"][i], arr["NU"][i] = E.ctypes.data, nu.ctypes.data
    h = _p()
    _check(L.sta_batch_create(k, nn, arr["X"], nt, arr["T"], arr["E"], arr["NU"],
                              C.byref(opt) if opt is not None else None, _stream_handle(stream),
                              C.byref(h)))
    _fixed.pop(h.value, None)  # a new context may reuse a destroyed one's address
    return h.value


def sta_batch_instance(h: int, i: int, owner=None):
    """(row_ptr, col, val) DeviceArrays of instance i in its own numbering, and its tet offset."""
    rp, cl, vl = _p(), _p(), _p()
    nr, nz, toff = _i64(), _i64(), _i64()
    _check(load_library().sta_batch_instance(h, int(i), C.byref(rp), C.byref(cl), C.byref(vl),
                                             C.byref(nr), C.byref(nz), C.byref(toff)))
    return (DeviceArray(rp.value or 0, (nr.value + 1,), "<i4", owner),
            DeviceArray(cl.value or 0, (nz.value,), "<i4", owner),
            DeviceArray(vl.value or 0, (nz.value,), "<f8", owner), int(toff.value))


def sta_batch_apply_edits(h: int, edits_per_instance, stream=None) -> None:
    """edits_per_instance: list of (m_i, 3) int32 arrays with instance-local tet ids."""
    parts = [_host(e, np.int32).reshape(-1, 3) for e in edits_per_instance]
    k = _sizes(h)["k"]
    if len(parts) != k:
        raise ValueError(f"one edit list per instance: {k} expected, got {len(parts)}")
    counts = (C.c_int64 * len(parts))(*[p.shape[0] for p in parts])
    allp = np.ascontiguousarray(np.concatenate(parts, 0)) if parts else np.zeros((0, 3), np.int32)
    _check(load_library().sta_batch_apply_edits(h, counts, allp.ctypes.data if allp.shape[0] else None,
                                                 _stream_handle(stream)))


# ----------------------------------------------------------------------------------------
# Convenience wrapper
# ----------------------------------------------------------------------------------------

class Assembler:
    """One superset mesh on the device: pattern, element cache, active mask and values."""

    def __init__(self, X, tets, E, nu, eps: float = 0.0, block_threads: int = 0,
                 blocks_per_sm: int = 0, stream=None):
        o = sta_default_options()
        o.eps, o.block_threads, o.blocks_per_sm = float(eps), int(block_threads), int(blocks_per_sm)
        self.h = sta_create(X, tets, E, nu, o, stream)
        s = sta_sizes(self.h)
        self.n_nodes, self.n_tets, self.nnz = s["n_nodes"], s["n_tets"], s["nnz"]
        self.n_rows = 3 * self.n_nodes

    def close(self):
        if getattr(self, "h", None):
            sta_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def full_rebuild(self, mask, stream=None):
        sta_full_rebuild(self.h, mask, stream)

    def apply_edits(self, edits, stream=None):
        sta_apply_edits(self.h, edits, stream)

    def refold(self, stream=None):
        sta_refold(self.h, stream)

    def last_touched(self, stream=None) -> int:
        return sta_last_touched(self.h, stream)

    def csr(self):
        """(row_ptr, col, val) torch tensors viewing the context's device memory."""
        return tuple(a.torch() for a in sta_csr(self.h, self))

    def values(self):
        return sta_csr(self.h, self)[2].torch()

    def scatter_map(self):
        return sta_scatter_map(self.h, self).torch()

    def mask(self):
        return sta_mask(self.h, self).torch()

    def recompute_elements(self, active_only=False, stream=None):
        sta_recompute_elements(self.h, active_only, stream)

    def set_params(self, X=None, E=None, nu=None, stream=None):
        sta_set_params(self.h, X, E, nu, stream)

    def element_matrices(self, tet_ids, stream=None):
        return sta_element_matrices(self.h, tet_ids, stream)

    def sizes(self) -> dict:
        return sta_sizes(self.h)

    def set_launch(self, block_threads: int = 0, blocks_per_sm: int = 0):
        sta_set_launch(self.h, block_threads, blocks_per_sm)

    def set_fold_depth(self, operands_in_flight: int = 4):
        """Operand loads in flight per lane of the rebuild fold (4 or 6; schedule only)."""
        sta_set_fold_depth(self.h, operands_in_flight)

    def set_rebuild_form(self, form: int = STA_REBUILD_AUTO):
        sta_set_rebuild_form(self.h, form)

    def rebuild_form(self) -> int:
        """STA_REBUILD_FUSED or STA_REBUILD_ZERO_FILL: the form of a rebuild issued now."""
        return sta_get_rebuild_form(self.h)

    def graph_enable(self, max_edited: int, stream=None):
        sta_graph_enable(self.h, max_edited, stream)

    def set_policy(self, policy: int, stream=None):
        sta_set_policy(self.h, policy, stream)

    def graph_disable(self, stream=None):
        sta_graph_disable(self.h, stream)

    def dyn_setup(self, rho: float, dt: float, f=None, clamped=None, stream=None):
        sta_dyn_setup(self.h, rho, dt, f, clamped, stream)

    def dyn_step(self, tol: float = 1e-10, max_iter: int = 1000, stream=None):
        return sta_dyn_step(self.h, tol, max_iter, stream)

    def dyn_apply(self, x, stream=None):
        return sta_dyn_apply(self.h, x, stream)

    def dyn_state(self):
        """(u, v, mass) torch tensors viewing the context's device memory."""
        return tuple(a.torch() for a in sta_dyn_state(self.h, self))

    def dyn_set_state(self, u=None, v=None, stream=None):
        sta_dyn_set_state(self.h, u, v, stream)


class BatchAssembler(Assembler):
    """k independent superset meshes in one context (batched form)."""

    def __init__(self, instances, eps: float = 0.0, block_threads: int = 0,
                 blocks_per_sm: int = 0, stream=None):
        o = sta_default_options()
        o.eps, o.block_threads, o.blocks_per_sm = float(eps), int(block_threads), int(blocks_per_sm)
        self.h = sta_batch_create(instances, o, stream)
        s = sta_sizes(self.h)
        self.n_nodes, self.n_tets, self.nnz = s["n_nodes"], s["n_tets"], s["nnz"]
        self.n_rows = 3 * self.n_nodes
        self.k = len(instances)

    def full_rebuild(self, masks, stream=None):
        """masks: list of per-instance masks, or one concatenated mask."""
        if isinstance(masks, (list, tuple)):
            masks = np.concatenate([np.asarray(m, np.uint8) for m in masks])
        sta_full_rebuild(self.h, masks, stream)

    def apply_edits(self, edits_per_instance, stream=None):
        sta_batch_apply_edits(self.h, edits_per_instance, stream)

    def instance_csr(self, i: int):
        rp, col, val, _ = sta_batch_instance(self.h, i, self)
        return rp.torch(), col.torch(), val.torch()


class ProxyAssembler(Assembler):
    """Graph-Laplacian proxy operator A_t = L_t + eps I of one superset mesh (node-level CSR,
    n rows).  Same edit, rebuild, graph and CSR calls as Assembler."""

    def __init__(self, n_nodes: int, tets, eps: float = 0.0, stream=None):
        self.h = sta_proxy_create(n_nodes, tets, eps, stream)
        s = sta_sizes(self.h)
        self.n_nodes, self.n_tets, self.nnz = s["n_nodes"], s["n_tets"], s["n_blocks"]
        self.n_rows = self.n_nodes

    def state(self):
        """(mult, degree) torch tensors viewing the context's device memory."""
        return tuple(a.torch() for a in sta_proxy_state(self.h, self))
