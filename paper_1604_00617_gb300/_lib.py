"""Thin ctypes binding of the C ABI declared in ``include/acr.h``.

Functions keep the C names and only marshal arguments: numpy arrays (host
memory) and torch tensors (host or device memory) are passed as raw pointers,
and status codes become :class:`AcrError`.  Every step of the solver runs in
the CUDA library; there is no Python or CPU code path.  Importing this module
loads ``_build/libacr.so`` and raises if it is missing.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libacr.so")

ACR_OK = 0
ACR_ERR_INVALID_ARG = -1
ACR_ERR_OOM = -2
ACR_ERR_SINGULAR = -3
ACR_ERR_NOT_CONVERGED = -4
ACR_ERR_CUDA = -5
ACR_ERR_TIMEOUT = -6

ACR_FP64 = 0
ACR_FP32TC_IR = 1
ACR_FP32_IR = 2

ACR_DENSE = 0
ACR_BANDED = 1

# tensor-core block products compiled into this build
TC_BUILT = True

ACR_REFINE_FGMRES = 0
ACR_REFINE_IR = 1
ACR_REFINE_NONE = 2

# largest rank for which the automatic choice continues in HODLR arithmetic
ACR_HRANK_SWITCH = 32

_NAMES = {0: "ACR_OK", -1: "ACR_ERR_INVALID_ARG", -2: "ACR_ERR_OOM", -3: "ACR_ERR_SINGULAR",
          -4: "ACR_ERR_NOT_CONVERGED", -5: "ACR_ERR_CUDA", -6: "ACR_ERR_TIMEOUT"}

# every symbol include/acr.h declares
EXPORTED = ["acr_default_opts", "acr_factor", "acr_factor_ex", "acr_solve", "acr_solve_ex",
            "acr_free", "acr_stats", "acr_factor_bytes", "acr_solve_bytes", "acr_last_error",
            "acr_block_inverse_noalloc", "acr_lowrank_truncate"]

# fixed scratch of acr_block_inverse_noalloc (ACR_NOALLOC_SCRATCH_BYTES)
ACR_NOALLOC_SCRATCH_BYTES = 16 << 20


class AcrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code
        self.msg = msg


class acr_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("input_kind", ctypes.c_int), ("leaf", ctypes.c_int),
                ("max_rank", ctypes.c_int), ("m_stop", ctypes.c_int), ("ir_tol", ctypes.c_double),
                ("ir_max_iter", ctypes.c_int), ("stream", ctypes.c_void_p), ("refine", ctypes.c_int),
                ("h_levels", ctypes.c_int), ("h_sketch", ctypes.c_int)]


class acr_stats_t(ctypes.Structure):
    _fields_ = [("nblk", ctypes.c_int), ("blksz", ctypes.c_int), ("levels", ctypes.c_int),
                ("precision", ctypes.c_int), ("compressed", ctypes.c_int),
                ("factor_bytes", ctypes.c_size_t), ("operator_bytes", ctypes.c_size_t),
                ("factor_flops", ctypes.c_double), ("factor_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("ir_iters", ctypes.c_int),
                ("ir_resid_max", ctypes.c_double), ("rank_max", ctypes.c_int * 32),
                ("rank_mean", ctypes.c_double * 32),
                ("gemm_ms", ctypes.c_double), ("gemm_flops", ctypes.c_double),
                ("inv_ms", ctypes.c_double), ("inv_flops", ctypes.c_double),
                ("sweep_ms", ctypes.c_double), ("sweep_bytes", ctypes.c_double),
                ("gemm_launches", ctypes.c_longlong), ("inv_launches", ctypes.c_longlong),
                ("sweep_launches", ctypes.c_longlong), ("launches_factor", ctypes.c_longlong),
                ("launches_solve", ctypes.c_longlong), ("compress_ms", ctypes.c_double),
                ("h_levels", ctypes.c_int), ("h_ms", ctypes.c_double), ("h_flops", ctypes.c_double),
                ("h_host_ms", ctypes.c_double), ("h_check", ctypes.c_double * 32),
                ("h_nodes", ctypes.c_longlong), ("h_sketch_redo", ctypes.c_longlong),
                ("sweep_passes", ctypes.c_longlong)]


def load(path: str = LIB_PATH):
    """Load the CUDA library; raise if it has not been built."""
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    i = ctypes.c_int
    lib.acr_default_opts.argtypes = [ctypes.POINTER(acr_opts)]
    lib.acr_default_opts.restype = None
    lib.acr_factor.argtypes = [i, i, vp, vp, vp, ctypes.c_double, ctypes.POINTER(vp)]
    lib.acr_factor.restype = i
    lib.acr_factor_ex.argtypes = [i, i, vp, vp, vp, ctypes.c_double, ctypes.POINTER(acr_opts),
                                  ctypes.POINTER(vp)]
    lib.acr_factor_ex.restype = i
    lib.acr_solve.argtypes = [vp, vp, i]
    lib.acr_solve.restype = i
    lib.acr_solve_ex.argtypes = [vp, vp, i, dp, ctypes.POINTER(i)]
    lib.acr_solve_ex.restype = i
    lib.acr_free.argtypes = [vp]
    lib.acr_free.restype = None
    lib.acr_stats.argtypes = [vp, ctypes.POINTER(acr_stats_t)]
    lib.acr_stats.restype = i
    lib.acr_factor_bytes.argtypes = [i, i, ctypes.c_double, ctypes.POINTER(acr_opts),
                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.acr_factor_bytes.restype = i
    lib.acr_solve_bytes.argtypes = [i, i, i, ctypes.POINTER(acr_opts), ctypes.POINTER(ctypes.c_size_t)]
    lib.acr_solve_bytes.restype = i
    lib.acr_last_error.argtypes = []
    lib.acr_last_error.restype = ctypes.c_char_p
    lib.acr_block_inverse_noalloc.argtypes = [i, i, vp, vp, vp]
    lib.acr_block_inverse_noalloc.restype = i
    lib.acr_lowrank_truncate.argtypes = [i, i, i, vp, vp, ctypes.c_double, i, i, vp, vp, vp, vp]
    lib.acr_lowrank_truncate.restype = i
    return lib


_lib = load()


def _ptr(x, nelem: int | None = None):
    """Raw pointer of a float64 numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64:
            raise TypeError("arrays must be float64")
        if not (x.flags.c_contiguous or x.flags.f_contiguous):
            raise ValueError("arrays must be contiguous")
        if nelem is not None and x.size < nelem:
            raise ValueError(f"array has {x.size} elements, need {nelem}")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64:
            raise TypeError("tensors must be float64")
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if nelem is not None and x.numel() < nelem:
            raise ValueError(f"tensor has {x.numel()} elements, need {nelem}")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(code: int):
    if code != ACR_OK:
        raise AcrError(code, acr_last_error())


def acr_last_error() -> str:
    return _lib.acr_last_error().decode()


def acr_default_opts() -> acr_opts:
    o = acr_opts()
    _lib.acr_default_opts(ctypes.byref(o))
    return o


def _sizes(nblk, blksz, kind):
    bb = blksz * blksz
    if kind == ACR_BANDED:
        return nblk * blksz, nblk * 3 * blksz
    return nblk * bb, nblk * bb


def acr_factor(nblk: int, blksz: int, A, D, C, tol: float = 0.0):
    """``acr_factor``: returns the handle (a ctypes void pointer)."""
    na, nd = _sizes(nblk, blksz, ACR_DENSE)
    h = ctypes.c_void_p()
    _check(_lib.acr_factor(nblk, blksz, _ptr(A, na if nblk > 1 else None), _ptr(D, nd),
                           _ptr(C, na if nblk > 1 else None), float(tol), ctypes.byref(h)))
    return h


def acr_factor_ex(nblk: int, blksz: int, A, D, C, tol: float = 0.0, opts: acr_opts | None = None):
    """``acr_factor_ex``: returns the handle."""
    o = opts if opts is not None else acr_default_opts()
    na, nd = _sizes(nblk, blksz, o.input_kind)
    h = ctypes.c_void_p()
    _check(_lib.acr_factor_ex(nblk, blksz, _ptr(A, na if nblk > 1 else None), _ptr(D, nd),
                              _ptr(C, na if nblk > 1 else None), float(tol), ctypes.byref(o),
                              ctypes.byref(h)))
    return h


def acr_solve(h, B, nrhs: int) -> None:
    """``acr_solve``: B (N x nrhs, column-major float64) is overwritten with X."""
    _check(_lib.acr_solve(h, _ptr(B), int(nrhs)))


def acr_solve_ex(h, B, nrhs: int):
    """``acr_solve_ex``: returns ``(resid, iters)``; B is overwritten with X.

    Raises AcrError on failure; for ACR_ERR_NOT_CONVERGED the exception carries
    ``resid`` and ``iters`` attributes and B holds the last iterate."""
    res = np.zeros(max(int(nrhs), 1))
    it = ctypes.c_int(0)
    code = _lib.acr_solve_ex(h, _ptr(B), int(nrhs), res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             ctypes.byref(it))
    if code != ACR_OK:
        err = AcrError(code, acr_last_error())
        err.resid = res[:nrhs].copy()
        err.iters = it.value
        raise err
    return res[:nrhs].copy(), it.value


def acr_free(h) -> None:
    _lib.acr_free(h)


def acr_stats(h) -> dict:
    s = acr_stats_t()
    _check(_lib.acr_stats(h, ctypes.byref(s)))
    d = {k: getattr(s, k) for k, _ in acr_stats_t._fields_}
    d["rank_max"] = list(s.rank_max)[: s.levels]
    d["rank_mean"] = list(s.rank_mean)[: s.levels]
    d["h_check"] = list(s.h_check)[: min(32, s.h_levels + 1)]
    return d


def acr_factor_bytes(nblk: int, blksz: int, tol: float = 0.0, opts: acr_opts | None = None) -> int:
    o = opts if opts is not None else acr_default_opts()
    out = ctypes.c_size_t(0)
    _check(_lib.acr_factor_bytes(nblk, blksz, float(tol), ctypes.byref(o), ctypes.byref(out)))
    return out.value


def acr_solve_bytes(nblk: int, blksz: int, nrhs: int, opts: acr_opts | None = None) -> int:
    o = opts if opts is not None else acr_default_opts()
    out = ctypes.c_size_t(0)
    _check(_lib.acr_solve_bytes(nblk, blksz, nrhs, ctypes.byref(o), ctypes.byref(out)))
    return out.value


def acr_block_inverse_noalloc(blksz: int, count: int, mats, info, stream=None) -> None:
    """``acr_block_inverse_noalloc``: invert ``count`` column-major blocks in
    place on the device without allocating (``mats``: float64 device tensor,
    ``info``: int32 device tensor of ``count``).  Queued on ``stream`` (a CUDA
    stream handle or None); returns without waiting."""
    if not hasattr(info, "data_ptr") or not hasattr(mats, "data_ptr"):
        raise TypeError("mats and info must be device tensors")
    import torch
    if info.dtype != torch.int32 or info.numel() < count:
        raise TypeError("info must be an int32 tensor with count elements")
    if not info.is_contiguous():
        raise ValueError("info must be contiguous")
    for name, t in (("mats", mats), ("info", info)):
        if t.device.type != "cuda" or (torch.cuda.is_available() and t.device.index != torch.cuda.current_device()):
            raise ValueError(f"{name} must be on the current CUDA device")
    iptr = ctypes.c_void_p(info.data_ptr())
    _check(_lib.acr_block_inverse_noalloc(int(blksz), int(count), _ptr(mats, blksz * blksz * count), iptr,
                                          ctypes.c_void_p(stream) if stream else None))


def acr_lowrank_truncate(U, V, tol: float, precision: int = ACR_FP64, sketch: int = 0):
    """``acr_lowrank_truncate`` on host arrays: U, V of shape (count, R, s)
    (node i's s x R factor column-major, i.e. numpy's [i, col, row]).  Returns
    (Uout, Vout, ranks, exact_redo) in the same layout."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    if U.ndim != 3 or U.shape != V.shape:
        raise ValueError("U and V must have the same shape (count, R, s)")
    count, R, s = U.shape
    Uo = np.zeros_like(U)
    Vo = np.zeros_like(V)
    rk = np.zeros(count, dtype=np.int32)
    redo = ctypes.c_int(0)
    _check(_lib.acr_lowrank_truncate(count, s, R, _ptr(U), _ptr(V), float(tol), int(precision), int(sketch),
                                     _ptr(Uo), _ptr(Vo), ctypes.c_void_p(rk.ctypes.data), ctypes.byref(redo)))
    return Uo, Vo, rk, redo.value
