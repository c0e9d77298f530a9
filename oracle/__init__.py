"""CPU oracle for block cyclic reduction -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The solver library never does, and the
oracle imports nothing from the solver: the two share no code.

``acr_oracle.c`` is plain C (FP64, loops, OpenMP across the independent blocks
of a level); this module compiles it with gcc on first use and wraps it with
ctypes.  Every function documents the passage of the paper it follows in the C
source.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "acr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_OK = 0
ORACLE_ERR_SINGULAR = -3


class OracleSingular(RuntimeError):
    def __init__(self, level, block):
        super().__init__(f"singular eliminated block: level {level}, block {block}")
        self.level = level
        self.block = block


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP); return its path.

    ``mutant > 0`` builds a copy with one planted mistake (see ORACLE_MUTANT in
    the C source); only the mutation test asks for it."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_PATH if mutant == 0 else os.path.join(_BUILD, f"liboracle_mutant{mutant}.so")
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _load(mutant: int = 0):
    global _lib
    with _lock:
        if mutant:
            return _bind(ctypes.CDLL(build(mutant=mutant)))
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i = ctypes.c_int
    lib.oracle_bcr_solve.argtypes = [i, i, dp, dp, dp, dp, i, dp, i, ip, ip]
    lib.oracle_bcr_reduce.argtypes = [i, i, dp, dp, dp, i, dp, dp, dp, ip]
    lib.oracle_dense_solve.argtypes = [i, dp, dp, i, dp]
    lib.oracle_residual.argtypes = [i, i, dp, dp, dp, dp, dp, i, dp]
    lib.oracle_bcr_schedule.argtypes = [i, i, ip, i]
    lib.oracle_num_threads.argtypes = []
    for f in (lib.oracle_bcr_solve, lib.oracle_bcr_reduce, lib.oracle_dense_solve,
              lib.oracle_residual, lib.oracle_bcr_schedule, lib.oracle_num_threads):
        f.restype = ctypes.c_int
    return lib


_active_mutant = 0


def use_mutant(mutant: int) -> None:
    """Route the wrappers below to a planted-mistake build (tests only);
    ``use_mutant(0)`` restores the real oracle."""
    global _active_mutant
    _active_mutant = int(mutant)


def _L():
    return _load(_active_mutant)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _blocks_colmajor(X):
    """(n, b, b) row/col matrices -> contiguous, each block column-major."""
    return np.ascontiguousarray(np.transpose(np.asarray(X, dtype=np.float64), (0, 2, 1)))


def _blocks_from_colmajor(X):
    return np.ascontiguousarray(np.transpose(X, (0, 2, 1)))


def num_threads() -> int:
    return _L().oracle_num_threads()


def bcr_solve(A, D, C, F, m_stop: int = 1):
    """Exact FP64 dense block cyclic reduction solve.

    ``A, D, C``: ``(n, b, b)`` row/col block matrices (``A[0]``, ``C[-1]``
    ignored).  ``F``: ``(N,)`` or ``(N, nrhs)``.  Returns ``X`` shaped like ``F``.
    """
    lib = _L()
    n, b, _ = np.shape(D)
    Fa = np.asarray(F, dtype=np.float64)
    F2 = np.asfortranarray(Fa.reshape(n * b, -1))
    nrhs = F2.shape[1]
    X = np.zeros_like(F2, order="F")
    Ac, Dc, Cc = _blocks_colmajor(A), _blocks_colmajor(D), _blocks_colmajor(C)
    el, eb = ctypes.c_int(-1), ctypes.c_int(-1)
    st = lib.oracle_bcr_solve(n, b, _dp(Ac), _dp(Dc), _dp(Cc), _dp(F2), nrhs, _dp(X), m_stop,
                              ctypes.byref(el), ctypes.byref(eb))
    if st == ORACLE_ERR_SINGULAR:
        raise OracleSingular(el.value, eb.value)
    if st != ORACLE_OK:
        raise RuntimeError(f"oracle_bcr_solve failed: {st}")
    return X.reshape(Fa.shape)


def bcr_reduce(A, D, C, nlev: int):
    """Apply ``nlev`` reduction levels; return ``(A', D', C')`` of the reduced
    system as ``(m, b, b)`` row/col matrices."""
    lib = _L()
    n, b, _ = np.shape(D)
    Ac, Dc, Cc = _blocks_colmajor(A), _blocks_colmajor(D), _blocks_colmajor(C)
    oD = np.zeros_like(Dc); oA = np.zeros_like(Dc); oC = np.zeros_like(Dc)
    m = ctypes.c_int(0)
    st = lib.oracle_bcr_reduce(n, b, _dp(Ac), _dp(Dc), _dp(Cc), nlev, _dp(oD), _dp(oA), _dp(oC),
                               ctypes.byref(m))
    if st != ORACLE_OK:
        raise RuntimeError(f"oracle_bcr_reduce failed: {st}")
    mm = m.value
    return (_blocks_from_colmajor(oA[:mm]), _blocks_from_colmajor(oD[:mm]),
            _blocks_from_colmajor(oC[:mm]))


def dense_solve(M, F):
    """Partial-pivoted LU solve of a dense ``(N, N)`` system."""
    lib = _L()
    Mf = np.asfortranarray(np.asarray(M, dtype=np.float64))
    Fa = np.asarray(F, dtype=np.float64)
    N = Mf.shape[0]
    F2 = np.asfortranarray(Fa.reshape(N, -1))
    X = np.zeros_like(F2, order="F")
    st = lib.oracle_dense_solve(N, _dp(Mf), _dp(F2), F2.shape[1], _dp(X))
    if st != ORACLE_OK:
        raise RuntimeError(f"oracle_dense_solve failed: {st}")
    return X.reshape(Fa.shape)


def residual(A, D, C, X, F):
    """Per-column ``||F - M X|| / ||F||`` in FP64 (dense blocks)."""
    lib = _L()
    n, b, _ = np.shape(D)
    Xa = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(n * b, -1))
    F2 = np.asfortranarray(np.asarray(F, dtype=np.float64).reshape(n * b, -1))
    rel = np.zeros(F2.shape[1])
    Ac, Dc, Cc = _blocks_colmajor(A), _blocks_colmajor(D), _blocks_colmajor(C)
    st = lib.oracle_residual(n, b, _dp(Ac), _dp(Dc), _dp(Cc), _dp(Xa), _dp(F2), F2.shape[1], _dp(rel))
    if st != ORACLE_OK:
        raise RuntimeError(f"oracle_residual failed: {st}")
    return rel


def bcr_schedule(n: int, m_stop: int = 1):
    """Original indices eliminated at each level (last entry: the top solve)."""
    lib = _L()
    cap = 4 * n + 64
    buf = (ctypes.c_int * cap)()
    nlev = lib.oracle_bcr_schedule(n, m_stop, buf, cap)
    if nlev < 0:
        raise RuntimeError("schedule buffer too small")
    out, pos = [], 0
    for _ in range(nlev):
        cnt = buf[pos]
        out.append([buf[pos + 1 + k] for k in range(cnt)])
        pos += 1 + cnt
    return out
