"""The C-ABI library builds, loads and exports every symbol include/acr.h
declares; argument validation answers without touching the GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "acr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(acr_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_00617_gb300 import build
    build()
    from paper_1604_00617_gb300 import _lib
    return _lib


def test_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib.LIB_PATH)
    declared = _declared()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(raw, name), f"{name} missing from libacr.so"
    assert set(declared) == set(lib.EXPORTED)


def test_default_opts(lib):
    o = lib.acr_default_opts()
    assert o.precision == lib.ACR_FP64 and o.input_kind == lib.ACR_DENSE
    assert o.m_stop == 1 and o.ir_tol == 1e-8 and o.ir_max_iter == 20 and not o.stream


def test_invalid_arguments_rejected_on_host(lib):
    import numpy as np
    D = np.zeros(4)
    with pytest.raises(lib.AcrError) as ei:
        lib.acr_factor(0, 2, D, D, D, 0.0)
    assert ei.value.code == lib.ACR_ERR_INVALID_ARG
    assert "nblk" in lib.acr_last_error()
    o = lib.acr_default_opts()
    o.precision = 7
    with pytest.raises(lib.AcrError) as ei:
        lib.acr_factor_ex(1, 2, None, D, None, 0.0, o)
    assert ei.value.code == lib.ACR_ERR_INVALID_ARG
    o = lib.acr_default_opts()
    o.m_stop = 4
    with pytest.raises(lib.AcrError):
        lib.acr_factor_ex(1, 2, None, D, None, 0.0, o)


def test_factor_bytes_plan(lib):
    # n = 8, b = 4, FP64: levels m = 8, 4, 2, 1
    # per level 3*ceil(m/2) + 2*floor(m/2) blocks, top level only its inverse
    # (every level's arrays start on a 256-byte boundary)
    def plan(es):
        off = 0
        for ne, nk, top in ((4, 4, False), (2, 2, False), (1, 1, False), (1, 0, True)):
            off += (ne + (0 if top else 2 * ne) + 2 * nk) * 16 * es
            off = (off + 255) // 256 * 256
        return off
    o = lib.acr_default_opts()
    got = lib.acr_factor_bytes(8, 4, 0.0, o)
    assert got == plan(8) + 3 * 8 * 16 * 8  # plus the FP64 operator copy
    o.precision = lib.ACR_FP32_IR
    o.input_kind = lib.ACR_BANDED
    assert lib.acr_factor_bytes(8, 4, 0.0, o) == plan(4) + 5 * 32 * 8


def test_solve_bytes_bound(lib):
    o = lib.acr_default_opts()
    o.precision = lib.ACR_FP32TC_IR
    o.ir_max_iter = 60                       # restart length 50
    N = 64 * 64
    b1 = lib.acr_solve_bytes(64, 64, 1, o)
    b8 = lib.acr_solve_bytes(64, 64, 8, o)
    assert b8 > b1 > 0
    assert b8 >= N * 8 * 8 * (50 + 51)       # the FGMRES bases V and Z alone
    o.refine = lib.ACR_REFINE_IR             # no Krylov bases
    assert lib.acr_solve_bytes(64, 64, 8, o) < b8
    with pytest.raises(lib.AcrError):
        lib.acr_solve_bytes(0, 64, 1, o)
    with pytest.raises(lib.AcrError):
        lib.acr_solve_bytes(64, 64, -1, o)


_CTYPES = {"int": ctypes.c_int, "size_t": ctypes.c_size_t, "double": ctypes.c_double,
           "long long": ctypes.c_longlong, "void *": ctypes.c_void_p}


def _header_struct(name):
    """(field, ctype) pairs of `typedef struct {...} name;` in include/acr.h."""
    src = open(os.path.join(ROOT, "include", "acr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        m = re.match(r"(long long|size_t|double|int|void)\s*(\*?)\s*(.*)", decl)
        base = m.group(1) + (" *" if m.group(2) else "")
        for var in m.group(3).split(","):
            var = var.strip()
            arr = re.match(r"(\w+)\[(\d+)\]", var)
            if arr:
                fields.append((arr.group(1), _CTYPES[base] * int(arr.group(2))))
            else:
                fields.append((var, _CTYPES[base]))
    return fields


@pytest.mark.parametrize("name", ["acr_opts", "acr_stats_t"])
def test_binding_structs_match_header(name):
    from paper_1604_00617_gb300 import _lib
    want = _header_struct(name)
    got = getattr(_lib, name)._fields_
    assert [f for f, _ in got] == [f for f, _ in want]
    for (f, tg), (_, tw) in zip(got, want):
        if hasattr(tw, "_length_"):
            assert tg._length_ == tw._length_ and tg._type_ is tw._type_, f
        else:
            assert tg is tw, f


def test_noalloc_rejects_host_memory_without_launching(lib):
    """acr_block_inverse_noalloc accepts only device memory of the current
    device; host buffers are refused before anything is queued (on a machine
    without a GPU the call fails the same way, with no current device)."""
    import numpy as np
    mats = np.eye(4).ravel().copy()
    info = np.zeros(1, dtype=np.int32)
    code = lib._lib.acr_block_inverse_noalloc(4, 1, ctypes.c_void_p(mats.ctypes.data),
                                              ctypes.c_void_p(info.ctypes.data), None)
    assert code == lib.ACR_ERR_INVALID_ARG
    assert "device" in lib.acr_last_error()
    assert (mats == np.eye(4).ravel()).all() and info[0] == 0
    with pytest.raises(TypeError):
        lib.acr_block_inverse_noalloc(4, 1, mats, info)


def test_lowrank_truncate_rejects_bad_arguments_on_host(lib):
    import numpy as np
    U = np.zeros((2, 3, 4))
    for kw, msg in ((dict(tol=-1.0), "tol"), (dict(tol=1.0), "tol"), (dict(tol=1e-3, precision=9), "precision"),
                    (dict(tol=1e-3, sketch=-2), "sketch")):
        with pytest.raises(lib.AcrError) as ei:
            lib.acr_lowrank_truncate(U, U, **kw)
        assert ei.value.code == lib.ACR_ERR_INVALID_ARG and msg in lib.acr_last_error()
    with pytest.raises(ValueError):
        lib.acr_lowrank_truncate(U, np.zeros((2, 3, 5)), 1e-3)
