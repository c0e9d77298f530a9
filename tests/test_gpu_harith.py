"""The reduction in HODLR arithmetic (Section 3: H-inverse of the eliminated
blocks, H-products and H-sums of the Schur complement of Eq. "fund",
truncated to tol), through the C ABI.

* Parity with the FP64 oracle: FP64 factors with compression reach a relative
  residual <= 10 tol without refinement on the workloads where that bound
  holds, and their error against the oracle is bounded; mixed precision
  refines to 1e-8.
* The number of levels done in HODLR arithmetic is reported and obeys
  ``h_levels``; every stopping level gives a correct factorization (the dense
  levels above it take over).
* The level-0 blocks are exactly rank 1 and remain so through the
  H-inverse (the inverse of a tridiagonal matrix is semiseparable).
"""

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1604_00617_gb300 import build
    build()
    from paper_1604_00617_gb300 import _lib
    return _lib


def factor(lib, P, tol, prec=0, **kw):
    a, D3, c = P.banded_abi()
    o = lib.acr_default_opts()
    o.precision = prec
    o.input_kind = lib.ACR_BANDED
    for k, v in kw.items():
        setattr(o, k, v)
    return lib.acr_factor_ex(P.nblk, P.b, a, D3, c, tol, o)


def solve(lib, h, F):
    B = np.asfortranarray(F.copy())
    res, it = lib.acr_solve_ex(h, B, F.shape[1])
    return B, res, it


def host_resid(P, X, F):
    return np.linalg.norm(F - P.matvec(X), axis=0) / np.linalg.norm(F, axis=0)


@pytest.mark.parametrize("idx,n,tol,leaf", [(0, 64, 1e-10, 16), (0, 128, 1e-8, 16), (1, 64, 1e-8, 16),
                                            (1, 128, 1e-6, 32), (2, 128, 1e-6, 32), (2, 96, 1e-7, 16),
                                            (0, 64, 1e-10, 4), (1, 64, 1e-8, 8), (2, 128, 1e-8, 8)])
def test_fp64_within_10_tol(lib, idx, n, tol, leaf):
    P = syn.make_config(idx, n)
    F = syn.rhs_uniform(P.N, 2, 2000 + idx)
    h = factor(lib, P, tol, leaf=leaf, refine=lib.ACR_REFINE_NONE, ir_tol=1.0)
    try:
        s = lib.acr_stats(h)
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert s["h_levels"] >= 1, s["h_levels"]
    r = host_resid(P, X, F)
    assert (r <= 10 * tol).all(), (r, s["h_levels"])
    A, D, C = P.dense_blocks()
    Xo = oracle.bcr_solve(A, D, C, F)
    err = np.linalg.norm(X - Xo, axis=0) / np.linalg.norm(Xo, axis=0)
    assert (err <= 1e4 * tol).all(), err
    print(f"cfg{idx} n={n} tol {tol:g}: {s['h_levels']} H levels of {s['levels']}, resid {r.max():.2e}, "
          f"err {err.max():.2e}, ranks {s['rank_max']}")


def test_fp64_deep_tree_helmholtz_refined(lib):
    """Leaf 4 under a 64-row block (4 tree levels) on the indefinite
    Helmholtz operator: the truncations of every tree level and every
    reduction level add up beyond 10 tol (the unrefined residual is recorded,
    bounded by 1e3 tol), and FGMRES brings the solve to 1e-11."""
    P = syn.make_config(3, 64)
    F = syn.rhs_uniform(P.N, 2, 2003)
    tol = 1e-10
    h = factor(lib, P, tol, leaf=4, refine=lib.ACR_REFINE_NONE, ir_tol=1.0)
    try:
        s = lib.acr_stats(h)
        X, _, _ = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert s["h_levels"] >= 1
    r0 = host_resid(P, X, F)
    assert (r0 <= 1e3 * tol).all(), r0
    h = factor(lib, P, tol, leaf=4, ir_tol=1e-11, ir_max_iter=40)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (host_resid(P, X, F) <= 2e-11).all(), (res, it)
    print(f"Helmholtz 64 leaf 4: unrefined {r0.max():.2e}, refined in {it} iterations")


@pytest.mark.parametrize("idx,n,tol,prec", [(1, 128, 1e-8, 0), (2, 128, 1e-8, 0), (3, 256, 1e-8, 1)])
def test_sketch_truncation_matches_exact(lib, idx, n, tol, prec):
    """The randomized first truncation pass and the exact one give factors
    that solve the system alike: the unrefined residuals agree within 10 tol
    (FP64) or both refine to 1e-8 (FP32)."""
    P = syn.make_config(idx, n)
    F = syn.rhs_uniform(P.N, 2, 2100 + idx)
    out = {}
    for sk in (0, 1):
        kw = dict(leaf=16, h_sketch=sk)
        if prec == 0:
            kw.update(refine=lib.ACR_REFINE_NONE, ir_tol=1.0)
        else:
            kw.update(ir_max_iter=60)
        h = factor(lib, P, tol, prec=prec, **kw)
        try:
            s = lib.acr_stats(h)
            X, res, it = solve(lib, h, F)
        finally:
            lib.acr_free(h)
        out[sk] = (s, host_resid(P, X, F), it)
    s0, s1 = out[0][0], out[1][0]
    assert s0["h_levels"] == s1["h_levels"] >= 1
    assert s0["h_sketch_redo"] == 0 and 0 <= s1["h_sketch_redo"] <= s1["h_nodes"]
    if prec == 0:
        assert (out[0][1] <= 10 * tol).all() and (out[1][1] <= 10 * tol).all(), (out[0][1], out[1][1])
    else:
        assert (out[0][1] <= 1.5e-8).all() and (out[1][1] <= 1.5e-8).all()
        assert out[1][2] <= out[0][2] + 3, (out[0][2], out[1][2])
    print(f"cfg{idx} n={n}: nodes {s1['h_nodes']}, exact redo {s1['h_sketch_redo']}, "
          f"resid exact {out[0][1].max():.2e} sketch {out[1][1].max():.2e}, h_ms {s0['h_ms']:.2f} -> {s1['h_ms']:.2f}")


@pytest.mark.parametrize("hl", [1, 2, 3, 5])
def test_every_switch_level_gives_the_solution(lib, hl):
    """h_levels = k: k levels in HODLR arithmetic, the rest dense; all agree."""
    P = syn.make_config(1, 64)
    F = syn.rhs_uniform(P.N, 2, 2001)
    tol = 1e-10
    h = factor(lib, P, tol, leaf=16, h_levels=hl, refine=lib.ACR_REFINE_NONE, ir_tol=1.0)
    try:
        s = lib.acr_stats(h)
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert s["h_levels"] == hl
    assert (host_resid(P, X, F) <= 10 * tol).all()


def test_h_levels_off_matches_previous_path(lib):
    """h_levels = -1: the dense reduction compressed afterwards; both forms
    solve the same system to the same tolerance."""
    P = syn.make_config(2, 64)
    F = syn.rhs_uniform(P.N, 2, 2002)
    X = {}
    for hl in (-1, 0):
        h = factor(lib, P, 1e-10, leaf=16, h_levels=hl, refine=lib.ACR_REFINE_NONE, ir_tol=1.0)
        try:
            s = lib.acr_stats(h)
            X[hl], _, _ = solve(lib, h, F)
        finally:
            lib.acr_free(h)
        assert (s["h_levels"] == 0) == (hl == -1)
    assert np.linalg.norm(X[0] - X[-1]) / np.linalg.norm(X[-1]) <= 1e-8


def test_all_levels_in_hodlr_arithmetic(lib):
    """Few, small blocks: the ranks stay low up to the top block, which is
    then inverted in HODLR arithmetic as well."""
    P = syn.make_config(0, 32)
    F = syn.rhs_uniform(P.N, 1, 2000)
    h = factor(lib, P, 1e-10, leaf=8, refine=lib.ACR_REFINE_NONE, ir_tol=1.0)
    try:
        s = lib.acr_stats(h)
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert s["h_levels"] == s["levels"]
    assert (host_resid(P, X, F) <= 1e-9).all()


def test_level0_rank_one(lib):
    P = syn.make_config(3, 128)
    h = factor(lib, P, 1e-8, leaf=16)
    try:
        s = lib.acr_stats(h)
    finally:
        lib.acr_free(h)
    assert s["h_levels"] >= 1 and s["rank_max"][0] == 1


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("idx,n", [(1, 128), (2, 128), (3, 128), (3, 256)])
def test_mixed_precision_refined(lib, prec, idx, n):
    P = syn.make_config(idx, n)
    F = syn.rhs_uniform(P.N, 3, 2000 + idx)
    h = factor(lib, P, 1e-6 if idx < 3 else 1e-8, prec=prec, leaf=32, ir_max_iter=60)
    try:
        s = lib.acr_stats(h)
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert s["h_levels"] >= 1
    assert (res <= 1e-8).all() and (host_resid(P, X, F) <= 1.5e-8).all(), (res, it)
    if n <= 128:
        A, D, C = P.dense_blocks()
        Xo = oracle.bcr_solve(A, D, C, F)
        assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) <= 1e-5
