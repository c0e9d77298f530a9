"""Parity of the CUDA block cyclic reduction (uncompressed blocks) with the FP64
CPU oracle, through the C ABI.

Bar: relative error <= 1e-10 against the oracle in FP64 with compression off;
relative residual <= ir_tol (1e-8) per column after refinement in the mixed
modes (error against the oracle reported and bounded).  Sizes span several
tiles, ragged tails (blksz not a multiple of any tile), odd block counts, the
shared-memory and the blocked inversion paths, and the full-size workloads.
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


def _cm(X):
    return np.ascontiguousarray(np.transpose(X, (0, 2, 1)))


def factor(lib, A, D, C, prec=0, device=False, **kw):
    n, b, _ = D.shape
    Ac, Dc, Cc = _cm(A), _cm(D), _cm(C)
    if device:
        import torch
        Ac, Dc, Cc = (torch.from_numpy(x).cuda() for x in (Ac, Dc, Cc))
    o = lib.acr_default_opts()
    o.precision = prec
    for k, v in kw.items():
        setattr(o, k, v)
    return lib.acr_factor_ex(n, b, Ac, Dc, Cc, 0.0, o)


def factor_banded(lib, P, prec=0, tol=0.0, **kw):
    a, D3, c = P.banded_abi()
    o = lib.acr_default_opts()
    o.precision = prec
    o.input_kind = lib.ACR_BANDED
    for k, v in kw.items():
        setattr(o, k, v)
    return lib.acr_factor_ex(P.nblk, P.b, a, D3, c, tol, o)


def solve(lib, h, F, device=False):
    F2 = F.reshape(F.shape[0], -1)
    if device:
        import torch
        B = torch.from_numpy(np.ascontiguousarray(F2.T)).cuda()  # column-major N x nrhs
        res, it = lib.acr_solve_ex(h, B, F2.shape[1])
        X = B.cpu().numpy().T
    else:
        B = np.asfortranarray(F2.copy())
        res, it = lib.acr_solve_ex(h, B, F2.shape[1])
        X = B
    return X.reshape(F.shape), res, it


def relerr(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


@pytest.mark.parametrize("n,b", [(1, 1), (1, 7), (2, 3), (3, 4), (5, 7), (8, 8), (7, 33),
                                 (13, 20), (16, 64), (33, 17), (6, 130), (4, 159)])
def test_dense_fp64_random_blocks(lib, n, b):
    A, D, C = syn.random_blocks(n, b, seed=100 + n * b)
    F = np.random.default_rng(n + b).uniform(-1, 1, (n * b, 3))
    h = factor(lib, A, D, C)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert relerr(X, oracle.bcr_solve(A, D, C, F)) <= 1e-10
    assert it == 0


@pytest.mark.parametrize("n,b", [(3, 170), (5, 200), (2, 257)])
def test_dense_fp64_blocked_inversion(lib, n, b):
    """blksz above the shared-memory limit takes the panel + update path."""
    A, D, C = syn.random_blocks(n, b, seed=7 + b)
    F = np.random.default_rng(b).uniform(-1, 1, (n * b, 2))
    h = factor(lib, A, D, C)
    try:
        X, _, _ = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert relerr(X, oracle.bcr_solve(A, D, C, F)) <= 1e-10


@pytest.mark.parametrize("idx,n", [(0, 64), (1, 64), (2, 64), (3, 64), (3, 47), (1, 96)])
@pytest.mark.parametrize("banded", [False, True])
def test_pde_fp64(lib, idx, n, banded):
    P = syn.make_config(idx, n)
    A, D, C = P.dense_blocks()
    F = syn.rhs_uniform(P.N, 2, 2000 + idx)
    h = factor_banded(lib, P) if banded else factor(lib, A, D, C)
    try:
        X, res, _ = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert relerr(X, oracle.bcr_solve(A, D, C, F)) <= 1e-10


@pytest.mark.parametrize("prec", [2])
@pytest.mark.parametrize("idx,n", [(0, 64), (1, 64), (2, 64), (3, 64), (1, 128)])
def test_pde_mixed_refinement(lib, prec, idx, n):
    P = syn.make_config(idx, n)
    A, D, C = P.dense_blocks()
    F = syn.rhs_uniform(P.N, 4, 2000 + idx)
    h = factor_banded(lib, P, prec=prec)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert it >= 1 and (res <= 1e-8).all(), (res, it)
    # residual recomputed independently (numpy banded product)
    r = np.linalg.norm(F - P.matvec(X), axis=0) / np.linalg.norm(F, axis=0)
    assert (r <= 1.5e-8).all()
    err = relerr(X, oracle.bcr_solve(A, D, C, F))
    assert err <= 1e-6, err


@pytest.mark.parametrize("nrhs", [1, 2, 5, 8, 16, 17, 64])
def test_nrhs_variants(lib, nrhs):
    A, D, C = syn.random_blocks(9, 24, seed=nrhs)
    F = np.random.default_rng(nrhs).uniform(-1, 1, (9 * 24, nrhs))
    h = factor(lib, A, D, C)
    try:
        X, _, _ = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert relerr(X, oracle.bcr_solve(A, D, C, F)) <= 1e-10


def test_device_pointers_match_host(lib):
    A, D, C = syn.random_blocks(10, 40, seed=3)
    F = np.random.default_rng(1).uniform(-1, 1, (400, 3))
    h1 = factor(lib, A, D, C)
    h2 = factor(lib, A, D, C, device=True)
    try:
        X1, _, _ = solve(lib, h1, F)
        X2, _, _ = solve(lib, h2, F, device=True)
    finally:
        lib.acr_free(h1)
        lib.acr_free(h2)
    assert np.array_equal(X1, X2)


def test_singular_block_reports_level_and_block(lib):
    A, D, C = syn.random_blocks(6, 5, seed=1)
    D[4] = 0.0
    with pytest.raises(lib.AcrError) as ei:
        factor(lib, A, D, C)
    assert ei.value.code == lib.ACR_ERR_SINGULAR
    assert "level 0, block 4" in ei.value.msg
    # singular Schur complement at level 1 (scalar blocks): 2 - 1 - 1 = 0
    A = np.array([0.0, 1.0, 1.0]).reshape(3, 1, 1)
    D = np.array([1.0, 2.0, 1.0]).reshape(3, 1, 1)
    C = np.array([1.0, 1.0, 0.0]).reshape(3, 1, 1)
    with pytest.raises(lib.AcrError) as ei:
        factor(lib, A, D, C)
    assert ei.value.code == lib.ACR_ERR_SINGULAR and "level 1, block 0" in ei.value.msg


def test_nan_input_rejected(lib):
    A, D, C = syn.random_blocks(4, 6, seed=2)
    D[1, 2, 3] = np.nan
    with pytest.raises(lib.AcrError) as ei:
        factor(lib, A, D, C)
    assert ei.value.code == lib.ACR_ERR_INVALID_ARG


def test_refinement_not_converged_reported(lib):
    P = syn.make_config(3, 64)
    F = syn.rhs_uniform(P.N, 2, 5)
    h = factor_banded(lib, P, prec=2, ir_max_iter=1, ir_tol=1e-15)
    try:
        with pytest.raises(lib.AcrError) as ei:
            solve(lib, h, F)
        assert ei.value.code == lib.ACR_ERR_NOT_CONVERGED
        assert ei.value.iters == 1
    finally:
        lib.acr_free(h)


@pytest.mark.parametrize("refine", [0, 1])
def test_refinement_methods_poisson(lib, refine):
    """FGMRES and classic refinement both reach 1e-8 on an SPD problem."""
    P = syn.make_config(0, 128)
    F = syn.rhs_uniform(P.N, 3, 2000)
    h = factor_banded(lib, P, prec=2, refine=refine)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all() and 1 <= it <= 10


def test_refinement_off_reports_not_converged(lib):
    P = syn.make_config(0, 128)
    F = syn.rhs_uniform(P.N, 2, 2000)
    h = factor_banded(lib, P, prec=2, refine=2)
    try:
        with pytest.raises(lib.AcrError) as ei:
            solve(lib, h, F)
        assert ei.value.code == lib.ACR_ERR_NOT_CONVERGED and ei.value.iters == 1
    finally:
        lib.acr_free(h)


def test_stats(lib):
    P = syn.make_config(0, 32)
    h = factor_banded(lib, P)
    try:
        s = lib.acr_stats(h)
        assert s["levels"] == 6 and s["nblk"] == 32 and s["blksz"] == 32
        assert s["factor_ms"] > 0 and s["factor_flops"] > 0
        # structured level 0 keeps diagonals only: below the dense-storage bound
        o = lib.acr_default_opts()
        o.input_kind = lib.ACR_BANDED
        bound = lib.acr_factor_bytes(32, 32, 0.0, o) - 5 * 32 * 32 * 8
        assert 0 < s["factor_bytes"] < bound
        assert s["launches_factor"] > 0
    finally:
        lib.acr_free(h)


@pytest.mark.parametrize("prec", [0, 2])
def test_full_size_convdiff_512(lib, prec):
    """512^2 convection-diffusion (N = 262144) at full size: the oracle cannot
    run here in seconds, so the check is the residual, recomputed with numpy."""
    P = syn.make_config(2)
    F = syn.rhs_uniform(P.N, 8, 2002)
    h = factor_banded(lib, P, prec=prec)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    r = np.linalg.norm(F - P.matvec(X), axis=0) / np.linalg.norm(F, axis=0)
    assert (r <= 1e-8).all(), r


def test_full_size_helmholtz_1m(lib):
    """The N = 1048576 Helmholtz workload: mixed precision + FGMRES refinement
    (the launch configuration the benchmark times).  Block cyclic reduction of
    this indefinite operator amplifies rounding (near-singular reduced
    blocks), so plain refinement diverges and FGMRES needs a few dozen
    preconditioner solves."""
    P = syn.make_config(3)
    F = syn.rhs_uniform(P.N, 8, 2003)
    h = factor_banded(lib, P, prec=2, ir_max_iter=60)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all(), res
    r = np.linalg.norm(F - P.matvec(X), axis=0) / np.linalg.norm(F, axis=0)
    assert (r <= 1.5e-8).all(), r


@pytest.mark.parametrize("n,b", [(2, 128), (3, 128), (5, 256), (4, 384), (9, 128)])
def test_tensor_core_products_match_simt(lib, n, b):
    """tcgen05 three-term TF32 products agree with the FP32 CUDA-core products
    to FP32 rounding (one sweep, no refinement), and refine to the oracle."""
    A, D, C = syn.random_blocks(n, b, seed=n + b)
    F = np.random.default_rng(n).uniform(-1, 1, (n * b, 3))
    X = {}
    for prec in (1, 2):
        h = factor(lib, A, D, C, prec=prec, refine=2, ir_tol=1.0)
        try:
            X[prec], _, _ = solve(lib, h, F)
        finally:
            lib.acr_free(h)
    assert relerr(X[1], X[2]) <= 1e-6
    h = factor(lib, A, D, C, prec=1)
    try:
        Xr, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all()
    assert relerr(Xr, oracle.bcr_solve(A, D, C, F)) <= 1e-9


@pytest.mark.parametrize("n,b", [(3, 256), (5, 384), (2, 512), (3, 640)])
def test_tensor_core_inversion_with_interchanges(lib, n, b):
    """Diagonal blocks whose rows are randomly permuted: every inversion must
    interchange rows, across the 128-column outer panels whose updates run
    on the tensor cores.  The FP32 tensor-core factor agrees with the FP32
    CUDA-core factor to FP32 rounding, and refines to the oracle."""
    rng = np.random.default_rng(7 * b + n)
    A, D, C = syn.random_blocks(n, b, seed=b + n)
    for i in range(n):
        D[i] = D[i][rng.permutation(b)]
    F = rng.uniform(-1, 1, (n * b, 2))
    X = {}
    for prec in (1, 2):
        h = factor(lib, A, D, C, prec=prec, refine=2, ir_tol=1.0)
        try:
            X[prec], _, _ = solve(lib, h, F)
        finally:
            lib.acr_free(h)
    assert relerr(X[1], X[2]) <= 1e-5
    h = factor(lib, A, D, C, prec=1)
    try:
        Xr, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all()
    assert relerr(Xr, oracle.bcr_solve(A, D, C, F)) <= 1e-9


@pytest.mark.parametrize("n,b", [(3, 300), (2, 520)])
def test_fp32_blocked_inversion_ragged(lib, n, b):
    """FP32 blocks above the shared-memory limit whose size is not a multiple
    of the 32-column panel: register panels (one row per thread up to 512
    rows, two above) that gather for their update themselves, then a narrow
    last panel through the generic panel kernel and the separate gather, with
    rows interchanged everywhere.  Refined to the oracle."""
    rng = np.random.default_rng(11 * b + n)
    A, D, C = syn.random_blocks(n, b, seed=3 * b + n)
    for i in range(n):
        D[i] = D[i][rng.permutation(b)]
    F = rng.uniform(-1, 1, (n * b, 2))
    h = factor(lib, A, D, C, prec=2)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all()
    assert relerr(X, oracle.bcr_solve(A, D, C, F)) <= 1e-9


@pytest.mark.parametrize("idx,n", [(1, 128), (2, 256), (3, 256)])
def test_pde_tensor_core_refinement(lib, idx, n):
    P = syn.make_config(idx, n)
    A, D, C = P.dense_blocks()
    F = syn.rhs_uniform(P.N, 4, 2000 + idx)
    h = factor_banded(lib, P, prec=1, ir_max_iter=60)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all(), (res, it)
    r = np.linalg.norm(F - P.matvec(X), axis=0) / np.linalg.norm(F, axis=0)
    assert (r <= 1.5e-8).all()
    if n <= 128:
        assert relerr(X, oracle.bcr_solve(A, D, C, F)) <= 1e-6


def test_full_size_helmholtz_1m_tensor_cores(lib):
    """The benchmark's launch configuration: N = 1048576 Helmholtz, FP32 factor
    with tcgen05 products, FGMRES to 1e-8."""
    P = syn.make_config(3)
    F = syn.rhs_uniform(P.N, 8, 2003)
    h = factor_banded(lib, P, prec=1, ir_max_iter=60)
    try:
        X, res, it = solve(lib, h, F)
    finally:
        lib.acr_free(h)
    assert (res <= 1e-8).all(), res
    r = np.linalg.norm(F - P.matvec(X), axis=0) / np.linalg.norm(F, axis=0)
    assert (r <= 1.5e-8).all(), r
