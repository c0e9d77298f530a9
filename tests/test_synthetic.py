"""Generator properties: the structure each workload's discretisation fixes."""

import math

import numpy as np
import pytest

import synthetic as syn


def test_exact_level0_structure():
    """D_i tridiagonal, A_i and C_i diagonal (Section 3)."""
    for idx in range(4):
        P = syn.make_config(idx, 12)
        A, D, C = P.dense_blocks()
        for i in range(P.nblk):
            assert np.count_nonzero(np.triu(D[i], 2)) == 0
            assert np.count_nonzero(np.tril(D[i], -2)) == 0
            assert np.count_nonzero(A[i] - np.diag(np.diag(A[i]))) == 0
            assert np.count_nonzero(C[i] - np.diag(np.diag(C[i]))) == 0
        assert not A[0].any() and not C[-1].any()


@pytest.mark.parametrize("idx,sym", [(0, True), (1, True), (2, False), (3, True)])
def test_symmetry(idx, sym):
    M = syn.make_config(idx, 10).assemble()
    assert np.allclose(M, M.T) == sym


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_m_matrix_sign_pattern(idx):
    M = syn.make_config(idx, 10).assemble()
    off = M - np.diag(np.diag(M))
    assert (np.diag(M) > 0).all() and (off <= 0).all()
    # weakly diagonally dominant by rows
    assert (np.diag(M) + 1e-12 >= np.abs(off).sum(1)).all()


def test_diffusion_contrast_and_harmonic_faces():
    n = 24
    g = syn.gaussian_random_field(n + 2, 1001)
    sigma = math.log(1e4) / (g.max() - g.min())
    kap = np.exp(sigma * (g - g.min()))
    assert math.isclose(kap.max() / kap.min(), 1e4, rel_tol=1e-12)
    P = syn.variable_diffusion(n, seed=1001)
    cell = kap[1:-1, 1:-1]
    # east face between (p=3, q=5) and (p=4, q=5): harmonic mean
    hm = 2 * cell[5, 3] * cell[5, 4] / (cell[5, 3] + cell[5, 4])
    assert math.isclose(-P.Du[5, 3], hm, rel_tol=1e-14)
    # row sum equals the boundary face coefficients only (interior rows: zero)
    M = P.assemble()
    rs = M.sum(1).reshape(n, n)
    assert np.allclose(rs[3:-3, 3:-3], 0, atol=1e-9 * kap.max())


def test_helmholtz_points_per_wavelength_and_indefinite():
    n = 40
    P = syn.helmholtz(n, seed=1003)
    h = 1.0 / (n + 1)
    kh = np.sqrt(4.0 - P.Dd)
    k0h = 2 * math.pi / 16
    assert np.all(kh >= 0.8 * k0h - 1e-12) and np.all(kh <= 1.2 * k0h + 1e-12)
    w = np.linalg.eigvalsh(P.assemble())
    assert w.min() < 0 < w.max()


def test_convection_upwind_coefficients():
    n = 16
    P = syn.convection_diffusion(n, seed=1002)
    h = 1.0 / (n + 1)
    # |beta| h = 1e3 h; diagonal minus 4 equals h(|bx| + |by|) <= sqrt(2) 1e3 h
    extra = P.Dd - 4.0
    assert (extra >= 1e3 * h - 1e-9).all() and (extra <= math.sqrt(2) * 1e3 * h + 1e-9).all()
    # the row sum of an interior row is zero (upwind differences of constants vanish)
    M = P.assemble()
    assert np.allclose(M.sum(1).reshape(n, n)[1:-1, 1:-1], 0, atol=1e-9)


def test_seeds_reproduce_bitwise():
    a = syn.make_config(1, 16); b = syn.make_config(1, 16)
    assert np.array_equal(a.Dd, b.Dd) and np.array_equal(a.a, b.a)
    r1 = syn.rhs_uniform(100, 3, 2001); r2 = syn.rhs_uniform(100, 3, 2001)
    assert np.array_equal(r1, r2) and r1.min() >= -1 and r1.max() <= 1


def test_banded_matvec_matches_assembled():
    P = syn.make_config(2, 9)
    x = np.random.default_rng(0).standard_normal((P.N, 2))
    assert np.allclose(P.matvec(x), P.assemble() @ x)


def _offdiag_rank(M, r0, c0, sz, tol):
    s = np.linalg.svd(M[r0:r0 + sz, c0:c0 + sz], compute_uv=False)
    return int((s > tol * s[0]).sum())


def test_strip_kernel_mid_ranks():
    # the regime the FP32 sketch test relies on: every off-diagonal node of
    # D^-1 and of the top block's inverse has rank 13..28 at 1e-6, so the
    # 16-column sketch saturates and the 32-column one resolves it
    A, D, C = syn.strip_kernel_blocks(3, 1024, seed=5)
    assert A.shape == D.shape == C.shape == (3, 1024, 1024)
    assert not A[0].any() and not C[-1].any()
    K = D[0] - (D[0, 0, 0] - 1.0) * np.eye(1024)  # K has a unit diagonal
    assert np.linalg.eigvalsh(K).min() > 0  # K is SPD
    Di = [np.linalg.inv(D[j]) for j in (0, 2)]
    top = np.linalg.inv(D[1] - A[1] @ Di[0] @ C[0] - C[1] @ Di[1] @ A[2])
    for M in (Di[0], Di[1], top):
        for l in range(1, 5):
            sz = 1024 >> l
            for r0, c0 in ((0, sz), (sz, 0)):
                assert 13 <= _offdiag_rank(M, r0, c0, sz, 1e-6) <= 28, (l, r0, c0)
