"""Pins for the CPU oracle: values fixed by the paper and by mathematics, not by
the oracle itself.

* dense LU of the assembled matrix and ``numpy.linalg.solve`` (brute force);
* ``b = 1``: the Thomas algorithm and textbook scalar cyclic reduction;
* the closed-form eigenpairs of the 5-point Laplacian;
* the DST diagonalisation of every reduced Poisson block (the principle behind
  FACR, Section 1): block cyclic reduction becomes ``b`` independent scalar
  reductions on ``tridiag(-1, mu_j, -1)``;
* the Schur complement ``H22 - H21 H11^-1 H12`` of the even/odd permuted
  matrix (Section 3, Eq. "fund") formed densely;
* the n = 8 reduction structure of Section 3 (``golden/n8_reduction.json``);
* manufactured solutions;
* singular eliminated blocks reported with their (level, block).

A mutation test builds the oracle with planted mistakes and checks that these
pins catch every one.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _assemble(A, D, C):
    n, b, _ = D.shape
    M = np.zeros((n * b, n * b))
    for i in range(n):
        s = slice(i * b, (i + 1) * b)
        M[s, s] = D[i]
        if i > 0:
            M[s, (i - 1) * b:i * b] = A[i]
        if i < n - 1:
            M[s, (i + 1) * b:(i + 2) * b] = C[i]
    return M


def _rel(x, y):
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


# ---------------------------------------------------------------- pin bodies
# Each returns an error figure; the tests assert it is small and the mutation
# test asserts that some figure becomes large under a planted mistake.

def pin_dense(n, b, seed, symmetric=False):
    A, D, C = syn.random_blocks(n, b, seed, symmetric=symmetric)
    F = np.random.default_rng(seed + 7).standard_normal((n * b, 3))
    X = oracle.bcr_solve(A, D, C, F)
    M = _assemble(A, D, C)
    return max(_rel(X, np.linalg.solve(M, F)), _rel(X, oracle.dense_solve(M, F)))


def pin_pivot(n, b, seed):
    """Brute force on blocks that need row interchanges: every D_i of a
    diagonally dominant system has its rows shifted cyclically by one and its
    new diagonal set to zero, so each block is a dominant permutation pattern
    whose LU needs a row swap at every step (Section 3 inverts each eliminated
    block with partial pivoting).  A singular report counts as an infinite
    error."""
    A, D, C = syn.random_blocks(n, b, seed)
    D = np.roll(D, 1, axis=1)
    D[:, np.arange(b), np.arange(b)] = 0.0
    F = np.random.default_rng(seed + 11).standard_normal((n * b, 2))
    try:
        X = oracle.bcr_solve(A, D, C, F)
    except oracle.OracleSingular:
        return math.inf
    return _rel(X, np.linalg.solve(_assemble(A, D, C), F))


def _thomas(lo, di, up, f):
    n = len(di)
    cp = np.zeros(n); dp = np.zeros(n)
    cp[0] = up[0] / di[0]; dp[0] = f[0] / di[0]
    for i in range(1, n):
        den = di[i] - lo[i] * cp[i - 1]
        cp[i] = up[i] / den if i < n - 1 else 0.0
        dp[i] = (f[i] - lo[i] * dp[i - 1]) / den
    x = np.zeros(n)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def _scalar_cr(lo, di, up, f):
    """Textbook scalar cyclic reduction (alpha/gamma multipliers), recursive."""
    m = len(di)
    if m == 1:
        return np.array([f[0] / di[0]])
    nk = m // 2
    d2 = np.zeros(nk); l2 = np.zeros(nk); u2 = np.zeros(nk); f2 = np.zeros(nk)
    for k in range(nk):
        i = 2 * k + 1
        al = -lo[i] / di[i - 1]
        ga = -up[i] / di[i + 1] if i + 1 < m else 0.0
        d2[k] = di[i] + al * up[i - 1] + (ga * lo[i + 1] if i + 1 < m else 0.0)
        l2[k] = al * lo[i - 1]
        u2[k] = ga * up[i + 1] if i + 1 < m else 0.0
        f2[k] = f[i] + al * f[i - 1] + (ga * f[i + 1] if i + 1 < m else 0.0)
    y = _scalar_cr(l2, d2, u2, f2)
    x = np.zeros(m)
    x[1::2] = y
    for j in range(0, m, 2):
        s = f[j]
        if j > 0:
            s -= lo[j] * x[j - 1]
        if j + 1 < m:
            s -= up[j] * x[j + 1]
        x[j] = s / di[j]
    return x


def pin_scalar(n, seed):
    rng = np.random.default_rng(seed)
    di = rng.uniform(3, 5, n)
    lo = rng.uniform(-1, 1, n); lo[0] = 0.0
    up = rng.uniform(-1, 1, n); up[-1] = 0.0
    f = rng.uniform(-1, 1, n)
    A = lo.reshape(n, 1, 1); D = di.reshape(n, 1, 1); C = up.reshape(n, 1, 1)
    x = oracle.bcr_solve(A, D, C, f)
    return max(_rel(x, _thomas(lo, di, up, f)), _rel(x, _scalar_cr(lo, di, up, f)))


def pin_eigen(n, j, k):
    """f = v_jk gives u = v_jk / lambda_jk exactly (h^2-scaled Laplacian)."""
    p = np.arange(1, n + 1)
    vx = np.sin(j * math.pi * p / (n + 1))
    vy = np.sin(k * math.pi * p / (n + 1))
    v = np.outer(vy, vx).reshape(-1)  # block q (y), row p (x)
    lam = 4 - 2 * math.cos(j * math.pi / (n + 1)) - 2 * math.cos(k * math.pi / (n + 1))
    P = syn.poisson(n)
    A, D, C = P.dense_blocks()
    u = oracle.bcr_solve(A, D, C, v)
    return _rel(u, v / lam)


def _dst(b):
    p = np.arange(1, b + 1)
    return math.sqrt(2.0 / (b + 1)) * np.sin(np.outer(p, p) * math.pi / (b + 1))


def _scalar_levels(n, mu, nlev):
    """Scalar reduction coefficients (d, a, c) after nlev levels, one mode."""
    d = np.full(n, mu); a = -np.ones(n); c = -np.ones(n)
    a[0] = 0.0; c[-1] = 0.0
    for _ in range(nlev):
        m = len(d)
        if m == 1:
            break
        nk = m // 2
        d2 = np.zeros(nk); a2 = np.zeros(nk); c2 = np.zeros(nk)
        for k in range(nk):
            i = 2 * k + 1
            al = -a[i] / d[i - 1]
            ga = -c[i] / d[i + 1] if i + 1 < m else 0.0
            d2[k] = d[i] + al * c[i - 1] + (ga * a[i + 1] if i + 1 < m else 0.0)
            a2[k] = al * a[i - 1]
            c2[k] = ga * c[i + 1] if i + 1 < m else 0.0
        d, a, c = d2, a2, c2
    return d, a, c


def pin_dst(n, b, nlev):
    """Every reduced Poisson block is S diag(.) S with the scalar-CR values."""
    S = _dst(b)
    mu = 4 - 2 * np.cos(np.arange(1, b + 1) * math.pi / (b + 1))
    D0 = np.tile((4 * np.eye(b) - np.eye(b, k=1) - np.eye(b, k=-1))[None], (n, 1, 1))
    A0 = np.tile(-np.eye(b)[None], (n, 1, 1)); A0[0] = 0
    C0 = np.tile(-np.eye(b)[None], (n, 1, 1)); C0[-1] = 0
    Ar, Dr, Cr = oracle.bcr_reduce(A0, D0, C0, nlev)
    m = Dr.shape[0]
    modes = [_scalar_levels(n, mu[j], nlev) for j in range(b)]
    err = 0.0
    for i in range(m):
        for X, which in ((Dr, 0), (Ar, 1), (Cr, 2)):
            ref = np.diag([modes[j][which][i] for j in range(b)])
            err = max(err, np.abs(S @ X[i] @ S - ref).max() / max(1.0, np.abs(ref).max()))
    return err, m


def pin_schur(n, b, seed):
    """One reduction level equals H22 - H21 H11^-1 H12 of the permuted matrix."""
    A, D, C = syn.random_blocks(n, b, seed)
    M = _assemble(A, D, C)
    even = np.concatenate([np.arange(j * b, (j + 1) * b) for j in range(0, n, 2)])
    odd = np.concatenate([np.arange(i * b, (i + 1) * b) for i in range(1, n, 2)])
    H11 = M[np.ix_(even, even)]; H12 = M[np.ix_(even, odd)]
    H21 = M[np.ix_(odd, even)]; H22 = M[np.ix_(odd, odd)]
    S = H22 - H21 @ np.linalg.solve(H11, H12)
    Ar, Dr, Cr = oracle.bcr_reduce(A, D, C, 1)
    Sr = _assemble(Ar, Dr, Cr)
    # the Schur complement is block tridiagonal: nothing outside the band
    return _rel(Sr, S)


def pin_manufactured(idx, n, seed=5):
    P = syn.make_config(idx, n)
    A, D, C = P.dense_blocks()
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (P.N, 2))
    F = P.matvec(u)
    x = oracle.bcr_solve(A, D, C, F)
    return _rel(x, u)


# ---------------------------------------------------------------- the tests

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 32])
def test_dense_lu_square(n):
    assert pin_dense(n, n, seed=n) < 1e-12


@pytest.mark.parametrize("n,b", [(7, 3), (6, 5), (9, 2), (13, 4), (4, 9)])
def test_dense_lu_ragged(n, b):
    assert pin_dense(n, b, seed=10 * n + b) < 1e-12
    assert pin_dense(n, b, seed=10 * n + b + 1, symmetric=True) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 31, 64, 100])
def test_scalar_b1_thomas_and_textbook_cr(n):
    assert pin_scalar(n, seed=n) < 1e-13


@pytest.mark.parametrize("n,j,k", [(8, 1, 1), (8, 3, 5), (15, 2, 14), (64, 1, 1), (64, 17, 40)])
def test_laplacian_eigenpairs(n, j, k):
    assert pin_eigen(n, j, k) < 1e-12


@pytest.mark.parametrize("n,b,nlev", [(8, 6, 1), (8, 6, 2), (8, 6, 3), (11, 5, 1), (11, 5, 2),
                                      (11, 5, 3), (16, 16, 4), (13, 7, 2)])
def test_dst_levels(n, b, nlev):
    err, m = pin_dst(n, b, nlev)
    assert err < 1e-12


@pytest.mark.parametrize("n,b", [(7, 3), (8, 3), (2, 4), (3, 2), (10, 2)])
def test_schur_complement_of_permuted_system(n, b):
    assert pin_schur(n, b, seed=n + b) < 1e-12


def test_n8_structure_golden():
    g = json.load(open(os.path.join(GOLDEN, "n8_reduction.json")))
    sched = oracle.bcr_schedule(8)
    assert sched[0] == g["level0_eliminated"]
    # relabel: at every level the surviving blocks are renumbered 0..m-1
    alive = list(range(8))
    sizes, relab = [], []
    for elim in sched:
        sizes.append(len(alive))
        relab.append([alive.index(o) for o in elim])
        alive = [o for o in alive if o not in elim]
    assert sizes == g["level_sizes"]
    assert relab == g["eliminated_relabelled"]
    assert sorted(set(range(8)) - set(g["level0_eliminated"])) == g["level0_kept"]
    # the reduced systems have the printed sizes
    P = syn.poisson(8)
    A, D, C = P.dense_blocks()
    for t, sz in enumerate(g["level_sizes"]):
        assert oracle.bcr_reduce(A, D, C, t)[1].shape[0] == sz


@pytest.mark.parametrize("idx,n", [(0, 64), (1, 32), (2, 32), (3, 32), (3, 20)])
def test_manufactured_solution(idx, n):
    assert pin_manufactured(idx, n) < 1e-10


def test_singular_block_reported():
    A, D, C = syn.random_blocks(6, 3, 1)
    D[4] = 0.0
    with pytest.raises(oracle.OracleSingular) as ei:
        oracle.bcr_solve(A, D, C, np.ones(18))
    assert (ei.value.level, ei.value.block) == (0, 4)
    # a Schur complement that is exactly singular at level 1 (scalar case):
    # d'_0 = 2 - 1*1/1 - 1*1/1 = 0
    A = np.array([0.0, 1.0, 1.0]).reshape(3, 1, 1)
    D = np.array([1.0, 2.0, 1.0]).reshape(3, 1, 1)
    C = np.array([1.0, 1.0, 0.0]).reshape(3, 1, 1)
    with pytest.raises(oracle.OracleSingular) as ei:
        oracle.bcr_solve(A, D, C, np.ones(3))
    assert ei.value.level == 1


def _all_pins():
    """Error figures of a fast subset of the pins (used by the mutation test)."""
    errs = [pin_dense(7, 3, 1), pin_dense(8, 4, 2), pin_scalar(9, 3), pin_eigen(8, 3, 5),
            pin_dst(11, 5, 2)[0], pin_dst(8, 6, 3)[0], pin_schur(7, 3, 4), pin_schur(8, 3, 5),
            pin_manufactured(2, 16), pin_pivot(7, 6, 3)]
    return errs


def test_pins_pass_on_real_oracle():
    assert max(_all_pins()) < 1e-10


@pytest.mark.parametrize("n,b,seed", [(7, 6, 3), (8, 5, 4), (5, 9, 1)])
def test_row_interchanges_brute_force(n, b, seed):
    assert pin_pivot(n, b, seed) < 1e-10


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7])
def test_pins_catch_planted_mistakes(mutant):
    """Each planted mistake makes at least one pin fail: a dropped Schur term,
    a wrong sign, a wrong index, a transposed operand, a dropped term of the
    right-hand-side reduction, a wrong neighbour in the back-substitution,
    and an LU without row interchanges."""
    oracle.use_mutant(mutant)
    try:
        errs = _all_pins()
    finally:
        oracle.use_mutant(0)
    assert max(errs) > 1e-6, errs


# ------------------------------------------------ residual and early stop pins

@pytest.mark.parametrize("n,b,seed", [(1, 5, 1), (4, 3, 2), (7, 6, 3), (12, 9, 4)])
def test_oracle_residual_against_assembled_matrix(n, b, seed):
    """``oracle.residual`` is ||F - M X||_2 / ||F||_2 per column; recomputed
    here with the assembled matrix and numpy, for arbitrary X (not a
    solution), and ~0 for the brute-force solution."""
    A, D, C = syn.random_blocks(n, b, seed)
    rng = np.random.default_rng(seed + 3)
    F = rng.standard_normal((n * b, 3))
    X = rng.standard_normal((n * b, 3))
    M = _assemble(A, D, C)
    want = np.linalg.norm(F - M @ X, axis=0) / np.linalg.norm(F, axis=0)
    got = oracle.residual(A, D, C, X, F)
    assert np.allclose(got, want, rtol=1e-12, atol=0), (got, want)
    Xs = np.linalg.solve(M, F)
    assert (oracle.residual(A, D, C, Xs, F) <= 1e-13).all()


@pytest.mark.parametrize("n,m_stop", [(8, 2), (8, 3), (11, 2), (11, 5), (16, 4), (9, 9), (6, 20)])
def test_early_stop_top_solve_brute_force(n, m_stop):
    """Section 3 allows the reduction to stop once the system is small
    enough; the remaining m <= m_stop blocks are then solved as one dense
    system.  Every stopping point gives the brute-force solution."""
    b = 5
    A, D, C = syn.random_blocks(n, b, seed=n + 17 * m_stop)
    F = np.random.default_rng(m_stop).standard_normal((n * b, 2))
    X = oracle.bcr_solve(A, D, C, F, m_stop=m_stop)
    assert _rel(X, np.linalg.solve(_assemble(A, D, C), F)) <= 1e-12
    # the schedule: the last entry lists the blocks of the top solve
    sched = oracle.bcr_schedule(n, m_stop)
    assert 1 <= len(sched[-1]) <= max(1, m_stop)
    assert sorted(i for lv in sched for i in lv) == list(range(n))
