"""Batched low-rank truncation (Section 3: the recompression after every
H-sum and H-product) through ``acr_lowrank_truncate``, node by node against a
host SVD of the same dense node M = U V^T:

* the kept rank is the number of singular values above tol * sigma_1, so
  sigma_{r+1} <= tol * sigma_1 < sigma_r;
* the kept right factor is orthonormal (Q^T Q = I) and zero beyond the rank;
* |M - U' V'^T|_2 is sigma_{r+1} up to rounding (the truncation is the
  optimal one);
* the randomized first pass gives the same ranks and bounds, and hands the
  nodes whose rank nears its width to the exact pass.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1604_00617_gb300 import build
    build()
    from paper_1604_00617_gb300 import _lib
    return _lib


def nodes(count, s, R, ranks, seed, tail=1e-8):
    """count nodes M_i = U_i V_i^T with singular values 1, q, q^2, ... down to
    rank ranks[i] (q = 0.7), then a tail from `tail` down by halves, given
    through non-orthogonal factors of width R.  Layout (count, R, s)."""
    rng = np.random.default_rng(seed)
    U = np.zeros((count, R, s))
    V = np.zeros((count, R, s))
    for i in range(count):
        k = min(s, R)
        A, _ = np.linalg.qr(rng.standard_normal((s, k)))
        B, _ = np.linalg.qr(rng.standard_normal((s, k)))
        sig = np.empty(k)
        r = ranks[i]
        sig[:r] = 0.7 ** np.arange(r)
        if r < k:
            sig[r:] = tail * 0.5 ** np.arange(k - r) if r > 0 else 0.0
        G = rng.standard_normal((k, R)) / np.sqrt(R) + np.eye(k, R)
        Gp = np.linalg.pinv(G).T                       # G Gp^T = I (k x k)
        U[i] = ((A * sig) @ G).T
        V[i] = (B @ Gp).T
    return U, V


def check(U, V, Uo, Vo, rk, tol, eps):
    for i in range(U.shape[0]):
        M = U[i].T @ V[i]
        sv = np.linalg.svd(M, compute_uv=False)
        if sv[0] == 0:
            assert rk[i] == 0 and not Uo[i].any() and not Vo[i].any()
            continue
        r = int(rk[i])
        want = int(np.sum(sv > tol * sv[0]))
        assert r == want, (i, r, want, sv[:want + 2] / sv[0])
        assert r == len(sv) or sv[r] <= tol * sv[0]
        Q = Vo[i, :r].T
        assert np.abs(Q.T @ Q - np.eye(r)).max() <= eps, i
        assert not Vo[i, r:].any() and not Uo[i, r:].any()
        err = np.linalg.norm(M - Uo[i].T @ Vo[i], 2)
        tail = sv[r] if r < len(sv) else 0.0
        assert err <= 1.01 * tail + eps * sv[0], (i, err, tail)


@pytest.mark.parametrize("s,R", [(64, 40), (48, 80), (128, 24), (32, 32)])
def test_exact_pass_fp64(lib, s, R):
    rng = np.random.default_rng(s * 1000 + R)
    k = min(s, R)
    ranks = rng.integers(0, k // 2 + 1, size=24)
    U, V = nodes(24, s, R, ranks, seed=s + R)
    U[3] = 0.0  # a zero node
    V[3] = 0.0
    tol = 1e-6
    Uo, Vo, rk, redo = lib.acr_lowrank_truncate(U, V, tol)
    assert redo == 0
    check(U, V, Uo, Vo, rk, tol, 1e-11)


def test_sketch_pass_fp64(lib):
    s, R = 96, 64
    ranks = np.array([1, 3, 6, 9, 10, 11, 12, 14, 20, 2] * 3)
    U, V = nodes(len(ranks), s, R, ranks, seed=7)
    tol = 1e-6
    Uo, Vo, rk, redo = lib.acr_lowrank_truncate(U, V, tol, sketch=16)
    check(U, V, Uo, Vo, rk, tol, 1e-11)
    # width 16: ranks above 10 are redone exactly, the others resolved by the sketch
    assert redo == int(np.sum(ranks > 10)), (redo, rk)
    Ue, Ve, rke, _ = lib.acr_lowrank_truncate(U, V, tol)
    assert (rke == rk).all()


@pytest.mark.parametrize("sketch", [0, 16])
def test_fp32_truncation(lib, sketch):
    s, R = 64, 48
    ranks = np.array([2, 5, 8, 12, 4, 7, 1, 9] * 2)
    U, V = nodes(len(ranks), s, R, ranks, seed=11, tail=1e-7)
    tol = 1e-5
    Uo, Vo, rk, redo = lib.acr_lowrank_truncate(U, V, tol, precision=lib.ACR_FP32TC_IR, sketch=sketch)
    check(U, V, Uo, Vo, rk, tol, 2e-5)


def test_tol_zero_keeps_everything(lib):
    """tol -> 0: the truncation is a refactorization, U' V'^T = U V^T to
    rounding (a few thousand units of FP64 for width 20 through two QRs and
    the Jacobi rotations)."""
    s, R = 48, 20
    U, V = nodes(6, s, R, [20] * 6, seed=3)
    Uo, Vo, rk, _ = lib.acr_lowrank_truncate(U, V, 0.0)
    assert (rk == 20).all()
    for i in range(6):
        M = U[i].T @ V[i]
        assert np.linalg.norm(M - Uo[i].T @ Vo[i]) <= 1e-12 * np.linalg.norm(M)
