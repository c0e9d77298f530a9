"""acr_block_inverse_noalloc: the batched block inversion for callers that
cannot allocate device memory (for example code running inside a framework's
memory pool that already holds almost all of the GPU, or latency-critical
paths that cannot absorb an allocation).  Its result must equal what the
solver's own entry points give for the same blocks: factoring the block-
diagonal system tridiag(0, D_i, 0) and solving with identity right-hand sides
yields every D_i^-1.  Two calls in a row with different blocks check that the
shared scratch keeps nothing that matters between calls.

This file is named to run last: a failure here leaves every other test run.
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


def _blocks(count, b, seed):
    rng = np.random.default_rng(seed)
    D = rng.uniform(-1, 1, (count, b, b)) + 2.0 * np.sqrt(b) * np.eye(b)[None]
    return D


def _colmajor(X):
    return np.ascontiguousarray(np.transpose(X, (0, 2, 1)))


def _reference_inverses(lib, D):
    """D_i^-1 through acr_factor / acr_solve on tridiag(0, D_i, 0)."""
    count, b, _ = D.shape
    Z = np.zeros_like(D)
    h = lib.acr_factor(count, b, _colmajor(Z), _colmajor(D), _colmajor(Z), 0.0)
    try:
        B = np.asfortranarray(np.tile(np.eye(b), (count, 1)))
        lib.acr_solve(h, B, b)
    finally:
        lib.acr_free(h)
    return np.stack([B[i * b:(i + 1) * b, :] for i in range(count)])


def test_noalloc_inverse_matches_factor_solve(lib):
    import torch
    stream = torch.cuda.current_stream()
    count, b = 3, 256  # blksz 256 takes the blocked path, which uses the scratch
    for seed in (11, 12):  # two calls in a row
        D = _blocks(count, b, seed)
        mats = torch.from_numpy(_colmajor(D)).cuda()
        info = torch.full((count,), -7, dtype=torch.int32, device="cuda")
        lib.acr_block_inverse_noalloc(b, count, mats, info, stream.cuda_stream)
        torch.cuda.synchronize()
        assert (info.cpu().numpy() == 0).all()
        X = np.transpose(mats.cpu().numpy(), (0, 2, 1))
        ref = _reference_inverses(lib, D)
        for i in range(count):
            err = np.linalg.norm(X[i] - ref[i]) / np.linalg.norm(ref[i])
            assert err <= 1e-10, (seed, i, err)


def test_noalloc_rejects_batches_beyond_the_scratch(lib):
    import torch
    b, count = 1024, 200  # needs far more than the fixed scratch
    mats = torch.zeros(b * b, dtype=torch.float64, device="cuda")  # never touched
    info = torch.zeros(count, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.AcrError) as ei:
        lib._check(lib._lib.acr_block_inverse_noalloc(b, count, lib._ptr(mats), lib.ctypes.c_void_p(info.data_ptr()),
                                                      None))
    assert ei.value.code == lib.ACR_ERR_INVALID_ARG and "scratch" in ei.value.msg
