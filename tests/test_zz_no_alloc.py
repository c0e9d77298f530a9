"""acr_block_inverse_noalloc: the batched block inversion for callers that
cannot allocate device memory when they need it (code running inside another
framework's memory pool that already holds almost all of the GPU, or
latency-critical paths that cannot absorb an allocation, its failure or the
synchronisation a free can cause).

Its inverses are checked element by element against ``numpy.linalg.inv`` of
the same blocks, computed on the host (LAPACK, not this library).  Two calls
in a row with different blocks check that the shared scratch array, which
keeps the previous call's contents, leaks nothing into the next result.

This file is named to run last: a failure here leaves every other test run.
It also passes alone in a fresh process (the first call on the device looks
up the scratch array's address).
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
    return rng.uniform(-1, 1, (count, b, b)) + 2.0 * np.sqrt(b) * np.eye(b)[None]


def _colmajor(X):
    return np.ascontiguousarray(np.transpose(X, (0, 2, 1)))


@pytest.mark.parametrize("b,count", [(256, 3), (200, 5)])
def test_noalloc_inverse_matches_numpy_inverse(lib, b, count):
    """blksz above the shared-memory kernel's limit (159 in FP64) takes the
    blocked path, whose pivots and panels live in the fixed scratch."""
    import torch
    stream = torch.cuda.current_stream()
    for seed in (11, 12):  # two calls in a row on the same scratch
        D = _blocks(count, b, seed + b)
        mats = torch.from_numpy(_colmajor(D)).cuda()
        info = torch.full((count,), -7, dtype=torch.int32, device="cuda")
        lib.acr_block_inverse_noalloc(b, count, mats, info, stream.cuda_stream)
        torch.cuda.synchronize()
        assert (info.cpu().numpy() == 0).all()
        X = np.transpose(mats.cpu().numpy(), (0, 2, 1))
        for i in range(count):
            ref = np.linalg.inv(D[i])
            # element by element: every entry within 1e-12 of the largest
            # entry of the reference inverse (the blocks are well conditioned:
            # diagonally dominant, condition number below 10)
            assert np.abs(X[i] - ref).max() <= 1e-12 * np.abs(ref).max(), (seed, i)
            assert np.linalg.norm(X[i] - ref) / np.linalg.norm(ref) <= 1e-12


def test_noalloc_reports_a_singular_block(lib):
    import torch
    b, count = 180, 2
    D = _blocks(count, b, 5)
    D[1][:, 7] = 0.0  # column 7 of block 1 is zero: no pivot in that column
    mats = torch.from_numpy(_colmajor(D)).cuda()
    info = torch.zeros(count, dtype=torch.int32, device="cuda")
    lib.acr_block_inverse_noalloc(b, count, mats, info, None)
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[0] == 0 and inf[1] > 0
    X0 = np.transpose(mats.cpu().numpy(), (0, 2, 1))[0]
    ref = np.linalg.inv(D[0])
    assert np.abs(X0 - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_batches_beyond_the_scratch(lib):
    import torch
    b, count = 1024, 200  # needs far more than the fixed scratch
    mats = torch.zeros(b * b, dtype=torch.float64, device="cuda")  # never touched
    info = torch.zeros(count, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.AcrError) as ei:
        lib._check(lib._lib.acr_block_inverse_noalloc(b, count, lib._ptr(mats), lib.ctypes.c_void_p(info.data_ptr()),
                                                      None))
    assert ei.value.code == lib.ACR_ERR_INVALID_ARG and "scratch" in ei.value.msg
