"""Failure paths on the GPU, in the forms that leave the device usable.

* Timeout: every mbarrier wait of the tensor-core product kernel is bounded.
  With ACR_TEST_TC_WITHHOLD=1 its producer issues no copies and the waits
  give up after a short limit; the factorization must return
  ACR_ERR_TIMEOUT, and the next factorization in the same process (the
  setting removed) must succeed.
* Out of memory: with nearly all of the GPU's memory taken by another
  allocator (torch), a factorization whose arena does not fit must return
  ACR_ERR_OOM and leak nothing; once the memory is released the same call
  succeeds.

Each scenario runs in a child process of its own, so neither the setting nor
the occupied memory reaches the other tests.
"""

import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(script, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.pop("ACR_TEST_TC_WITHHOLD", None)
    if env_extra:
        env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(script)], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1604_00617_gb300 import build
    build()


def test_tensor_core_wait_timeout_is_reported_and_device_stays_usable():
    out = _run("""
        import os
        import numpy as np
        import synthetic as syn
        from paper_1604_00617_gb300 import _lib as acr

        def cm(X):
            return np.ascontiguousarray(np.transpose(X, (0, 2, 1)))

        A, D, C = syn.random_blocks(3, 256, seed=9)
        F = np.random.default_rng(9).uniform(-1, 1, (3 * 256, 2))
        o = acr.acr_default_opts()
        o.precision = acr.ACR_FP32TC_IR
        os.environ["ACR_TEST_TC_WITHHOLD"] = "1"
        try:
            acr.acr_factor_ex(3, 256, cm(A), cm(D), cm(C), 0.0, o)
            print("NO ERROR")
        except acr.AcrError as e:
            print("CODE", e.code)
        del os.environ["ACR_TEST_TC_WITHHOLD"]
        h = acr.acr_factor_ex(3, 256, cm(A), cm(D), cm(C), 0.0, o)
        B = np.asfortranarray(F.copy())
        res, it = acr.acr_solve_ex(h, B, 2)
        acr.acr_free(h)
        print("AFTER", float(res.max()))
    """)
    lines = dict(ln.split(" ", 1) for ln in out.strip().splitlines() if " " in ln)
    assert lines.get("CODE") == "-6", out  # ACR_ERR_TIMEOUT
    assert float(lines["AFTER"]) <= 1e-8, out


def test_device_out_of_memory_is_reported_and_recovers():
    out = _run("""
        import numpy as np
        import torch
        import synthetic as syn
        from paper_1604_00617_gb300 import _lib as acr

        P = syn.make_config(3, 512)
        a, D3, c = P.banded_abi()
        F = syn.rhs_uniform(P.N, 1, 2003)
        o = acr.acr_default_opts()
        o.precision = acr.ACR_FP32TC_IR
        o.input_kind = acr.ACR_BANDED
        o.ir_max_iter = 60
        need = acr.acr_factor_bytes(P.nblk, P.b, 0.0, o)
        torch.cuda.init()
        free, total = torch.cuda.mem_get_info()
        hold = torch.empty(free - (256 << 20), dtype=torch.uint8, device="cuda")
        print("NEED", need)
        try:
            acr.acr_factor_ex(P.nblk, P.b, a, D3, c, 0.0, o)
            print("NO ERROR")
        except acr.AcrError as e:
            print("CODE", e.code)
        del hold
        torch.cuda.empty_cache()
        h = acr.acr_factor_ex(P.nblk, P.b, a, D3, c, 0.0, o)
        B = np.asfortranarray(F.copy())
        res, it = acr.acr_solve_ex(h, B, 1)
        acr.acr_free(h)
        print("AFTER", float(res.max()))
    """)
    lines = dict(ln.split(" ", 1) for ln in out.strip().splitlines() if " " in ln)
    assert int(lines["NEED"]) > (256 << 20)
    assert lines.get("CODE") == "-2", out  # ACR_ERR_OOM
    assert float(lines["AFTER"]) <= 1e-8, out
