"""The serving loop on the GPU: a mixed stream of diffusion and
convection-diffusion systems with interleaved solves, admitted and overlapped
on several streams; each solve's result must equal the result of the same
system factored and the same right-hand side solved alone (nrhs = 1)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _alone(lib, req, rhs, srv):
    o = lib.acr_default_opts()
    o.precision = srv.precision
    o.input_kind = lib.ACR_BANDED
    o.ir_tol = srv.ir_tol
    o.ir_max_iter = srv.ir_max_iter
    o.leaf = req.leaf
    h = lib.acr_factor_ex(req.nblk, req.blksz, req.a, req.D3, req.c, req.tol, o)
    try:
        out = []
        for f in rhs:
            B = np.asfortranarray(f.reshape(-1, 1).copy())
            res, _ = lib.acr_solve_ex(h, B, 1)
            out.append((B[:, 0], float(res[0])))
        return out
    finally:
        lib.acr_free(h)


@pytest.mark.parametrize("tol", [0.0, 1e-6])
def test_mix_equals_alone(tol):
    from paper_1604_00617_gb300 import _lib as lib
    from paper_1604_00617_gb300 import serving
    ev = serving.make_requests(48, rate=3000.0, seed=11, sizes=(64, 128, 256), probs=(0.4, 0.4, 0.2),
                               max_solves=10, tol=tol)
    srv = serving.Server(budget_bytes=16 << 30, slots=4, keep_results=True)
    recs, wall = srv.run(ev)
    assert not srv.errors, srv.errors
    assert all(r.ok for r in recs.values())
    solves = [r for _, r in ev if isinstance(r, serving.SolveRequest)]
    assert all(recs[r.rid].resid <= 1e-8 for r in solves)
    # the mix really overlapped and coalesced
    assert srv.peak_active > 1
    assert max(recs[r.rid].batch for r in solves) > 1
    systems = [r for _, r in ev if isinstance(r, serving.SystemRequest)]
    for s in systems:
        mine = [r for r in solves if r.sys_rid == s.rid]
        alone = _alone(lib, s, [r.rhs for r in mine], srv)
        for r, (x, res) in zip(mine, alone):
            got = srv.results[r.rid]
            assert res <= 1e-8
            d = np.max(np.abs(got - x)) / np.max(np.abs(x))
            assert np.array_equal(got, x), f"system {s.rid} n={s.nblk} solve {r.rid}: rel diff {d:.3e}"


def test_budget_respected_on_device():
    import torch
    from paper_1604_00617_gb300 import _lib as lib
    from paper_1604_00617_gb300 import serving
    ev = serving.make_requests(24, rate=5000.0, seed=5, sizes=(256,), probs=(1.0,), max_solves=4, tol=1e-6)
    one = serving.peak_bytes(ev[0][1], lib.ACR_FP32TC_IR)
    budget = 2 * one
    torch.cuda.synchronize()
    srv = serving.Server(budget_bytes=budget, slots=6)
    recs, wall = srv.run(ev)
    assert all(r.ok for r in recs.values())
    assert srv.peak_reserved <= budget
    st = serving.summarize(recs, wall)
    assert st["solves_per_s"] > 0 and st["failed"] == 0
