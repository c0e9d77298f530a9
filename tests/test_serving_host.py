"""Host-side tests of the serving loop's scheduling: admission under the
memory budget, continuous batching, right-hand-side coalescing and failure
propagation, with the CUDA library replaced by a fake that sleeps."""

import threading
import time

import numpy as np
import pytest

from paper_1604_00617_gb300 import _lib as acr
from paper_1604_00617_gb300 import serving


class FakeStream:
    cuda_stream = 0


class FakeLib:
    """Factor and solve calls that take `tf` / `ts` seconds; a solve returns
    2 * B; systems whose block count is in `fail` fail to factor."""

    def __init__(self, tf=0.05, ts=0.01, fail=(), held=1 << 20):
        self.tf, self.ts, self.fail, self.held = tf, ts, set(fail), held
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0
        self.solve_calls = []   # (system id, nrhs)
        self.freed = []

    def acr_default_opts(self):
        return acr.acr_default_opts()

    def _enter(self):
        with self.lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)

    def _leave(self):
        with self.lock:
            self.live -= 1

    def acr_factor_ex(self, nblk, blksz, a, D3, c, tol, o):
        self._enter()
        time.sleep(self.tf)
        self._leave()
        if nblk in self.fail:
            raise acr.AcrError(acr.ACR_ERR_SINGULAR, "planted failure")
        return {"id": int(a[0]), "n": nblk}

    def acr_stats(self, h):
        return {"factor_bytes": self.held, "operator_bytes": 0}

    def acr_solve_ex(self, h, B, nrhs):
        self._enter()
        with self.lock:
            self.solve_calls.append((h["id"], nrhs))
        time.sleep(self.ts)
        B *= 2.0
        self._leave()
        return np.zeros(nrhs), 1

    def acr_free(self, h):
        with self.lock:
            self.freed.append(h["id"])


def _system(rid, t, n, nsolve, tag=None):
    a = np.full(n * n, float(rid if tag is None else tag))
    return serving.SystemRequest(rid, t, n, n, a, np.zeros(3 * n * n), np.zeros(n * n), nsolve, 0.0, 0, "x")


def _stream(spec, seed=0):
    """spec: list of (arrival, n, solve arrivals) -> events."""
    rng = np.random.default_rng(seed)
    ev, rid = [], 0
    for t, n, solves in spec:
        sid = rid
        ev.append((t, _system(sid, t, n, len(solves))))
        rid += 1
        for ts in solves:
            ev.append((ts, serving.SolveRequest(rid, sid, ts, rng.uniform(-1, 1, n * n))))
            rid += 1
    return ev


def test_all_served_and_results_routed():
    lib = FakeLib()
    ev = _stream([(0.0, 8, [0.001, 0.002, 0.06]), (0.01, 16, [0.02]), (0.03, 8, [0.031, 0.032])])
    srv = serving.Server(1 << 40, slots=4, lib=lib, new_stream=FakeStream, keep_results=True)
    recs, wall = srv.run(ev)
    assert all(r.ok for r in recs.values())
    for _, r in ev:
        if isinstance(r, serving.SolveRequest):
            np.testing.assert_array_equal(srv.results[r.rid], 2.0 * r.rhs)
    assert sorted(lib.freed) == [0, 4, 6]
    assert srv.reserved == 0 and not srv.handles


def test_continuous_admission_overlaps():
    # system 1 arrives while system 0 factors: it starts before 0 finishes
    lib = FakeLib(tf=0.3)
    ev = _stream([(0.0, 8, [0.35]), (0.02, 8, [0.36])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream, solve_slots=0)
    recs, _ = srv.run(ev)
    assert recs[2].start < recs[0].done
    assert lib.max_live == 2 and srv.peak_active == 2


def test_solve_slot_kept_free_of_factorizations():
    # system 0 is resident at 0.3; systems 1 and 2 queue at 0.31 / 0.32 and
    # its solve arrives at 0.35.  With one of two slots kept for solves, system
    # 1 factors alone, system 2 waits, and the solve starts at once instead of
    # waiting for a factorization to end.
    lib = FakeLib(tf=0.3, ts=0.01)
    ev = _stream([(0.0, 8, [0.35]), (0.31, 8, [0.9]), (0.32, 8, [0.95])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream)
    recs, _ = srv.run(ev)
    solve0, fac1, fac2 = recs[1], recs[2], recs[4]
    assert solve0.start < fac1.done and solve0.start - solve0.arrival < 0.1
    assert fac2.start >= fac1.done  # never two factorizations at once
    assert all(r.ok for r in recs.values())


def test_solves_coalesced_while_factoring():
    lib = FakeLib(tf=0.2)
    ev = _stream([(0.0, 8, [0.01 + 0.01 * i for i in range(10)])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream, max_batch=64)
    recs, _ = srv.run(ev)
    assert lib.solve_calls[0] == (0, 10)
    assert all(r.batch == 10 for r in recs.values() if r.kind == "solve")


def test_max_batch_splits():
    lib = FakeLib(tf=0.2)
    ev = _stream([(0.0, 8, [0.01 + 0.001 * i for i in range(10)])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream, max_batch=4)
    srv.run(ev)
    assert [c[1] for c in lib.solve_calls] == [4, 4, 2]


def test_budget_bounds_reservation():
    lib = FakeLib(tf=0.05)
    reqs = [_system(0, 0, 16, 0)]
    one = serving.peak_bytes(reqs[0], acr.ACR_FP32TC_IR)
    ev = _stream([(0.001 * i, 16, []) for i in range(6)])
    budget = 2 * one + one // 2   # room for two factorizations in flight
    srv = serving.Server(budget, slots=6, lib=lib, new_stream=FakeStream)
    recs, _ = srv.run(ev)
    assert all(r.ok for r in recs.values())
    assert srv.peak_reserved <= budget
    assert lib.max_live <= 2


def test_oversized_request_still_admitted_alone():
    lib = FakeLib(tf=0.02)
    ev = _stream([(0.0, 16, [0.001])])
    srv = serving.Server(1, slots=2, lib=lib, new_stream=FakeStream)
    recs, _ = srv.run(ev)
    assert all(r.ok for r in recs.values())


def test_failed_factor_fails_its_solves_only():
    lib = FakeLib(tf=0.05, fail={12})
    ev = _stream([(0.0, 12, [0.001, 0.2]), (0.0, 8, [0.01])])
    srv = serving.Server(1 << 40, slots=4, lib=lib, new_stream=FakeStream)
    recs, _ = srv.run(ev)
    assert [recs[i].ok for i in range(3)] == [False, False, False]
    assert recs[3].ok and recs[4].ok
    assert len(srv.errors) == 1 and "planted" in srv.errors[0][1]


class RaisingLib(FakeLib):
    """FakeLib whose factor of block count `bad_factor`, statistics of
    `bad_stats` and solve of `bad_solve` raise errors that are not the
    library's own."""

    def __init__(self, bad_factor, bad_stats, bad_solve, **kw):
        super().__init__(**kw)
        self.bad_factor, self.bad_stats, self.bad_solve = bad_factor, bad_stats, bad_solve

    def acr_factor_ex(self, nblk, blksz, a, D3, c, tol, o):
        if nblk == self.bad_factor:
            raise MemoryError("planted host failure")
        return super().acr_factor_ex(nblk, blksz, a, D3, c, tol, o)

    def acr_stats(self, h):
        if h["n"] == self.bad_stats:
            raise RuntimeError("planted stats failure")
        return super().acr_stats(h)

    def acr_solve_ex(self, h, B, nrhs):
        if h["n"] == self.bad_solve:
            raise ValueError("planted solve failure")
        return super().acr_solve_ex(h, B, nrhs)


def test_unexpected_exceptions_fail_requests_not_the_loop():
    lib = RaisingLib(bad_factor=12, bad_stats=10, bad_solve=8, tf=0.02, ts=0.005)
    ev = _stream([(0.0, 12, [0.001]), (0.0, 10, [0.002]), (0.0, 8, [0.003, 0.004]), (0.0, 6, [0.005])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream)
    done = []
    th = threading.Thread(target=lambda: done.append(srv.run(ev)), daemon=True)
    th.start()
    th.join(timeout=20)
    assert done, "serving loop did not finish"
    recs, _ = done[0]
    # system 0: factor raises; system 2: statistics raise; system 4: its
    # solves raise (its factor is fine); system 7 is untouched
    assert not any(recs[i].ok for i in (0, 1, 2, 3, 5, 6))
    assert recs[4].ok and recs[7].ok and recs[8].ok
    # the handle whose statistics failed was freed; nothing stays reserved
    assert 2 in lib.freed
    assert srv.reserved == 0 and srv.active == 0 and srv.solving == 0
    assert len(srv.errors) == 3


def test_summary():
    lib = FakeLib(tf=0.01, ts=0.005)
    ev = _stream([(0.0, 8, [0.001 * i for i in range(1, 6)])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream)
    recs, wall = srv.run(ev)
    s = serving.summarize(recs, wall)
    assert s["solve"]["count"] == 5 and s["factor"]["count"] == 1
    assert s["solve"]["p50_ms"] <= s["solve"]["p99_ms"]
    assert s["failed"] == 0 and s["solves_per_s"] > 0


def test_summary_splits_solves_by_residency():
    """Solves that arrive after their system's factorization has finished are
    reported apart from those that also wait for it."""
    lib = FakeLib(tf=0.05, ts=0.002)
    # two solves arrive during the 50 ms factorization, two well after it
    ev = _stream([(0.0, 8, [0.001, 0.002, 0.2, 0.21])])
    srv = serving.Server(1 << 40, slots=2, lib=lib, new_stream=FakeStream)
    recs, wall = srv.run(ev)
    s = serving.summarize(recs, wall)
    assert s["solve_before_factor_done"]["count"] == 2 and s["solve_resident"]["count"] == 2
    assert s["solve_resident"]["p99_ms"] < 40 < s["solve_before_factor_done"]["p50_ms"]


def test_request_stream_seeded():
    e1 = serving.make_requests(30, rate=100.0, seed=3, sizes=(8, 16), probs=(0.5, 0.5), max_solves=5)
    e2 = serving.make_requests(30, rate=100.0, seed=3, sizes=(8, 16), probs=(0.5, 0.5), max_solves=5)
    assert len(e1) == 30 and [t for t, _ in e1] == [t for t, _ in e2]
    times = [t for t, _ in e1]
    assert times == sorted(times)
    nsys = [r for _, r in e1 if isinstance(r, serving.SystemRequest)]
    for s in nsys:
        solves = [r for _, r in e1 if isinstance(r, serving.SolveRequest) and r.sys_rid == s.rid]
        assert len(solves) == s.nsolve >= 1
        assert s.leaf == 32 and s.tol == 1e-6


def test_capacity_sweep_rescales_arrivals():
    ev = serving.make_requests(24, rate=100.0, seed=1, sizes=(8,), probs=(1.0,), max_solves=4)
    seen = []

    def fake_serve(events, rate):
        seen.append((rate, [t for t, _ in events]))
        return {"wall_s": 2.0 if rate == float("inf") else 1.0}

    cap, res = serving.capacity_sweep(ev, 100.0, (0.5, 1.0), fake_serve)
    assert cap == pytest.approx(len(ev) / 2.0)
    assert seen[0][1] == [0.0] * len(ev)                       # the burst
    t0 = [t for t, _ in ev]
    for (rate, ts), f in zip(seen[1:], (0.5, 1.0)):
        assert rate == pytest.approx(f * cap)
        assert ts == pytest.approx([t * 100.0 / (f * cap) for t in t0])
    assert [r["capacity_fraction"] for r in res] == [0.5, 1.0]


def test_solve_workspace_counts_against_budget():
    # room for the factorization, then for the resident factor (1 MB in the
    # fake) plus the workspace of 4 right-hand sides -- not of 16
    lib = FakeLib(tf=0.05, ts=0.01)
    n = 64
    req = _system(0, 0.0, n, 0)
    fac = serving.peak_bytes(req, acr.ACR_FP32TC_IR)
    four = serving.solve_bytes(n, n, 4, acr.ACR_FP32TC_IR, 60)
    assert serving.solve_bytes(n, n, 8, acr.ACR_FP32TC_IR, 60) > four
    budget = max(fac, lib.held + four)
    ev = _stream([(0.0, n, [0.001 * (i + 1) for i in range(16)])])
    srv = serving.Server(budget, slots=2, lib=lib, new_stream=FakeStream, max_batch=64)
    recs, _ = srv.run(ev)
    assert all(r.ok for r in recs.values())
    assert sum(c[1] for c in lib.solve_calls) == 16
    assert max(c[1] for c in lib.solve_calls) < 16      # batches were cut to fit
    assert srv.peak_reserved <= budget
    assert srv.reserved == 0
