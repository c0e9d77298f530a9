"""Continuous-batching serving loop over the C ABI.

Requests arrive as a Poisson stream.  A *system* request brings a block
tridiagonal operator (banded 5-point form) and asks for its factorization;
it is followed by solve requests (one right-hand side each) against that
factorization.  The loop

* admits a system when a worker slot is free and the device-memory budget
  has room for the factorization's peak working set (a bound computed from
  ``acr_factor_bytes``); the reservation shrinks to the bytes the handle
  keeps once the factorization returns (the compressed size when tol > 0).
  Every solve call reserves its workspace (``acr_solve_bytes``) while it
  runs.  Requests that arrive while others run are admitted as slots and
  memory free up -- nothing waits for the current batch to drain;
* runs each admitted piece of work in its own host thread (the C calls drop
  the Python lock) on the stream of its system, every resident system having
  a stream of its own, so factorizations and solves of different systems
  overlap on the device;
* keeps each factorization resident until its last solve has been served and
  coalesces the solve requests queued for one factorization into a single
  multi-right-hand-side ``acr_solve_ex`` call (at most ``max_batch``);
* records per-request latency (arrival to completion) and reports p50 / p99
  per request kind and solves per second.

A request's result does not depend on what it is batched or overlapped
with: the library computes each right-hand-side column with the same
per-column arithmetic whatever the call's column count, and freezes a column
once its residual has converged, so a solve in the mix returns what the same
solve returns alone.
"""

from __future__ import annotations

import collections
import ctypes
import dataclasses
import heapq
import threading
import time

import numpy as np

from . import _lib as acr


@dataclasses.dataclass
class SystemRequest:
    """A factorization request: banded operator arrays in the C-ABI layout
    (``a``, ``c``: nblk*blksz diagonals; ``D3``: [sub, diag, super] per
    block), the compression tolerance and HODLR leaf for this system."""
    rid: int
    arrival: float
    nblk: int
    blksz: int
    a: np.ndarray
    D3: np.ndarray
    c: np.ndarray
    nsolve: int           # solve requests that follow
    tol: float = 0.0
    leaf: int = 0
    kind: str = ""


@dataclasses.dataclass
class SolveRequest:
    rid: int
    sys_rid: int
    arrival: float
    rhs: np.ndarray       # (N,) float64


@dataclasses.dataclass
class Record:
    rid: int
    kind: str             # "factor" | "solve"
    arrival: float
    size: int = 0         # grid n of the system
    start: float = 0.0
    done: float = 0.0
    ok: bool = True
    resid: float = 0.0
    iters: int = 0
    batch: int = 1
    sys_rid: int = -1     # a solve's system


def peak_bytes(req: SystemRequest, precision: int) -> int:
    """Upper bound on the device bytes a factorization holds while it runs:
    the dense level arena and operator copy (``acr_factor_bytes``), the staged
    host input, the ping-pong level temporaries (at most half the arena) and,
    with compression, the sketch panels of every tree level (two
    b x k panels per block per level, k = 32) and the node pool (at most the
    arena)."""
    o = acr.acr_default_opts()
    o.precision = precision
    o.input_kind = acr.ACR_BANDED
    fb = acr.acr_factor_bytes(req.nblk, req.blksz, 0.0, o)
    N = req.nblk * req.blksz
    est = fb + fb // 2 + 5 * N * 8
    if req.tol > 0:
        b = req.blksz
        leaf = max(req.leaf, 1)
        L = 0
        while (b >> (L + 1)) >= leaf and (b >> L) % 2 == 0:
            L += 1
        est += fb * 2 * L * 32 // b + fb
    return int(est)


def solve_bytes(nblk: int, blksz: int, nrhs: int, precision: int, ir_max_iter: int) -> int:
    """Upper bound of one solve call's device workspace (acr_solve_bytes)."""
    o = acr.acr_default_opts()
    o.precision = precision
    o.input_kind = acr.ACR_BANDED
    o.ir_max_iter = ir_max_iter
    return acr.acr_solve_bytes(nblk, blksz, nrhs, o)


class Server:
    """Admission by memory budget, resident factorizations, solve batching."""

    def __init__(self, budget_bytes: int, slots: int = 4, precision: int = acr.ACR_FP32TC_IR,
                 ir_tol: float = 1e-8, ir_max_iter: int = 60, max_batch: int = 64,
                 keep_results: bool = False, lib=None, new_stream=None, solve_slots: int = 1):
        # `lib` and `new_stream` replace the CUDA library and torch's stream
        # constructor (host-side tests of the scheduling)
        self.lib = lib if lib is not None else acr
        if new_stream is None:
            import torch
            new_stream = torch.cuda.Stream
            self._sync = torch.cuda.synchronize
        else:
            self._sync = lambda: None
        self.new_stream = new_stream
        self.budget = int(budget_bytes)
        self.slots = slots
        # slots factorizations may not take: solves on resident systems never
        # wait behind a full set of factorizations (with one slot, none is kept)
        self.solve_slots = min(max(0, solve_slots), max(0, slots - 1))
        self.factoring = 0
        self.precision = precision
        self.ir_tol = ir_tol
        self.ir_max_iter = ir_max_iter
        self.max_batch = max_batch
        self.keep_results = keep_results
        self.cv = threading.Condition(threading.Lock())
        self.reserved = 0
        self.peak_reserved = 0
        self.active = 0
        self.peak_active = 0
        self.handles = {}            # sys rid -> (handle, bytes held, stream)
        self.dims = {}               # sys rid -> (nblk, blksz)
        self.solving = 0             # solve calls in flight
        self.pending = collections.defaultdict(collections.deque)
        self.remaining = {}          # sys rid -> solves still to serve
        self.busy = set()            # systems with a solve batch in flight
        self.sys_queue = collections.deque()
        self.records = {}
        self.results = {}
        self.errors = []
        self.stream_pool = []

    # ---------------------------------------------------------------- helpers
    def _stream(self):
        return self.stream_pool.pop() if self.stream_pool else self.new_stream()

    def _opts(self, req: SystemRequest, stream):
        o = self.lib.acr_default_opts()
        o.precision = self.precision
        o.input_kind = acr.ACR_BANDED
        o.ir_tol = self.ir_tol
        o.ir_max_iter = self.ir_max_iter
        o.leaf = req.leaf
        o.stream = ctypes.c_void_p(stream.cuda_stream)
        return o

    def _release(self, sys_rid):
        h, held, stream = self.handles.pop(sys_rid)
        self.lib.acr_free(h)
        self.reserved -= held
        self.stream_pool.append(stream)

    def _finish(self):
        self.active -= 1
        self.cv.notify_all()

    # ---------------------------------------------------------------- work
    def _run_factor(self, req: SystemRequest, est: int, stream):
        rec = self.records[req.rid]
        rec.start = time.perf_counter()
        h, held = None, 0
        try:
            h = self.lib.acr_factor_ex(req.nblk, req.blksz, req.a, req.D3, req.c, req.tol, self._opts(req, stream))
            st = self.lib.acr_stats(h)
            held = int(st["factor_bytes"] + st["operator_bytes"])
        except Exception as e:  # any failure fails the request; the loop's bookkeeping still runs
            if h is not None:
                self.lib.acr_free(h)
                h = None
            rec.ok = False
            self.errors.append((req.rid, str(e)))
        rec.done = time.perf_counter()
        with self.cv:
            self.factoring -= 1
            self.reserved -= est
            if h is not None:
                self.reserved += held
                self.handles[req.rid] = (h, held, stream)
                if self.remaining.get(req.rid, 0) == 0:
                    self._release(req.rid)
            else:
                self.stream_pool.append(stream)
                self._drop_solves(req.rid)
            self._finish()

    def _drop_solves(self, sys_rid):
        """A failed factorization fails its solves (called with the lock)."""
        self.remaining[sys_rid] = -1
        for r in self.pending.pop(sys_rid, ()):
            rec = self.records[r.rid]
            rec.ok, rec.done = False, time.perf_counter()

    def _run_solves(self, sys_rid: int, batch: list, ws: int):
        t0 = time.perf_counter()
        ok, B, res, it = True, None, None, 0
        try:
            h = self.handles[sys_rid][0]
            B = np.asfortranarray(np.stack([r.rhs for r in batch], axis=1))
            res, it = self.lib.acr_solve_ex(h, B, B.shape[1])
        except Exception as e:  # any failure fails the batch; the loop's bookkeeping still runs
            ok = False
            res = getattr(e, "resid", None)
            it = getattr(e, "iters", 0)
            self.errors.append((sys_rid, str(e)))
        if res is None or len(res) < len(batch):
            res = np.full(len(batch), np.nan)
        t1 = time.perf_counter()
        for q, r in enumerate(batch):
            rec = self.records[r.rid]
            rec.start, rec.done, rec.ok = t0, t1, ok
            rec.resid, rec.iters, rec.batch = float(res[q]), it, len(batch)
            if self.keep_results and B is not None:
                self.results[r.rid] = B[:, q].copy()
        with self.cv:
            self.busy.discard(sys_rid)
            self.reserved -= ws
            self.solving -= 1
            self.remaining[sys_rid] -= len(batch)
            if self.remaining[sys_rid] == 0:
                self._release(sys_rid)
            self._finish()

    # ---------------------------------------------------------------- loop
    def _dispatch(self):
        """Start whatever can start now (called with the lock held)."""
        started = []
        # solve batches first: finishing a system frees its memory.  A batch
        # reserves its workspace; it is halved until that fits the budget, and
        # runs over budget only when no other solve is in flight (resident
        # factorizations free their memory only after their solves)
        for sys_rid, q in list(self.pending.items()):
            if self.active >= self.slots:
                break
            if q and sys_rid in self.handles and sys_rid not in self.busy:
                nblk, blksz = self.dims[sys_rid]
                nb = min(len(q), self.max_batch)
                ws = solve_bytes(nblk, blksz, nb, self.precision, self.ir_max_iter)
                while nb > 1 and self.reserved + ws > self.budget:
                    nb = (nb + 1) // 2
                    ws = solve_bytes(nblk, blksz, nb, self.precision, self.ir_max_iter)
                if self.reserved + ws > self.budget and self.solving > 0:
                    continue
                batch = [q.popleft() for _ in range(nb)]
                self.busy.add(sys_rid)
                self.active += 1
                self.solving += 1
                self.reserved += ws
                self.peak_reserved = max(self.peak_reserved, self.reserved)
                self.peak_active = max(self.peak_active, self.active)
                started.append(threading.Thread(target=self._run_solves, args=(sys_rid, batch, ws)))
        while self.sys_queue and self.active < self.slots and self.factoring < self.slots - self.solve_slots:
            req = self.sys_queue[0]
            est = peak_bytes(req, self.precision)
            if self.reserved + est > self.budget and self.reserved > 0:
                break  # wait until memory is released (admission stays in arrival order)
            self.sys_queue.popleft()
            self.dims[req.rid] = (req.nblk, req.blksz)
            self.reserved += est
            self.peak_reserved = max(self.peak_reserved, self.reserved)
            self.active += 1
            self.factoring += 1
            self.peak_active = max(self.peak_active, self.active)
            started.append(threading.Thread(target=self._run_factor, args=(req, est, self._stream())))
        for t in started:
            t.start()
        return started

    def run(self, events):
        """Serve a list of (arrival seconds, request) in real time; returns
        (records, wall seconds)."""
        self._sync()
        heap = [(ev[0], i, ev[1]) for i, ev in enumerate(events)]
        heapq.heapify(heap)
        for _, _, r in heap:
            if isinstance(r, SystemRequest):
                self.remaining[r.rid] = r.nsolve
        threads = []
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            with self.cv:
                while heap and heap[0][0] <= now:
                    _, _, r = heapq.heappop(heap)
                    if isinstance(r, SystemRequest):
                        self.records[r.rid] = Record(r.rid, "factor", t0 + r.arrival, r.nblk)
                        self.sys_queue.append(r)
                    else:
                        self.records[r.rid] = Record(r.rid, "solve", t0 + r.arrival, sys_rid=r.sys_rid)
                        if self.remaining.get(r.sys_rid, 0) < 0:
                            self.records[r.rid].ok = False
                            self.records[r.rid].done = time.perf_counter()
                        else:
                            self.pending[r.sys_rid].append(r)
                threads += self._dispatch()
                if not heap and not self.sys_queue and self.active == 0 and not any(self.pending.values()):
                    break
                wait = (heap[0][0] - now) if heap else 0.05
                self.cv.wait(timeout=max(0.0002, min(wait, 0.05)))
        wall = time.perf_counter() - t0
        for t in threads:
            t.join()
        with self.cv:
            for rid in list(self.handles):
                self._release(rid)
        return self.records, wall


def summarize(records, wall: float) -> dict:
    """p50 / p99 / mean latency (ms) per request kind, solves per second over
    the wall time, failures and the mean solve batch."""
    out = {}
    for kind in ("factor", "solve"):
        lat = np.array([(r.done - r.arrival) * 1e3 for r in records.values() if r.kind == kind and r.ok])
        if lat.size:
            out[kind] = {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}
    # solves whose system was already factored when they arrived (resident):
    # their latency is the solve's own wait and run, while the others also
    # wait for their system's factorization
    def fdone(r):
        f = records.get(r.sys_rid)
        return f.done if f is not None and f.kind == "factor" and f.ok else float("inf")
    for name, sel in (("solve_resident", lambda r: fdone(r) <= r.arrival),
                      ("solve_before_factor_done", lambda r: fdone(r) > r.arrival)):
        lat = np.array([(r.done - r.arrival) * 1e3 for r in records.values()
                        if r.kind == "solve" and r.ok and sel(r)])
        if lat.size:
            out[name] = {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}
    nsolve = sum(1 for r in records.values() if r.kind == "solve" and r.ok)
    out["solves_per_s"] = nsolve / wall if wall > 0 else 0.0
    out["failed"] = sum(1 for r in records.values() if not r.ok)
    batches = [r.batch for r in records.values() if r.kind == "solve"]
    out["mean_solve_batch"] = float(np.mean(batches)) if batches else 0.0
    return out


def make_requests(nreq: int, rate: float, seed: int, sizes=(128, 256, 512, 1024), probs=(0.4, 0.3, 0.2, 0.1),
                  max_solves: int = 64, tol: float = 1e-6):
    """The seeded request mix: each system a variable-coefficient diffusion
    or a convection-diffusion operator (50/50, fields seeded per system) on an
    n x n grid, n drawn from ``sizes`` with ``probs``, HODLR leaf 32 up to
    n = 256 and 64 above, then 1..max_solves single right-hand sides
    uniform[-1, 1]; Poisson arrivals at ``rate`` requests per second, systems
    and solves counted alike.  Returns a time-ordered list of
    (arrival, request)."""
    import synthetic as syn
    rng = np.random.default_rng(seed)
    events = []
    t = 0.0
    rid = 0
    while rid < nreq:
        n = int(rng.choice(sizes, p=probs))
        kind = "diffusion" if rng.random() < 0.5 else "convdiff"
        fseed = int(rng.integers(1 << 30))
        P = syn.variable_diffusion(n, seed=fseed) if kind == "diffusion" else syn.convection_diffusion(n, seed=fseed)
        a, D3, c = P.banded_abi()
        ns = min(int(rng.integers(1, max_solves + 1)), max(1, nreq - rid - 1))
        t += rng.exponential(1.0 / rate)
        sys_rid = rid
        events.append((t, SystemRequest(sys_rid, t, n, n, a, D3, c, ns, tol, 32 if n <= 256 else 64, kind)))
        rid += 1
        for _ in range(ns):
            t += rng.exponential(1.0 / rate)
            events.append((t, SolveRequest(rid, sys_rid, t, rng.uniform(-1.0, 1.0, P.N))))
            rid += 1
    return events


def serve(nreq: int = 2000, rate: float = 100.0, seed: int = 42, budget_gb: float = 150.0, slots: int = 4,
          max_batch: int = 64, events=None) -> dict:
    """Serve the seeded mix at an offered `rate` (requests/s) and summarise."""
    ev = events if events is not None else make_requests(nreq, rate, seed)
    srv = Server(int(budget_gb * 1e9), slots=slots, max_batch=max_batch)
    recs, wall = srv.run(ev)
    out = summarize(recs, wall)
    out.update({"requests": len(ev), "offered_rate": rate, "wall_s": wall, "slots": slots,
                "budget_gb": budget_gb, "peak_reserved_gb": srv.peak_reserved / 1e9,
                "peak_active": srv.peak_active,
                "systems": sum(1 for _, r in ev if isinstance(r, SystemRequest)),
                "errors": srv.errors[:3]})
    return out


def capacity_sweep(events, rate: float, fractions=(0.5, 0.8, 1.0), serve_fn=None):
    """Capacity, then offered loads relative to it: the mix is served with
    every request arriving at t = 0 (capacity = requests / wall time), then
    with its arrival times rescaled to each fraction of that capacity.
    `events` were drawn at `rate` requests/s; `serve_fn(events, rate)` returns
    a summary with "wall_s" (serve() with the defaults).  Returns
    (capacity, [summary per fraction])."""
    serve_fn = serve_fn or (lambda ev, r: serve(rate=r, events=ev))
    burst = [(0.0, dataclasses.replace(r, arrival=0.0)) for _, r in events]
    first = serve_fn(burst, float("inf"))
    capacity = len(events) / first["wall_s"]
    out = []
    for f in fractions:
        sm = serve_fn(_rescale(events, rate, f * capacity), f * capacity)
        sm["capacity_fraction"] = f
        sm["capacity_rps"] = capacity
        out.append(sm)
    return capacity, out


def _rescale(events, rate_from: float, rate_to: float):
    """The same requests with arrival times scaled to another offered rate."""
    k = rate_from / rate_to
    out = []
    for t, r in events:
        r = dataclasses.replace(r, arrival=t * k)
        out.append((t * k, r))
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="serve the seeded diffusion / convection-diffusion mix")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rates", type=str, default="100", help="comma-separated offered rates, requests/s")
    ap.add_argument("--seed", type=int, default=42)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--capacity", type=str, default="",
                    help="comma-separated fractions of the measured capacity to offer instead of --rates")
    a = ap.parse_args()
    rates = [float(x) for x in a.rates.split(",")]
    base = make_requests(a.requests, rates[0], a.seed)
    if a.capacity:
        fr = [float(x) for x in a.capacity.split(",")]
        cap, res = capacity_sweep(base, rates[0], fr, lambda ev, r: serve(
            rate=r, budget_gb=a.budget_gb, slots=a.slots, max_batch=a.max_batch, events=ev))
        print(json.dumps({"capacity_requests_per_s": cap}), flush=True)
        for sm in res:
            print(json.dumps(sm), flush=True)
        raise SystemExit(0)
    for rate in rates:
        ev = base if rate == rates[0] else _rescale(base, rates[0], rate)
        print(json.dumps(serve(rate=rate, budget_gb=a.budget_gb, slots=a.slots, max_batch=a.max_batch, events=ev)),
              flush=True)
