"""Serving orchestration on top of the native request server (spx_server_*):
keeps request buffers alive, replays an arrival trace, and summarises
latency and throughput.  Scheduling, admission and the solves themselves run
in the C++/CUDA library."""
from __future__ import annotations

import time

import numpy as np

from . import spx


class Server:
    def __init__(self, ctx: int, budget_bytes: int = 0, max_slots: int = 8, batch_rows: int | None = None,
                 keep_x: bool = True):
        self.h = spx.spx_server_create(ctx, budget_bytes, max_slots)
        self.batch_rows = spx.spx_server_set_batching(self.h, batch_rows) if batch_rows is not None else None
        self.live = {}      # id -> (arrays kept alive, x)
        self.results = {}   # id -> result dict
        self.keep_x = keep_x  # False: drop each solution once its request completes (long traces)

    def submit(self, rp, col, val, b, solver="cg", tol=1e-8, max_iter=100000, precision="mixed") -> int:
        x = np.zeros(b.shape[0])
        rid = spx.spx_server_submit(self.h, rp, col, val, b, x, solver, tol, max_iter, 30, precision)
        self.live[rid] = (rp, col, val, b, x)
        return rid

    def submit_matrix(self, A: int, b, solver="cg", tol=1e-8, max_iter=100000, precision="mixed") -> int:
        """A request on a resident matrix handle (kept alive by the caller)."""
        x = np.zeros(b.shape[0])
        rid = spx.spx_server_submit_matrix(self.h, A, b, x, solver, tol, max_iter, 30, precision)
        self.live[rid] = (A, None, None, b, x)
        return rid

    def poll(self, wait_ms: int = 0) -> int:
        got = spx.spx_server_poll(self.h, 1024, wait_ms)
        for r in got:
            x = self.live.pop(r["id"])[4]
            if self.keep_x:
                r["x"] = x
            self.results[r["id"]] = r
        return len(got)

    def drain(self, timeout_s: float = 600.0):
        t = time.time()
        while self.live and time.time() - t < timeout_s:
            self.poll(wait_ms=50)
        if self.live:
            raise TimeoutError(f"{len(self.live)} requests did not complete")

    def close(self):
        if self.h:
            spx.spx_server_destroy(self.h)
            self.h = None


def poisson_trace(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return np.array(out)
        out.append(t)


def replay(server: Server, trace_s: np.ndarray, requests: list, solver_of, tol=1e-8, precision="mixed"):
    """Submit requests[i] at wall time trace_s[i] (relative to the start) while
    collecting completions; returns the wall time of the run."""
    t0 = time.perf_counter()
    ids = []
    for i, ta in enumerate(trace_s):
        while True:
            now = time.perf_counter() - t0
            if now >= ta:
                break
            server.poll(wait_ms=0)
            time.sleep(min(0.0005, ta - now))
        rp, col, val, b = requests[i]
        ids.append(server.submit(rp, col, val, b, solver=solver_of(i), tol=tol, precision=precision))
        server.poll(wait_ms=0)
    server.drain()
    return time.perf_counter() - t0, ids


def replay_lazy(server: Server, trace_s: np.ndarray, make, max_pending_bytes: float, tol=1e-8, precision="mixed"):
    """Open-loop replay whose request payloads are built on demand: request i
    is due at trace_s[i] (s after the start); make(i) returns (kind, payload,
    solver, nbytes) with kind "host" (payload = rp, col, val, b) or "handle"
    (payload = matrix handle, b).  A due request is submitted once the host
    bytes of the requests already submitted and not yet completed leave room
    for it (max_pending_bytes), so a backlogged server holds a bounded amount
    of host memory; its latency still counts from its due time.  While the
    server's queue is not empty that wait changes neither the order nor the
    moment of any admission.  Returns (wall time, ids, delays in ms)."""
    t0 = time.perf_counter()
    ids, delays = [], []
    pending = {}  # id -> bytes
    held = 0.0

    def collect(wait_ms=0):
        nonlocal held
        server.poll(wait_ms=wait_ms)
        for rid in [r for r in pending if r in server.results]:
            held -= pending.pop(rid)

    for i, ta in enumerate(trace_s):
        while True:
            now = time.perf_counter() - t0
            if now >= ta:
                break
            collect()
            time.sleep(min(0.0005, ta - now))
        kind, payload, solver, nbytes = make(i)
        while pending and held + nbytes > max_pending_bytes:
            collect(wait_ms=2)
        delays.append((time.perf_counter() - t0 - ta) * 1e3)
        if kind == "host":
            rp, col, val, b = payload
            rid = server.submit(rp, col, val, b, solver=solver, tol=tol, precision=precision)
        else:
            A, b = payload
            rid = server.submit_matrix(A, b, solver=solver, tol=tol, precision=precision)
        ids.append(rid)
        pending[rid] = nbytes
        held += nbytes
        collect()
    server.drain()
    return time.perf_counter() - t0, ids, delays


def latency_stats(results: list[dict], delays_ms=None) -> dict:
    """Latency from arrival to completion (plus each request's client-side
    delay before its submission, if given) and queue wait before admission."""
    d = np.zeros(len(results)) if delays_ms is None else np.asarray(delays_ms, dtype=np.float64)
    lat = np.array([r["done_ms"] - r["submit_ms"] for r in results]) + d
    wait = np.array([r["admit_ms"] - r["submit_ms"] for r in results]) + d
    return {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "queue_wait_p50_ms": float(np.percentile(wait, 50)),
            "queue_wait_p99_ms": float(np.percentile(wait, 99))}
