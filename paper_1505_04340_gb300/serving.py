"""Continuous-batching solve server over resident SLR preconditioners.

Requests (a matrix id and 1..nrhs_max right-hand sides) arrive over time.  The
server keeps one SLR handle per matrix resident on the device: it is set up on
the first request for that matrix, admitted only while free device memory (and
the server's own capacity, if one is given) covers it, and least recently used
idle handles are evicted to make room.  Every pending request of a matrix is
packed into the columns of one multi-RHS SLR-PCG solve; solves of different
matrices run at the same time, each on its own CUDA stream in its own worker
thread (the library releases the interpreter lock while it runs).  A request
that arrives while its matrix is being solved joins the next batch of that
matrix as soon as the running solve returns; one that arrives for an idle
matrix starts as soon as a worker slot is free.

Each column of a multi-RHS solve is an independent CG run with its own scalars,
convergence mask and fixed-order reductions, so a request's answer does not
depend on what it was batched or overlapped with.

The solver is the C library (``slr.SLR``); this module only schedules.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass

import numpy as np

from .slr import SLR, SLRError


@dataclass
class MatrixSpec:
    """A matrix the server may be asked to solve with (CSR, partition, rank)."""
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    part: np.ndarray
    nparts: int
    k: int
    lanczos_steps: int = 0

    @property
    def n(self):
        return len(self.rowptr) - 1


@dataclass
class Request:
    rid: int
    matrix: object                 # key into the server's matrix table
    b: np.ndarray                  # (n,) or (n, r) float64, original order
    arrival: float                 # seconds after the start of the run
    x: np.ndarray | None = None
    iterations: np.ndarray | None = None
    relres: np.ndarray | None = None
    status: int = -1               # slr_status of the solve, -1 = not served
    error: str = ""
    start: float = 0.0             # when its solve began
    done: float = 0.0              # when its solution was back on the host
    batch: int = 0                 # columns in the solve it was part of
    cold: bool = False             # its matrix was set up for it

    @property
    def ncols(self):
        return 1 if self.b.ndim == 1 else self.b.shape[1]

    @property
    def latency(self):
        return self.done - self.arrival


class _Slot:
    """A resident handle and its stream."""

    def __init__(self, handle, stream, footprint):
        self.handle = handle
        self.stream = stream
        self.footprint = int(footprint)
        self.last_used = time.perf_counter()


class CudaBackend:
    """Handles of the SLR library on the current GPU, one CUDA stream each."""

    def __init__(self, precision="mixed", nrhs_max=8, setup_kw=None):
        import torch
        self.torch = torch
        self.precision, self.nrhs_max = precision, int(nrhs_max)
        self.setup_kw = dict(setup_kw or {})

    def free_bytes(self):
        return self.torch.cuda.mem_get_info()[0]

    def setup(self, spec):
        stream = self.torch.cuda.Stream()
        h = SLR(spec.rowptr, spec.colind, spec.val, spec.part, spec.nparts, k=spec.k,
                lanczos_steps=spec.lanczos_steps, precision=self.precision, nrhs_max=self.nrhs_max,
                flexible_cg=(self.precision == "mixed"), stream=stream, **self.setup_kw)
        stream.synchronize()
        return _Slot(h, stream, h.info["device_bytes"])

    def solve(self, slot, B, tol, maxit):
        """B: (n, r) float64 host array -> (X host array, iterations, relres, status)."""
        torch = self.torch
        with torch.cuda.stream(slot.stream):
            bd = torch.from_numpy(B).pin_memory().to("cuda", non_blocking=True)
            x, its, rel, st = slot.handle.pcg(bd, tol=tol, maxit=maxit, stream=slot.stream, check=False)
            xh = x.cpu().numpy()                   # waits for this stream only
        return xh, its, rel, st

    def release(self, slot):
        slot.handle.close()


class SolveServer:
    """Schedules SLR-PCG solves of a request stream on the current GPU.

    matrices: key -> MatrixSpec.
    precision, nrhs_max, tol, maxit: for every handle and solve ("mixed" uses
        flexible CG around the FP32 apply).
    backend: what sets up handles and runs solves (default: CudaBackend).
    max_concurrent: solves (worker threads, streams) in flight at once.
    reserve_bytes: device memory left free when a new handle is admitted.
    capacity_bytes: device memory all resident handles may hold (None: no cap
        beyond free memory).
    log: a text stream that receives one line per failed setup or solve.
    """

    def __init__(self, matrices: dict, precision="mixed", nrhs_max=8, tol=1e-8, maxit=300,
                 max_concurrent=4, reserve_bytes=1 << 30, capacity_bytes=None, setup_kw=None, backend=None,
                 log=None):
        self.backend = backend or CudaBackend(precision, nrhs_max, setup_kw)
        self.matrices = matrices
        self.precision = precision
        self.nrhs_max = int(nrhs_max)
        self.tol, self.maxit = float(tol), int(maxit)
        self.max_concurrent = int(max_concurrent)
        self.reserve = int(reserve_bytes)
        self.capacity = capacity_bytes
        self.log = log
        self.errors: list = []           # (seconds, key, message)
        self.slots: dict = {}            # key -> _Slot (resident handles)
        self.footprints: dict = {}       # key -> device bytes seen at its last setup
        self.claimed: dict = {}          # key -> bytes admitted for a setup in progress
        self.cv = threading.Condition()
        self.setups = 0
        self.evictions = 0
        self.batches = 0
        self.max_inflight = 0

    # ------------------------------------------------------------ residency
    def _need(self, key):
        if key in self.footprints:
            return self.footprints[key]
        spec = self.matrices[key]
        nnz = int(spec.rowptr[-1])
        # factors and workspaces grow with n, nnz and the RHS block; the first
        # setup of a matrix records its real figure
        return int(spec.n * (400 + 64 * self.nrhs_max) + 24 * nnz + (64 << 20))

    def _resident_bytes(self):
        return sum(s.footprint for s in self.slots.values()) + sum(self.claimed.values())

    def _admit(self, key):
        """Make room for `key` (called with the lock held; False: wait for a running solve)."""
        need = self._need(key)
        while True:
            ok = self.backend.free_bytes() - sum(self.claimed.values()) - need >= self.reserve
            if self.capacity is not None:
                ok = ok and self._resident_bytes() + need <= self.capacity
            if ok:
                self.claimed[key] = need
                return True
            idle = [(s.last_used, k) for k, s in self.slots.items() if k not in self.busy and not self.pending.get(k)]
            if not idle:
                idle = [(s.last_used, k) for k, s in self.slots.items() if k not in self.busy]
            if not idle:
                if self.busy - {key}:
                    return False                   # a running solve may free memory: wait
                self.claimed[key] = need           # nothing could free memory: try anyway
                return True
            _, victim = min(idle, key=lambda t: t[0])
            self.backend.release(self.slots.pop(victim))
            self.evictions += 1

    # ------------------------------------------------------------ solving
    def _solve(self, key, slot, reqs, cold):
        n = self.matrices[key].n
        B = np.ascontiguousarray(np.concatenate([r.b.reshape(n, -1) for r in reqs], axis=1))
        start = time.perf_counter() - self.t0
        xh, its, rel, st = self.backend.solve(slot, B, self.tol, self.maxit)
        done = time.perf_counter() - self.t0
        c = 0
        for r in reqs:
            w = r.ncols
            r.x = xh[:, c:c + w].reshape(r.b.shape).copy()
            r.iterations, r.relres = its[c:c + w].copy(), rel[c:c + w].copy()
            # the library's status covers the whole block: a request whose own
            # columns all met the tolerance has converged
            r.status = 0 if st == 0 or bool(np.all(r.relres <= self.tol)) else int(st)
            r.start, r.done, r.batch, r.cold = start, done, B.shape[1], cold
            c += w

    def _take_batch(self, key):
        q = self.pending.get(key)
        batch, cols = [], 0
        while q and (not batch or cols + q[0].ncols <= self.nrhs_max):
            r = q.popleft()
            batch.append(r)
            cols += r.ncols
        return batch

    def _worker(self, key):
        cold = False
        batch = []
        try:
            with self.cv:
                slot = self.slots.get(key)
                while slot is None and not self._admit(key):
                    self.cv.wait(0.05)
            if slot is None:
                try:
                    slot = self.backend.setup(self.matrices[key])
                finally:
                    with self.cv:
                        self.claimed.pop(key, None)
                cold = True
                with self.cv:
                    self.slots[key] = slot
                    self.footprints[key] = slot.footprint
                    self.setups += 1
            while True:
                with self.cv:
                    batch = self._take_batch(key)
                    if not batch:
                        break
                    self.batches += 1
                self._solve(key, slot, batch, cold)
                cold = False
                slot.last_used = time.perf_counter()
        except (SLRError, RuntimeError) as e:            # this matrix's requests fail, the server goes on
            t = time.perf_counter() - self.t0
            with self.cv:
                self.errors.append((t, key, f"{type(e).__name__}: {e}"))
                if self.log is not None:
                    print(f"[serving] {t:.3f}s matrix {key}: {type(e).__name__}: {e}", file=self.log, flush=True)
                for r in batch + list(self.pending.pop(key, deque())):
                    if r.status == -1:
                        r.status = e.status if isinstance(e, SLRError) else 4
                        r.error, r.done = str(e), time.perf_counter() - self.t0
        finally:
            with self.cv:
                self.busy.discard(key)
                self.cv.notify_all()

    # ------------------------------------------------------------ the loop
    def run(self, requests: list, realtime=True):
        """Serve `requests` and return them, completed.

        realtime: release each request at its arrival time; otherwise all are
        released at once (their latencies then count from their arrival times
        all the same, for a backlog)."""
        self.t0 = time.perf_counter()
        for r in requests:
            if r.matrix not in self.matrices or r.ncols > self.nrhs_max or r.b.shape[0] != self.matrices[r.matrix].n:
                r.status, r.error = 1, "unknown matrix, wrong length or more columns than nrhs_max"
        arrivals = deque(sorted((r for r in requests if r.status == -1), key=lambda r: r.arrival))
        self.pending: dict = {}
        self.busy: set = set()
        threads = []
        with self.cv:
            while True:
                now = time.perf_counter() - self.t0
                while arrivals and (not realtime or arrivals[0].arrival <= now):
                    r = arrivals.popleft()
                    self.pending.setdefault(r.matrix, deque()).append(r)
                # oldest waiting request first, one worker per matrix
                ready = sorted(((q[0].arrival, k) for k, q in self.pending.items() if q and k not in self.busy),
                               key=lambda t: t[0])
                for _, key in ready:
                    if len(self.busy) >= self.max_concurrent:
                        break
                    self.busy.add(key)
                    th = threading.Thread(target=self._worker, args=(key,), daemon=True)
                    th.start()
                    threads.append(th)
                self.max_inflight = max(self.max_inflight, len(self.busy))
                if not arrivals and not self.busy and not any(self.pending.values()):
                    break
                wait = None if not arrivals else max(arrivals[0].arrival - now, 0.0)
                self.cv.wait(wait if wait is not None else 0.5)
        for th in threads:
            th.join()
        return requests

    def close(self):
        for s in self.slots.values():
            self.backend.release(s)
        self.slots.clear()


def latency_stats(reqs):
    """Latency percentiles (all requests, and those whose matrix was already
    resident), queueing and service time, CG iterations and throughput."""
    served = [r for r in reqs if r.status in (0, 5)]
    ms = lambda v: np.array(v, dtype=np.float64) * 1e3
    lat = ms([r.latency for r in served])
    warm = ms([r.latency for r in served if not r.cold])
    queue = ms([r.start - r.arrival for r in served])
    service = ms([r.done - r.start for r in served])
    its = np.concatenate([np.atleast_1d(r.iterations) for r in served]) if served else np.zeros(0)
    span = max(r.done for r in served) - min(r.arrival for r in served)
    cols = sum(r.ncols for r in served)
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    return {"requests": len(reqs), "served": len(served), "solves": cols,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "warm_p50_ms": pct(warm, 50), "warm_p99_ms": pct(warm, 99),
            "queue_p50_ms": pct(queue, 50), "service_p50_ms": pct(service, 50), "service_p99_ms": pct(service, 99),
            "iterations_mean": float(its.mean()) if len(its) else None, "iterations_max": int(its.max()) if len(its) else None,
            "solves_per_s": cols / span, "requests_per_s": len(served) / span, "span_s": span}
