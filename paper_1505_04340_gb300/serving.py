"""Continuous-batching solve server over resident SLR preconditioners.

Requests (a matrix id and 1..nrhs_max right-hand sides) arrive over time.  The
server keeps one SLR handle per matrix resident on the device: it is set up on
the first request for that matrix, admitted only while free device memory (and
the server's own capacity, if one is given) covers it, and least recently used
idle handles are evicted to make room.

Batching is continuous at iteration granularity.  A handle's nrhs_max CG
columns are slots (``slr_cg_*``): a worker per active matrix starts the columns
of waiting requests in free slots, advances every occupied slot a few CG
iterations (``iters_per_step``), collects the columns that have converged,
frees their slots and starts waiting columns in them, and so on until the
matrix has no work.  A request that arrives while its matrix is being solved
therefore joins at the next iteration boundary, and a converged column's slot
is refilled without waiting for the rest of its batch.  Workers of different
matrices run at once, each on its own CUDA stream in its own thread (the
library releases the interpreter lock while it runs).

Each slot is an independent CG run with its own scalars, convergence mask and
fixed-order reductions, so a request's answer does not depend on what it ran
beside.

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
    start: float = 0.0             # when its first column started
    done: float = 0.0              # when its last column was back on the host
    batch: int = 0                 # slots occupied on its matrix when it started
    cold: bool = False             # its matrix was set up for it

    @property
    def ncols(self):
        return 1 if self.b.ndim == 1 else self.b.shape[1]

    @property
    def latency(self):
        return self.done - self.arrival


class Resident:
    """A resident handle and its stream."""

    def __init__(self, handle, stream, footprint):
        self.handle = handle
        self.stream = stream
        self.footprint = int(footprint)
        self.last_used = time.perf_counter()


class CudaBackend:
    """Handles of the SLR library on the current GPU, one CUDA stream each; the CG
    slots of a handle through slr_cg_slot_start / slr_cg_advance / slr_cg_slot_result."""

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
        return Resident(h, stream, h.info["device_bytes"])

    def start(self, res, slots, B, tol, maxit):
        """Start the columns B[:, i] (host, original order) in the given slots; returns
        the device copy, which the caller keeps until the next advance has run."""
        torch = self.torch
        with torch.cuda.stream(res.stream):
            bd = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory().to("cuda", non_blocking=True)
            for i, j in enumerate(slots):
                res.handle.cg_start(j, bd[i], tol=tol, maxit=maxit, stream=res.stream)
        return bd

    def advance(self, res, iters, width):
        """(active, iterations, relres, status) of slots 0 .. width-1 after `iters` iterations."""
        return res.handle.cg_advance(iters, width, stream=res.stream)

    def results(self, res, slots):
        """x of the given slots as an (n, len(slots)) host array."""
        torch = self.torch
        with torch.cuda.stream(res.stream):
            X = torch.empty((len(slots), res.handle.n), dtype=torch.float64, device="cuda")
            for i, j in enumerate(slots):
                res.handle.cg_result(j, out=X[i], stream=res.stream)
            return X.cpu().numpy().T                 # waits for this stream only

    def release(self, res):
        res.handle.close()


class SolveServer:
    """Schedules SLR-PCG solves of a request stream on the current GPU.

    matrices: key -> MatrixSpec.
    precision, nrhs_max, tol, maxit: for every handle and solve ("mixed" uses
        flexible CG around the FP32 apply); nrhs_max is the number of CG slots.
    backend: what sets up handles and runs the slots (default: CudaBackend).
    max_concurrent: matrices (worker threads, streams) served at once.
    reserve_bytes: device memory left free when a new handle is admitted.
    capacity_bytes: device memory all resident handles may hold (None: no cap
        beyond free memory).
    log: a text stream that receives one line per failed setup or solve.
    iters_per_step: CG iterations every occupied slot runs between two looks at
        the slots (completions, admissions).
    """

    def __init__(self, matrices: dict, precision="mixed", nrhs_max=8, tol=1e-8, maxit=300,
                 max_concurrent=4, reserve_bytes=1 << 30, capacity_bytes=None, setup_kw=None, backend=None,
                 log=None, iters_per_step=4):
        self.backend = backend or CudaBackend(precision, nrhs_max, setup_kw)
        self.matrices = matrices
        self.precision = precision
        self.nrhs_max = int(nrhs_max)
        self.tol, self.maxit = float(tol), int(maxit)
        self.max_concurrent = int(max_concurrent)
        self.reserve = int(reserve_bytes)
        self.capacity = capacity_bytes
        self.log = log
        self.iters_per_step = int(iters_per_step)
        self.errors: list = []           # (seconds, key, message)
        self.slots: dict = {}            # key -> Resident (resident handles)
        self.footprints: dict = {}       # key -> device bytes seen at its last setup
        self.claimed: dict = {}          # key -> bytes admitted for a setup in progress
        self.cv = threading.Condition()
        self.setups = 0
        self.evictions = 0
        self.batches = 0                 # admissions of waiting requests into free slots
        self.steps = 0                   # advances of a matrix's slots
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
    def _take_columns(self, key, free):
        """Waiting requests of `key` whose columns fit the free slots, oldest first
        (called with the lock held); each with the slots it gets."""
        q = self.pending.get(key)
        taken = []
        while q and q[0].ncols <= len(free):
            r = q.popleft()
            taken.append((r, [free.pop(0) for _ in range(r.ncols)]))
        return taken

    def _run_matrix(self, key, res, cold, started):
        """The slot loop of one matrix: admit, advance, collect, until it has no work."""
        n = self.matrices[key].n
        free = list(range(self.nrhs_max))
        owner = {}                       # slot -> (request, column)
        left = {}                        # rid -> columns not finished
        keep = []                        # device copies of started columns, until the next advance
        while True:
            with self.cv:
                taken = self._take_columns(key, free)
                if taken:
                    self.batches += 1
            if taken:
                now = time.perf_counter() - self.t0
                for r, sl in taken:
                    started.append(r)
                    keep.append(self.backend.start(res, sl, r.b.reshape(n, -1), self.tol, self.maxit))
                    for c, j in enumerate(sl):
                        owner[j] = (r, c)
                    left[r.rid] = r.ncols
                    r.x = np.zeros(r.b.shape)
                    r.iterations = np.zeros(r.ncols, np.int32)
                    r.relres = np.zeros(r.ncols)
                    r.status, r.start, r.cold = 0, now, cold
                for r, _ in taken:
                    r.batch = len(owner)
                cold = False
            if not owner:
                return
            width = max(owner) + 1
            act, its, rel, sts = self.backend.advance(res, self.iters_per_step, width)
            self.steps += 1
            keep.clear()
            done = sorted(j for j in owner if not act[j])
            if done:
                X = self.backend.results(res, done)
                t = time.perf_counter() - self.t0
                for i, j in enumerate(done):
                    r, c = owner.pop(j)
                    free.append(j)
                    if r.b.ndim == 1:
                        r.x[:] = X[:, i]
                    else:
                        r.x[:, c] = X[:, i]
                    r.iterations[c], r.relres[c] = its[j], rel[j]
                    if sts[j] == 2:
                        r.status = 6                       # SLR_ERR_BREAKDOWN
                    elif sts[j] != 1 and r.status == 0:
                        r.status = 5                       # SLR_ERR_NOT_CONVERGED (maxit)
                    left[r.rid] -= 1
                    if left[r.rid] == 0:
                        r.done = t
                free.sort()
            res.last_used = time.perf_counter()

    def _worker(self, key):
        started = []
        try:
            with self.cv:
                slot = self.slots.get(key)
                while slot is None and not self._admit(key):
                    self.cv.wait(0.05)
            cold = False
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
            self._run_matrix(key, slot, cold, started)
        except (SLRError, RuntimeError) as e:            # this matrix's requests fail, the server goes on
            t = time.perf_counter() - self.t0
            with self.cv:
                self.errors.append((t, key, f"{type(e).__name__}: {e}"))
                if self.log is not None:
                    print(f"[serving] {t:.3f}s matrix {key}: {type(e).__name__}: {e}", file=self.log, flush=True)
                unfinished = [r for r in started if r.done == 0.0] + list(self.pending.pop(key, deque()))
                for r in unfinished:
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
                    self.cv.notify_all()               # a running worker of that matrix may take it
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
