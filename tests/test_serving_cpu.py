"""Scheduling logic of the solve server, on the CPU with a fake backend.

The fake backend stands in for the device: it keeps a byte count for each
resident "handle", sleeps for a setup or an advance of the CG slots, lets each
started column run a set number of iterations, and returns x = b / diag(A) so
that the column bookkeeping can be checked exactly.
"""
import threading
import time

import numpy as np
import pytest

from paper_1505_04340_gb300 import serving
from paper_1505_04340_gb300.slr import SLRError
import slrgen


class FakeBackend:
    def __init__(self, total, setup_s=0.02, step_s=0.01, fail=(), need=lambda b: 8):
        self.total, self.used, self.max_used = total, 0, 0
        self.setup_s, self.step_s, self.fail, self.need = setup_s, step_s, set(fail), need
        self.lock = threading.Lock()
        self.inflight = self.max_inflight = 0
        self.steps = []                          # (key, width, occupied, start, end)

    def free_bytes(self):
        with self.lock:
            return self.total - self.used

    def setup(self, spec):
        if spec.k in self.fail:
            raise SLRError(2, "fake setup")
        fp = spec.n * 100
        with self.lock:
            self.used += fp
            self.max_used = max(self.max_used, self.used)
        time.sleep(self.setup_s)
        diag = np.array([spec.val[spec.rowptr[i]:spec.rowptr[i + 1]][spec.colind[spec.rowptr[i]:spec.rowptr[i + 1]] == i][0]
                         for i in range(spec.n)])
        return serving.Resident(handle={"k": spec.k, "diag": diag, "slots": {}}, stream=None, footprint=fp)

    def start(self, res, slots, B, tol, maxit):
        for i, j in enumerate(slots):
            assert j not in res.handle["slots"] or not res.handle["slots"][j]["active"]
            res.handle["slots"][j] = {"b": B[:, i].copy(), "its": 0, "need": self.need(B[:, i]), "active": True}
        return None

    def advance(self, res, iters, width):
        with self.lock:
            self.inflight += 1
            self.max_inflight = max(self.max_inflight, self.inflight)
        t = time.perf_counter()
        time.sleep(self.step_s)
        act, its, rel, sts = (np.zeros(width, np.int32), np.zeros(width, np.int32), np.zeros(width),
                              np.zeros(width, np.int32))
        occupied = 0
        for j, st in res.handle["slots"].items():
            if j >= width:
                continue
            if st["active"]:
                occupied += 1
                st["its"] = min(st["its"] + iters, st["need"])
                st["active"] = st["its"] < st["need"]
            act[j], its[j] = st["active"], st["its"]
            rel[j], sts[j] = (0.5, 0) if st["active"] else (1e-9, 1)
        with self.lock:
            self.inflight -= 1
            self.steps.append((res.handle["k"], width, occupied, t, time.perf_counter()))
        return act, its, rel, sts

    def results(self, res, slots):
        d = res.handle["diag"]
        return np.stack([res.handle["slots"][j]["b"] / d for j in slots], axis=1)

    def release(self, res):
        with self.lock:
            self.used -= res.footprint


def _matrices(count=4):
    mats = {}
    for i in range(count):
        side = 12 + 4 * i
        p = slrgen.make_problem(f"m{i}", (side, side), (2, 2), 4, kind="fv", coef_range=(1e-2, 1e2),
                                matrix_seed=50 + i)
        mats[i] = serving.MatrixSpec(p.rowptr, p.colind, p.val, p.part, p.nparts, k=i)
    return mats


def _requests(mats, specs):
    out = []
    for rid, (key, ncols, t) in enumerate(specs):
        b = slrgen.uniform_pm1(100 + rid, mats[key].n * ncols).reshape(mats[key].n, ncols)
        out.append(serving.Request(rid=rid, matrix=key, b=b[:, 0] if ncols == 1 else b, arrival=t))
    return out


def _diag(spec):
    return np.array([spec.val[spec.rowptr[i]:spec.rowptr[i + 1]][spec.colind[spec.rowptr[i]:spec.rowptr[i + 1]] == i][0]
                     for i in range(spec.n)])


def _check_answers(mats, reqs):
    for r in reqs:
        assert r.status == 0, (r.rid, r.status, r.error)
        d = _diag(mats[r.matrix])
        want = r.b / (d if r.b.ndim == 1 else d[:, None])
        assert np.array_equal(r.x, want), r.rid
        assert r.x.shape == r.b.shape


def test_backlog_is_batched_per_matrix_and_bounded():
    mats = _matrices()
    rng = slrgen.uniform01(7, 60).reshape(30, 2)
    specs = [(int(u[0] * 4), 1 + int(u[1] * 3), 0.0) for u in rng]
    reqs = _requests(mats, specs)
    be = FakeBackend(total=1 << 40)
    srv = serving.SolveServer(mats, nrhs_max=8, max_concurrent=3, reserve_bytes=0, backend=be)
    srv.run(reqs, realtime=False)
    _check_answers(mats, reqs)
    assert be.max_inflight <= 3 and srv.max_inflight <= 3
    assert all(w <= 8 and occ <= 8 for _, w, occ, _, _ in be.steps)
    assert srv.setups == 4 and srv.evictions == 0
    # a backlog shares the slots: some request started beside others
    assert any(r.batch > r.ncols for r in reqs)
    st = serving.latency_stats(reqs)
    assert st["served"] == 30 and st["solves"] == sum(r.ncols for r in reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"]


def test_late_arrivals_join_at_an_iteration_boundary():
    mats = _matrices(2)
    # r0 on matrix 0 at t=0 needs 40 iterations; r1, r2 on matrix 0 and r3 on matrix 1
    # arrive while it runs: they start in free slots before r0 finishes
    reqs = _requests(mats, [(0, 2, 0.0), (0, 1, 0.08), (0, 3, 0.09), (1, 1, 0.08)])
    need = lambda b: 40 if abs(b[0] - reqs[0].b[0, 0]) < 1e-15 or abs(b[0] - reqs[0].b[0, 1]) < 1e-15 else 8
    be = FakeBackend(total=1 << 40, setup_s=0.05, step_s=0.02, need=need)
    srv = serving.SolveServer(mats, nrhs_max=8, max_concurrent=2, reserve_bytes=0, backend=be)
    srv.run(reqs, realtime=True)
    _check_answers(mats, reqs)
    r0, r1, r2, r3 = reqs
    assert r0.batch == 2
    assert r1.start < r0.done and r2.start < r0.done      # joined the running slots
    assert r1.done < r0.done                              # and finished first
    assert r3.start < r0.done                             # the other matrix did not wait for matrix 0
    assert be.max_inflight == 2


def test_converged_slot_is_refilled():
    mats = _matrices(1)
    # two slots; r0 needs 40 iterations, r1 8, r2 waits for a slot: it takes r1's when r1 converges
    reqs = _requests(mats, [(0, 1, 0.0), (0, 1, 0.0), (0, 1, 0.0)])
    first = reqs[0].b[0]
    be = FakeBackend(total=1 << 40, setup_s=0.0, step_s=0.01, need=lambda b: 40 if b[0] == first else 8)
    srv = serving.SolveServer(mats, nrhs_max=2, max_concurrent=1, reserve_bytes=0, backend=be)
    srv.run(reqs, realtime=False)
    _check_answers(mats, reqs)
    r0, r1, r2 = reqs
    assert r1.done <= r2.start < r0.done


def test_capacity_forces_lru_eviction():
    mats = _matrices(4)
    fp = [m.n * 100 for m in mats.values()]
    cap = fp[2] + fp[3] + 10                  # any two handles fit, never three
    order = [0, 1, 2, 3, 0, 1, 3, 2, 0, 0, 1]
    reqs = _requests(mats, [(k, 1, 0.01 * i) for i, k in enumerate(order)])
    be = FakeBackend(total=1 << 40, setup_s=0.01, step_s=0.005)
    srv = serving.SolveServer(mats, nrhs_max=4, max_concurrent=2, reserve_bytes=0, capacity_bytes=cap, backend=be)
    srv.footprints = {k: fp[k] for k in mats}
    srv.run(reqs, realtime=True)
    _check_answers(mats, reqs)
    assert be.max_used <= cap
    assert srv.evictions > 0 and srv.setups > 4


def test_rejects_and_failures_do_not_stop_the_server():
    mats = _matrices(3)
    big = serving.Request(rid=90, matrix=0, b=np.ones((mats[0].n, 9)), arrival=0.0)     # 9 > nrhs_max
    unknown = serving.Request(rid=91, matrix=7, b=np.ones(5), arrival=0.0)
    reqs = _requests(mats, [(0, 1, 0.0), (1, 2, 0.0), (2, 1, 0.0), (1, 1, 0.01)])
    be = FakeBackend(total=1 << 40, fail={1})                                           # matrix 1 fails setup
    srv = serving.SolveServer(mats, nrhs_max=8, max_concurrent=2, reserve_bytes=0, backend=be)
    srv.run(reqs + [big, unknown], realtime=True)
    assert big.status == 1 and unknown.status == 1
    assert reqs[1].status == 2 and reqs[3].status == 2 and "fake setup" in reqs[1].error
    _check_answers(mats, [reqs[0], reqs[2]])


def test_request_stream_recipe():
    rq = slrgen.serving_requests(count=256, seed=3, nspecs=32, rate=50.0)
    assert len(rq) == 256 and rq[0]["arrival"] == 0.0
    t = np.array([r["arrival"] for r in rq])
    assert np.all(np.diff(t) >= 0)
    # Poisson arrivals: mean gap 1/rate (256 samples: within 20 %)
    assert abs(np.diff(t).mean() * 50.0 - 1.0) < 0.2
    assert {r["nrhs"] for r in rq} == set(range(1, 9))
    assert {r["spec"] for r in rq} <= set(range(32))
    specs = slrgen.serving_specs(32, seed=3)
    for s in specs:
        nparts = int(np.prod(s["boxes"]))
        assert 16 <= nparts <= 256 and s["k"] in (16, 32, 64)
        side = s["dims"][0]
        assert (64 <= side <= 512) if len(s["dims"]) == 2 else (32 <= side <= 64)
