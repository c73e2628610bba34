"""The solve server on the GPU: requests served in a concurrent, batched mix give
the same answers as the same requests served alone.

Each column of a multi-RHS solve is its own CG run (own scalars, own mask,
fixed-order reductions), and setup is deterministic, so the expected difference
is zero; the stated tolerance is 1e-12 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import slrgen

pytestmark = pytest.mark.gpu

MIX_TOL = 1e-12


def _pool():
    from paper_1505_04340_gb300 import serving
    shapes = [((40, 40), (4, 4), 8), ((64, 64), (2, 2), 16), ((14, 14, 14), (2, 2, 2), 8),
              ((18, 18, 18), (3, 3, 3), 16)]
    mats, probs = {}, {}
    for i, (dims, boxes, k) in enumerate(shapes):
        p = slrgen.make_problem(f"pool{i}", dims, boxes, k, kind="fv", coef_range=(1e-2, 1e2), matrix_seed=200 + i)
        probs[i] = p
        mats[i] = serving.MatrixSpec(p.rowptr, p.colind, p.val, p.part, p.nparts, k=k)
    return mats, probs


def _stream(mats, probs, count=24, rate=300.0):
    from paper_1505_04340_gb300 import serving
    reqs = []
    for d in slrgen.serving_requests(count=count, seed=11, nspecs=len(mats), rate=rate):
        nr = 1 + (d["nrhs"] - 1) % 4
        _, b = slrgen.request_rhs(probs[d["spec"]], nr, d["rhs_seed"])
        reqs.append(serving.Request(rid=d["rid"], matrix=d["spec"], b=b[:, 0] if nr == 1 else b,
                                    arrival=d["arrival"]))
    return reqs


def _fresh(reqs):
    from paper_1505_04340_gb300 import serving
    return [serving.Request(rid=r.rid, matrix=r.matrix, b=r.b, arrival=0.0) for r in reqs]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_mix_equals_alone(precision):
    from paper_1505_04340_gb300 import serving
    mats, probs = _pool()
    reqs = _stream(mats, probs)
    srv = serving.SolveServer(mats, precision=precision, nrhs_max=8, max_concurrent=3, reserve_bytes=0)
    try:
        srv.run(reqs, realtime=True)
    finally:
        srv.close()
    assert all(r.status == 0 for r in reqs), [(r.rid, r.status, r.error) for r in reqs if r.status]
    assert srv.setups == len(mats)
    assert srv.max_inflight >= 2                       # solves of different matrices overlapped
    for r in reqs:
        A = sp.csr_matrix((probs[r.matrix].val, probs[r.matrix].colind, probs[r.matrix].rowptr))
        B, X = r.b.reshape(A.shape[0], -1), r.x.reshape(A.shape[0], -1)
        res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
        assert np.all(res <= 1e-7), (r.rid, res)

    # the same requests one at a time on a second server (its own setups)
    alone = _fresh(reqs)
    srv2 = serving.SolveServer(mats, precision=precision, nrhs_max=8, max_concurrent=1, reserve_bytes=0)
    try:
        for r in alone:
            srv2.run([r], realtime=False)
    finally:
        srv2.close()
    worst, same = 0.0, 0
    for a, m in zip(alone, reqs):
        assert a.status == 0 and a.batch == a.ncols
        d = np.max(np.abs(a.x - m.x)) / np.max(np.abs(a.x))
        worst = max(worst, d)
        same += np.array_equal(a.x, m.x)
        assert np.array_equal(a.iterations, m.iterations), a.rid
    assert worst <= MIX_TOL, worst
    print(f"{precision}: {same}/{len(reqs)} requests bitwise equal alone and in the mix, worst {worst:.2e}")


def test_backlog_with_eviction_matches():
    from paper_1505_04340_gb300 import serving
    mats, probs = _pool()
    reqs = _stream(mats, probs, count=20)
    srv = serving.SolveServer(mats, precision="mixed", nrhs_max=8, max_concurrent=2, reserve_bytes=0)
    try:
        srv.run(reqs, realtime=False)
        fps = dict(srv.footprints)
    finally:
        srv.close()
    assert any(r.batch > r.ncols for r in reqs)        # the backlog was packed
    cap = sorted(fps.values())[-1] + sorted(fps.values())[-2] + 1
    again = _fresh(reqs)
    srv2 = serving.SolveServer(mats, precision="mixed", nrhs_max=8, max_concurrent=2, reserve_bytes=0,
                               capacity_bytes=cap)
    srv2.footprints = fps
    try:
        srv2.run(again, realtime=False)
    finally:
        srv2.close()
    assert srv2.evictions > 0
    for a, m in zip(again, reqs):
        assert a.status == 0
        assert np.max(np.abs(a.x - m.x)) <= MIX_TOL * np.max(np.abs(m.x)), a.rid


def test_concurrent_handles_of_different_widths():
    """Two threads solve with operators of very different band widths at once.

    The band kernel's shared-memory limit is process-wide; a per-launch limit
    raced between threads (one thread's launch after another's lower setting)."""
    import threading
    import torch
    from paper_1505_04340_gb300 import SLR
    wide = slrgen.make_problem("wide", (32, 32, 32), (2, 2, 2), 8)            # planes of 15 x 15
    narrow = slrgen.make_problem("narrow", (64, 64), (8, 8), 8)               # planes of 7
    errors, outs = [], {}

    def work(name, P, prec):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, precision=prec, nrhs_max=4,
                        flexible_cg=(prec == "mixed"), stream=st)
                b = torch.tensor(P.b[:, 0], device="cuda")
                B = torch.stack([b, 2 * b, -b], dim=1)
                res = []
                for _ in range(20):
                    x, its, rel, s = h.pcg(B, stream=st)
                    assert s == 0, (name, s, rel)
                    res.append(x.cpu().numpy())
                h.close()
            assert all(np.array_equal(res[0], r) for r in res), name
            outs[name] = res[0]
        except BaseException as e:                                       # reported by the main thread
            errors.append(f"{name}: {type(e).__name__}: {e}")

    for prec in ("fp64", "mixed"):
        th = [threading.Thread(target=work, args=(nm + prec, P, prec)) for nm, P in (("wide", wide), ("narrow", narrow))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors, errors
    for nm in ("wide", "narrow"):
        P = wide if nm == "wide" else narrow
        x = outs[nm + "fp64"][:, 0]
        assert np.linalg.norm(x - P.xstar[:, 0]) / np.linalg.norm(P.xstar[:, 0]) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cg_slots_equal_pcg_solve(precision):
    """Columns started in CG slots at different iteration boundaries (one refilling a
    converged column's slot) give bitwise the answers and iteration counts of
    slr_pcg_solve on each column alone: a slot starts with p = 0 and a unit rho
    placeholder, so its first preconditioner update yields p = z exactly."""
    import torch
    from paper_1505_04340_gb300 import SLR
    P = slrgen.make_problem("slots", (18, 17, 16), (3, 2, 2), 8, kind="fv", coef_range=(1e-2, 1e2), nrhs=3)
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps, precision=precision,
            nrhs_max=4, flexible_cg=(precision == "mixed"))
    B = [torch.tensor(np.ascontiguousarray(P.b[:, j]), device="cuda") for j in range(3)]
    ref = [h.pcg(b) for b in B]                             # (x, its, rel, status) of each column alone
    holder = {0: 0}                                         # slot -> column it runs
    h.cg_start(0, B[0])
    act, its, rel, st = h.cg_advance(3, 1)
    assert act[0] == 1 and its[0] == 3
    h.cg_start(2, B[1])                                     # slot 1 stays idle; slot 2 joins at iteration 3
    holder[2] = 1
    out, queue = {}, [2]                                    # column 2 waits for a free slot
    for _ in range(300):
        act, its, rel, st = h.cg_advance(2, 3)
        assert act[1] == 0                                  # the idle slot never runs
        for slot in list(holder):
            if not act[slot]:
                out[holder.pop(slot)] = (h.cg_result(slot).cpu().numpy(), int(its[slot]), int(st[slot]))
                if queue:                                   # refill the converged column's slot
                    holder[slot] = queue.pop(0)
                    h.cg_start(slot, B[holder[slot]])
        if not holder:
            break
    assert sorted(out) == [0, 1, 2]
    for j in range(3):
        x, it, s_ = out[j]
        xr, itr, _, sr = ref[j]
        assert s_ == 1 and sr == 0
        assert it == int(itr[0]), (j, it, itr)
        assert np.array_equal(x, xr.cpu().numpy()), j
