"""Failure paths of the library on the GPU, made to happen without a GPU fault.

* A bounded device wait that runs out: the cooperative C solve's grid barrier
  is given a poll budget of one (``spin_limit``), so its waits give up; the
  kernels still finish (every index they use comes from the factor's
  structure), the status word reports it, the calls return SLR_ERR_TIMEOUT, and
  the context stays usable for the next handle.
* A device allocation that fails: the host-side hook ``slr_inject_alloc_failure``
  makes the nth allocation report out-of-memory; setup returns SLR_ERR_OOM and
  releases everything it held, an update of the low-rank part that fails keeps
  the old one.
"""
import ctypes as C

import numpy as np
import pytest

import slrgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1505_04340_gb300 import SLR, slr  # noqa: E402
from paper_1505_04340_gb300.slr import SLRError  # noqa: E402

TIMEOUT, OOM = 7, 3


def _problem():
    return slrgen.make_problem("3d", (20, 19, 18), (3, 2, 2), 8)


def _handle(P, **kw):
    return SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps, **kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_barrier_wait_runs_out(precision):
    P = _problem()
    b = torch.tensor(P.b[:, 0], device="cuda")
    opts = dict(precision=precision, c_persistent=True, c_top_zone=False, spin_limit=1)
    # setup: the Lanczos H applies run the cooperative C solve and report the expiry
    with pytest.raises(SLRError) as ei:
        _handle(P, **opts)
    assert ei.value.status == TIMEOUT and "grid-barrier" in str(ei.value)
    # rank 0 needs no Lanczos: setup succeeds, the solve's waits run out
    hp = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=0, **opts)
    assert hp.get_info()["c_persistent"] == 1 and hp.get_info()["c_levels"] > 2
    x, its, rel, st = hp.pcg(b, maxit=5, check=False)
    assert st == TIMEOUT
    assert b"grid-barrier" in slr.load().slr_last_error_message()
    assert hp.device_status() == TIMEOUT
    # an apply on the timed-out operator: the status word is cleared by the call and set again
    r = torch.randn(P.n, dtype=torch.float64, device="cuda")
    hp.apply(r)
    assert hp.device_status() == TIMEOUT
    hp.close()
    # the context is unharmed: a handle with the default budget solves, status clear
    h = _handle(P, precision=precision, c_persistent=True)
    x, its, rel, st = h.pcg(b)
    assert st == 0 and rel[0] <= 1e-8
    assert h.device_status() == 0
    h.close()


def test_status_clear_after_normal_calls():
    P = _problem()
    h = _handle(P, c_persistent=True)
    r = torch.randn(P.n, dtype=torch.float64, device="cuda")
    h.apply(r)
    h.bsolve(torch.randn(h.n_interior, dtype=torch.float64, device="cuda"))
    assert h.device_status() == 0
    h.close()


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("nth", [1, 5, 25])
def test_injected_allocation_failure_in_setup(nth):
    P = _problem()
    lib = slr.load()
    h0 = _handle(P)                 # warm the context and the kernels' one-time state
    h0.close()
    free0 = _free_bytes()
    lib.slr_inject_alloc_failure(nth)
    try:
        with pytest.raises(SLRError) as ei:
            _handle(P, precision="mixed")
        assert ei.value.status == OOM and "injected" in str(ei.value)
    finally:
        lib.slr_inject_alloc_failure(0)
    assert abs(_free_bytes() - free0) <= 4 << 20      # everything the failed setup held was released
    h = _handle(P, precision="mixed")                # and the next setup succeeds
    x, its, rel, st = h.pcg(torch.tensor(P.b[:, 0], device="cuda"))
    assert st == 0
    h.close()


def test_injected_allocation_failure_keeps_lowrank():
    P = _problem()
    lib = slr.load()
    h = _handle(P)
    Z, lam, theta = h.get_lowrank()
    r = torch.randn(P.n, dtype=torch.float64, device="cuda")
    z0 = h.apply(r).cpu().numpy()
    lib.slr_inject_alloc_failure(1)
    try:
        with pytest.raises(SLRError) as ei:
            h.set_lowrank(Z[:, :3], lam[:3], lam[3])
        assert ei.value.status == OOM
    finally:
        lib.slr_inject_alloc_failure(0)
    z1 = h.apply(r).cpu().numpy()
    assert np.array_equal(z0, z1)                     # the old pairs still serve the apply
    h.close()
