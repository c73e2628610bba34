"""Partitions with vertex separators (Section 2.1: the method applies to them as
well as to the edge-based partitions) through the C ABI, against the oracle:
part = -1 marks a separator vertex, the separators form the interface, and a
part's vertices coupled only to their own part and to separators are interior.

Tolerances as in test_gpu_parity: 1e-10 relative (max-norm) in FP64, 1e-4 for the
FP32 apply; PCG iteration counts within 1 of the oracle's.
"""
import numpy as np
import pytest

import slrgen
from oracle.slr_oracle import SLR as OracleSLR, slr_pcg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1505_04340_gb300 import SLR  # noqa: E402

TOL64 = 1e-10
from tolerances import tol32  # noqa: E402

CASES = {
    "2d-vsep": ((32, 32), (2, 2), 8),
    "3d-vsep": ((16, 16, 16), (2, 2, 2), 8),
    "3d-vsep-ragged": ((19, 14, 11), (3, 2, 2), 6),
}


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def cu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def problem(name):
    dims, boxes, k = CASES[name]
    return slrgen.make_problem(name, dims, boxes, k, separators=True)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vsep_solves_and_apply_parity(name, precision):
    P = problem(name)
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, lanczos_steps=P.lanczos_steps)
    g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps, precision=precision,
            nrhs_max=2)
    tol = TOL64 if precision == "fp64" else tol32(g.get_info())
    assert np.array_equal(g.perm(), o.order.perm)
    assert g.get_info()["s"] == int(np.sum(P.part < 0))
    rng = np.random.default_rng(7)
    f = rng.standard_normal((o.order.n_I, 2))
    assert rel(g.bsolve(cu(f)).cpu().numpy(), o.bsolve.solve(f)) <= tol
    gg = rng.standard_normal((o.order.s, 2))
    assert rel(g.csolve(cu(gg)).cpu().numpy(), o.cfac.solve(gg)) <= tol
    g.set_lowrank(o.Z(), o.lam, o.theta)
    r = rng.standard_normal((o.App.shape[0], 2))
    assert rel(g.apply(cu(r)).cpu().numpy(), o.apply(r)) <= tol


@pytest.mark.parametrize("name", list(CASES))
def test_vsep_pcg_matches_oracle(name):
    P = problem(name)
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, lanczos_steps=P.lanczos_steps)
    _, its_o, _, ok_o = slr_pcg(o, P.b[:, 0])
    g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps)
    x, its, rels, st = g.pcg(cu(P.b[:, 0]))
    assert st == 0 and ok_o[0] and abs(int(its[0]) - its_o[0]) <= 1
    xs = P.xstar[:, 0]
    assert np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs) < 1e-6
