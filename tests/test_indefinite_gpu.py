"""Symmetric indefinite problems with an SPD interface (Section 1; the shifted
problems -Laplacian u - c u = f of Section 6) through the C ABI, against the
oracle: B solves with indefinite B_i (factored as L S L^T, S the pivot signs, on
the device and on the host), the apply with the oracle's eigenpairs (lambda may
exceed 1), and SLR-preconditioned GMRES(40).

Tolerances as in test_gpu_parity: 1e-10 relative (max-norm) in FP64, 1e-4 for the
FP32 apply.  GMRES iteration counts may differ from the oracle's by rounding
(flexible vs plain right preconditioning, Gram-Schmidt variants): within 2.
"""
import numpy as np
import pytest

import slrgen
from oracle.slr_oracle import SLR as OracleSLR, slr_gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1505_04340_gb300 import SLR  # noqa: E402
from paper_1505_04340_gb300.slr import SLRError  # noqa: E402

TOL64 = 1e-10
# The blocks B_i = L S L^T are indefinite and factored without pivoting, so the
# FP32 solves can carry element growth that the SPD bound of tests/tolerances.py
# does not cover; the mixed path is held to 1e-4 here and its error is printed
# beside that bound.
TOL32 = 1e-4

CASES = {
    # name: (dims, boxes, shift, k); B_i indefinite, C SPD (checked by the oracle pins)
    "2d-shift": ((32, 32), (2, 2), 0.2, 8),
    "3d-shift": ((16, 16, 16), (2, 2, 2), 0.6, 8),
}


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def cu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def problem(name):
    dims, boxes, shift, k = CASES[name]
    return slrgen.make_problem(name, dims, boxes, k, shift=shift)


def handle(P, precision="fp64", nrhs_max=4, **kw):
    return SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps,
               precision=precision, indefinite=True, nrhs_max=nrhs_max, **kw)


def oracle(P):
    return OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, lanczos_steps=P.lanczos_steps,
                     indefinite=True)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("factor", ["auto", "host"])
def test_indefinite_bsolve_parity(name, precision, factor):
    P = problem(name)
    o = oracle(P)
    g = handle(P, precision, band_factor=factor)
    assert g.get_info()["band_on_device"] == (1 if factor == "auto" else 0)
    f = np.random.default_rng(1).standard_normal((o.order.n_I, 3))
    t = g.bsolve(cu(f)).cpu().numpy()
    err = rel(t, o.bsolve.solve(f))
    print(f"indefinite bsolve {precision}: {err:.2e}")
    assert err <= (TOL64 if precision == "fp64" else TOL32)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_indefinite_apply_parity_with_oracle_pairs(name, precision):
    P = problem(name)
    o = oracle(P)
    g = handle(P, precision)
    g.set_lowrank(o.Z(), o.lam, o.theta)       # lambda_1 > 1 here: accepted in indefinite mode
    r = np.random.default_rng(3).standard_normal((o.App.shape[0], 2))
    z = g.apply(cu(r)).cpu().numpy()
    err = rel(z, o.apply(r))
    print(f"indefinite apply {precision}: {err:.2e}")
    assert err <= (TOL64 if precision == "fp64" else TOL32)


@pytest.mark.parametrize("name", list(CASES))
def test_indefinite_theta_reading_and_ritz_values(name):
    """The device Lanczos finds the same leading Ritz values, some above 1, and keeps
    theta = lambda_{k+1} only while it is below 1."""
    P = problem(name)
    o = oracle(P)
    g = handle(P)
    lam = np.asarray(g.ritz())[: P.k]
    assert lam[0] > 1.0
    assert np.allclose(lam[:3], o.ritz_values[:3], rtol=1e-8, atol=1e-10)
    inf = g.get_info()
    assert inf["theta"] < 1.0
    if o.ritz_values[P.k] >= 1.0:
        assert inf["theta"] == 0.0


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gmres_converges_like_the_oracle(name, precision):
    P = problem(name)
    o = oracle(P)
    _, its_o, rel_o, ok_o = slr_gmres(o, P.b[:, 0])
    assert ok_o[0]
    g = handle(P, precision)
    x, its, rels, st = g.gmres(cu(P.b[:, 0]))
    assert st == 0 and rels[0] <= 1e-8
    if precision == "fp64":
        assert abs(int(its[0]) - its_o[0]) <= 2, (its, its_o)
    else:
        assert int(its[0]) <= its_o[0] + 4, (its, its_o)
    xs = P.xstar[:, 0]
    assert np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs) < 1e-5


def test_gmres_restart_and_columns():
    """A shorter restart converges in more iterations, as the oracle's does (GMRES(5)
    stagnates on this indefinite problem: 767 oracle iterations), columns are
    independent runs, and each column of a block equals the column solved alone."""
    P = slrgen.make_problem("3d-shift-2rhs", (16, 16, 16), (2, 2, 2), 8, shift=0.6, nrhs=2)
    g = handle(P, nrhs_max=2)
    B = cu(P.b)
    x, its, rels, st = g.gmres(B)
    assert st == 0 and np.all(rels <= 1e-8)
    x1, its1, _, _ = g.gmres(cu(P.b[:, 1]))
    assert int(its1[0]) == int(its[1])
    assert np.array_equal(x1.cpu().numpy(), x.cpu().numpy()[:, 1])
    o = oracle(P)
    _, its_o, _, ok_o = slr_gmres(o, P.b[:, 0], restart=15)
    x15, its15, rels15, st15 = g.gmres(cu(P.b[:, 0]), restart=15)
    assert st15 == 0 and ok_o[0] and rels15[0] <= 1e-8 and int(its15[0]) > int(its[0])
    assert abs(int(its15[0]) - its_o[0]) <= 3


def test_gmres_on_spd_problem_matches_oracle_gmres():
    """The accelerator also works for SPD A (the same iterations as the oracle's GMRES)."""
    P = slrgen.make_problem("spd", (32, 32), (2, 2), 8)
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 8)
    _, its_o, _, ok_o = slr_gmres(o, P.b[:, 0])
    g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=8, lanczos_steps=P.lanczos_steps)
    _, its, rels, st = g.gmres(cu(P.b[:, 0]))
    assert st == 0 and ok_o[0] and abs(int(its[0]) - its_o[0]) <= 2


def test_gmres_reports_not_converged_and_rejects_bad_arguments():
    P = problem("3d-shift")
    g = handle(P)
    _, its, rels, st = g.gmres(cu(P.b[:, 0]), maxit=3, check=False)
    assert st == 5 and int(its[0]) == 3 and rels[0] > 1e-8
    with pytest.raises(SLRError, match="INVALID_ARG"):
        g.gmres(cu(P.b[:, 0]), restart=0)


def test_indefinite_needs_the_option():
    """Without the indefinite option an indefinite B_i is refused as not SPD."""
    P = problem("2d-shift")
    with pytest.raises(SLRError, match="SLR_ERR_NOT_SPD"):
        SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps)
