"""The low-rank products of Eq. 4.7 on the tensor cores (u_dtype TF32 or BF16).

For a block of 8 or more right-hand sides, the FP32 apply forms U_k^T W and
U_k (d o V) with tcgen05 MMAs on TF32- or BF16-rounded operands, accumulating
in FP32.  The checks isolate the low-rank correction
corr = S~^{-1} g - (1 - theta)^{-1} C^{-1} g = L^{-T} U_k (d o U_k^T L^{-1} g)
and compare it with the FP64 oracle's: rounding the inputs of the two products
to a unit round-off u moves each product by at most about 2u relative to the
sum of its terms' magnitudes, so the correction stays within 16 u of the
oracle's (u = 2^-11 for TF32, 2^-8 for BF16), while an operand laid out wrong
in shared memory or tensor memory would miss by O(1).  End to end, mixed PCG
with the tensor-core products reaches 1e-8 on every column and its solution
lies within 1e-7 of the FP64 oracle's.
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

U_TC = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}
CASES = {
    # name: (dims, boxes, k)
    "3d-lap": ((20, 19, 18), (3, 2, 2), 8),
    "2d-fv": ((61, 47), (3, 4), 24),
    "3d-k100": ((24, 24, 24), (2, 2, 2), 100),
}


def cu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _problem(name, nrhs=1):
    dims, boxes, k = CASES[name]
    kind, cr = ("fv", (1e-2, 1e2)) if name.startswith("2d-fv") else ("laplacian", None)
    return slrgen.make_problem(name, dims, boxes, k, kind=kind, coef_range=cr, nrhs=nrhs)


_oracles = {}


def _oracle(name):
    if name not in _oracles:
        P = _problem(name)
        _oracles[name] = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, P.lanczos_steps)
    return _oracles[name]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("u_dtype", ["tf32", "bf16"])
@pytest.mark.parametrize("nrhs", [8, 16, 40])
def test_lowrank_correction_matches_oracle(name, u_dtype, nrhs):
    P = _problem(name)
    o = _oracle(name)
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=0, precision="mixed", nrhs_max=nrhs, u_dtype=u_dtype)
    h.set_lowrank(o.Z(), o.lam, o.theta)
    G = np.random.default_rng(11).standard_normal((o.order.s, nrhs))
    y = h.stilde_solve(cu(G)).cpu().numpy()
    c = h.csolve(cu(G)).cpu().numpy()
    corr = y - c / (1.0 - o.theta)
    corr_o = o.stilde_inv(G) - o.cfac.solve(G) / (1.0 - o.theta)
    err = np.abs(corr - corr_o).max(axis=0) / np.abs(corr_o).max(axis=0)
    print(f"{name} {u_dtype} nrhs {nrhs}: correction error {err.max():.2e} (u = {U_TC[u_dtype]:.1e})")
    assert err.max() <= 16 * U_TC[u_dtype], err


@pytest.mark.parametrize("u_dtype", ["tf32", "bf16"])
def test_mixed_pcg_with_tensor_core_lowrank(u_dtype):
    name = "3d-lap"
    P = _problem(name, nrhs=8)
    o = _oracle(name)
    X_o = np.stack([slr_pcg(o, P.b[:, j])[0] for j in range(8)], axis=1)
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps, precision="mixed",
            nrhs_max=8, flexible_cg=True, u_dtype=u_dtype)
    x, its, rel, st = h.pcg(cu(P.b))
    X = x.cpu().numpy()
    assert st == 0 and np.all(rel <= 1e-8)
    diff = np.linalg.norm(X - X_o, axis=0) / np.linalg.norm(X_o, axis=0)
    h32 = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps, precision="mixed",
              nrhs_max=8, flexible_cg=True)
    _, its32, _, _ = h32.pcg(cu(P.b))
    print(f"{u_dtype}: iterations {its.tolist()} (FP32 products {its32.tolist()}), x vs oracle {diff.max():.2e}")
    assert diff.max() <= 1e-7


# ---------------------------------------------------------------- the band solve
BAND_CASES = {
    # name: (dims, boxes, k): plane widths 63 (one M-tile), 90 and 156-180 (two M-tiles, ragged)
    "2d-fv": ((61, 47), (3, 4), 8),
    "3d-lap": ((20, 19, 18), (3, 2, 2), 8),
    "3d-wide": ((30, 28, 13), (2, 2, 1), 6),
}


def _band_problem(name, nrhs=1):
    dims, boxes, k = BAND_CASES[name]
    kind, cr = ("fv", (1e-2, 1e2)) if name.startswith("2d-fv") else ("laplacian", None)
    return slrgen.make_problem(name, dims, boxes, k, kind=kind, coef_range=cr, nrhs=nrhs)


_kappas = {}


def _kappa_L(name, o):
    """Largest 2-norm condition number of the Cholesky factors L_i of the B_i:
    sqrt(kappa(B_i)), with B_i = L_i L_i^T rebuilt from the oracle's band factor."""
    if name not in _kappas:
        worst = 1.0
        for blk in o.bsolve.blocks:
            lo = blk.cb                                  # lower band storage: lo[d, j] = L[j + d, j]
            m, w = lo.shape[1], lo.shape[0] - 1
            L = np.zeros((m, m))
            for d in range(w + 1):
                L[np.arange(d, m), np.arange(0, m - d)] = lo[d, :m - d]
            ev = np.linalg.eigvalsh(L @ L.T)
            worst = max(worst, float(np.sqrt(ev[-1] / ev[0])))
        _kappas[name] = worst
    return _kappas[name]


@pytest.mark.parametrize("name", list(BAND_CASES))
@pytest.mark.parametrize("mma", ["tf32", "bf16"])
@pytest.mark.parametrize("nrhs", [8, 32, 40])
def test_band_solve_on_tensor_cores_matches_oracle(name, mma, nrhs):
    """t = B^{-1} F with the factor and the plane vectors rounded to TF32 / BF16.
    Rounding an input moves each product term by at most u relative (factor and
    vector: 2u per term, FP32 accumulation adds far less); these diagonally
    dominant blocks keep the plane sums well conditioned and the chain contractive,
    so the solve stays within a few u of the exact one, while a block left out or
    misplaced moves it by O(1).  Bound 16 u; kappa(L) u, the worst-case bound, is
    printed beside it (it runs to 0.3 for TF32 on the FV blocks)."""
    P = _band_problem(name)
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0)
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=0, precision="mixed", nrhs_max=nrhs, band_mma=mma)
    assert h.get_info()["band_mma"] == {"tf32": 1, "bf16": 2}[mma]
    F = np.random.default_rng(21).standard_normal((o.order.n_I, nrhs))
    T = h.bsolve(cu(F)).cpu().numpy()
    To = np.stack([o.bsolve.solve(F[:, j]) for j in range(nrhs)], axis=1)
    err = float((np.abs(T - To).max(axis=0) / np.abs(To).max(axis=0)).max())
    tol = 16 * U_TC[mma]
    print(f"{name} {mma} nrhs {nrhs}: band solve error {err:.2e} (bound {tol:.2e}; kappa(L) u = "
          f"{_kappa_L(name, o) * U_TC[mma]:.2e})")
    assert err <= tol


@pytest.mark.parametrize("mma", ["tf32", "bf16"])
@pytest.mark.parametrize("nrhs", [8, 16, 24])
def test_band_solve_on_tensor_cores_two_ctas_per_sm(mma, nrhs):
    """More subdomains (180) than SMs, so two CTAs share each SM, and planes of up
    to 144 rows (two M-tiles of 128): the accumulators and staged operands of both
    M-tiles of both CTAs must stay in their own tensor-memory columns, for N padded
    to 16 (8 and 16 right-hand sides) as well as to 32.  A column written into the
    other CTA's allocation moves the solve by O(1); the bound is the 16 u of the
    small-case test.  The reference is the oracle's banded Cholesky solves alone
    (its C factor is not needed here)."""
    from oracle.slr_oracle import BSolver, dd_order, split_blocks
    P = slrgen.make_problem("3d-many", (78, 78, 20), (6, 6, 5), 8, kind="laplacian", nrhs=1)
    order = dd_order(P.rowptr, P.colind, P.part, P.nparts)
    bs = BSolver(split_blocks(P.rowptr, P.colind, P.val, order)[0], order.int_off)
    assert P.nparts > 152 and max(b.cb.shape[0] - 1 for b in bs.blocks) > 128
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=0, precision="mixed", nrhs_max=nrhs, band_mma=mma)
    F = np.random.default_rng(23).standard_normal((order.n_I, nrhs))
    T = h.bsolve(cu(F)).cpu().numpy()
    To = np.stack([bs.solve(F[:, j]) for j in range(nrhs)], axis=1)
    err = float((np.abs(T - To).max(axis=0) / np.abs(To).max(axis=0)).max())
    print(f"{mma} nrhs {nrhs}: band solve error {err:.2e} (bound {16 * U_TC[mma]:.2e})")
    assert err <= 16 * U_TC[mma]
    h.close()


def test_apply_does_not_depend_on_block_width():
    """The whole mixed apply with tensor-core band solves and low-rank products, on
    a workload with more subdomains than SMs and two M-tiles per plane: the first
    8 and 16 columns of a 32-column block match the same columns applied alone.
    Each output column of an MMA depends only on its own operand column, so the
    agreement is exact in practice; the bound is the band solve's 16 u."""
    P = slrgen.make_problem("3d-many", (78, 78, 20), (6, 6, 5), 8, kind="laplacian", nrhs=1)
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=8, precision="mixed", nrhs_max=32,
            band_mma="tf32", u_dtype="tf32")
    R = cu(np.random.default_rng(37).standard_normal((P.rowptr.size - 1, 32)))
    z = h.apply(R).cpu().numpy()
    for w in (8, 16):
        zw = h.apply(R[:, :w].contiguous()).cpu().numpy()
        err = float((np.abs(zw - z[:, :w]).max(axis=0) / np.abs(z[:, :w]).max(axis=0)).max())
        print(f"first {w} of 32 columns vs alone: {err:.2e}")
        assert err <= 16 * U_TC["tf32"]
    h.close()


@pytest.mark.parametrize("mma", ["tf32", "bf16"])
def test_apply_with_tensor_core_band_solve(mma):
    """The whole apply (Eq. 4.1) with both B-solves on the tensor cores, the second
    one subtracting from its base (u = t - B^{-1} E y), against the same operator's
    CUDA-core FP32 apply on 16 columns: within 16 u of the operand type relative to
    the largest entry, as each B-solve is (a base misapplied moves it by O(1))."""
    P = _problem("3d-lap", nrhs=16)
    kw = dict(k=P.k, lanczos_steps=P.lanczos_steps, precision="mixed", nrhs_max=16)
    h0 = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, **kw)
    h1 = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, band_mma=mma, **kw)
    R = cu(np.random.default_rng(31).standard_normal((P.rowptr.size - 1, 16)))
    z0, z1 = h0.apply(R).cpu().numpy(), h1.apply(R).cpu().numpy()
    err = float((np.abs(z1 - z0).max(axis=0) / np.abs(z0).max(axis=0)).max())
    print(f"apply with the {mma} band solve: {err:.2e} (bound {16 * U_TC[mma]:.2e})")
    assert err <= 16 * U_TC[mma]
    h0.close()
    h1.close()


@pytest.mark.parametrize("mma", ["tf32", "bf16"])
def test_mixed_pcg_with_tensor_core_band_solve(mma):
    """Flexible CG absorbs the rounded factor: every column reaches 1e-8 and the
    solution matches the FP64 oracle's to 1e-7."""
    name = "3d-lap"
    P = _problem(name, nrhs=16)
    o = _oracle(name)
    X_o = np.stack([slr_pcg(o, P.b[:, j])[0] for j in range(16)], axis=1)
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps, precision="mixed",
            nrhs_max=16, flexible_cg=True, band_mma=mma, u_dtype=mma)
    x, its, rel, st = h.pcg(cu(P.b))
    X = x.cpu().numpy()
    assert st == 0 and np.all(rel <= 1e-8)
    diff = np.linalg.norm(X - X_o, axis=0) / np.linalg.norm(X_o, axis=0)
    print(f"band {mma}: iterations {its.tolist()}, x vs oracle {diff.max():.2e}")
    assert diff.max() <= 1e-7
