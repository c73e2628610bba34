"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Kernel level: B^{-1} (Section 5.2), C^{-1}, S~^{-1} (Eq. 4.7) and the full
apply M^{-1} (Eq. 4.1) on the same seeded inputs, element by element, with the
low-rank pairs handed over from the oracle (they are ordering independent as
Z_k = L^{-T} U_k, Proposition 4.3).  End to end: the GPU's own Lanczos Ritz
values and PCG iteration counts against the oracle's.

Tolerances (FP64 path): 1e-10 relative (max-norm) on every apply; the band
solve uses explicitly inverted triangular blocks, whose rounding is bounded by
kappa(D_J) eps ~ 1e-13 on these problems.  Mixed path (FP32 apply): the
probabilistic bound 4 sqrt(N) u of ``tests/tolerances.py`` (N the longest sum).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import slrgen
from oracle.slr_oracle import SLR as OracleSLR, THETA_LAMBDA_K1, THETA_ZERO, BSolver, slr_pcg, split_blocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1505_04340_gb300 import SLR  # noqa: E402

from tolerances import TOL64, tol32  # noqa: E402


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def cu(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


PROBLEMS = {
    # name: (dims, boxes, k, kind, coef_range)
    "c1-lap32": ((32, 32), (2, 2), 8, "laplacian", None),
    "fv-ragged": ((61, 47), (3, 4), 8, "fv", (1e-3, 1e3)),
    "3d-lap": ((20, 19, 18), (3, 2, 2), 8, "laplacian", None),
    "3d-wide": ((36, 36, 12), (2, 2, 1), 6, "laplacian", None),      # plane width 289 > 256 threads
    "one-part": ((20, 20), (1, 1), 4, "laplacian", None),            # no interface at all
}


# band-layout cases run only by the ring/split test: 14 x 14 planes split in 2 or
# 4 slices, where the upper and lower blocks break into different chunk counts
EXTRA = {
    "3d-196": ((30, 30, 8), (2, 2, 1), 6, "laplacian", None),
}


def make(name, nrhs=1):
    dims, boxes, k, kind, cr = PROBLEMS[name] if name in PROBLEMS else EXTRA[name]
    return slrgen.make_problem(name, dims, boxes, k, kind=kind, coef_range=cr, nrhs=nrhs)


_oracles = {}


def oracle(name, theta_mode=THETA_LAMBDA_K1):
    key = (name, theta_mode)
    if key not in _oracles:
        P = make(name)
        _oracles[key] = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, P.lanczos_steps,
                                  theta_mode=theta_mode)
    return _oracles[key]


def gpu_handle(P, precision="fp64", nrhs_max=4, theta="lambda_k1", **kw):
    return SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps,
               theta=theta, precision=precision, nrhs_max=nrhs_max, **kw)


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("factor", ["auto", "host"])
def test_bsolve_parity(name, precision, factor):
    """B^{-1} with the B_i factored on the device (planes up to 256 wide; the 324-wide
    3-D case falls back to the host) and on the host."""
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P, precision, band_factor=factor)
    inf = g.get_info()
    W = max(b for b in slrgen_plane_widths(P))
    assert inf["band_on_device"] == (1 if factor == "auto" and 0 < W <= 256 else 0)
    assert np.array_equal(g.perm(), o.order.perm)
    nI = o.order.n_I
    f = np.random.default_rng(1).standard_normal((nI, 3))
    t = g.bsolve(cu(f)).cpu().numpy()
    want = o.bsolve.solve(f)
    assert rel(t, want) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))


def slrgen_plane_widths(P):
    """Half-bandwidth of each B_i in DD order (natural order inside each box)."""
    A = sp.csr_matrix((P.val, P.colind, P.rowptr))
    out = [0]
    for q in range(P.nparts):
        idx = np.flatnonzero(P.part == q)
        inner = [i for i in idx if all(P.part[j] == q for j in A.indices[A.indptr[i]:A.indptr[i + 1]])]
        if not inner:
            continue
        B = A[sorted(inner)][:, sorted(inner)].tocoo()
        out.append(int(np.max(np.abs(B.row - B.col))) if B.nnz else 0)
    return out


def test_device_band_factor_matches_host_factor():
    """The device factorization and the host's band Cholesky give the same B solves
    to rounding (both exact Cholesky factors, different operation orders)."""
    P = make("3d-lap")
    f = cu(np.random.default_rng(5).standard_normal((gpu_handle(P).info["n_interior"], 2)))
    td = gpu_handle(P, band_factor="auto").bsolve(f).cpu().numpy()
    th = gpu_handle(P, band_factor="host").bsolve(f).cpu().numpy()
    assert rel(td, th) <= 1e-12


def test_device_band_factor_detects_non_spd_block():
    from paper_1505_04340_gb300.slr import SLRError
    rp, ci, v = slrgen.laplacian((6, 5))
    v = v.copy()
    diag = np.array([q for i in range(30) for q in range(rp[i], rp[i + 1]) if ci[q] == i])
    v[diag[7]] = -4.0                                # an interior node of part 0 loses positivity
    part = slrgen.box_partition((6, 5), (2, 1))
    with pytest.raises(SLRError, match="SLR_ERR_NOT_SPD"):
        SLR(rp, ci, v, part, 2, k=2, lanczos_steps=4)


@pytest.mark.parametrize("name,split,slots,nt", [("3d-196", 2, 5, 512), ("3d-196", 4, 5, 512), ("3d-196", 1, 2, 512),
                                                  ("3d-196", 2, 8, 512), ("3d-wide", 2, 8, 512), ("3d-wide", 4, 3, 512),
                                                  ("fv-ragged", 1, 8, 512), ("fv-ragged", 2, 2, 512),
                                                  ("3d-196", 2, 2, 256), ("3d-196", 1, 3, 256),
                                                  ("3d-wide", 2, 2, 256), ("fv-ragged", 1, 2, 256),
                                                  ("fv-ragged", 1, 2, 32), ("c1-lap32", 1, 2, 32)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bsolve_ring_and_split(name, split, slots, nt, precision):
    """B^{-1} with the factor streamed through 2..8 buffers, 1, 2 or 4 CTAs per subdomain,
    and CTAs of 512 or 256 threads, or one warp per subdomain (planes of at most 64 rows)."""
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P, precision, band_split=split, band_slots=slots, band_threads=nt)
    assert g.get_info()["band_threads"] == nt
    f = np.random.default_rng(2).standard_normal((o.order.n_I, 4))
    t = g.bsolve(cu(f)).cpu().numpy()
    assert rel(t, o.bsolve.solve(f)) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warp_band_solve_column_alone_equals_block(precision):
    """The warp-per-subdomain band solve (the default for planes of at most 64 rows):
    parity with the oracle, and a column solved alone equals its column of a block of
    five (one launch of four columns, then one of one) bit for bit."""
    P = make("fv-ragged")
    o = oracle("fv-ragged")
    g = gpu_handle(P, precision, nrhs_max=5)
    assert g.get_info()["band_threads"] == 32
    f = np.random.default_rng(9).standard_normal((o.order.n_I, 5))
    t = g.bsolve(cu(f)).cpu().numpy()
    assert rel(t, o.bsolve.solve(f)) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))
    for c in (0, 3, 4):
        assert np.array_equal(g.bsolve(cu(f[:, c])).cpu().numpy(), t[:, c]), c


def test_warp_band_solve_needs_narrow_planes():
    """band_threads = 32 asks for a warp per subdomain; planes wider than 64 rows keep
    the automatic CTA size."""
    g = gpu_handle(make("3d-wide"), "fp64", band_threads=32)             # planes of 289 rows
    assert g.get_info()["band_threads"] in (256, 512)


@pytest.mark.parametrize("name", ["fv-ragged", "3d-lap"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("factor", ["auto", "host"])
def test_band_order_is_bitwise_neutral(name, precision, factor):
    """The launch order of the subdomain clusters (subdomains of unequal work here)
    changes only which subdomains share SMs: B^{-1}, the Ritz values and the apply
    are the same bit for bit in every order, with the factor packed on the device
    (blocks located by subdomain id) or on the host."""
    P = make(name)
    f = cu(np.random.default_rng(4).standard_normal((oracle(name).order.n_I, 3)))
    r = cu(np.random.default_rng(5).standard_normal((P.rowptr.size - 1, 2)))
    ref = None
    for order in (1, 2, 3):
        g = gpu_handle(P, precision, band_factor=factor, band_order=order, band_split=2)
        got = (g.bsolve(f).cpu().numpy(), np.asarray(g.ritz()), g.apply(r).cpu().numpy())
        tol = TOL64 if precision == "fp64" else tol32(g.get_info())
        g.close()
        if ref is None:
            ref = got
            assert rel(got[0], oracle(name).bsolve.solve(f.cpu().numpy())) <= tol
        else:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), order


@pytest.mark.parametrize("name", [n for n in PROBLEMS if n != "one-part"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("zone", [True, False])
def test_csolve_parity(name, precision, persistent, zone):
    """C^{-1} by the per-level kernels and the persistent one (one cooperative launch per
    direction), with the factor's top levels solved by their explicit inverse or level by level."""
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P, precision, nrhs_max=5, c_persistent=persistent, c_top_zone=zone)
    if not zone:
        assert g.get_info()["c_top_levels"] == 0
    gg = np.random.default_rng(2).standard_normal((o.order.s, 5))
    y = g.csolve(cu(gg)).cpu().numpy()
    assert rel(y, o.cfac.solve(gg)) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))
    # a column alone gives the same numbers as in the block: column 1 is solved in a
    # block of four right-hand sides, column 4 after it, on its own
    for c in (1, 4):
        assert np.array_equal(g.csolve(cu(gg[:, c])).cpu().numpy(), y[:, c]), c


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_csolve_medium_with_fused_levels(precision):
    """C^{-1} on a 40^3 Laplacian with 4^3 boxes (s = 24,696): its two lowest levels
    hold more than 152 small supernodes each and run as fused one-CTA-per-supernode
    steps; both the per-level and the persistent path against the oracle's factor."""
    from oracle.slr_oracle import dd_order, split_blocks, CFactor
    P = slrgen.make_problem("m40", (40, 40, 40), (4, 4, 4), 4)
    order = dd_order(P.rowptr, P.colind, P.part, P.nparts)
    C = split_blocks(P.rowptr, P.colind, P.val, order)[2]
    want_fn = CFactor(C, route="sparse").solve
    gg = np.random.default_rng(6).standard_normal((order.s, 2))
    want = want_fn(gg)
    for persistent in (False, True):
        for zone in (True, False):
            g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=2, lanczos_steps=4, precision=precision,
                    nrhs_max=2, c_persistent=persistent, c_top_zone=zone)
            inf = g.get_info()
            # the zone takes some top levels but leaves level steps below it
            assert (0 < inf["c_top_levels"] < inf["c_levels"]) if zone else inf["c_top_levels"] == 0
            y = g.csolve(cu(gg)).cpu().numpy()
            assert rel(y, want) <= (TOL64 if precision == "fp64" else tol32(g.get_info())), (persistent, zone)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("persistent", [False, True])
def test_csolve_wide_block_fused_levels(precision, persistent):
    """C^{-1} of a block of 11 right-hand sides on the 40^3 problem: the fused small
    levels take blocks of 8 or more through their tiled paths (a group of 8 and a
    ragged group of 3, padded).  Parity with the oracle's factor, and a column solved
    alone (by the row-per-thread paths) equals its column of the block bit for bit."""
    from oracle.slr_oracle import dd_order, split_blocks, CFactor
    P = slrgen.make_problem("m40", (40, 40, 40), (4, 4, 4), 4)
    order = dd_order(P.rowptr, P.colind, P.part, P.nparts)
    C = split_blocks(P.rowptr, P.colind, P.val, order)[2]
    gg = np.random.default_rng(12).standard_normal((order.s, 11))
    want = CFactor(C, route="sparse").solve(gg)
    g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=2, lanczos_steps=4, precision=precision,
            nrhs_max=11, c_persistent=persistent, c_top_zone=False)
    y = g.csolve(cu(gg)).cpu().numpy()
    assert rel(y, want) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))
    for c in (0, 9, 10):
        assert np.array_equal(g.csolve(cu(gg[:, c])).cpu().numpy(), y[:, c]), c
    g.close()


def test_pcg_with_persistent_c_solve_matches_per_level():
    P = make("3d-lap")
    b = cu(P.b[:, 0])
    x1, it1, _, s1 = gpu_handle(P).pcg(b)
    x2, it2, _, s2 = gpu_handle(P, c_persistent=True).pcg(b)
    assert s1 == s2 == 0 and abs(int(it1[0]) - int(it2[0])) <= 1
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("name", [n for n in PROBLEMS if n != "one-part"])
@pytest.mark.parametrize("theta_mode", [THETA_LAMBDA_K1, THETA_ZERO])
def test_stilde_and_apply_parity_with_oracle_pairs(name, theta_mode):
    P = make(name)
    o = oracle(name, theta_mode)
    g = gpu_handle(P, theta="lambda_k1" if theta_mode == THETA_LAMBDA_K1 else "zero")
    g.set_lowrank(o.Z(), o.lam, o.theta)
    gg = np.random.default_rng(3).standard_normal((o.order.s, 2))
    assert rel(g.stilde_solve(cu(gg)).cpu().numpy(), o.stilde_inv(gg)) <= TOL64
    r = np.random.default_rng(4).standard_normal((P.n, 3))
    z = g.apply(cu(r)).cpu().numpy()
    assert rel(z, o.apply(r)) <= TOL64
    # one column at a time gives the same numbers as the block (fixed-order arithmetic)
    z0 = g.apply(cu(r[:, 0])).cpu().numpy()
    assert np.array_equal(z0, z[:, 0])


@pytest.mark.parametrize("name", ["c1-lap32", "fv-ragged", "3d-lap"])
def test_mixed_apply_close_to_oracle(name):
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P, "mixed")
    g.set_lowrank(o.Z(), o.lam, o.theta)
    r = np.random.default_rng(5).standard_normal(P.n)
    assert rel(g.apply(cu(r)).cpu().numpy(), o.apply(r)) <= tol32(g.get_info())


def test_get_lowrank_roundtrip():
    P = make("fv-ragged")
    o = oracle("fv-ragged")
    g = gpu_handle(P)
    g.set_lowrank(o.Z(), o.lam, o.theta)
    Z, lam, th = g.get_lowrank()
    assert rel(Z, o.Z()) <= 1e-10
    assert np.allclose(lam[:P.k], o.lam) and th == o.theta


def test_full_rank_exact_eigenpairs_give_one_iteration():
    """k = s exact pairs make S~ = S and M = A: PCG converges in one step (Section 4)."""
    P = make("c1-lap32")
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 10 ** 6, eig="dense")
    g = gpu_handle(P)
    g.set_lowrank(o.Z(), o.lam, 0.0)
    A = sp.csr_matrix((P.val, P.colind, P.rowptr))
    x = np.random.default_rng(6).standard_normal(P.n)
    App = o.App
    z = g.apply(cu(App @ x)).cpu().numpy()
    assert rel(z, x) <= 1e-9
    xs, its, res, st = g.pcg(cu(P.b[:, 0]))
    assert st == 0 and its[0] == 1
    del A


@pytest.mark.parametrize("name", ["c1-lap32", "fv-ragged", "3d-lap"])
def test_lanczos_ritz_values_match(name):
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P)
    rg = g.ritz()
    ro = o.ritz_values
    assert len(rg) == len(ro)
    # converged extreme Ritz values agree; near-multiple pairs converge at a
    # rate set by rounding, so only the leading well-resolved ones are compared
    lead = 5 if name != "fv-ragged" else P.k
    assert np.abs(rg[:lead] - ro[:lead]).max() <= 1e-8
    assert rg.max() < 1.0 and rg.min() > -1e-12


@pytest.mark.parametrize("name", ["c1-lap32", "fv-ragged", "3d-lap", "one-part"])
@pytest.mark.parametrize("theta", ["lambda_k1", "zero"])
def test_pcg_end_to_end(name, theta):
    """SLR-PCG (Section 6) against the oracle's.

    With the oracle's low-rank pairs imported both runs apply the same
    preconditioner, so their CG iterates agree: same iteration count (+-1) and
    solutions within a hundredth of their own error.  With the GPU's own Lanczos pairs (near-degenerate
    Ritz pairs converge at a rate set by rounding, Section 5.1) the iteration
    count stays within one and the solution is as accurate as the oracle's."""
    P = make(name, nrhs=2)
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, P.lanczos_steps,
                  theta_mode=THETA_LAMBDA_K1 if theta == "lambda_k1" else THETA_ZERO)
    xo, its_o, _, _ = slr_pcg(o, P.b)
    A = sp.csr_matrix((P.val, P.colind, P.rowptr))
    # same preconditioner
    g = gpu_handle(P, theta=theta)
    g.set_lowrank(o.Z(), o.lam, o.theta)
    x, its, relres, st = g.pcg(cu(P.b))
    assert st == 0 and np.all(relres <= 1e-8)
    assert np.all(np.abs(its - np.array(its_o)) <= 1), (its, its_o)
    err_o = np.linalg.norm(xo - P.xstar) / np.linalg.norm(P.xstar)
    if np.array_equal(its, its_o):
        # same operator in another summation order: the iterates agree to within 1%
        # of the solution's own error (CG amplifies rounding by about cond(A))
        assert rel(x.cpu().numpy(), xo) <= max(1e-10, 1e-2 * err_o)
    # own Lanczos pairs
    g = gpu_handle(P, theta=theta)
    x, its, relres, st = g.pcg(cu(P.b))
    assert st == 0 and np.all(relres <= 1e-8)
    assert np.all(np.abs(its - np.array(its_o)) <= 1), (its, its_o)
    xn = x.cpu().numpy()
    assert np.linalg.norm(P.b - A @ xn) <= 2.2e-8 * np.linalg.norm(P.b)
    err = np.linalg.norm(xn - P.xstar) / np.linalg.norm(P.xstar)
    assert err <= max(1e-7, 10 * err_o), (err, err_o)


@pytest.mark.parametrize("name", ["c1-lap32", "3d-lap", "fv-ragged"])
@pytest.mark.parametrize("flexible", [False, True])
def test_mixed_pcg_reaches_1e8(name, flexible):
    """FP32 apply, FP64 outer CG: 1e-8 residual, solution within 1e-7 of the FP64 oracle.

    A 1e-8 residual fixes x only to about cond(A) 1e-8; where that exceeds 1e-7
    (the FV problem with 1e6 coefficient contrast) the mixed solution must be
    no farther from the oracle's than the oracle's is from x*."""
    P = make(name, nrhs=1)
    o = oracle(name)
    xo, its_o, _, _ = slr_pcg(o, P.b)
    g = gpu_handle(P, "mixed", flexible_cg=flexible)
    x, its, relres, st = g.pcg(cu(P.b[:, 0]))
    assert st == 0 and relres[0] <= 1e-8
    A = sp.csr_matrix((P.val, P.colind, P.rowptr))
    xn = x.cpu().numpy()
    assert np.linalg.norm(P.b[:, 0] - A @ xn) <= 2e-8 * np.linalg.norm(P.b[:, 0])
    own = np.linalg.norm(xo[:, 0] - P.xstar[:, 0]) / np.linalg.norm(P.xstar[:, 0])
    diff = np.linalg.norm(xn - xo[:, 0]) / np.linalg.norm(xo[:, 0])
    assert diff <= max(1e-7, own), (diff, own)
    if name != "fv-ragged":
        assert diff <= 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_loop_equals_host_loop(precision):
    """The CUDA-graph CG loop runs the same kernels in the same order as the host loop."""
    P = make("3d-lap", nrhs=3)
    a = gpu_handle(P, precision, flexible_cg=(precision == "mixed"))
    b = gpu_handle(P, precision, flexible_cg=(precision == "mixed"), host_loop=True)
    xa, ia, ra, sa = a.pcg(cu(P.b))
    xb, ib, rb, sb = b.pcg(cu(P.b))
    assert sa == sb == 0 and np.array_equal(ia, ib)
    assert torch.equal(xa, xb) and np.array_equal(ra, rb)
    xa2, ia2, _, _ = a.pcg(cu(P.b))                 # cached graph, second launch
    assert torch.equal(xa, xa2) and np.array_equal(ia, ia2)


def test_pcg_rhs_zero_and_maxit():
    P = make("c1-lap32")
    g = gpu_handle(P)
    x, its, res, st = g.pcg(cu(np.zeros(P.n)))
    assert st == 0 and its[0] == 0 and float(x.abs().max()) == 0.0
    x, its, res, st = g.pcg(cu(P.b[:, 0]), maxit=2)
    assert st == 5 and its[0] == 2 and res[0] > 1e-8


@pytest.mark.slow
def test_full_size_3d_laplace_64_properties():
    """3-D 64^3, 4x4x4 boxes, k=32: properties that hold at any size, plus sampled blocks."""
    P = slrgen.config2()
    g = gpu_handle(P, nrhs_max=2)
    from oracle.slr_oracle import dd_order
    order = dd_order(P.rowptr, P.colind, P.part, P.nparts)
    assert np.array_equal(g.perm(), order.perm)
    Bi, E, C, App = split_blocks(P.rowptr, P.colind, P.val, order)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(order.n_I)
    t = g.bsolve(cu(f)).cpu().numpy()
    for q in (0, 21, 63):                     # sampled subdomains through the oracle
        a, b = order.int_off[q], order.int_off[q + 1]
        want = BSolver([Bi[q]], np.array([0, b - a])).solve(f[a:b])
        assert rel(t[a:b], want) <= TOL64
    gg = rng.standard_normal(order.s)
    y = g.csolve(cu(gg)).cpu().numpy()
    assert np.linalg.norm(C @ y - gg) <= 1e-12 * np.linalg.norm(gg) * 10
    r1, r2 = rng.standard_normal(P.n), rng.standard_normal(P.n)
    z1 = g.apply(cu(r1)).cpu().numpy()
    z2 = g.apply(cu(r2)).cpu().numpy()
    assert abs(z1 @ r2 - z2 @ r1) <= 1e-10 * abs(z1 @ r2)      # M^{-1} symmetric
    assert z1 @ r1 > 0
    x, its, relres, st = g.pcg(cu(P.b[:, 0]))
    A = sp.csr_matrix((P.val, P.colind, P.rowptr))
    assert st == 0 and np.linalg.norm(P.b[:, 0] - A @ x.cpu().numpy()) <= 2e-8 * np.linalg.norm(P.b[:, 0])


@pytest.mark.parametrize("name", ["3d-lap", "3d-196"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_handle(name, precision):
    """Setup with autotune: the choice is reported, cached for the next handle of the
    same shape, and the tuned operator keeps parity with the oracle."""
    P = make(name)
    o = oracle(name)
    fl = precision == "mixed"
    g = gpu_handle(P, precision, autotune=True, flexible_cg=fl)
    inf = g.get_info()
    assert inf["tuned"] == 1 and inf["band_split"] in (1, 2, 4) and inf["band_slots"] in (2, 3, 4)
    g2 = gpu_handle(P, precision, autotune=True, flexible_cg=fl)
    inf2 = g2.get_info()
    assert inf2["tune_seconds"] == 0.0                 # taken from the cache
    assert (inf2["band_split"], inf2["band_slots"], inf2["c_persistent"]) == \
           (inf["band_split"], inf["band_slots"], inf["c_persistent"])
    f = np.random.default_rng(8).standard_normal((o.order.n_I, 2))
    assert rel(g.bsolve(cu(f)).cpu().numpy(), o.bsolve.solve(f)) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))
    gg = np.random.default_rng(9).standard_normal((o.order.s, 2))
    assert rel(g.csolve(cu(gg)).cpu().numpy(), o.cfac.solve(gg)) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))
    b = cu(P.b[:, 0])
    _, it1, _, s1 = g.pcg(b)
    _, it2, _, s2 = gpu_handle(P, precision, flexible_cg=fl).pcg(b)
    assert s1 == 0 and s2 == 0 and abs(int(it1[0]) - int(it2[0])) <= 1


@pytest.mark.parametrize("name,K", [("c1-lap32", 3), ("c1-lap32", 10), ("3d-lap", 4), ("fv-ragged", 20)])
def test_target_condition_number_rank(name, K):
    """Rank rule of Section 4 (Eq. condk): the GPU keeps the same number of Ritz values
    above 1 - 1/K as the oracle, and a tighter K never needs more iterations."""
    P = make(name)
    cap = 40
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, cap, P.lanczos_steps, target_kappa=K)
    near = np.abs(o.ritz_values - (1 - 1 / K)).min()
    if near < 1e-6:
        pytest.skip("a Ritz value sits on the threshold")
    g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=cap, lanczos_steps=P.lanczos_steps, target_kappa=K)
    assert g.get_info()["k"] == o.k
    b = cu(P.b[:, 0])
    _, it_k, _, st = g.pcg(b)
    loose = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=cap, lanczos_steps=P.lanczos_steps,
                target_kappa=4 * K)
    _, it_loose, _, st2 = loose.pcg(b)
    assert st == 0 and st2 == 0
    assert loose.get_info()["k"] <= o.k and int(it_k[0]) <= int(it_loose[0]) + 1


@pytest.mark.parametrize("name", ["c1-lap32", "3d-lap"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_add_vectors_matches_oracle_improvement(name, precision):
    """Section 5.3: vectors from a deflated Lanczos run are appended, the old ones kept;
    the Ritz values match the oracle's improved preconditioner and PCG gets no slower."""
    P = make(name)
    k0, j = 2, 4
    o = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k0, 20)
    o.improve(j, lanczos_steps=24)
    fl = precision == "mixed"
    g = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=k0, lanczos_steps=20, precision=precision,
            nrhs_max=1, flexible_cg=fl)
    b = cu(P.b[:, 0])
    _, it0, _, st0 = g.pcg(b)
    Z0, _, _ = g.get_lowrank()
    assert g.add_vectors(j, lanczos_steps=24) == j
    assert g.get_info()["k"] == k0 + j
    Z1, lam, th = g.get_lowrank()
    assert np.abs(Z1[:, :k0] - Z0).max() <= 1e-12 * np.abs(Z0).max()     # old vectors kept
    assert np.allclose(lam[:k0 + j], o.lam, rtol=1e-8, atol=1e-10), (lam[:k0 + j], o.lam)
    assert th == pytest.approx(o.theta, rel=1e-8)
    _, it1, _, st1 = g.pcg(b)
    its_o = int(np.atleast_1d(slr_pcg(o, P.b[:, 0])[1])[0])
    assert st0 == st1 == 0 and int(it1[0]) <= int(it0[0]) and abs(int(it1[0]) - its_o) <= 1


@pytest.mark.parametrize("name", ["3d-lap", "3d-wide", "fv-ragged"])
@pytest.mark.parametrize("nt", [512, 256])
def test_bsolve_wide_rhs_block_mixed(name, nt):
    """FP32 B^{-1} on 11 right-hand sides (column groups of 8, 2 and 1 per CTA, where they
    fit): parity with the oracle, and each column alone equals its column of the block."""
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P, "mixed", nrhs_max=11, band_threads=nt)
    f = np.random.default_rng(12).standard_normal((o.order.n_I, 11))
    t = g.bsolve(cu(f)).cpu().numpy()
    assert rel(t, o.bsolve.solve(f)) <= tol32(g.get_info())
    for c in (0, 7, 8, 10):
        assert np.array_equal(g.bsolve(cu(f[:, c])).cpu().numpy(), t[:, c]), c


@pytest.mark.parametrize("name", ["c1-lap32", "fv-ragged", "3d-lap"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zform_apply_matches_oracle(name, precision):
    """The Z-form apply (Proposition 4.3, Eq. 4.15: (1-theta)^{-1} C^{-1} g' + Z_k (d o Z_k^T g'),
    the product Z_k^T g' on a second stream beside the C solves) against the oracle's
    Z-form apply with the same pairs, one and several columns."""
    P = make(name)
    o = oracle(name)
    g = gpu_handle(P, precision, zform=True)
    g.set_lowrank(o.Z(), o.lam, o.theta)
    r = np.random.default_rng(9).standard_normal((P.n, 3))
    z = g.apply(cu(r)).cpu().numpy()
    zo = np.stack([o.apply(r[:, j], zform=True) for j in range(3)], axis=1)
    assert rel(z, zo) <= (TOL64 if precision == "fp64" else tol32(g.get_info()))
    z0 = g.apply(cu(r[:, 0])).cpu().numpy()
    assert np.array_equal(z0, z[:, 0])


@pytest.mark.parametrize("name", ["c1-lap32", "3d-lap"])
def test_zform_pcg_matches_uform(name):
    """The same preconditioner in both forms: PCG iteration counts equal (±1), both to 1e-8."""
    P = make(name)
    b = cu(P.b[:, 0])
    hu = gpu_handle(P)
    hz = gpu_handle(P, zform=True)
    xu, itu, relu, stu = hu.pcg(b)
    xz, itz, relz, stz = hz.pcg(b)
    assert stu == 0 and stz == 0 and relz[0] <= 1e-8
    assert abs(int(itu[0]) - int(itz[0])) <= 1
    assert rel(xz.cpu().numpy(), xu.cpu().numpy()) <= 1e-7
