"""Pins of the CPU oracle to the mathematics and to the paper's printed numbers.

Each test checks the oracle against something other than itself: published
test vectors, closed forms (Proposition 3.3), printed values (figure of
kappa(theta) in Section 4), lemmas and propositions (Lemma 3.1, Lemma 3.2,
Propositions 4.1-4.3), dense brute force on tiny inputs, and library solves.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import slrgen
from oracle import brute
from oracle.slr_oracle import (SLR, THETA_LAMBDA_K1, THETA_ZERO, BandCholesky, BandLU, BSolver, CFactor,
                               dd_order, gmres, h_apply, lanczos, pcg, ritz, slr_gmres, slr_pcg, split_blocks)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            key, *val = line.split()
            out[key] = float(val[0]) if val else key
    return out


def small_fv(dims=(20, 18), boxes=(3, 2), k=6, seed=7, lo=1e-2, hi=1e2):
    return slrgen.make_problem("fv", dims, boxes, k, kind="fv", coef_range=(lo, hi),
                               matrix_seed=seed)


# ---------------------------------------------------------------- inputs

def test_splitmix64_published_vectors():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = [int(x) for x in slrgen.splitmix64(0, 3)]
    assert got == want
    # counter-based: a window of the stream equals the slice of a longer draw
    assert np.array_equal(slrgen.splitmix64(5, 4, start=3), slrgen.splitmix64(5, 7)[3:])


def test_generators_shape_and_symmetry():
    rp, ci, v = slrgen.laplacian((5, 4, 3))
    A = sp.csr_matrix((v, ci, rp)).toarray()
    assert np.array_equal(A, A.T)
    assert np.allclose(np.diag(A), 6.0)
    # interior row of the 7-point stencil sums to zero
    assert abs(A[1 + 5 * 1 + 20 * 1].sum()) < 1e-15
    rp, ci, v = slrgen.diffusion_fv((6, 5), slrgen.loguniform(3, 30, 1e-3, 1e3))
    A = sp.csr_matrix((v, ci, rp)).toarray()
    assert np.allclose(A, A.T)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    part = slrgen.box_partition((32, 32), (2, 2))
    assert np.bincount(part).tolist() == [256] * 4


# ---------------------------------------------------------------- Section 2.1

def _iface_count_boxes(dims, boxes):
    """Interface size of a box partition by inclusion-exclusion over the axes."""
    sets = []
    for ax, (nd, b) in enumerate(zip(dims, boxes)):
        cuts = [c * nd // b for c in range(1, b)]
        cols = set()
        for c in cuts:
            cols |= {c - 1, c}
        sets.append(len(cols))
    n = np.prod(dims)
    frac = [s / d for s, d in zip(sets, dims)]
    # |X u Y u Z| = n (1 - prod(1 - frac))
    return int(round(n * (1.0 - np.prod([1.0 - f for f in frac]))))


@pytest.mark.parametrize("dims,boxes", [((32, 32), (2, 2)), ((30, 17), (3, 2)),
                                        ((12, 11, 10), (2, 3, 2)), ((16, 16, 16), (4, 4, 4))])
def test_dd_order_interface_and_permutation(dims, boxes):
    rp, ci, v = slrgen.laplacian(dims)
    part = slrgen.box_partition(dims, boxes)
    p = int(np.prod(boxes))
    o = dd_order(rp, ci, part, p)
    assert o.s == _iface_count_boxes(dims, boxes)
    if dims == (32, 32):
        assert o.s == 124
    assert np.array_equal(np.sort(o.perm), np.arange(len(part)))
    # interiors of part q, then interfaces of part q, each ascending
    for q in range(p):
        seg = o.perm[o.int_off[q]:o.int_off[q + 1]]
        assert np.all(part[seg] == q) and np.all(np.diff(seg) > 0)
        seg = o.perm[o.n_I + o.ifc_off[q]:o.n_I + o.ifc_off[q + 1]]
        assert np.all(part[seg] == q) and np.all(np.diff(seg) > 0)
    Bi, E, C, App = split_blocks(rp, ci, v, o)
    # B is block diagonal: interior nodes of different parts never couple
    B = App[:o.n_I, :o.n_I].tocoo()
    owner = np.searchsorted(o.int_off, np.arange(o.n_I), side="right") - 1
    assert np.all(owner[B.row] == owner[B.col])


# ---------------------------------------------------------------- Section 5.2

@pytest.mark.parametrize("m,w", [(37, 5), (64, 8), (10, 1), (9, 12)])
def test_band_cholesky_solve_vs_dense(m, w):
    rng = np.random.default_rng(m * 100 + w)
    M = np.zeros((m, m))
    for d in range(1, min(w, m - 1) + 1):
        off = rng.uniform(-1, 0, m - d)
        M += np.diag(off, d) + np.diag(off, -d)
    M += np.diag(np.abs(M).sum(1) + rng.uniform(0.1, 1, m))
    bc = BandCholesky(sp.csr_matrix(M))
    f = rng.standard_normal((m, 3))
    assert np.allclose(bc.solve(f), np.linalg.solve(M, f), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- Section 3.1

def test_cfactor_dense_and_sparse_routes_agree():
    P = small_fv((24, 22), (3, 3))
    o = dd_order(P.rowptr, P.colind, P.part, P.nparts)
    _, E, C, _ = split_blocks(P.rowptr, P.colind, P.val, o)
    fd, fs = CFactor(C, "dense"), CFactor(C, "sparse")
    Cd = C.toarray()
    I = np.eye(C.shape[0])
    for f in (fd, fs):
        # L L^T = C: L = L^{-1}-inverse applied to I, so check C L^{-T} L^{-1} = I
        Li = f.solve_L(I)
        assert np.allclose(Li @ Cd @ Li.T, I, atol=1e-11)
    g = np.random.default_rng(1).standard_normal(C.shape[0])
    assert np.allclose(fd.solve(g), np.linalg.solve(Cd, g), rtol=1e-11)
    assert np.allclose(fs.solve(g), np.linalg.solve(Cd, g), rtol=1e-11)


# ---------------------------------------------------------------- Section 3.2 (P8, P9)

def _two_domain(nx, ny):
    """Blocks of Eq. 3.6: Omega_1, Omega_2 (n_x x n_y each) and the 1-row separator."""
    rp, ci, v = slrgen.laplacian((nx, 2 * ny + 1))
    A = sp.csr_matrix((v, ci, rp))
    rows = np.arange(nx * (2 * ny + 1)) // nx
    u = np.where(rows != ny)[0]            # Omega_1 then Omega_2 in grid order
    g = np.where(rows == ny)[0]
    B = A[u][:, u].tocsr()
    E = A[u][:, g].tocsr()
    C = A[g][:, g].tocsr()
    half = nx * ny
    Bi = [B[:half, :half].tocsr(), B[half:, half:].tocsr()]
    return Bi, B, E, C, np.array([0, half, 2 * half])


@pytest.mark.parametrize("nx,ny", [(15, 7), (65, 32)])
def test_two_domain_closed_form(nx, ny):
    """Proposition 3.3: spectrum of the oracle's H equals zeta/(1+zeta)."""
    Bi, B, E, C, off = _two_domain(nx, ny)
    assert np.allclose(C.toarray(), np.diag(np.full(nx, 4.0)) - np.eye(nx, k=1) - np.eye(nx, k=-1))
    bs, cf = BSolver(Bi, off), CFactor(C, "dense")
    H = h_apply(np.eye(nx), E, bs, cf)
    lam = np.sort(np.linalg.eigvalsh((H + H.T) / 2))[::-1]
    want = np.sort(brute.two_domain_lambda(nx, ny))[::-1]
    assert np.allclose(lam, want, rtol=0, atol=1e-13)
    # gamma_k are the eigenvalues of S^{-1} - C^{-1} (Eq. 3.10), by brute force
    S = brute.schur(B.toarray(), E.toarray(), C.toarray())
    D = np.linalg.inv(S) - np.linalg.inv(C.toarray())
    g, _, _ = brute.gamma_two_domain(nx, ny)
    assert np.allclose(np.sort(np.linalg.eigvalsh(D)), np.sort(g), atol=1e-13)


def test_fig_kappa_printed_values():
    """The printed lambda_s, lambda_{k+1} and kappa of the figure in Section 4."""
    gold = _golden("fig_kappa.txt")
    nx, k = int(gold["nx"]), int(gold["k"])
    lam = np.sort(brute.two_domain_lambda(nx, 127))[::-1]
    assert abs(lam[-1] - gold["lambda_s"]) < 5e-6
    assert abs(lam[k] - gold["lambda_k1"]) < 5e-6
    kap = float(brute.kappa(0.5 * (lam[-1] + lam[k]), lam[-1], lam[k]))
    assert abs(kap - gold["kappa"]) < 5e-5


@pytest.mark.slow
def test_fig_kappa_through_oracle_h():
    """The same printed numbers from the oracle's own B, C solves at full size."""
    gold = _golden("fig_kappa.txt")
    nx, k = int(gold["nx"]), int(gold["k"])
    Bi, _, E, C, off = _two_domain(nx, 127)
    bs, cf = BSolver(Bi, off), CFactor(C, "dense")
    H = h_apply(np.eye(nx), E, bs, cf)
    lam = np.sort(np.linalg.eigvalsh((H + H.T) / 2))[::-1]
    assert abs(lam[-1] - gold["lambda_s"]) < 5e-6
    assert abs(lam[k] - gold["lambda_k1"]) < 5e-6
    assert abs((1 - lam[-1]) / (1 - lam[k]) - gold["kappa"]) < 5e-5


# ---------------------------------------------------------------- Section 3.1 lemmas (P2, P3)

@pytest.mark.parametrize("prob", ["lap", "fv"])
def test_lemmas_eigH_and_X(prob):
    P = slrgen.config1() if prob == "lap" else small_fv(lo=1e-3, hi=1e3)
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0)
    B, E, C = brute.dense_blocks(slr)
    H = slr.h_dense()
    assert np.allclose(H, H.T, atol=1e-13)
    lam = np.linalg.eigvalsh((H + H.T) / 2)
    assert lam.min() >= -1e-13 and lam.max() < 1.0          # Lemma 3.1
    assert np.allclose(np.sort(lam), np.sort(np.linalg.eigvalsh(brute.h_from_blocks(B, E, C))),
                       atol=1e-12)
    # Lemma 3.2 via Eq. 3.4: X = L^T (S^{-1} - C^{-1}) L has eigenvalues lambda/(1-lambda)
    S = brute.schur(B, E, C)
    L = np.linalg.cholesky(C)
    X = L.T @ (np.linalg.inv(S) - np.linalg.inv(C)) @ L
    assert np.allclose(np.sort(np.linalg.eigvalsh((X + X.T) / 2)), np.sort(lam / (1 - lam)),
                       rtol=1e-9, atol=1e-11)


# ---------------------------------------------------------------- Section 4 (P4, P5, P6, P7)

@pytest.mark.parametrize("theta_mode", [THETA_LAMBDA_K1, THETA_ZERO])
def test_prop_eigSS(theta_mode):
    """Proposition 4.1 with Eq. 4.12: eig(S S~^{-1}) = 1 (i<=k), (1-lambda_i)/(1-theta)."""
    P = small_fv()
    k = 5
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, theta_mode=theta_mode, eig="dense")
    B, E, C = brute.dense_blocks(slr)
    S = brute.schur(B, E, C)
    Sti = slr.stilde_inv(np.eye(S.shape[0]))
    sig = np.sort(np.linalg.eigvals(S @ Sti).real)
    lam = slr.ritz_values
    theta = lam[k] if theta_mode == THETA_LAMBDA_K1 else 0.0
    assert slr.theta == pytest.approx(theta)
    want = np.sort(np.concatenate([np.ones(k), (1 - lam[k:]) / (1 - theta)]))
    assert np.allclose(sig, want, rtol=1e-9, atol=1e-10)
    # Proposition 4.2: the condition number equals the piecewise formula
    kap = sig.max() / sig.min()
    assert kap == pytest.approx(float(brute.kappa(theta, lam[-1], lam[k])), rel=1e-8)


@pytest.mark.parametrize("K", [1.5, 3.0, 10.0, 40.0])
def test_rank_rule_bounds_condition_number(K):
    """Rank rule of Section 4 (Eq. condk): with exact eigenpairs, k = #{lambda_i > 1 - 1/K}
    (counted on an H formed densely from the blocks, not by the oracle) and, with
    theta = lambda_{k+1}, the condition number of S S~^{-1} is at most K."""
    P = small_fv()
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 10 ** 6, eig="dense", target_kappa=K)
    B, E, C = brute.dense_blocks(slr)
    lam = np.sort(np.linalg.eigvalsh(brute.h_from_blocks(B, E, C)))[::-1]
    assert not np.any(np.abs(lam - (1 - 1 / K)) < 1e-9)          # no tie at the threshold
    assert slr.k == int(np.sum(lam > 1 - 1 / K))
    S = brute.schur(B, E, C)
    sig = np.linalg.eigvals(S @ slr.stilde_inv(np.eye(S.shape[0]))).real
    assert sig.max() / sig.min() <= K * (1 + 1e-9)
    # the rule picks the smallest such rank: one vector fewer breaks the bound
    if slr.k > 0:
        fewer = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, slr.k - 1, eig="dense")
        sig2 = np.linalg.eigvals(S @ fewer.stilde_inv(np.eye(S.shape[0]))).real
        assert sig2.max() / sig2.min() > K


def test_rank_rule_with_lanczos_caps_at_k():
    """With Lanczos (Section 5.1) the rule counts Ritz values; the requested k is a cap."""
    P = slrgen.config1()
    full = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 8, lanczos_steps=40)
    lam = full.ritz_values
    K = 4.0
    want = min(8, int(np.sum(lam > 1 - 1 / K)))
    got = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 8, lanczos_steps=40, target_kappa=K)
    assert got.k == want and np.allclose(got.lam, lam[:want])
    assert got.theta == pytest.approx(lam[want])
    capped = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 2, lanczos_steps=40, target_kappa=1.05)
    assert capped.k == 2


@pytest.mark.parametrize("theta_mode", [THETA_LAMBDA_K1, THETA_ZERO])
def test_improve_by_deflation_adds_the_next_eigenpairs(theta_mode):
    """Section 5.3: with exact U_k, a full deflated Lanczos run appends exactly the next
    eigenpairs of H (a densely formed H, not the oracle's); the extended set keeps
    U orthonormal and gives Proposition 4.1's spectrum of S S~^{-1} for rank k + j."""
    P = small_fv()
    k, j = 3, 4
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, theta_mode=theta_mode, eig="dense")
    B, E, C = brute.dense_blocks(slr)
    lam = np.sort(np.linalg.eigvalsh(brute.h_from_blocks(B, E, C)))[::-1]
    s = len(lam)
    added = slr.improve(j, lanczos_steps=s - k)
    assert added == j and slr.k == k + j
    assert np.allclose(slr.lam, lam[:k + j], atol=1e-10)
    assert np.allclose(slr.U.T @ slr.U, np.eye(k + j), atol=1e-10)
    theta = lam[k + j] if theta_mode == THETA_LAMBDA_K1 else 0.0
    assert slr.theta == pytest.approx(theta, abs=1e-10)
    S = brute.schur(B, E, C)
    sig = np.sort(np.linalg.eigvals(S @ slr.stilde_inv(np.eye(s))).real)
    want = np.sort(np.concatenate([np.ones(k + j), (1 - lam[k + j:]) / (1 - theta)]))
    assert np.allclose(sig, want, rtol=1e-8, atol=1e-9)


def test_improve_with_lanczos_lowers_iterations():
    """Adding vectors to a Lanczos-built preconditioner keeps the old ones and helps PCG."""
    P = slrgen.config1()
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 2, lanczos_steps=20)
    U0 = slr.U.copy()
    its0 = slr_pcg(slr, P.b[:, 0])[1]
    slr.improve(6, lanczos_steps=40)
    assert slr.k == 8 and np.array_equal(slr.U[:, :2], U0)
    assert np.abs(slr.U[:, :2].T @ slr.U[:, 2:]).max() < 1e-10
    assert slr_pcg(slr, P.b[:, 0])[1] < its0


def test_prop_kappa_piecewise_sweep():
    lam = np.sort(brute.two_domain_lambda(40, 19))[::-1]
    k = 6
    for theta in np.linspace(0, 0.95, 40):
        sig = np.concatenate([np.ones(k), (1 - lam[k:]) / (1 - theta)])
        assert sig.max() / sig.min() == pytest.approx(float(brute.kappa(theta, lam[-1], lam[k])),
                                                      rel=1e-12)


@pytest.mark.parametrize("theta_mode", [THETA_LAMBDA_K1, THETA_ZERO])
def test_prop_skt_zform_equals_uform(theta_mode):
    """Proposition 4.3 holds for any orthonormal U_k, so also for Lanczos Ritz vectors."""
    P = small_fv()
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 6, lanczos_steps=20,
              theta_mode=theta_mode)
    g = np.random.default_rng(3).standard_normal((slr.order.s, 2))
    a, b = slr.stilde_inv(g), slr.stilde_inv_zform(g)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())
    r = np.random.default_rng(4).standard_normal(P.n)
    assert np.allclose(slr.apply(r), slr.apply(r, zform=True), rtol=1e-11, atol=1e-12)


def test_full_rank_gives_exact_inverse():
    """k = s with exact eigenpairs: S~ = S, M = A, PCG converges in one step."""
    P = slrgen.config1()
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 10 ** 6, eig="dense")
    assert slr.k == slr.order.s
    x = np.random.default_rng(5).standard_normal(P.n)
    assert np.allclose(slr.apply(slr.App @ x), x, rtol=1e-10, atol=1e-10)
    _, its, rel, ok = slr_pcg(slr, P.b[:, 0])
    assert its == [1] and ok[0]


def test_rank_zero_is_block_lu_with_C():
    """k = 0, theta = 0: S~ = C and M = [[I,0],[E^T B^{-1},I]] [[B,E],[0,C]] (Eq. 4.1)."""
    P = small_fv((14, 13), (2, 2))
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0, theta_mode=THETA_ZERO)
    B, E, C = brute.dense_blocks(slr)
    nI = B.shape[0]
    s = C.shape[0]
    L1 = np.block([[np.eye(nI), np.zeros((nI, s))], [E.T @ np.linalg.inv(B), np.eye(s)]])
    U1 = np.block([[B, E], [np.zeros((s, nI)), C]])
    r = np.random.default_rng(6).standard_normal(P.n)
    assert np.allclose(slr.apply(r), np.linalg.solve(L1 @ U1, r), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("theta_mode", [THETA_LAMBDA_K1, THETA_ZERO])
def test_apply_is_inverse_of_dense_M(theta_mode):
    """Eq. 4.1 formed densely from the blocks, M = [[B, E], [E^T, E^T B^{-1} E + S~]],
    with S~^{-1} = L^{-T} ((1-theta)^{-1} I + U_k ((I-Lambda_k)^{-1} - (1-theta)^{-1} I) U_k^T) L^{-1}
    (Eq. 4.7 with Eqs. 4.10-4.11) from a dense eigensolve of H (Eq. 3.2, dense Cholesky
    of C in DD order): the apply is M^{-1}.  Random coefficients keep lambda_k and
    lambda_{k+1} apart, so U_k is unique up to signs, which cancel."""
    P = small_fv()
    k = 5
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, theta_mode=theta_mode, eig="dense")
    B, E, C = brute.dense_blocks(slr)
    H = brute.h_from_blocks(B, E, C)
    w, V = np.linalg.eigh((H + H.T) / 2)
    lam, U = w[::-1], V[:, ::-1][:, :k]
    assert lam[k - 1] - lam[k] > 1e-6 * lam[0]
    theta = lam[k] if theta_mode == THETA_LAMBDA_K1 else 0.0
    Linv = np.linalg.inv(np.linalg.cholesky(C))
    G = np.eye(C.shape[0]) / (1 - theta) + U @ np.diag(1 / (1 - lam[:k]) - 1 / (1 - theta)) @ U.T
    St = np.linalg.inv(Linv.T @ G @ Linv)
    M = np.block([[B, E], [E.T, E.T @ np.linalg.solve(B, E) + St]])
    r = np.random.default_rng(8).standard_normal((P.n, 2))
    want = np.linalg.solve(M, r)
    assert np.allclose(slr.apply(r), want, rtol=1e-9, atol=1e-11 * np.abs(want).max())


def test_apply_symmetric_positive():
    """M^{-1} is symmetric (M = [[B,E],[E^T, E^T B^{-1} E + S~]]) and here positive definite."""
    P = small_fv()
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 6)
    Mi = slr.apply(np.eye(P.n))
    assert np.allclose(Mi, Mi.T, atol=1e-11 * np.abs(Mi).max())
    assert np.linalg.eigvalsh((Mi + Mi.T) / 2).min() > 0


# ---------------------------------------------------------------- Section 5.1

def test_lanczos_full_steps_reproduces_spectrum():
    P = small_fv(lo=1e-3, hi=1e3)
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0)
    s = slr.order.s
    H = slr.h_dense()
    a, b, V = lanczos(lambda v: H @ v, np.random.default_rng(8).standard_normal(s), s)
    lam, U = ritz(a, b, V)
    assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)
    ex = np.sort(np.linalg.eigvalsh((H + H.T) / 2))[::-1]
    assert np.allclose(lam[:10], ex[:10], atol=1e-11)
    res = np.linalg.norm(H @ U[:, :10] - U[:, :10] * lam[:10], axis=0)
    assert res.max() < 1e-10


def test_lanczos_start_vector_makes_ritz_ordering_invariant():
    """v_1 = L^{-1} C z makes Z_k = L^{-T} U_k independent of how C is factored."""
    P = small_fv((24, 22), (3, 3), k=4)
    kw = dict(lanczos_steps=30, seed=11)
    a = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 4, c_route="dense", **kw)
    b = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 4, c_route="sparse", **kw)
    assert np.allclose(a.ritz_values[:5], b.ritz_values[:5], rtol=1e-10)
    Za, Zb = a.Z(), b.Z()
    assert np.allclose(np.abs(np.sum(Za * Zb, 0) / np.sqrt(np.sum(Za * Za, 0) * np.sum(Zb * Zb, 0))),
                       1.0, atol=1e-8)


# ---------------------------------------------------------------- Section 6

def test_pcg_converges_and_rank_helps():
    P = slrgen.config1()
    its = {}
    for k in (0, 8):
        slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, P.lanczos_steps)
        x, it, rel, ok = slr_pcg(slr, P.b[:, 0])
        A = sp.csr_matrix((P.val, P.colind, P.rowptr))
        assert ok[0] and rel[0] <= 1e-8
        assert np.linalg.norm(P.b[:, 0] - A @ x) <= 2e-8 * np.linalg.norm(P.b[:, 0])
        its[k] = it[0]
    assert its[8] < its[0]


def test_pcg_identity_preconditioner_is_cg():
    """With M = I the iteration is plain CG: it terminates in <= n steps on SPD A."""
    rng = np.random.default_rng(9)
    Q = np.linalg.qr(rng.standard_normal((12, 12)))[0]
    A = Q @ np.diag(np.arange(1.0, 13.0)) @ Q.T
    b = rng.standard_normal(12)
    x, it, rel, ok = pcg(A, b, lambda r: r.copy(), tol=1e-12)
    assert ok and it <= 12 and np.allclose(A @ x, b, atol=1e-10)


def test_lanczos_three_term_recurrence_without_reorth():
    """Before orthogonality is lost the plain recurrence gives V^T H V = T (Section 5.1)."""
    P = small_fv()
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0)
    H = slr.h_dense()
    a, b, V = lanczos(lambda v: H @ v, np.random.default_rng(2).standard_normal(H.shape[0]), 6,
                      reorth_passes=0)
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    assert np.allclose(V.T @ H @ V, T, atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(6), atol=1e-12)


# ---------------------------------------------------------------------------
# Symmetric indefinite problems (Section 6, -Laplacian u - c u = f; SPD interface
# assumed, Section 1) and the GMRES(40) accelerator
# ---------------------------------------------------------------------------

def _shifted(dims, boxes, shift, k=8):
    return slrgen.make_problem("shifted", dims, boxes, k, shift=shift)


def test_shifted_problem_is_indefinite_with_spd_interface():
    """The test workload: A has negative eigenvalues, C (interface) is SPD and some B_i
    are indefinite, so the B solves need a symmetric indefinite factorisation."""
    P = _shifted((32, 32), (2, 2), 0.2)
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 4, indefinite=True)
    B, E, C = brute.dense_blocks(slr)
    assert np.linalg.eigvalsh(slr.App.toarray()).min() < 0
    assert np.linalg.eigvalsh(C).min() > 0
    assert np.linalg.eigvalsh(B).min() < 0


@pytest.mark.parametrize("m,w", [(40, 3), (64, 8)])
def test_band_lu_solve_vs_dense_indefinite(m, w):
    rng = np.random.default_rng(m)
    D = np.zeros((m, m))
    for d in range(1, w + 1):
        v = rng.standard_normal(m - d)
        D += np.diag(v, d) + np.diag(v, -d)
    D += np.diag(rng.uniform(-2, 2, m))                      # symmetric, indefinite
    f = rng.standard_normal((m, 3))
    got = BandLU(sp.csr_matrix(D)).solve(f)
    assert np.allclose(got, np.linalg.solve(D, f), rtol=1e-10, atol=1e-10)


def test_gmres_solves_nonsymmetric_system_and_restarts():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.4
    b = rng.standard_normal(n)
    want = np.linalg.solve(A, b)
    for restart in (60, 7):                                    # full and restarted
        x, its, rel, ok = gmres(sp.csr_matrix(A), b, lambda v: v, tol=1e-10, maxit=2000, restart=restart)
        assert ok and rel <= 1e-10
        assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) == pytest.approx(rel, rel=1e-6)
        assert np.allclose(x, want, rtol=1e-8, atol=1e-9)
    # without restarts GMRES terminates in at most n steps (exact arithmetic: the Krylov space is full)
    _, its, _, ok = gmres(sp.csr_matrix(A), b, lambda v: v, tol=1e-10, maxit=2000, restart=n)
    assert ok and its <= n
    # an exact preconditioner: one step
    Ainv = np.linalg.inv(A)
    _, its, rel, ok = gmres(sp.csr_matrix(A), b, lambda v: Ainv @ v, tol=1e-10)
    assert ok and its == 1


def test_gmres_minimises_residual_over_krylov_space():
    """At step j the GMRES iterate minimises ||b - A x|| over x in K_j (checked by a
    dense least-squares problem on the Krylov basis)."""
    rng = np.random.default_rng(4)
    n = 30
    A = np.diag(np.linspace(-1, 3, n)) + 0.1 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    for j in (3, 8):
        x, its, rel, _ = gmres(sp.csr_matrix(A), b, lambda v: v, tol=1e-14, maxit=j, restart=40)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(j)], axis=1)
        y, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
        best = np.linalg.norm(b - A @ K @ y) / np.linalg.norm(b)
        assert its == j and rel == pytest.approx(best, rel=1e-6)


@pytest.mark.parametrize("theta_mode", [THETA_LAMBDA_K1, THETA_ZERO])
def test_prop_eigSS_indefinite(theta_mode):
    """Proposition 4.1 is algebraic (S = L(I - H)L^T for any symmetric H): with an
    indefinite B, eig(S S~^{-1}) is still 1 (i <= k) and (1 - lambda_i)/(1 - theta)."""
    P = _shifted((24, 24), (2, 2), 0.3)
    k = 5
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, theta_mode=theta_mode, eig="dense", indefinite=True)
    B, E, C = brute.dense_blocks(slr)
    lam = np.sort(np.linalg.eigvalsh(brute.h_from_blocks(B, E, C)))[::-1]
    assert lam[0] > 1.0                                        # H has eigenvalues above 1
    S = brute.schur(B, E, C)
    sig = np.sort(np.linalg.eigvals(S @ slr.stilde_inv(np.eye(S.shape[0]))).real)
    theta = slr.theta
    assert theta == pytest.approx(lam[k] if (theta_mode == THETA_LAMBDA_K1 and lam[k] < 1) else 0.0)
    want = np.sort(np.concatenate([np.ones(k), (1 - lam[k:]) / (1 - theta)]))
    assert np.allclose(sig, want, rtol=1e-8, atol=1e-9)


def test_theta_falls_back_to_zero_when_lambda_k1_reaches_one():
    """Reading for the indefinite case: theta = lambda_{k+1} only while it is below 1."""
    P = _shifted((24, 24), (2, 2), 0.3)
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0, eig="dense", indefinite=True)
    B, E, C = brute.dense_blocks(slr)
    lam = np.sort(np.linalg.eigvalsh(brute.h_from_blocks(B, E, C)))[::-1]
    assert lam[0] >= 1.0 and slr.theta == 0.0                  # k = 0: lambda_1 >= 1
    k = int(np.sum(lam >= 1.0))
    slr2 = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, eig="dense", indefinite=True)
    assert slr2.theta == pytest.approx(lam[k])


def test_full_rank_indefinite_gives_exact_inverse_and_one_gmres_step():
    P = _shifted((16, 16), (2, 2), 0.5)
    slr0 = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0, indefinite=True)
    s = slr0.order.s
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, s, eig="dense", indefinite=True)
    A = slr.App.toarray()
    M = np.stack([slr.apply(e) for e in np.eye(A.shape[0])], axis=1)
    assert np.allclose(M @ A, np.eye(A.shape[0]), atol=1e-9)
    x, its, rel, oks = slr_gmres(slr, P.b[:, 0])
    assert its[0] == 1 and oks[0]


def test_slr_gmres_converges_on_shifted_problem_and_rank_helps():
    P = _shifted((32, 32), (2, 2), 0.2)
    res = {}
    for k in (0, 8):
        slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k, indefinite=True)
        x, its, rels, oks = slr_gmres(slr, P.b[:, 0])
        assert oks[0] and rels[0] <= 1e-8
        assert np.linalg.norm(x - P.xstar[:, 0]) / np.linalg.norm(P.xstar[:, 0]) < 1e-5
        res[k] = its[0]
    assert res[8] < res[0]


# ---------------------------------------------------------------------------
# Vertex-separator partitions (Section 2.1: the method also applies to them)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,boxes,want", [((32, 32), (2, 2), 2 * 32 - 1), ((17, 17), (3, 3), 2 * 2 * 17 - 4),
                                             ((12, 12, 12), (2, 2, 2), 3 * 12 * 12 - 3 * 12 + 1)])
def test_vertex_separator_interface_counts_and_block_diagonal_B(dims, boxes, want):
    """The interface is exactly the separator planes (closed-form counts by
    inclusion-exclusion) and B has no coupling between different parts' interiors."""
    rp, ci, v = slrgen.laplacian(dims)
    part = slrgen.box_partition_vsep(dims, boxes)
    p = int(np.prod(boxes))
    o = dd_order(rp, ci, part, p)
    assert o.s == want == int(np.sum(part < 0))
    Bi, E, C, App = split_blocks(rp, ci, v, o)
    B = App[:o.n_I, :o.n_I].tocoo()
    owner = np.repeat(np.arange(p), np.diff(o.int_off))
    assert np.all(owner[B.row] == owner[B.col])
    assert E.nnz > 0


def test_vertex_separator_slr_full_rank_is_exact_and_pcg_converges():
    P = slrgen.make_problem("vsep", (20, 20), (2, 2), 4, separators=True)
    s = dd_order(P.rowptr, P.colind, P.part, P.nparts).s
    full = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, s, eig="dense")
    A = full.App.toarray()
    M = np.stack([full.apply(e) for e in np.eye(A.shape[0])], axis=1)
    assert np.allclose(M @ A, np.eye(A.shape[0]), atol=1e-9)
    slr = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 4)
    x, its, rels, oks = slr_pcg(slr, P.b[:, 0])
    assert oks[0] and np.linalg.norm(x - P.xstar[:, 0]) / np.linalg.norm(P.xstar[:, 0]) < 1e-6
