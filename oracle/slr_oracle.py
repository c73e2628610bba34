"""Plain FP64 CPU oracle of SLR-preconditioned CG (Li, Xi & Saad, arXiv 1505.04340).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this file;
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU baseline
leg and its ``--impl reference`` arm) may use it.  It shares no code with the
CUDA library: the two meet only in the seeded inputs of ``slrgen``.

Every step is written in the paper's order and notation, slow and direct:

* ``dd_order``      - vertex-based partition, interface detection, global DD
                      reordering [u_1..u_p, y_1..y_p]        (Section 2.1, Eqs. 2.1-2.3)
* ``split_blocks``  - A_pp = [[B, E], [E^T, C]], B = diag(B_i) (Eq. 2.3)
* ``BandCholesky``  - direct solves with each B_i            (Section 5.2)
* ``CFactor``       - C = L L^T                               (Section 3.1, Eq. 3.1)
* ``h_apply``       - H = L^{-1} E^T B^{-1} E L^{-T}          (Eq. 3.2)
* ``lanczos``       - Lanczos on H with full reorthogonalisation, Ritz pairs
                                                               (Section 5.1)
* ``SLR.apply``     - z = M^{-1} r with M of Eq. 4.1 and S~^{-1} of Eq. 4.7,
                      Lambda~ of Eq. 4.11 (theta = lambda_{k+1}) or Eq. 4.10
                      (theta = 0)
* ``SLR.stilde_inv_zform`` - the same S~^{-1} through Proposition 4.3 (Eq. 4.15)
* ``pcg``           - preconditioned CG, stop at ||r|| <= 1e-8 ||b||, 300 its
                                                               (Section 6)
* ``gmres``         - right-preconditioned GMRES(40) for the symmetric indefinite
                      problems of Section 6 (B_i may be indefinite, C is SPD:
                      the SPD-interface assumption of Section 1)

Readings where the paper is silent (they are listed with reasons in the design
notes):  the Lanczos start vector is v_1 = L^{-1} C z / ||L^{-1} C z|| (= L^T z
normalised) with z uniform[-1,1) from a seeded SplitMix64 stream in DD interface
order, which makes the Ritz pairs independent of the ordering used to factor C;
reorthogonalisation is full (two classical Gram-Schmidt passes); B_i and C are
factored exactly (the paper's experiments use incomplete factors).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

THETA_LAMBDA_K1 = 0      # theta = lambda_{k+1}   (Eq. 4.11, the paper's choice)
THETA_ZERO = 1           # theta = 0              (Eq. 4.10)


# ---------------------------------------------------------------------------
# Section 2.1: vertex-based partition and the global DD ordering
# ---------------------------------------------------------------------------

@dataclass
class DDOrder:
    perm: np.ndarray        # new -> old (int64 [n])
    iperm: np.ndarray       # old -> new
    is_iface: np.ndarray    # bool [n], original numbering
    int_off: np.ndarray     # [p+1] offsets of u_i inside u
    ifc_off: np.ndarray     # [p+1] offsets of y_i inside y
    n_I: int                # interior unknowns (length of u)
    s: int                  # interface unknowns (length of y)


def dd_order(rowptr, colind, part, nparts) -> DDOrder:
    """Interface detection (Section 2.1) and the reordering of Eqs. 2.2-2.3.

    A node is a local interface node iff it is coupled (a structural
    off-diagonal entry) to a node of another part; otherwise it is interior.
    The new order lists u_1, ..., u_p (interiors of part 0..p-1) and then
    y_1, ..., y_p (interfaces of part 0..p-1); inside each group nodes keep
    ascending original index.

    Vertex separators (Section 2.1 notes the method applies to them too): part
    id -1 marks a separator vertex; separator vertices are interface nodes listed
    after y_p (beyond ifc_off[p]), and a node of a part is interface only if it
    is coupled to another part's node (coupling to a separator keeps it interior).
    """
    n = len(rowptr) - 1
    part = np.asarray(part, dtype=np.int64)
    is_iface = np.zeros(n, dtype=bool)
    for i in range(n):
        if part[i] < 0:
            is_iface[i] = True
            continue
        for q in range(rowptr[i], rowptr[i + 1]):
            j = colind[q]
            if j != i and part[j] >= 0 and part[j] != part[i]:
                is_iface[i] = True
                break
    interior = [[] for _ in range(nparts)]
    iface = [[] for _ in range(nparts)]
    separator = []
    for i in range(n):
        if part[i] < 0:
            separator.append(i)
        else:
            (iface if is_iface[i] else interior)[part[i]].append(i)
    perm = []
    int_off = [0]
    for q in range(nparts):
        perm += interior[q]
        int_off.append(len(perm))
    n_I = len(perm)
    ifc_off = [0]
    for q in range(nparts):
        perm += iface[q]
        ifc_off.append(len(perm) - n_I)
    perm += separator
    perm = np.array(perm, dtype=np.int64)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    return DDOrder(perm, iperm, is_iface, np.array(int_off), np.array(ifc_off), n_I, n - n_I)


def split_blocks(rowptr, colind, val, order: DDOrder):
    """Blocks of the reordered matrix P A P^T = [[B, E], [E^T, C]] (Eq. 2.3).

    Returns (list of B_i as dense-banded-capable CSR, E (n_I x s), C (s x s),
    A_pp (n x n)) as scipy CSR matrices.
    """
    n = len(rowptr) - 1
    A = sp.csr_matrix((val, colind, rowptr), shape=(n, n))
    App = A[order.perm][:, order.perm].tocsr()
    nI = order.n_I
    B = App[:nI, :nI].tocsr()
    E = App[:nI, nI:].tocsr()
    C = App[nI:, nI:].tocsr()
    Bi = [B[order.int_off[q]:order.int_off[q + 1], order.int_off[q]:order.int_off[q + 1]].tocsr()
          for q in range(len(order.int_off) - 1)]
    return Bi, E, C, App


# ---------------------------------------------------------------------------
# Section 5.2: solves with B = diag(B_i)
# ---------------------------------------------------------------------------

class BandCholesky:
    """Direct solver for one SPD block B_i: banded Cholesky in natural order.

    The half-bandwidth w is the largest |i - j| over the stored entries of B_i.
    Factor and solve are LAPACK's banded Cholesky (dpbtrf / dpbtrs).
    """

    def __init__(self, Bi):
        m = Bi.shape[0]
        self.m = m
        if m == 0:
            self.w = 0
            return
        coo = Bi.tocoo()
        self.w = int(np.max(np.abs(coo.row - coo.col))) if coo.nnz else 0
        ab = np.zeros((self.w + 1, m))            # lower band storage: ab[i-j, j] = B[i, j]
        low = coo.row >= coo.col
        ab[coo.row[low] - coo.col[low], coo.col[low]] = coo.data[low]
        self.cb = sla.cholesky_banded(ab, lower=True)

    def solve(self, f):
        if self.m == 0:
            return f.copy()
        return sla.cho_solve_banded((self.cb, True), f)


class BandLU:
    """Direct solver for one symmetric, possibly indefinite block B_i: LAPACK's
    banded LU with partial pivoting (dgbsv) on the full band.  An independent
    method from any symmetric factorisation; used when A is indefinite."""

    def __init__(self, Bi):
        m = Bi.shape[0]
        self.m = m
        if m == 0:
            self.w = 0
            return
        coo = Bi.tocoo()
        self.w = w = int(np.max(np.abs(coo.row - coo.col))) if coo.nnz else 0
        self.ab = np.zeros((2 * w + 1, m))      # ab[w + i - j, j] = B[i, j]
        self.ab[w + coo.row - coo.col, coo.col] = coo.data

    def solve(self, f):
        if self.m == 0:
            return f.copy()
        return sla.solve_banded((self.w, self.w), self.ab, f)


class BSolver:
    """t = B^{-1} f as p independent solves (Section 5.2); ``indefinite`` takes
    banded LU instead of banded Cholesky."""

    def __init__(self, Bi, int_off, indefinite=False):
        self.blocks = [BandLU(b) if indefinite else BandCholesky(b) for b in Bi]
        self.off = int_off

    def solve(self, f):
        t = np.empty_like(f)
        for q, blk in enumerate(self.blocks):
            a, b = self.off[q], self.off[q + 1]
            t[a:b] = blk.solve(f[a:b])
        return t


# ---------------------------------------------------------------------------
# Section 3.1: C = L L^T
# ---------------------------------------------------------------------------

class CFactor:
    """Cholesky factor of the interface matrix C (Eq. 3.1).

    ``route='dense'``: numpy's dense Cholesky of C in DD order, L lower
    triangular.  ``route='sparse'``: SuperLU with a symmetric minimum-degree
    ordering and no pivoting gives P C P^T = L_1 D L_1^T; then L = P^T L_1 D^{1/2}
    (a row-permuted triangular matrix with C = L L^T).  The two routes give
    different L but the same C^{-1} and the same spectrum of H (Eq. 3.2).
    """

    def __init__(self, C, route="auto"):
        s = C.shape[0]
        self.s = s
        if route == "auto":
            route = "dense" if s <= 6000 else "sparse"
        self.route = route
        if s == 0:
            return
        if route == "dense":
            self.L = np.linalg.cholesky(C.toarray())
        else:
            lu = spla.splu(sp.csc_matrix(C), permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                           options=dict(SymmetricMode=True))
            pr = lu.perm_r
            pc = lu.perm_c
            # Pr A Pc = L U with Pr[perm_r[i], i] = 1 and Pc[i, perm_c[i]] = 1;
            # symmetric elimination needs the same order on rows and columns.
            if not np.array_equal(pr, pc):
                raise RuntimeError("SuperLU pivoted off the diagonal; C is not SPD")
            d = lu.U.diagonal()
            if np.any(d <= 0):
                raise np.linalg.LinAlgError("C is not positive definite")
            self.p = pr                        # position of original row i in the factor
            self.L1 = sp.csc_matrix(lu.L)      # unit lower
            self.L1T = sp.csc_matrix(lu.L.T)
            self.sqd = np.sqrt(d)

    def solve_L(self, x):
        """L^{-1} x."""
        if self.s == 0:
            return x.copy()
        if self.route == "dense":
            return sla.solve_triangular(self.L, x, lower=True)
        xp = np.empty_like(x)
        xp[self.p] = x
        y = spla.spsolve_triangular(self.L1, xp, lower=True, unit_diagonal=True)
        return (y.T / self.sqd).T

    def solve_Lt(self, y):
        """L^{-T} y."""
        if self.s == 0:
            return y.copy()
        if self.route == "dense":
            return sla.solve_triangular(self.L, y, lower=True, trans="T")
        z = spla.spsolve_triangular(self.L1T, (y.T / self.sqd).T, lower=False,
                                    unit_diagonal=True)
        return z[self.p]

    def solve(self, g):
        """C^{-1} g = L^{-T} L^{-1} g."""
        return self.solve_Lt(self.solve_L(g))


# ---------------------------------------------------------------------------
# Section 5.1: Lanczos on H = L^{-1} E^T B^{-1} E L^{-T}
# ---------------------------------------------------------------------------

def h_apply(v, E, bsolve, cfac):
    """H v with H of Eq. 3.2, applied right to left, never formed."""
    y = cfac.solve_Lt(v)
    t = bsolve.solve(E @ y)
    return cfac.solve_L(E.T @ t)


def lanczos(hop, v1, m, reorth_passes=2, breakdown=1e-12):
    """m steps of symmetric Lanczos with full reorthogonalisation.

    Three-term recurrence w = H v_j - beta_{j-1} v_{j-1}, alpha_j = v_j^T w,
    w -= alpha_j v_j, then ``reorth_passes`` classical Gram-Schmidt passes
    against all previous basis vectors, beta_j = ||w||.  Stops early when
    beta_j <= breakdown * max|alpha| (an invariant subspace was found).
    Returns (alpha, beta, V) with V of shape [s, m_eff].
    """
    s = v1.shape[0]
    m = min(m, s)
    V = np.zeros((s, m))
    alpha = np.zeros(m)
    beta = np.zeros(m)
    V[:, 0] = v1 / np.linalg.norm(v1)
    m_eff = m
    for j in range(m):
        w = hop(V[:, j])
        if j > 0:
            w = w - beta[j - 1] * V[:, j - 1]
        alpha[j] = V[:, j] @ w
        w = w - alpha[j] * V[:, j]
        for _ in range(reorth_passes):
            w = w - V[:, :j + 1] @ (V[:, :j + 1].T @ w)
        beta[j] = np.linalg.norm(w)
        if j + 1 == m:
            break
        if beta[j] <= breakdown * np.max(np.abs(alpha[:j + 1])):
            m_eff = j + 1
            break
        V[:, j + 1] = w / beta[j]
    return alpha[:m_eff], beta[:m_eff], V[:, :m_eff]


def ritz(alpha, beta, V):
    """Ritz values (descending) and Ritz vectors V Y of the tridiagonal T."""
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    lam, Y = np.linalg.eigh(T)
    order = np.argsort(-lam, kind="stable")
    return lam[order], V @ Y[:, order]


def lanczos_start(cfac, C, seed):
    """v_1 = L^{-1} C z (= L^T z), z uniform[-1,1) from SplitMix64 stream ``seed``."""
    from slrgen import uniform_pm1
    z = uniform_pm1(seed, C.shape[0])
    return cfac.solve_L(C @ z)


# ---------------------------------------------------------------------------
# Section 4: the SLR preconditioner
# ---------------------------------------------------------------------------

class SLR:
    """Setup and apply of the Schur-complement low-rank preconditioner.

    ``eig='lanczos'`` follows Section 5.1 (m = lanczos_steps, default 5k);
    ``eig='dense'`` takes exact eigenpairs of a densely formed H (tiny
    problems only; used for the rank-s identity checks).  ``target_kappa``:
    choose the rank by the rule of Section 4 (Eq. condk), k = the number of
    eigenvalue estimates above 1 - 1/K, at most ``k``.
    """

    def __init__(self, rowptr, colind, val, part, nparts, k, lanczos_steps=None,
                 theta_mode=THETA_LAMBDA_K1, seed=1, eig="lanczos", c_route="auto", target_kappa=None,
                 indefinite=False):
        self.order = dd_order(rowptr, colind, part, nparts)
        Bi, E, C, App = split_blocks(rowptr, colind, val, self.order)
        self.E, self.C, self.App = E, C, App
        self.indefinite = indefinite
        self.bsolve = BSolver(Bi, self.order.int_off, indefinite)
        self.cfac = CFactor(C, c_route)
        s = self.order.s
        self.k = k = int(min(k, s))
        self.theta_mode = theta_mode
        self.seed = seed
        self.improvements = 0
        if k == 0 or s == 0:
            lam = np.zeros(1)
            U = np.zeros((s, 0))
        elif eig == "dense":
            H = self.h_dense()
            lam, Uf = np.linalg.eigh(H)
            order = np.argsort(-lam, kind="stable")
            lam, U = lam[order], Uf[:, order]
        else:
            m = lanczos_steps if lanczos_steps is not None else 5 * k
            v1 = lanczos_start(self.cfac, C, seed)
            a, b, V = lanczos(lambda v: h_apply(v, E, self.bsolve, self.cfac), v1, m)
            lam, U = ritz(a, b, V)
        self.k = k = min(k, U.shape[1])
        if target_kappa is not None and k > 0:
            # rank rule of Section 4 (Eq. condk): the condition number of S S~^{-1} stays below K
            # when lambda_{k+1} <= 1 - 1/K, i.e. k = number of eigenvalues above 1 - 1/K (capped)
            self.k = k = min(k, int(np.sum(lam > 1.0 - 1.0 / target_kappa)))
        self.ritz_values = lam
        self.lam = lam[:k].copy()
        self.U = U[:, :k].copy()
        if theta_mode == THETA_LAMBDA_K1 and len(lam) > k and lam[k] < 1.0:
            self.theta = float(lam[k])
        else:
            # theta = 0 (Eq. 4.10); with an indefinite B, H can have eigenvalues >= 1, and
            # theta = lambda_{k+1} >= 1 would flip the sign of the C^{-1} term of Eq. 4.7
            self.theta = 0.0

    # -- Section 5.3: improve the preconditioner by adding vectors, keeping U_k
    def improve(self, k_add, lanczos_steps=None):
        """Append k_add eigenvector estimates of H without discarding U_k.

        Deflation: Lanczos (Section 5.1, full reorthogonalisation) on
        P H P with P = I - U_k U_k^T, started from L^{-1} C z (stream seed + 1 +
        the number of earlier improvements) projected out of span(U_k).  Its
        leading Ritz pairs approximate lambda_{k+1}, ...; they are appended to
        (Lambda_k, U_k) and theta = lambda_{k+1} moves to the next Ritz value of
        the deflated run (theta = 0 stays 0).
        """
        s = self.order.s
        U = self.U
        m = lanczos_steps if lanczos_steps is not None else 5 * k_add

        def proj(x):
            for _ in range(2):                       # two classical Gram-Schmidt passes
                x = x - U @ (U.T @ x)
            return x

        self.improvements += 1
        v1 = proj(lanczos_start(self.cfac, self.C, self.seed + self.improvements))
        m = min(m, s - U.shape[1])
        a, b, V = lanczos(lambda v: proj(h_apply(v, self.E, self.bsolve, self.cfac)), v1, m)
        lam2, U2 = ritz(a, b, V)
        j = min(k_add, U2.shape[1])
        self.U = np.hstack([U, U2[:, :j]])
        self.lam = np.concatenate([self.lam, lam2[:j]])
        self.k += j
        self.ritz_values = np.concatenate([self.lam, lam2[j:]])
        if self.theta_mode == THETA_LAMBDA_K1:
            self.theta = float(lam2[j]) if len(lam2) > j else 0.0
        return j

    # H formed column by column (brute force aid for tiny problems)
    def h_dense(self):
        s = self.order.s
        return np.stack([h_apply(e, self.E, self.bsolve, self.cfac) for e in np.eye(s)], axis=1)

    def Z(self):
        """Z_k = L^{-T} U_k (Proposition 4.3)."""
        return self.cfac.solve_Lt(self.U)

    # -- S~^{-1} g  (Eq. 4.7 with Lambda~ = diag(lambda_1..lambda_k, theta, ..., theta))
    def stilde_inv(self, g):
        w = self.cfac.solve_L(g)
        v = self.U.T @ w
        corr_k = (1.0 / (1.0 - self.lam) - 1.0)                  # (I - Lambda_k)^{-1} - I
        corr_w = 1.0 / (1.0 - self.theta) - 1.0                  # (1 - theta)^{-1} - 1
        # U [(I - Lambda~)^{-1} - I] U^T w with U = [U_k, W], W W^T = I - U_k U_k^T
        wk = self.U @ (corr_k[:, None] * v if v.ndim == 2 else corr_k * v)
        ww = corr_w * (w - self.U @ v)
        return self.cfac.solve_Lt(w + wk + ww)

    # -- S_{k,theta}^{-1} g through Proposition 4.3
    def stilde_inv_zform(self, g, Z=None):
        Z = self.Z() if Z is None else Z
        c = 1.0 / (1.0 - self.theta)
        dvec = 1.0 / (1.0 - self.lam) - c
        v = Z.T @ g
        return c * self.cfac.solve(g) + Z @ (dvec[:, None] * v if v.ndim == 2 else dvec * v)

    def apply(self, r, zform=False):
        """z = M^{-1} r, r in DD order (Eq. 4.1 with the block LU of Eq. 2.4).

        M = [[I, 0], [E^T B^{-1}, I]] [[B, E], [0, S~]]:
        t = B^{-1} f;  g' = g - E^T t;  y = S~^{-1} g';  u = t - B^{-1} (E y).
        """
        nI = self.order.n_I
        f, g = r[:nI], r[nI:]
        t = self.bsolve.solve(f)
        gp = g - self.E.T @ t
        y = self.stilde_inv_zform(gp) if zform else self.stilde_inv(gp)
        u = t - self.bsolve.solve(self.E @ y)
        return np.concatenate([u, y])

    def to_dd(self, x):
        return x[self.order.perm]

    def from_dd(self, x):
        out = np.empty_like(x)
        out[self.order.perm] = x
        return out


# ---------------------------------------------------------------------------
# Section 6: the CG accelerator
# ---------------------------------------------------------------------------

def pcg(A, b, minv, tol=1e-8, maxit=300):
    """Preconditioned CG from x_0 = 0 for one right-hand side.

    Stops when the recurrence residual satisfies ||r_j|| <= tol ||b||
    (Section 6: residual reduced by 8 orders, at most 300 iterations).
    Returns (x, iterations, ||r_j||/||b||, converged).  The iteration count
    is the number of products with A.
    """
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    z = minv(r)
    p = z.copy()
    rho = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        pq = p @ q
        if pq <= 0.0:
            return x, it, np.linalg.norm(r) / bnorm, False
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, it, rel, True
        z = minv(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, maxit, np.linalg.norm(r) / bnorm, False


def gmres(A, b, minv, tol=1e-8, maxit=300, restart=40):
    """Right-preconditioned GMRES(restart) from x_0 = 0 for one right-hand side
    (Saad & Schultz 1986): Arnoldi on A M^{-1} with modified Gram-Schmidt, the
    least-squares problem by Givens rotations, x = M^{-1} (V y) at each restart
    or at convergence.  Stops when the residual estimate ||r_j|| <= tol ||b||
    (with right preconditioning it is the residual of A x = b); at most
    ``maxit`` products with A.  Returns (x, iterations, ||b - A x||/||b||,
    converged)."""
    n = len(b)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    its = 0
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or its >= maxit:
            return x, its, beta / bnorm, beta <= tol * bnorm
        m = restart
        V = np.zeros((n, m + 1))
        Hh = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        j_done = 0
        for j in range(m):
            w = A @ minv(V[:, j])
            its += 1
            for i in range(j + 1):                       # modified Gram-Schmidt
                Hh[i, j] = V[:, i] @ w
                w = w - Hh[i, j] * V[:, i]
            Hh[j + 1, j] = np.linalg.norm(w)
            if Hh[j + 1, j] > 0.0:
                V[:, j + 1] = w / Hh[j + 1, j]
            for i in range(j):                           # earlier rotations on the new column
                t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
                Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
                Hh[i, j] = t
            d = np.hypot(Hh[j, j], Hh[j + 1, j])         # new rotation zeroes H[j+1, j]
            cs[j], sn[j] = (Hh[j, j] / d, Hh[j + 1, j] / d) if d > 0.0 else (1.0, 0.0)
            Hh[j, j] = d
            Hh[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j_done = j + 1
            if abs(g[j + 1]) <= tol * bnorm or its >= maxit:
                break
        y = sla.solve_triangular(Hh[:j_done, :j_done], g[:j_done])
        x = x + minv(V[:, :j_done] @ y)


def slr_gmres(slr: SLR, b, tol=1e-8, maxit=300, restart=40):
    """Solve A x = b (original order) with SLR-preconditioned GMRES(restart) in DD order."""
    xs, its, rels, oks = [], [], [], []
    b2 = b.reshape(len(b), -1)
    for j in range(b2.shape[1]):
        x, it, rel, ok = gmres(slr.App, slr.to_dd(b2[:, j]), slr.apply, tol, maxit, restart)
        xs.append(slr.from_dd(x))
        its.append(it)
        rels.append(rel)
        oks.append(ok)
    return np.stack(xs, axis=1).reshape(b.shape), its, rels, oks


def slr_pcg(slr: SLR, b, tol=1e-8, maxit=300):
    """Solve A x = b (original order) with SLR-preconditioned CG run in DD order."""
    xs, its, rels, oks = [], [], [], []
    b2 = b.reshape(len(b), -1)
    for j in range(b2.shape[1]):
        x, it, rel, ok = pcg(slr.App, slr.to_dd(b2[:, j]), slr.apply, tol, maxit)
        xs.append(slr.from_dd(x))
        its.append(it)
        rels.append(rel)
        oks.append(ok)
    return np.stack(xs, axis=1).reshape(b.shape), its, rels, oks
