"""Brute-force and closed-form companions of the oracle (TEST INFRASTRUCTURE ONLY).

Dense forms of the quantities the SLR method never builds, for tiny problems,
and the paper's closed forms for the two-domain model problem.  Used only by
``tests/`` to pin ``oracle.slr_oracle`` to the mathematics.

* ``dense_blocks``      - B, E, C of Eq. 2.3 as dense arrays
* ``schur``             - S = C - E^T B^{-1} E                       (Eq. 2.4)
* ``h_from_blocks``     - H = L^{-1} E^T B^{-1} E L^{-T}, L = chol(C) (Eqs. 3.1-3.2)
* ``eta``, ``gamma_two_domain`` - Eqs. 3.9 and 3.10 (Proposition 3.3)
* ``kappa``             - kappa(theta) of Proposition 4.2 (Eq. 4.14)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def dense_blocks(slr):
    nI = slr.order.n_I
    App = slr.App.toarray()
    return App[:nI, :nI], App[:nI, nI:], App[nI:, nI:]


def schur(B, E, C):
    """S = C - E^T B^{-1} E (Eq. 2.4)."""
    return C - E.T @ np.linalg.solve(B, E)


def h_from_blocks(B, E, C):
    """H of Eq. 3.2 with L the dense lower Cholesky factor of C."""
    L = np.linalg.cholesky(C)
    K = E.T @ np.linalg.solve(B, E)
    X = sla.solve_triangular(L, K, lower=True)
    return sla.solve_triangular(L, X.T, lower=True).T


def eta(nx):
    """Eigenvalues of T^_x / 2 (Eq. 3.9): 1 + 2 sin^2(k pi / (2 (n_x + 1)))."""
    k = np.arange(1, nx + 1)
    return 1.0 + 2.0 * np.sin(k * np.pi / (2.0 * (nx + 1))) ** 2


def gamma_two_domain(nx, ny):
    """Eigenvalues gamma_k of S_Gamma^{-1} - T^_x^{-1} (Proposition 3.3, Eq. 3.10).

    theta_k = arccosh(eta_k);
    gamma_k = sinh(n_y theta_k) / (eta_k [sinh((n_y + 2) theta_k) - sinh(n_y theta_k)]).
    Returns (gamma, zeta = 2 eta gamma, eta); zeta_k are the eigenvalues of
    S_Gamma^{-1} T^_x - I, i.e. of X in Eq. 3.4.
    """
    e = eta(nx)
    th = np.arccosh(e)
    # Same ratio with numerator and denominator multiplied by 2 exp(-n_y theta),
    # so that large n_y theta cannot overflow: sinh(x) = (e^x - e^-x) / 2.
    q = np.exp(-2.0 * ny * th)
    g = (1.0 - q) / (e * (np.exp(2.0 * th) - 1.0 - q * (np.exp(-2.0 * th) - 1.0)))
    return g, 2.0 * e * g, e


def two_domain_lambda(nx, ny):
    """Eigenvalues of H for the two-domain problem: lambda = zeta / (1 + zeta).

    From Eq. 3.4, X = (I - H)^{-1} - I has eigenvalues lambda/(1 - lambda)
    (Lemma 3.2); in the two-domain setting those are the zeta_k.
    """
    _, z, _ = gamma_two_domain(nx, ny)
    return z / (1.0 + z)


def kappa(theta, lam_s, lam_k1):
    """Spectral condition number of S S~^{-1} as a function of theta (Eq. 4.14)."""
    theta = np.asarray(theta, dtype=np.float64)
    return np.where(theta < lam_s, (1.0 - theta) / (1.0 - lam_k1),
                    np.where(theta <= lam_k1, (1.0 - lam_s) / (1.0 - lam_k1),
                             (1.0 - lam_s) / (1.0 - theta)))
