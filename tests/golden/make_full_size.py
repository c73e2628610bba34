"""Writes the expected values of the full-size parity tests from the CPU oracle.

The oracle cannot run the 2-D FV 1024^2 and the 3-D anisotropic 96^3 workloads
inside a GPU test (its setup of the 96^3 problem alone takes minutes), so this
script runs it once and stores what the tests compare against, at sampled
positions:

* the apply z = M^{-1} r (Eq. 4.1 with S~^{-1} of Eq. 4.7) of two seeded
  vectors r, and
* preconditioned CG (Section 6: x_0 = 0, ||r_j|| <= 1e-8 ||b||) on the first
  right-hand sides b = A x*: iteration count, final relative residual and x.

Both use a seeded low-rank part instead of Lanczos pairs, so that the GPU test
can hand the library exactly the same pairs without storing them:
Z = X R^{-1} with X uniform[-1, 1) (SplitMix64 streams ``seed + j``) and
R^T R = X^T C X (so Z^T C Z = I, the C-orthonormal Z_k of Proposition 4.3),
lambda_i = theta + 0.1 u_i (u uniform[0, 1) from stream ``seed + k``, sorted
descending), so every d_i = 1/(1 - lambda_i) - 1/(1 - theta) >= 0 and the
preconditioner stays SPD.  C is the interface block of the reordered matrix
(Eq. 2.3) from the oracle's DD order.

Only ``oracle/`` and the input generators of ``slrgen`` are called.  Run
``python tests/golden/make_full_size.py config3 config4`` (about half an hour
on 8 cores); it writes ``tests/golden/full_<config>.json``.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import slrgen  # noqa: E402

# per workload: rank of the seeded low-rank part, theta, right-hand sides solved, PCG cap
SPECS = {
    "config2": dict(k=32, theta=0.3, cols=1, maxit=300),
    "config3": dict(k=64, theta=0.3, cols=1, maxit=3000),
    "config4": dict(k=64, theta=0.3, cols=2, maxit=300),
}
PAIR_SEED = 5000          # streams of the seeded low-rank part
VEC_SEED = 6000           # streams of the applied vectors (one per vector)
SAMPLE_SEED = 7000        # stream of the sampled positions
NSAMPLE = 4096            # draws; every 4th distinct position is kept


def problem(name):
    return getattr(slrgen, name)()


def seeded_pairs(C, k, theta, seed=PAIR_SEED):
    """(Z, lambda) as described in the module docstring; C in DD interface order."""
    s = C.shape[0]
    X = np.stack([slrgen.uniform_pm1(seed + j, s) for j in range(k)], axis=1)
    G = X.T @ (C @ X)
    R = np.linalg.cholesky(G).T                       # upper, R^T R = X^T C X
    Z = sla.solve_triangular(R, X.T, trans="T", lower=False).T
    lam = np.sort(theta + 0.1 * slrgen.uniform01(seed + k, k))[::-1].copy()
    return Z, lam


def sample_positions(n, seed=SAMPLE_SEED):
    return np.unique((slrgen.uniform01(seed, NSAMPLE) * n).astype(np.int64))[::4]


def applied_vectors(n):
    return [slrgen.uniform_pm1(VEC_SEED + j, n) for j in range(2)]


def oracle_with_pairs(P, k, theta):
    """The oracle's SLR of P with the seeded pairs in place of its Lanczos ones."""
    from oracle.slr_oracle import SLR
    ora = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, 0)
    Z, lam = seeded_pairs(ora.C, k, theta)
    ora.U = ora.cfac.solve_L(ora.C @ Z)               # U_k = L^{-1} C Z_k (Z_k = L^{-T} U_k)
    ora.lam = lam
    ora.k = k
    ora.theta = theta
    return ora


def write(name):
    from oracle.slr_oracle import slr_pcg
    spec = SPECS[name]
    P = problem(name)
    t0 = time.time()
    ora = oracle_with_pairs(P, spec["k"], spec["theta"])
    print(f"{name}: oracle setup {time.time() - t0:.0f} s", flush=True)
    idx = sample_positions(P.n)
    out = dict(workload=P.name, n=P.n, k=spec["k"], theta=spec["theta"], pair_seed=PAIR_SEED,
               vec_seed=VEC_SEED, sample_seed=SAMPLE_SEED, idx=idx.tolist(), apply=[], pcg=[])
    for r in applied_vectors(P.n):
        z = ora.apply(r)
        out["apply"].append(dict(z=z[idx].tolist(), norm2=float(np.linalg.norm(z)), maxabs=float(np.abs(z).max())))
    print(f"{name}: applies done {time.time() - t0:.0f} s", flush=True)
    for j in range(spec["cols"]):
        x, its, rels, oks = slr_pcg(ora, P.b[:, j], tol=1e-8, maxit=spec["maxit"])
        out["pcg"].append(dict(column=j, iterations=int(its[0]), relres=float(rels[0]), converged=bool(oks[0]),
                               x=x[idx].tolist(), norm2=float(np.linalg.norm(x))))
        print(f"{name}: column {j}: {its[0]} iterations, relres {rels[0]:.2e} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, f"full_{name}.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["config3", "config4"]:
        write(nm)
