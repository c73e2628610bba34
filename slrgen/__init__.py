"""Seeded synthetic inputs for SLR-preconditioned CG (Li, Xi & Saad, arXiv 1505.04340).

This module produces *inputs only*: the sparse symmetric matrix A of Eq. (1.1)
in CSR form, a geometric box partition (the vertex-based partitioning of
Section 2.1), right-hand sides b = A x*, and the seeded uniform vectors that the
method itself draws (the Lanczos start vector of Section 5.1 is built from one
of them).  It contains none of the preconditioner's arithmetic, so both the
CPU oracle and the CUDA library can consume it without sharing method code.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used
as a counter-based generator: output i (0-based) of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15 mod 2**64)`` with the published
finaliser ``mix``.  A double in [0, 1) is ``(x >> 11) * 2**-53``.

Model problems follow Section 6.1 (5-/7-point centred differences on the unit
square/cube, Dirichlet boundary, the 1/h**2 factor omitted as in Section 3.2)
and their variable-coefficient and anisotropic variants.  Grid index of a node
is ``x + nx*y + nx*ny*z`` (x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """Doubles in [-1, 1): ``2u - 1``."""
    return 2.0 * uniform01(seed, count) - 1.0


def loguniform(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    """Log-uniform doubles in [lo, hi): ``lo * (hi/lo)**u``."""
    return lo * (hi / lo) ** uniform01(seed, count)


# ---------------------------------------------------------------------------
# matrices
# ---------------------------------------------------------------------------

def _grid_index(dims):
    return np.arange(int(np.prod(dims)), dtype=np.int64).reshape(tuple(reversed(dims)))


def _to_csr(n, rows, cols, vals):
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))


def laplacian(dims, coef=None):
    """Centred-difference -div(c grad u) with constant axis coefficients c.

    2-D (5-point) or 3-D (7-point), Dirichlet, no 1/h**2 scaling: the diagonal
    is ``2*sum(c)`` and each neighbour coupling is ``-c_axis``.  ``coef=None``
    is the plain Laplacian of Section 6.1; ``(1, 1, 1e-2)`` is the anisotropic
    variant (z the slowest index).
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    coef = (1.0,) * nd if coef is None else tuple(float(c) for c in coef)
    n = int(np.prod(dims))
    idx = _grid_index(dims)
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [np.full(n, 2.0 * sum(coef))]
    for ax in range(nd):
        arr_axis = nd - 1 - ax           # numpy axis of grid axis `ax`
        lo = [slice(None)] * nd
        hi = [slice(None)] * nd
        lo[arr_axis] = slice(0, dims[ax] - 1)
        hi[arr_axis] = slice(1, dims[ax])
        a = idx[tuple(lo)].ravel()
        b = idx[tuple(hi)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, -coef[ax])] * 2
    return _to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def diffusion_fv(dims, a):
    """Cell-centred finite volumes for -div(a grad u), Dirichlet boundary.

    ``a`` holds one positive coefficient per cell (grid order).  An interior
    face between cells i and j has transmissibility ``2 a_i a_j / (a_i + a_j)``
    (harmonic mean); a boundary face of cell i has ``2 a_i``.  Row i: the
    diagonal is the sum of the transmissibilities of its faces, each interior
    neighbour gets ``-T_ij``.
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    n = int(np.prod(dims))
    a = np.asarray(a, dtype=np.float64).reshape(n)
    idx = _grid_index(dims)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for ax in range(nd):
        arr_axis = nd - 1 - ax
        lo = [slice(None)] * nd
        hi = [slice(None)] * nd
        lo[arr_axis] = slice(0, dims[ax] - 1)
        hi[arr_axis] = slice(1, dims[ax])
        i = idx[tuple(lo)].ravel()
        j = idx[tuple(hi)].ravel()
        t = 2.0 * a[i] * a[j] / (a[i] + a[j])
        np.add.at(diag, i, t)
        np.add.at(diag, j, t)
        rows += [i, j]
        cols += [j, i]
        vals += [-t, -t]
        first = [slice(None)] * nd
        last = [slice(None)] * nd
        first[arr_axis] = 0
        last[arr_axis] = dims[ax] - 1
        for b in (idx[tuple(first)].ravel(), idx[tuple(last)].ravel()):
            np.add.at(diag, b, 2.0 * a[b])
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    return _to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def box_partition(dims, boxes):
    """Geometric box partition: box id per axis ``floor(coord * B_ax / N_ax)``.

    Part id = ``bx + Bx*by + Bx*By*bz``; returns int32 [n] in grid order.
    """
    dims = tuple(int(d) for d in dims)
    boxes = tuple(int(b) for b in boxes)
    coords = np.meshgrid(*[np.arange(d) for d in reversed(dims)], indexing="ij")
    coords = list(reversed(coords))          # coords[ax] has grid-axis `ax`
    part = np.zeros(coords[0].shape, dtype=np.int64)
    stride = 1
    for ax in range(len(dims)):
        part += (coords[ax] * boxes[ax] // dims[ax]) * stride
        stride *= boxes[ax]
    return part.ravel().astype(np.int32)


def box_partition_vsep(dims, boxes):
    """Box partition with vertex separators: the first grid plane of every box but
    the first along each axis (where ``floor(coord * B_ax / N_ax)`` steps up) is a
    separator (part id -1); the other vertices keep their box id.  With 5/7-point
    stencils the separator planes disconnect the boxes."""
    dims = tuple(int(d) for d in dims)
    boxes = tuple(int(b) for b in boxes)
    part = box_partition(dims, boxes).astype(np.int64)
    coords = np.meshgrid(*[np.arange(d) for d in reversed(dims)], indexing="ij")
    coords = list(reversed(coords))
    sep = np.zeros(coords[0].shape, dtype=bool)
    for ax in range(len(dims)):
        c = coords[ax]
        sep |= (c > 0) & ((c * boxes[ax]) // dims[ax] > ((c - 1) * boxes[ax]) // dims[ax])
    part = part.reshape(coords[0].shape)
    part[sep] = -1
    return part.ravel().astype(np.int32)


def csr_matvec(rowptr, colind, val, x):
    A = sp.csr_matrix((val, colind, rowptr), shape=(len(rowptr) - 1,) * 2)
    return A @ x


# ---------------------------------------------------------------------------
# problems
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """One SLR test problem: CSR A, partition, rank and right-hand sides."""
    name: str
    dims: tuple
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    part: np.ndarray
    nparts: int
    k: int
    lanczos_steps: int
    xstar: np.ndarray            # [n, nrhs]
    b: np.ndarray                # [n, nrhs] = A @ xstar
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.rowptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def make_problem(name, dims, boxes, k, *, kind="laplacian", coef=None, coef_range=None,
                 nrhs=1, matrix_seed=1, rhs_seed=2, lanczos_steps=None, shift=0.0, separators=False):
    """Build a Problem; ``kind`` is 'laplacian' (constant axis coefficients) or 'fv'.

    x* column j is uniform[-1,1) from stream ``rhs_seed + j``; b = A x*.
    For 'fv' the cell coefficients are log-uniform in ``coef_range`` from
    stream ``matrix_seed``.  ``shift`` s > 0 subtracts s I (the shifted,
    symmetric indefinite problems of Section 6: -Laplacian u - c u = f).
    ``separators``: a vertex-separator partition (``box_partition_vsep``) instead
    of the edge-based one.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    if kind == "laplacian":
        rowptr, colind, val = laplacian(dims, coef)
    elif kind == "fv":
        lo, hi = coef_range
        rowptr, colind, val = diffusion_fv(dims, loguniform(matrix_seed, n, lo, hi))
    else:
        raise ValueError(kind)
    if shift:
        val = val.copy()
        rows = np.repeat(np.arange(n), np.diff(rowptr))
        val[colind == rows] -= shift
    part = box_partition_vsep(dims, boxes) if separators else box_partition(dims, boxes)
    xstar = np.stack([uniform_pm1(rhs_seed + j, n) for j in range(nrhs)], axis=1)
    b = csr_matvec(rowptr, colind, val, xstar)
    return Problem(name=name, dims=dims, rowptr=rowptr, colind=colind, val=val, part=part,
                   nparts=int(np.prod(boxes)), k=int(k),
                   lanczos_steps=int(lanczos_steps if lanczos_steps is not None else 5 * k),
                   xstar=xstar, b=np.ascontiguousarray(b),
                   meta=dict(boxes=tuple(boxes), kind=kind, coef=coef, coef_range=coef_range, shift=shift,
                             separators=separators))


# The five workloads (grid, partition, rank, right-hand sides).
def config1():
    """2-D 5-point Laplacian 32x32, 2x2 boxes, k=8 from 40 Lanczos steps."""
    return make_problem("2d-laplace-32x32-p4-k8", (32, 32), (2, 2), 8, lanczos_steps=40)


def config2():
    """3-D 7-point Laplacian 64^3, 4x4x4 boxes of 16^3, k=32."""
    return make_problem("3d-laplace-64^3-p64-k32", (64, 64, 64), (4, 4, 4), 32)


def config3():
    """2-D FV diffusion 1024^2, a log-uniform in [1e-3,1e3], 16x16 boxes, k=64."""
    return make_problem("2d-fv-1024^2-p256-k64", (1024, 1024), (16, 16), 64, kind="fv",
                        coef_range=(1e-3, 1e3))


def config4(nrhs=32):
    """3-D anisotropic Laplacian 96^3, coefficients (1,1,1e-2), 6x6x6 boxes, k=64, 32 RHS."""
    return make_problem("3d-aniso-96^3-p216-k64-r32", (96, 96, 96), (6, 6, 6), 64,
                        coef=(1.0, 1.0, 1e-2), nrhs=nrhs)


def serving_specs(count=32, seed=3):
    """A pool of ``count`` serving matrix specs drawn from stream ``seed``.

    Each spec: 2-D (side in 64..512) or 3-D (side in 32..64) FV diffusion with
    coefficients log-uniform in [1e-2, 1e2], boxes chosen so the part count is
    in 16..256, k in {16, 32, 64}, 1-8 right-hand sides per request.
    """
    u = uniform01(seed, 8 * count).reshape(count, 8)
    specs = []
    for i in range(count):
        three_d = u[i, 0] < 0.5
        if three_d:
            side = 32 + int(u[i, 1] * 33)
            bpa = (3, 4, 5, 6)[int(u[i, 2] * 4)]       # 27..216 parts
            dims, boxes = (side,) * 3, (bpa,) * 3
        else:
            side = 64 + int(u[i, 1] * 449)
            bpa = (4, 8, 12, 16)[int(u[i, 2] * 4)]     # 16..256 parts
            dims, boxes = (side,) * 2, (bpa,) * 2
        k = (16, 32, 64)[int(u[i, 3] * 3)]
        specs.append(dict(dims=dims, boxes=boxes, k=k, matrix_seed=1000 + i))
    return specs


def serving_problem(spec):
    """The matrix of one serving spec: FV diffusion with coefficients log-uniform in [1e-2, 1e2]."""
    d = spec["dims"]
    name = ("3d" if len(d) == 3 else "2d") + f"-fv-{d[0]}^{len(d)}-p{int(np.prod(spec['boxes']))}-k{spec['k']}"
    return make_problem(name, d, spec["boxes"], spec["k"], kind="fv", coef_range=(1e-2, 1e2),
                        matrix_seed=spec["matrix_seed"])


def serving_requests(count=256, seed=3, nspecs=32, rate=50.0):
    """The request stream: ``count`` requests with Poisson arrivals at ``rate`` per second.

    Request i asks for matrix ``spec`` (uniform over ``nspecs`` serving specs)
    with ``nrhs`` in 1..8 right-hand sides; x* column j of request i is
    uniform[-1,1) from stream ``rhs_seed + j``.  Inter-arrival gaps are
    ``-log(1-u)/rate`` from stream ``seed + 1``; the first request arrives at 0.
    Returns a list of dicts (rid, spec, nrhs, arrival, rhs_seed).
    """
    u = uniform01(seed + 1, 3 * count).reshape(count, 3)
    gaps = -np.log1p(-u[:, 0]) / rate
    arrival = np.concatenate([[0.0], np.cumsum(gaps[1:])])
    out = []
    for i in range(count):
        out.append(dict(rid=i, spec=int(u[i, 1] * nspecs), nrhs=1 + int(u[i, 2] * 8),
                        arrival=float(arrival[i]), rhs_seed=1_000_000 + 16 * i))
    return out


def request_rhs(prob, nrhs, rhs_seed):
    """b = A x* for one request, x* columns uniform[-1,1) from ``rhs_seed + j``."""
    xstar = np.stack([uniform_pm1(rhs_seed + j, prob.n) for j in range(nrhs)], axis=1)
    return xstar, np.ascontiguousarray(csr_matvec(prob.rowptr, prob.colind, prob.val, xstar))
