"""Parity tolerances of the FP32 (mixed) apply against the FP64 oracle.

The longest sum in the apply is either a band-solve row (a plane's two block
products, N = 2 (W + 1) terms, W the plane width) or a row of the explicit
inverse of the top levels of C's factor (up to the zone's n_T positions).  With
rounding errors that behave as independent zero-mean variables (Higham & Mary,
SIAM J. Sci. Comput. 41 (2019)) such a sum is within lambda sqrt(N) u of the sum
of its terms' magnitudes, with overwhelming probability for lambda about 4, u =
2^-24; the plane chain of diagonally dominant B_i is contractive and the
interface solves and coupling products add sums of similar length.  Hence the
bound 4 sqrt(N) u (N at least 64): 1.9e-6 for planes of 32 rows, 5.1e-6 for the
3-D boxes of 16^3.
"""
import math

U32 = 2.0 ** -24
TOL64 = 1e-10


def tol32(info):
    """FP32 apply (or its B or C solve) against FP64, relative in the max norm."""
    W = info["band_entries"] / max(info["n_interior"], 1) - 1.0
    N = max(2.0 * (W + 1.0), float(info["c_top_positions"]), 64.0)
    return 4.0 * math.sqrt(N) * U32
