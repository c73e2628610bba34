"""slr_apply_noalloc through the C ABI, against slr_apply.

The allocation-free apply serves callers that cannot call cudaMalloc while
they run (inside a global-mode stream capture, or under an allocator they do
not control).  It runs the same kernels as slr_apply with its scratch in the
library's fixed 32 MiB device array, so its result must equal slr_apply's
within the parity tolerance, call after call, and sizes beyond the array must
be refused before anything is launched.  This file is named so that pytest
collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import slrgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1505_04340_gb300 import SLR, slr  # noqa: E402

TOL = {"fp64": 1e-10, "mixed": 1e-4}        # the parity tolerances of the apply tests


def _colmajor(x):
    return x.t().contiguous()                # (nrhs, n) buffer = n x nrhs column-major


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["3d-levels", "3d-persistent", "c2-top-zone"])
def test_noalloc_apply_matches_apply_twice(precision, case):
    """The per-level C solve, the cooperative one (its barrier counter lives in the
    array) and a problem whose C factor has a top zone (its arrival counters too)."""
    if case == "c2-top-zone":
        P = slrgen.config2()
        nr, steps = 1, P.k + 1
    else:
        P = slrgen.make_problem("3d", (20, 19, 18), (3, 2, 2), 8, nrhs=2)
        nr, steps = 2, P.lanczos_steps
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=steps,
            precision=precision, nrhs_max=2, c_persistent=(case == "3d-persistent"))
    info = h.get_info()
    assert info["c_persistent"] == (case == "3d-persistent")
    if case == "c2-top-zone":
        assert info["c_top_positions"] > 0
    lib = slr.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    r = _colmajor(torch.tensor(np.random.default_rng(3).standard_normal((P.n, nr)), device="cuda"))
    z_ref = torch.empty_like(r)
    assert lib.slr_apply(h._h, C.c_void_p(r.data_ptr()), C.c_void_p(z_ref.data_ptr()), nr, P.n, stream) == 0
    for _ in range(2):                       # the array keeps the previous call's contents
        z = torch.full_like(r, float("nan"))
        st = lib.slr_apply_noalloc(h._h, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), nr, P.n, stream)
        assert st == 0, lib.slr_last_error_message()
        torch.cuda.synchronize()
        err = float((z - z_ref).abs().max() / z_ref.abs().max())
        assert err <= TOL[precision], err
    h.close()


def test_noalloc_refuses_scratch_beyond_its_array():
    P = slrgen.config2()                     # 3-D 64^3: about 6 MB of scratch per column
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.k + 1, nrhs_max=8)
    lib = slr.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    r = torch.zeros((8, P.n), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    st = lib.slr_apply_noalloc(h._h, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), 8, P.n, stream)
    assert st == 8 and b"bytes" in lib.slr_last_error_message()
    st = lib.slr_apply_noalloc(h._h, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), 1, P.n, stream)
    assert st == 0, lib.slr_last_error_message()
    torch.cuda.synchronize()
    h.close()
