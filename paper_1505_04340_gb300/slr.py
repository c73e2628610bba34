"""Python binding of the SLR C ABI (include/slr.h): argument marshalling only.

Every step of the preconditioner runs in the CUDA library ``lib/libslr.so``;
this module converts numpy host arrays and torch CUDA tensors to pointers and
status codes to exceptions.  There is no CPU fallback: if the library is not
built, loading it raises.

Vector convention: a vector is a float64 CUDA tensor of shape (n,); a block of
right-hand sides is a tensor of shape (n, nrhs) in any memory layout (it is
passed to the library as a column-major buffer).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libslr.so")

OK = 0
STATUS = {0: "SLR_OK", 1: "SLR_ERR_INVALID_ARG", 2: "SLR_ERR_NOT_SPD", 3: "SLR_ERR_OOM",
          4: "SLR_ERR_CUDA", 5: "SLR_ERR_NOT_CONVERGED", 6: "SLR_ERR_BREAKDOWN", 7: "SLR_ERR_TIMEOUT",
          8: "SLR_ERR_UNSUPPORTED"}
THETA = {"lambda_k1": 0, "zero": 1}
PRECISION = {"fp64": 0, "mixed": 1}

# every symbol include/slr.h declares
EXPORTS = ["slr_default_opts", "slr_setup", "slr_apply", "slr_pcg_solve", "slr_bsolve", "slr_csolve",
           "slr_stilde_solve", "slr_set_lowrank", "slr_get_lowrank", "slr_get_ritz", "slr_get_perm",
           "slr_get_info", "slr_dd_order", "slr_kernel_launches", "slr_destroy", "slr_status_str",
           "slr_last_error_message", "slr_apply_noalloc", "slr_add_vectors", "slr_gmres_solve",
           "slr_device_status", "slr_inject_alloc_failure", "slr_cg_slot_start", "slr_cg_advance",
           "slr_cg_slot_result"]


U_DTYPE = {"fp32": 0, "tf32": 1, "bf16": 2}


class Opts(C.Structure):
    _fields_ = [("k", C.c_int32), ("lanczos_steps", C.c_int32), ("theta_mode", C.c_int32),
                ("precision", C.c_int32), ("nrhs_max", C.c_int32), ("flexible_cg", C.c_int32),
                ("seed", C.c_uint64), ("c_leaf", C.c_int32), ("verbose", C.c_int32),
                ("target_kappa", C.c_int32), ("indefinite", C.c_int32), ("u_dtype", C.c_int32),
                ("band_split", C.c_int32), ("band_slots", C.c_int32), ("band_threads", C.c_int32),
                ("band_order", C.c_int32), ("band_factor_host", C.c_int32), ("c_persistent", C.c_int32),
                ("c_levels_only", C.c_int32), ("host_loop", C.c_int32), ("autotune", C.c_int32),
                ("zform", C.c_int32), ("band_mma", C.c_int32), ("spin_limit", C.c_int32),
                ("reserved", C.c_int32 * 6)]


class Info(C.Structure):
    _fields_ = [(f, C.c_int64) for f in (
        "n", "n_interior", "s", "nparts", "k", "lanczos_steps", "nnz_A", "nnz_E", "nnz_C",
        "band_entries", "c_diag_entries", "c_panel_entries", "c_supernodes", "c_levels",
        "bytes_per_apply", "flops_per_apply", "device_bytes")] + [
        ("theta", C.c_double), ("setup_seconds", C.c_double * 5), ("precision", C.c_int32),
        ("theta_mode", C.c_int32), ("band_split", C.c_int32), ("band_slots", C.c_int32),
        ("c_persistent", C.c_int32), ("tuned", C.c_int32), ("tune_seconds", C.c_double),
        ("band_threads", C.c_int32), ("c_top_levels", C.c_int32), ("c_top_positions", C.c_int32),
        ("c_top_entries", C.c_int64), ("band_on_device", C.c_int32), ("lanczos_seconds", C.c_double * 3),
        ("band_mma", C.c_int32), ("u_dtype", C.c_int32), ("vector_bytes_per_column", C.c_int64)]


class SLRError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.slr_last_error_message().decode(errors="replace") if _lib else ""
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")


_lib = None


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"SLR CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, f64 = C.c_void_p, C.c_int32, C.c_double
    P = C.POINTER
    sig = {
        "slr_default_opts": (None, [P(Opts)]),
        "slr_setup": (i32, [i32, vp, vp, vp, i32, vp, P(Opts), vp, P(vp)]),
        "slr_apply": (i32, [vp, vp, vp, i32, i32, vp]),
        "slr_apply_noalloc": (i32, [vp, vp, vp, i32, i32, vp]),
        "slr_pcg_solve": (i32, [vp, vp, vp, i32, i32, f64, i32, vp, vp, vp]),
        "slr_gmres_solve": (i32, [vp, vp, vp, i32, i32, f64, i32, i32, vp, vp, vp]),
        "slr_bsolve": (i32, [vp, vp, vp, i32, i32, vp]),
        "slr_csolve": (i32, [vp, vp, vp, i32, i32, vp]),
        "slr_stilde_solve": (i32, [vp, vp, vp, i32, i32, vp]),
        "slr_set_lowrank": (i32, [vp, i32, vp, vp, f64, vp]),
        "slr_add_vectors": (i32, [vp, i32, i32, vp, vp]),
        "slr_get_lowrank": (i32, [vp, vp, vp, vp, vp]),
        "slr_get_ritz": (i32, [vp, vp, vp]),
        "slr_get_perm": (i32, [vp, vp]),
        "slr_get_info": (i32, [vp, P(Info)]),
        "slr_dd_order": (i32, [i32, vp, vp, i32, vp, vp, vp, vp, vp]),
        "slr_kernel_launches": (C.c_int64, []),
        "slr_device_status": (i32, [vp, vp]),
        "slr_cg_slot_start": (i32, [vp, i32, vp, f64, i32, vp]),
        "slr_cg_advance": (i32, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "slr_cg_slot_result": (i32, [vp, i32, vp, vp]),
        "slr_inject_alloc_failure": (None, [C.c_int64]),
        "slr_destroy": (None, [vp]),
        "slr_status_str": (C.c_char_p, [i32]),
        "slr_last_error_message": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, where):
    if status != OK:
        raise SLRError(status, where)


def _host_ptr(a):
    return C.c_void_p(a.ctypes.data) if a.size else None


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _as_colmajor(x, n, name):
    """(n,) or (n, r) float64 CUDA tensor -> (buffer of shape (r, n) contiguous, r, was_1d)."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if x.dim() == 1:
        if x.shape[0] != n:
            raise ValueError(f"{name} has length {x.shape[0]}, expected {n}")
        return x.contiguous().view(1, n), 1, True
    if x.dim() != 2 or x.shape[0] != n:
        raise ValueError(f"{name} must have shape ({n},) or ({n}, nrhs)")
    return x.t().contiguous(), x.shape[1], False


def _back(buf, was_1d):
    return buf.view(-1) if was_1d else buf.t()


def kernel_launches():
    """Kernels the library has launched in this process so far."""
    return int(load().slr_kernel_launches())


def dd_order(rowptr, colind, part, nparts):
    """Host-only interface detection and DD order (Eq. 2.2) through the library."""
    lib = load()
    rowptr, colind, part = _i32(rowptr), _i32(colind), _i32(part)
    n = len(rowptr) - 1
    perm = np.empty(n, np.int32)
    io = np.empty(nparts + 1, np.int32)
    fo = np.empty(nparts + 1, np.int32)
    s = C.c_int32(0)
    _check(lib.slr_dd_order(n, _host_ptr(rowptr), _host_ptr(colind), nparts, _host_ptr(part),
                            _host_ptr(perm), _host_ptr(io), _host_ptr(fo), C.byref(s)), "slr_dd_order")
    return perm, io, fo, s.value


class SLR:
    """An SLR preconditioner resident on the current CUDA device (``slr_setup``)."""

    def __init__(self, rowptr, colind, val, part, nparts, k=16, lanczos_steps=0, theta="lambda_k1",
                 precision="fp64", nrhs_max=1, flexible_cg=False, seed=1, c_leaf=64, verbose=False,
                 band_split=0, host_loop=False, band_slots=0, c_persistent=False, autotune=False, target_kappa=0,
                 band_threads=0, c_top_zone=True, band_factor="auto", indefinite=False, band_order=0,
                 u_dtype="fp32", band_mma="off", spin_limit=0, zform=False, stream=None):
        lib = load()
        self._lib = lib
        self._h = None
        o = Opts()
        lib.slr_default_opts(C.byref(o))
        o.k, o.lanczos_steps = int(k), int(lanczos_steps)
        o.theta_mode, o.precision = THETA[theta], PRECISION[precision]
        o.nrhs_max, o.flexible_cg, o.seed = int(nrhs_max), int(bool(flexible_cg)), int(seed)
        o.c_leaf, o.verbose = int(c_leaf), int(bool(verbose))
        o.band_split = int(band_split)          # CTAs per subdomain in the band solve, 0 = automatic
        o.host_loop = int(bool(host_loop))      # CG loop driven from the host instead of a CUDA graph
        o.band_slots = int(band_slots)          # band-solve stream buffers, 0 = automatic
        o.c_persistent = int(bool(c_persistent))  # C solves in one cooperative launch per direction
        o.autotune = int(bool(autotune))        # time the candidates at setup and keep the fastest
        o.target_kappa = int(target_kappa)      # rank by the rule lambda_{k+1} <= 1 - 1/K (0 = off)
        o.band_threads = int(band_threads)      # threads per band-solve CTA: 512, 256, 32 or 0 (automatic)
        o.c_levels_only = 0 if c_top_zone else 1  # explicit inverse of the factor's top levels
        o.band_factor_host = {"auto": 0, "host": 1}[band_factor]   # B_i factored on the device or the host
        o.indefinite = int(bool(indefinite))    # symmetric indefinite A with an SPD interface
        o.band_order = int(band_order)          # band-solve cluster launch order, 0 = automatic
        o.u_dtype = U_DTYPE[u_dtype]            # low-rank products on RHS blocks: fp32, tf32, bf16
        o.band_mma = {"off": 0, "tf32": 1, "bf16": 2}[band_mma]   # band solve of RHS blocks on tensor cores
        o.zform = int(bool(zform))              # S~^{-1} in the Z-form of Proposition 4.3
        o.spin_limit = int(spin_limit)          # polls of a grid-barrier wait, 0 = default
        self.rowptr, self.colind = _i32(rowptr), _i32(colind)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.part = _i32(part)
        self.n = len(self.rowptr) - 1
        h = C.c_void_p()
        _check(lib.slr_setup(self.n, _host_ptr(self.rowptr), _host_ptr(self.colind), _host_ptr(self.val),
                             int(nparts), _host_ptr(self.part), C.byref(o), _stream_ptr(stream),
                             C.byref(h)), "slr_setup")
        self._h = h
        self.nrhs_max = int(nrhs_max)
        self.info = self.get_info()
        self.s = self.info["s"]
        self.n_interior = self.info["n_interior"]

    # -- lifetime
    def close(self):
        if self._h is not None:
            self._lib.slr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- info
    def get_info(self):
        inf = Info()
        _check(self._lib.slr_get_info(self._h, C.byref(inf)), "slr_get_info")
        d = {f: getattr(inf, f) for f, _ in Info._fields_}
        d["setup_seconds"] = list(inf.setup_seconds)
        d["lanczos_seconds"] = list(inf.lanczos_seconds)
        return d

    def perm(self):
        p = np.empty(self.n, np.int32)
        _check(self._lib.slr_get_perm(self._h, _host_ptr(p)), "slr_get_perm")
        return p

    def ritz(self):
        lam = np.empty(max(self.info["lanczos_steps"], 1), np.float64)
        cnt = C.c_int32(0)
        _check(self._lib.slr_get_ritz(self._h, _host_ptr(lam), C.byref(cnt)), "slr_get_ritz")
        return lam[:cnt.value].copy()

    def get_lowrank(self, stream=None):
        k = self.get_info()["k"]
        Z = np.empty((k, self.s), np.float64)        # column-major s x k
        lam = np.empty(k + 1, np.float64)
        th = C.c_double(0)
        _check(self._lib.slr_get_lowrank(self._h, _host_ptr(Z) if k else None, _host_ptr(lam), C.byref(th),
                                         _stream_ptr(stream)), "slr_get_lowrank")
        return Z.T.copy(), lam, th.value

    def set_lowrank(self, Z, lam, theta, stream=None):
        Z = np.asarray(Z, dtype=np.float64)
        k = Z.shape[1] if Z.ndim == 2 else 0
        Zc = np.ascontiguousarray(Z.T)               # column-major s x k
        lam = np.ascontiguousarray(lam[:k], dtype=np.float64)
        _check(self._lib.slr_set_lowrank(self._h, k, _host_ptr(Zc) if k else None,
                                         _host_ptr(lam) if k else None, float(theta), _stream_ptr(stream)),
               "slr_set_lowrank")
        self.info = self.get_info()

    def add_vectors(self, k_add, lanczos_steps=0, stream=None):
        """Improve the preconditioner by k_add more eigenvector estimates of H, keeping
        the ones it has (Section 5.3, deflated Lanczos).  Returns how many were added."""
        added = C.c_int32(0)
        _check(self._lib.slr_add_vectors(self._h, int(k_add), int(lanczos_steps), _stream_ptr(stream),
                                         C.byref(added)), "slr_add_vectors")
        self.info = self.get_info()
        return added.value

    # -- the operator
    def _call(self, fn, x, rows, name, stream, out=None):
        buf, r, one = _as_colmajor(x, rows, name)
        res = buf if out is None else _as_colmajor(out, rows, "out")[0]
        if out is None:
            import torch
            res = torch.empty_like(buf)
        _check(fn(self._h, C.c_void_p(buf.data_ptr()), C.c_void_p(res.data_ptr()), r, rows,
                  _stream_ptr(stream)), fn.__name__)
        return _back(res, one)

    def apply(self, r, stream=None):
        """z = M^{-1} r in DD order (Eq. 4.1)."""
        return self._call(self._lib.slr_apply, r, self.n, "r", stream)

    def apply_noalloc(self, r, stream=None):
        """z = M^{-1} r with the scratch in the library's fixed device array (no allocation)."""
        return self._call(self._lib.slr_apply_noalloc, r, self.n, "r", stream)

    def device_status(self, stream=None):
        """Status of the device's bounded waits in the calls enqueued so far
        (0, or 7 = SLR_ERR_TIMEOUT: the last call's outputs are invalid)."""
        return int(self._lib.slr_device_status(self._h, _stream_ptr(stream)))

    def bsolve(self, f, stream=None):
        """t = B^{-1} f on the interior unknowns (DD order)."""
        return self._call(self._lib.slr_bsolve, f, self.n_interior, "f", stream)

    def csolve(self, g, stream=None):
        """y = C^{-1} g on the interface unknowns (DD order)."""
        return self._call(self._lib.slr_csolve, g, self.s, "g", stream)

    def stilde_solve(self, g, stream=None):
        """y = S~^{-1} g (Eq. 4.7) on the interface unknowns (DD order)."""
        return self._call(self._lib.slr_stilde_solve, g, self.s, "g", stream)

    def gmres(self, b, tol=1e-8, maxit=300, restart=40, stream=None, check=True):
        """Solve A x = b (original order) by SLR-preconditioned flexible GMRES(restart)
        (Section 6, the symmetric indefinite problems).

        Returns (x, iterations[nrhs], relres[nrhs], status)."""
        import torch
        buf, r, one = _as_colmajor(b, self.n, "b")
        x = torch.empty_like(buf)
        its = np.zeros(r, np.int32)
        rel = np.zeros(r, np.float64)
        st = self._lib.slr_gmres_solve(self._h, C.c_void_p(buf.data_ptr()), C.c_void_p(x.data_ptr()), r,
                                       self.n, float(tol), int(maxit), int(restart), _stream_ptr(stream),
                                       _host_ptr(its), _host_ptr(rel))
        if check and st not in (OK, 5):
            _check(st, "slr_gmres_solve")
        return _back(x, one), its, rel, st

    # -- continuous batching: CG slots (slr_cg_*)
    def cg_start(self, slot, b, tol=1e-8, maxit=300, stream=None):
        """Start slot `slot` on the right-hand side b (float64 CUDA tensor (n,), original order)."""
        b = b.contiguous()
        if not (b.is_cuda and b.dtype.is_floating_point and b.numel() == self.n):
            raise ValueError("b must be a float64 CUDA vector of length n")
        _check(self._lib.slr_cg_slot_start(self._h, int(slot), C.c_void_p(b.data_ptr()), float(tol), int(maxit),
                                          _stream_ptr(stream)), "slr_cg_slot_start")
        return b

    def cg_advance(self, iters, width, stream=None):
        """Run `iters` iterations over slots 0 .. width-1; returns (active, iterations,
        relres, status) per slot (numpy arrays)."""
        act = np.zeros(width, np.int32)
        its = np.zeros(width, np.int32)
        rel = np.zeros(width, np.float64)
        sts = np.zeros(width, np.int32)
        _check(self._lib.slr_cg_advance(self._h, int(iters), int(width), _stream_ptr(stream), _host_ptr(act),
                                        _host_ptr(its), _host_ptr(rel), _host_ptr(sts)), "slr_cg_advance")
        return act, its, rel, sts

    def cg_result(self, slot, out=None, stream=None):
        """x of a slot (original order) as a float64 CUDA tensor (n,)."""
        import torch
        x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(self._lib.slr_cg_slot_result(self._h, int(slot), C.c_void_p(x.data_ptr()), _stream_ptr(stream)),
               "slr_cg_slot_result")
        return x

    def pcg(self, b, tol=1e-8, maxit=300, stream=None, check=True):
        """Solve A x = b (original order) by SLR-preconditioned CG.

        Returns (x, iterations[nrhs], relres[nrhs], status)."""
        import torch
        buf, r, one = _as_colmajor(b, self.n, "b")
        x = torch.empty_like(buf)
        its = np.zeros(r, np.int32)
        rel = np.zeros(r, np.float64)
        st = self._lib.slr_pcg_solve(self._h, C.c_void_p(buf.data_ptr()), C.c_void_p(x.data_ptr()), r,
                                     self.n, float(tol), int(maxit), _stream_ptr(stream), _host_ptr(its),
                                     _host_ptr(rel))
        if check and st not in (OK, 5):
            _check(st, "slr_pcg_solve")
        return _back(x, one), its, rel, st
