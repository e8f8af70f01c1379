"""Thin Python binding of libkchol (include/kchol.h).

Argument marshalling only: every step runs in the library's sm_103a kernels.
PyTorch supplies device memory (tensors) and the CUDA stream; no torch type
crosses the C ABI.  There is no CPU fallback: if the shared library is
missing, importing the binding's functions raises.

Function names follow the C entry points without the ``kc_`` prefix.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libkchol.so")

KC_OK, KC_EINVAL, KC_ENOMEM, KC_ECUDA, KC_ETIMEOUT, KC_ENOTCONV, KC_ERANKDEF, KC_EINDEF = range(8)
RULE_MAX, RULE_MIN = 0, 1
FP64, FP32_FORM = 0, 1
_STATUS = {0: "KC_OK", 1: "KC_EINVAL", 2: "KC_ENOMEM", 3: "KC_ECUDA", 4: "KC_ETIMEOUT",
           5: "KC_ENOTCONV", 6: "KC_ERANKDEF", 7: "KC_EINDEF"}


class KcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


MATERN, CAUCHY = 0, 1


class kc_kernel(C.Structure):
    _fields_ = [("nu", C.c_double), ("ell", C.c_double), ("sigma2", C.c_double), ("nugget", C.c_double),
                ("family", C.c_int32), ("alpha", C.c_double), ("beta", C.c_double)]


class kc_pattern(C.Structure):
    _fields_ = [("N", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("colptr", C.c_void_p), ("rowidx", C.c_void_p), ("slot", C.c_void_p), ("order", C.c_void_p),
                ("depth", C.c_int32), ("level", C.c_void_p)]


class kc_opts(C.Structure):
    _fields_ = [("spin_limit_cycles", C.c_int64), ("rows_per_task", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("warps_per_cta", C.c_int32), ("test_hold_column", C.c_int32), ("lanes_per_row", C.c_int32),
                ("unroll", C.c_int32), ("adaptive_chunks", C.c_int32), ("stage_bytes", C.c_int32)]


_lib = None
ABI_VERSION = 5  # KC_ABI_VERSION of include/kchol.h that these signatures follow


def lib():
    """Load libkchol.so (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libkchol.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        P = C.POINTER
        L.kc_last_error.restype = C.c_char_p
        L.kc_abi_version.restype = i32
        if L.kc_abi_version() != ABI_VERSION:
            raise ImportError(f"libkchol.so has interface version {L.kc_abi_version()}, this binding needs "
                              f"{ABI_VERSION}; rebuild it with __graft_entry__.build()")
        L.kc_launch_count.restype = i64
        L.kc_last_factor_kernel_ms.restype = dbl
        sigs = {
            "kc_order_points": [vp, i64, i32, vp, vp, vp, vp],
            "kc_pattern_count": [vp, vp, i64, i32, dbl, i32, vp, P(C.c_int64), vp],
            "kc_pattern_fill": [vp, vp, i64, i32, dbl, i32, vp, vp, vp],
            "kc_pattern_begin": [vp, vp, i64, i32, dbl, i32, vp, P(C.c_int64), P(vp), vp],
            "kc_pattern_end": [vp, vp],
            "kc_schedule": [i64, vp, vp, vp, i32, vp, vp, vp, vp, vp, P(C.c_int32), vp],
            "kc_factor": [P(kc_pattern), vp, i32, P(kc_kernel), i32, vp, vp, P(C.c_int64), P(kc_opts), vp],
            "kc_solve": [P(kc_pattern), i32, vp, vp, P(kc_kernel), vp, vp, i32, vp, P(kc_opts), vp],
            "kc_solve_noalloc": [P(kc_pattern), i32, vp, vp, P(kc_kernel), vp, vp, i32, vp, vp],
            "kc_refine": [P(kc_pattern), vp, i32, P(kc_kernel), i32, vp, vp, vp, vp, i32, dbl, i32, vp,
                          P(C.c_int32), P(C.c_double), P(kc_opts), vp],
            "kc_pca_truncate": [P(kc_pattern), i32, vp, vp, i32, vp, vp],
            "kc_pca_error": [vp, i64, i32, P(kc_kernel), i32, vp, vp, i32, P(C.c_double), vp],
            "kc_factor_plan_create": [P(kc_pattern), vp, i32, P(kc_kernel), i32, vp, i32, P(kc_opts),
                                      P(vp), vp],
            "kc_factor_plan_launch": [vp, vp, vp, vp],
            "kc_factor_plan_finish": [vp, P(C.c_int64), vp],
            "kc_factor_plan_tune": [vp, vp, vp, P(C.c_int32), P(C.c_int32), P(C.c_double), vp],
            "kc_pattern_concat": [i32, P(vp), P(vp), P(C.c_int64), vp, vp, vp, vp],
            "kc_points_concat": [i32, P(vp), P(C.c_int64), P(C.c_int32), i32, vp, vp],
            "kc_index_concat": [i32, P(vp), P(C.c_int64), vp, vp],
            "kc_kernel_eval": [P(kc_kernel), i32, vp, i64, vp, vp],
            "kc_l_matvec": [P(kc_pattern), i32, vp, vp, vp, vp, i32, vp, vp],
            "kc_lt_matvec": [P(kc_pattern), i32, vp, vp, vp, vp, i32, vp, vp],
            "kc_llt_matvec": [P(kc_pattern), i32, vp, vp, vp, vp, i32, vp, vp],
            "kc_logdet": [P(kc_pattern), vp, P(C.c_double), P(C.c_int64), vp],
            "kc_pattern_reverse": [i64, vp, vp, vp, vp, vp],
            "kc_gather_entries": [i64, vp, vp, vp, vp, vp, vp, vp, P(C.c_int64), vp],
            "kc_factor_given": [P(kc_pattern), vp, i32, vp, vp, P(C.c_int64), P(kc_opts), vp],
            "kc_supernodal_count": [vp, vp, i32, dbl, P(kc_pattern), vp, vp, vp, vp, vp, vp, P(C.c_int64), vp],
            "kc_supernodal_fill": [vp, vp, i32, dbl, P(kc_pattern), vp, vp, vp],
            "kc_supernodal": [vp, vp, i32, dbl, P(kc_pattern), vp, vp, vp, vp, vp, vp, vp, i64, P(C.c_int64), vp],
            "kc_pattern_validate": [P(kc_pattern), vp],
            "kc_scratch_trim": [i64],
            "kc_factor_blocked": [P(kc_pattern), vp, i32, P(kc_kernel), i32, vp, vp, P(C.c_int64), P(kc_opts), vp],
            "kc_frob_error": [P(kc_pattern), i32, vp, vp, vp, i32, P(kc_kernel), vp, vp, vp, i64, vp, P(C.c_double),
                              P(C.c_double), P(C.c_int64), vp],
            "kc_refine_sparse": [P(kc_pattern), i32, vp, vp, vp, vp, vp, vp, vp, i32, dbl, i32, vp, P(C.c_int32),
                                 P(C.c_double), P(kc_opts), vp],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.kc_factor_plan_destroy.argtypes = [vp]
        L.kc_factor_plan_destroy.restype = None
        L.kc_pattern_abort.argtypes = [vp]
        L.kc_pattern_abort.restype = None
        _lib = L
    return _lib


EXPORTED = ("kc_last_error", "kc_abi_version", "kc_launch_count", "kc_last_factor_kernel_ms", "kc_order_points", "kc_pattern_count", "kc_pattern_fill",
            "kc_schedule", "kc_factor", "kc_solve", "kc_solve_noalloc", "kc_refine", "kc_pca_truncate", "kc_pca_error",
            "kc_factor_plan_create", "kc_factor_plan_launch", "kc_factor_plan_finish", "kc_factor_plan_tune",
            "kc_factor_plan_destroy", "kc_pattern_concat", "kc_points_concat", "kc_index_concat", "kc_kernel_eval",
            "kc_l_matvec", "kc_lt_matvec", "kc_llt_matvec", "kc_logdet", "kc_pattern_reverse",
            "kc_gather_entries", "kc_factor_given", "kc_refine_sparse", "kc_supernodal_count",
            "kc_supernodal_fill", "kc_supernodal", "kc_pattern_validate", "kc_scratch_trim",
            "kc_frob_error", "kc_factor_blocked", "kc_pattern_begin", "kc_pattern_end", "kc_pattern_abort")


def launch_count() -> int:
    """Kernels launched by libkchol in this process so far."""
    return int(lib().kc_launch_count())


def scratch_trim(keep_bytes: int = 0):
    """Release the current device's scratch pool down to keep_bytes."""
    _check(lib().kc_scratch_trim(int(keep_bytes)))


def last_factor_kernel_ms() -> float:
    """Device time of the last persistent factor kernel (CUDA events)."""
    return float(lib().kc_last_factor_kernel_ms())


def _check(st: int):
    if st != KC_OK:
        raise KcError(st, lib().kc_last_error().decode(errors="replace"))


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


@dataclass
class Kernel:
    """Covariance function: the Matern class (smoothness nu in (0, 50],
    length scale ell, variance sigma2) or, with family=CAUCHY, the Cauchy
    class (ell, alpha in (0, 2], beta > 0, sigma2); nugget on the diagonal."""
    nu: float = 1.5
    ell: float = 0.2
    sigma2: float = 1.0
    nugget: float = 0.0
    family: int = MATERN
    alpha: float = 1.0
    beta: float = 1.0

    def c(self):
        return kc_kernel(self.nu, self.ell, self.sigma2, self.nugget, self.family, self.alpha, self.beta)


def make_opts(spin_limit_cycles=0, rows_per_task=0, ctas_per_sm=0, warps_per_cta=0, test_hold_column=-1,
              lanes_per_row=0, unroll=0, adaptive_chunks=0, stage_bytes=0):
    return kc_opts(spin_limit_cycles, rows_per_task, ctas_per_sm, warps_per_cta, test_hold_column + 1,
                   lanes_per_row, unroll, adaptive_chunks, stage_bytes)


# ----------------------------------------------------------------- a2, a3, a4

def order_points(x: torch.Tensor, stream=None):
    """Maximin ordering of x (N, d) float64 on the GPU -> (perm int32, l float64, x_ord float64)."""
    _dev(x, torch.float64, "x")
    N, d = x.shape
    perm = torch.empty(N, dtype=torch.int32, device=x.device)
    l = torch.empty(N, dtype=torch.float64, device=x.device)
    xo = torch.empty_like(x)
    _check(lib().kc_order_points(_ptr(x), N, d, _ptr(perm), _ptr(l), _ptr(xo), _stream(stream)))
    return perm, l, xo


def pattern_count(x_ord, l, rho, rule=RULE_MAX, stream=None):
    _dev(x_ord, torch.float64, "x_ord")
    _dev(l, torch.float64, "l")
    N, d = x_ord.shape
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=x_ord.device)
    nnz = C.c_int64(0)
    _check(lib().kc_pattern_count(_ptr(x_ord), _ptr(l), N, d, float(rho), int(rule), _ptr(rowptr),
                                  C.byref(nnz), _stream(stream)))
    return rowptr, int(nnz.value)


def pattern_fill(x_ord, l, rho, rowptr, nnz, rule=RULE_MAX, stream=None):
    N, d = x_ord.shape
    _dev(rowptr, torch.int64, "rowptr")
    col = torch.empty(nnz, dtype=torch.int32, device=x_ord.device)
    _check(lib().kc_pattern_fill(_ptr(x_ord), _ptr(l), N, d, float(rho), int(rule), _ptr(rowptr), _ptr(col),
                                 _stream(stream)))
    return col


class Pattern:
    """Device CSR/CSC pattern of L plus its dependency schedule."""

    def __init__(self, rowptr, col, colptr, rowidx, slot, level, order, depth):
        self.rowptr, self.col, self.colptr, self.rowidx, self.slot = rowptr, col, colptr, rowidx, slot
        self.level, self.order, self.depth = level, order, depth
        self.N = rowptr.numel() - 1
        self.nnz = col.numel()
        self._c = kc_pattern(self.N, self.nnz, rowptr.data_ptr(), col.data_ptr(), colptr.data_ptr(),
                             rowidx.data_ptr(), slot.data_ptr(), order.data_ptr(), depth, level.data_ptr())

    def c(self):
        return C.byref(self._c)


def schedule(rowptr, col, x_ord=None, stream=None) -> Pattern:
    """CSC view, levels and the column order; with the points x_ord (N, d)
    the columns of each level go in Morton order of their points."""
    _dev(rowptr, torch.int64, "rowptr")
    _dev(col, torch.int32, "col")
    if x_ord is not None:
        _dev(x_ord, torch.float64, "x_ord")
    N = rowptr.numel() - 1
    nnz = col.numel()
    dev = rowptr.device
    colptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    rowidx = torch.empty(nnz, dtype=torch.int32, device=dev)
    slot = torch.empty(nnz, dtype=torch.int64, device=dev)
    level = torch.empty(N, dtype=torch.int32, device=dev)
    order = torch.empty(N, dtype=torch.int32, device=dev)
    depth = C.c_int32(0)
    d = int(x_ord.shape[1]) if x_ord is not None else 0
    _check(lib().kc_schedule(N, _ptr(rowptr), _ptr(col), _ptr(x_ord) if x_ord is not None else None, d,
                             _ptr(colptr), _ptr(rowidx), _ptr(slot), _ptr(level), _ptr(order), C.byref(depth),
                             _stream(stream)))
    return Pattern(rowptr, col, colptr, rowidx, slot, level, order, int(depth.value))


def pattern_validate(pat: Pattern, stream=None):
    """Raise KcError (KC_EINVAL) if the pattern or its schedule is malformed."""
    _check(lib().kc_pattern_validate(pat.c(), _stream(stream)))


# ------------------------------------------------------------------ a5, a6

def factor(pat: Pattern, x_ord, kern: Kernel, prec=FP32_FORM, opts: kc_opts | None = None, val=None, diag=None,
           stream=None):
    """ICHOL(0) -> (val [nnz] float64|float32, diag [N] float64, zero_pivots)."""
    _dev(x_ord, torch.float64, "x_ord")
    d = x_ord.shape[1]
    dt = torch.float64 if prec == FP64 else torch.float32
    if val is None:
        val = torch.empty(pat.nnz, dtype=dt, device=x_ord.device)
    if diag is None:
        diag = torch.empty(pat.N, dtype=torch.float64, device=x_ord.device)
    zp = C.c_int64(0)
    k = kern.c()
    _check(lib().kc_factor(pat.c(), _ptr(x_ord), d, C.byref(k), int(prec), _ptr(val), _ptr(diag), C.byref(zp),
                           C.byref(opts) if opts is not None else None, _stream(stream)))
    return val, diag, int(zp.value)


def factor_blocked(pat: Pattern, x_ord, kern: Kernel, prec=FP32_FORM, opts: kc_opts | None = None, val=None,
                   diag=None, stream=None):
    """The same factor by column groups (kc_factor_blocked) -> (val, diag, zero_pivots)."""
    _dev(x_ord, torch.float64, "x_ord")
    d = x_ord.shape[1]
    dt = torch.float64 if prec == FP64 else torch.float32
    if val is None:
        val = torch.empty(pat.nnz, dtype=dt, device=x_ord.device)
    if diag is None:
        diag = torch.empty(pat.N, dtype=torch.float64, device=x_ord.device)
    zp = C.c_int64(0)
    k = kern.c()
    _check(lib().kc_factor_blocked(pat.c(), _ptr(x_ord), d, C.byref(k), int(prec), _ptr(val), _ptr(diag),
                                   C.byref(zp), C.byref(opts) if opts is not None else None, _stream(stream)))
    return val, diag, int(zp.value)


# ------------------------------------------------------------- a7, a8, a9

def solve(pat: Pattern, prec, val, diag, kern: Kernel, perm, b, opts=None, stream=None):
    """x = (L L^T)^{-1} b; b is (nrhs, N) float64 in original order (row r = rhs r)."""
    _dev(b, torch.float64, "b")
    if b.dim() == 1:
        b = b[None]
    nrhs = b.shape[0]
    x = torch.empty_like(b)
    k = kern.c()
    _check(lib().kc_solve(pat.c(), int(prec), _ptr(val), _ptr(diag), C.byref(k), _ptr(perm), _ptr(b), nrhs,
                          _ptr(x), C.byref(opts) if opts is not None else None, _stream(stream)))
    return x


def solve_noalloc(pat: Pattern, prec, val, diag, kern: Kernel, perm, b, out=None, stream=None):
    """Same result as solve(), for callers that may not allocate device memory
    during the call: the library takes its scratch from a fixed device array
    (limits N <= 2^20 and N * nrhs <= 2^20).  Pass ``out`` (nrhs, N) float64 to
    keep this call free of allocations on the Python side too.  Calls that
    overlap on the GPU share that array and race: serialise them."""
    _dev(b, torch.float64, "b")
    if b.dim() == 1:
        b = b[None]
    nrhs = b.shape[0]
    x = torch.empty_like(b) if out is None else _dev(out, torch.float64, "out")
    k = kern.c()
    _check(lib().kc_solve_noalloc(pat.c(), int(prec), _ptr(val), _ptr(diag), C.byref(k), _ptr(perm), _ptr(b), nrhs,
                                  _ptr(x), _stream(stream)))
    return x


def refine(pat: Pattern, x_ord, kern: Kernel, prec, val, diag, perm, b, rtol=1e-10, maxit=200, opts=None,
           stream=None):
    """CG on the dense Theta preconditioned by L L^T -> (x, iters, relres per rhs, status)."""
    _dev(b, torch.float64, "b")
    if b.dim() == 1:
        b = b[None]
    nrhs = b.shape[0]
    x = torch.empty_like(b)
    it = C.c_int32(0)
    rr = (C.c_double * nrhs)()
    k = kern.c()
    st = lib().kc_refine(pat.c(), _ptr(x_ord), x_ord.shape[1], C.byref(k), int(prec), _ptr(val), _ptr(diag),
                         _ptr(perm), _ptr(b), nrhs, float(rtol), int(maxit), _ptr(x), C.byref(it), rr,
                         C.byref(opts) if opts is not None else None, _stream(stream))
    if st not in (KC_OK, KC_ENOTCONV, KC_EINDEF):
        _check(st)
    return x, int(it.value), [rr[i] for i in range(nrhs)], st


def pca_truncate(pat: Pattern, prec, val, perm, k, stream=None):
    """First k columns of L, rows in original order -> (k, N) float32."""
    Lk = torch.empty((k, pat.N), dtype=torch.float32, device=val.device)
    _check(lib().kc_pca_truncate(pat.c(), int(prec), _ptr(val), _ptr(perm), int(k), _ptr(Lk), _stream(stream)))
    return Lk


def pca_error(x, kern: Kernel, Lk, v0, iters=50, stream=None):
    """Power-iteration estimate of ||Theta - Lk^T Lk||_2 (x in original order)."""
    N, d = x.shape
    est = C.c_double(0.0)
    kk = kern.c()
    _check(lib().kc_pca_error(_ptr(x), N, d, C.byref(kk), Lk.shape[0], _ptr(Lk), _ptr(v0), int(iters),
                              C.byref(est), _stream(stream)))
    return float(est.value)


def kernel_eval(kern: Kernel, prec, r, stream=None):
    """The covariance function at distances r (float64 tensor), as the factor
    evaluates its entries in precision prec (no nugget)."""
    _dev(r, torch.float64, "r")
    out = torch.empty_like(r)
    k = kern.c()
    _check(lib().kc_kernel_eval(C.byref(k), int(prec), _ptr(r), r.numel(), _ptr(out), _stream(stream)))
    return out


def _factor_mv(fn, pat, prec, val, diag, perm, v, stream):
    _dev(v, torch.float64, "vector")
    one = v.dim() == 1
    if one:
        v = v[None]
    y = torch.empty_like(v)
    _check(fn(pat.c(), int(prec), _ptr(val), _ptr(diag), _ptr(perm), _ptr(v), v.shape[0], _ptr(y), _stream(stream)))
    return y[0] if one else y


def l_matvec(pat: Pattern, prec, val, diag, perm, z, stream=None):
    """y = P L P^T z; z (nrhs, N) or (N,) float64 in original order.  For
    z ~ N(0, I), y is a sample of N(0, L L^T) (task (4))."""
    return _factor_mv(lib().kc_l_matvec, pat, prec, val, diag, perm, z, stream)


def lt_matvec(pat: Pattern, prec, val, diag, perm, v, stream=None):
    """y = P L^T P^T v."""
    return _factor_mv(lib().kc_lt_matvec, pat, prec, val, diag, perm, v, stream)


def llt_matvec(pat: Pattern, prec, val, diag, perm, v, stream=None):
    """y = P L L^T P^T v, the factor's approximation of Theta v (task (1))."""
    return _factor_mv(lib().kc_llt_matvec, pat, prec, val, diag, perm, v, stream)


def logdet(pat: Pattern, diag, stream=None):
    """(log det(L L^T) over the kept pivots, number of dropped pivots): task (3)."""
    _dev(diag, torch.float64, "diag")
    v = C.c_double(0.0)
    z = C.c_int64(0)
    _check(lib().kc_logdet(pat.c(), _ptr(diag), C.byref(v), C.byref(z), _stream(stream)))
    return float(v.value), int(z.value)


def frob_error(pat: Pattern, prec, val, diag, x_ord, kern: Kernel, perm, pi, pj, keep=None, stream=None):
    """The sampled error estimator of Section 4.4 on the device: pairs pi, pj
    (int64, original numbering), optional int8 keep mask.  Returns (num2,
    den2, kept); E = sqrt(num2 / den2)."""
    _dev(x_ord, torch.float64, "x_ord")
    _dev(pi, torch.int64, "pi")
    _dev(pj, torch.int64, "pj")
    if keep is not None:
        _dev(keep, torch.int8, "keep")
    a, b, c = C.c_double(0.0), C.c_double(0.0), C.c_int64(0)
    kk = kern.c()
    _check(lib().kc_frob_error(pat.c(), int(prec), _ptr(val), _ptr(diag), _ptr(x_ord), x_ord.shape[1], C.byref(kk),
                               _ptr(perm), _ptr(pi), _ptr(pj), pi.numel(), _ptr(keep), C.byref(a), C.byref(b),
                               C.byref(c), _stream(stream)))
    return float(a.value), float(b.value), int(c.value)


# ------------------------------------------------------------------ the path

def pattern_rows(x_ord, l, rho, rule=RULE_MAX, stream=None):
    """The CSR rows of S_rho (rowptr int64, col int32) with one search
    (kc_pattern_begin / kc_pattern_end); the same arrays as pattern_count
    followed by pattern_fill."""
    _dev(x_ord, torch.float64, "x_ord")
    _dev(l, torch.float64, "l")
    N, d = x_ord.shape
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=x_ord.device)
    nnz = C.c_int64(0)
    h = C.c_void_p()
    _check(lib().kc_pattern_begin(_ptr(x_ord), _ptr(l), N, d, float(rho), int(rule), _ptr(rowptr), C.byref(nnz),
                                  C.byref(h), _stream(stream)))
    try:
        col = torch.empty(int(nnz.value), dtype=torch.int32, device=x_ord.device)
    except BaseException:
        lib().kc_pattern_abort(h)
        raise
    _check(lib().kc_pattern_end(h, _ptr(col)))
    return rowptr, col


def build_pattern(x_ord, l, rho, rule=RULE_MAX, stream=None) -> Pattern:
    rowptr, col = pattern_rows(x_ord, l, rho, rule, stream)
    return schedule(rowptr, col, x_ord, stream)


def pipeline(x, rho, kern: Kernel, prec=FP32_FORM, rule=RULE_MAX, opts=None, stream=None):
    """order -> pattern -> schedule -> factor, all on the device."""
    perm, l, xo = order_points(x, stream)
    pat = build_pattern(xo, l, rho, rule, stream)
    val, diag, zp = factor(pat, xo, kern, prec, opts, stream=stream)
    return dict(perm=perm, l=l, x_ord=xo, pat=pat, val=val, diag=diag, zero_pivots=zp)


# ------------------------------- supernodal multicolour ordering and pattern

def supernodal(x_ord, l, rho, pat: Pattern, with_schedule=True, stream=None):
    """The supernodal multicolour ordering and pattern from the maximin order
    (x_ord, l) and its max-rule pattern pat of the same rho -> dict with newm
    (maximin position of every new position), level, node, color, x_new,
    rowptr, col and (with_schedule) the scheduled pattern of the new order."""
    _dev(x_ord, torch.float64, "x_ord")
    _dev(l, torch.float64, "l")
    N, d = x_ord.shape
    dev = x_ord.device
    newm = torch.empty(N, dtype=torch.int32, device=dev)
    level = torch.empty(N, dtype=torch.int32, device=dev)
    node = torch.empty(N, dtype=torch.int32, device=dev)
    color = torch.empty(N, dtype=torch.int32, device=dev)
    x_new = torch.empty_like(x_ord)
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(0)
    # one pass when the guess holds the pattern (about 1.3x the max-rule one), else a second
    cap = 2 * pat.nnz + N
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    _check(lib().kc_supernodal(_ptr(x_ord), _ptr(l), d, float(rho), pat.c(), _ptr(newm), _ptr(level), _ptr(node),
                               _ptr(color), _ptr(x_new), _ptr(rowptr), _ptr(col), cap, C.byref(nnz),
                               _stream(stream)))
    if nnz.value > cap:
        col = torch.empty(int(nnz.value), dtype=torch.int32, device=dev)
        _check(lib().kc_supernodal_fill(_ptr(x_ord), _ptr(l), d, float(rho), pat.c(), _ptr(rowptr), _ptr(col),
                                        _stream(stream)))
    else:
        col = col[:nnz.value]
    spat = schedule(rowptr, col, x_new, stream) if with_schedule else None
    return dict(newm=newm, level=level, node=node, color=color, x_new=x_new, rowptr=rowptr, col=col, pat=spat)


def supernodal_pipeline(x, rho, kern: Kernel, prec=FP32_FORM, opts=None, stream=None):
    """order -> max-rule pattern -> supernodal ordering and pattern -> factor;
    ``perm`` maps a new position to the original index."""
    perm0, l, xo = order_points(x, stream)
    pat0 = build_pattern(xo, l, rho, RULE_MAX, stream)
    sn = supernodal(xo, l, rho, pat0, stream=stream)
    perm = perm0[sn["newm"].long()].contiguous()
    val, diag, zp = factor(sn["pat"], sn["x_new"], kern, prec, opts, stream=stream)
    return dict(perm=perm, sn=sn, pat=sn["pat"], x_new=sn["x_new"], val=val, diag=diag, zero_pivots=zp)


# ------------------------------------- Section 6: given matrix, reverse order

def pattern_reverse(pat: Pattern, x_ord=None, stream=None) -> Pattern:
    """The symmetric pattern of pat in the reversed order (position q holds
    position N-1-q of pat's order), scheduled; x_ord: pat's points, whose
    reversal orders each level spatially."""
    N = pat.N
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=pat.rowptr.device)
    col = torch.empty(pat.nnz, dtype=torch.int32, device=pat.rowptr.device)
    _check(lib().kc_pattern_reverse(N, _ptr(pat.colptr), _ptr(pat.rowidx), _ptr(rowptr), _ptr(col),
                                    _stream(stream)))
    xr = x_ord.flip(0).contiguous() if x_ord is not None else None
    return schedule(rowptr, col, xr, stream)


def gather_entries(pat: Pattern, orig, a_rowptr, a_col, a_val, count_outside=True, stream=None):
    """(aval float64[nnz], outside): the matrix A (CSR in original numbering,
    columns ascending) at every pattern position; orig maps a position to
    its original index.  outside = A's off-diagonal entries not in the
    pattern (None unless count_outside)."""
    _dev(orig, torch.int32, "orig")
    _dev(a_rowptr, torch.int64, "a_rowptr")
    _dev(a_col, torch.int32, "a_col")
    _dev(a_val, torch.float64, "a_val")
    aval = torch.empty(pat.nnz, dtype=torch.float64, device=orig.device)
    out = C.c_int64(0)
    _check(lib().kc_gather_entries(pat.N, _ptr(pat.rowptr), _ptr(pat.col), _ptr(orig), _ptr(a_rowptr), _ptr(a_col),
                                   _ptr(a_val), _ptr(aval), C.byref(out) if count_outside else None,
                                   _stream(stream)))
    return aval, (int(out.value) if count_outside else None)


def factor_given(pat: Pattern, aval, prec=FP32_FORM, opts: kc_opts | None = None, val=None, diag=None,
                 stream=None):
    """ICHOL(0) of the symmetric matrix given on the pattern (aval, CSR
    layout) -> (val, diag, zero_pivots)."""
    _dev(aval, torch.float64, "aval")
    dt = torch.float64 if prec == FP64 else torch.float32
    if val is None:
        val = torch.empty(pat.nnz, dtype=dt, device=aval.device)
    if diag is None:
        diag = torch.empty(pat.N, dtype=torch.float64, device=aval.device)
    zp = C.c_int64(0)
    _check(lib().kc_factor_given(pat.c(), _ptr(aval), int(prec), _ptr(val), _ptr(diag), C.byref(zp),
                                 C.byref(opts) if opts is not None else None, _stream(stream)))
    return val, diag, int(zp.value)


def refine_sparse(pat: Pattern, prec, val, diag, perm, a_rowptr, a_col, a_val, b, rtol=1e-10, maxit=200,
                  opts=None, stream=None):
    """CG on the given sparse A (CSR, original numbering) preconditioned by its
    factor -> (x, iters, relres per rhs, status)."""
    _dev(b, torch.float64, "b")
    if b.dim() == 1:
        b = b[None]
    nrhs = b.shape[0]
    x = torch.empty_like(b)
    it = C.c_int32(0)
    rr = (C.c_double * nrhs)()
    st = lib().kc_refine_sparse(pat.c(), int(prec), _ptr(val), _ptr(diag), _ptr(perm), _ptr(a_rowptr), _ptr(a_col),
                                _ptr(a_val), _ptr(b), nrhs, float(rtol), int(maxit), _ptr(x), C.byref(it), rr,
                                C.byref(opts) if opts is not None else None, _stream(stream))
    if st not in (KC_OK, KC_ENOTCONV, KC_EINDEF):
        _check(st)
    return x, int(it.value), list(rr), st


def reverse_factor(x, a_rowptr, a_col, a_val, rho, prec=FP32_FORM, opts=None, stream=None):
    """Section 6 on the device: maximin ordering of the points x, the
    min-rule pattern, reversed, the matrix A (CSR, original numbering)
    gathered onto it and factored.  ``orig`` (position -> original index)
    is the permutation the solves take."""
    perm, l, xo = order_points(x, stream)
    pat = build_pattern(xo, l, rho, RULE_MIN, stream)
    rpat = pattern_reverse(pat, xo, stream)
    orig = perm.flip(0).contiguous()
    aval, outside = gather_entries(rpat, orig, a_rowptr, a_col, a_val, stream=stream)
    val, diag, zp = factor_given(rpat, aval, prec, opts, stream=stream)
    return dict(perm=perm, l=l, x_ord=xo, orig=orig, pat=rpat, aval=aval, outside=outside, val=val, diag=diag,
                zero_pivots=zp)


# ------------------------------------------------------ plans and batching

class FactorPlan:
    """A factorisation plan: task list and counters of one pattern kept on the
    device, so that each factorisation is one persistent launch with no
    allocation and no host synchronisation (it can be recorded in a CUDA
    graph).  ``kerns`` has one Kernel per set and ``col_set`` (int32[N]) the
    set of every column when several sets are concatenated."""

    def __init__(self, pat: Pattern, x_ord, kerns, col_set=None, prec=FP32_FORM, opts=None, stream=None):
        _dev(x_ord, torch.float64, "x_ord")
        kerns = list(kerns)
        arr = (kc_kernel * len(kerns))(*[k.c() for k in kerns])
        h = C.c_void_p()
        self._keep = (pat, x_ord, col_set)
        self.prec = prec
        _check(lib().kc_factor_plan_create(pat.c(), _ptr(x_ord), x_ord.shape[1], arr, len(kerns), _ptr(col_set),
                                           int(prec), C.byref(opts) if opts is not None else None, C.byref(h),
                                           _stream(stream)))
        self._h = h

    def launch(self, val, diag, stream=None):
        _check(lib().kc_factor_plan_launch(self._h, _ptr(val), _ptr(diag), _stream(stream)))

    def finish(self, stream=None) -> int:
        zp = C.c_int64(0)
        _check(lib().kc_factor_plan_finish(self._h, C.byref(zp), _stream(stream)))
        return int(zp.value)

    def tune(self, val, diag, stream=None):
        """Time lanes-per-row x staging-depth once each and keep the fastest."""
        L, U, ms = C.c_int32(0), C.c_int32(0), C.c_double(0)
        _check(lib().kc_factor_plan_tune(self._h, _ptr(val), _ptr(diag), C.byref(L), C.byref(U), C.byref(ms),
                                         _stream(stream)))
        return {"lanes_per_row": L.value, "unroll": U.value, "ms": ms.value}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.kc_factor_plan_destroy(h)
            self._h = None


def _ptr_array(ts):
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def pattern_concat(rowptrs, cols, stream=None):
    """Block-diagonal concatenation -> (rowptr int64, col int32, set int32 per position)."""
    Ns = [r.numel() - 1 for r in rowptrs]
    tot = sum(Ns)
    nnz = sum(c.numel() for c in cols)
    dev = rowptrs[0].device
    rowptr = torch.empty(tot + 1, dtype=torch.int64, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    sets = torch.empty(tot, dtype=torch.int32, device=dev)
    _check(lib().kc_pattern_concat(len(Ns), _ptr_array(rowptrs), _ptr_array(cols), (C.c_int64 * len(Ns))(*Ns),
                                   _ptr(rowptr), _ptr(col), _ptr(sets), _stream(stream)))
    return rowptr, col, sets


def points_concat(xs, dout=None, stream=None):
    """Concatenate (N_s, d_s) float64 point sets, zero-padded to dout columns."""
    Ns = [x.shape[0] for x in xs]
    ds = [x.shape[1] for x in xs]
    dout = dout or max(ds)
    out = torch.empty((sum(Ns), dout), dtype=torch.float64, device=xs[0].device)
    _check(lib().kc_points_concat(len(xs), _ptr_array(xs), (C.c_int64 * len(Ns))(*Ns), (C.c_int32 * len(ds))(*ds),
                                  dout, _ptr(out), _stream(stream)))
    return out


def index_concat(idxs, stream=None):
    """Concatenate int32 index arrays, shifting set s by the sizes before it."""
    Ns = [t.numel() for t in idxs]
    out = torch.empty(sum(Ns), dtype=torch.int32, device=idxs[0].device)
    _check(lib().kc_index_concat(len(idxs), _ptr_array(idxs), (C.c_int64 * len(Ns))(*Ns), _ptr(out),
                                 _stream(stream)))
    return out
