"""Thin ctypes binding of libgencd (include/gencd.h).

Argument marshalling only: every step of GenCD runs in the CUDA library.
Functions keep the C names.  Host buffers are numpy arrays; device buffers are
CUDA torch tensors (their data pointer is passed with GENCD_DEVICE).  The CUDA
stream defaults to torch's current stream.

Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgencd.so")

GENCD_OK = 0
GENCD_NOT_CONVERGED = 1
GENCD_EINVAL = -1
GENCD_ENOMEM = -2
GENCD_ECUDA = -3
GENCD_ETIMEOUT = -4
GENCD_EDIVERGED = -5
GENCD_ESTATE = -6

GENCD_LOSS_SQUARED, GENCD_LOSS_LOGISTIC = 0, 1
GENCD_SHOTGUN, GENCD_THREAD_GREEDY, GENCD_GREEDY, GENCD_COLORING, GENCD_TOP_GREEDY, GENCD_SHOTGUN_BLOCKS = \
    0, 1, 2, 3, 4, 5
GENCD_F64, GENCD_F32, GENCD_BF16, GENCD_BINARY = 0, 1, 2, 3
GENCD_HOST, GENCD_DEVICE = 0, 1

LOSSES = {"squared": GENCD_LOSS_SQUARED, "logistic": GENCD_LOSS_LOGISTIC}
VARIANTS = {"shotgun": GENCD_SHOTGUN, "thread_greedy": GENCD_THREAD_GREEDY, "greedy": GENCD_GREEDY,
            "coloring": GENCD_COLORING, "top_greedy": GENCD_TOP_GREEDY, "shotgun_blocks": GENCD_SHOTGUN_BLOCKS}
PRECISIONS = {"f64": GENCD_F64, "f32": GENCD_F32, "bf16": GENCD_BF16, "binary": GENCD_BINARY}
KERNELS = ["propose_all", "finalize", "accept", "update", "refresh", "propose_list", "coloring_iter",
           "objective", "setup", "propose_light", "propose_slabs", "scale_heavy", "propose_fused"]

# every symbol include/gencd.h declares
EXPORTS = ["gencd_create", "gencd_destroy", "gencd_set_lambda", "gencd_set_loss", "gencd_lambda_max",
           "gencd_default_params", "gencd_set_params", "gencd_get_params", "gencd_solve",
           "gencd_iterate", "gencd_set_iteration", "gencd_get_iteration", "gencd_get_w",
           "gencd_set_w", "gencd_get_z", "gencd_objective", "gencd_propose_at", "gencd_propose_all",
           "gencd_spectral_radius", "gencd_color", "gencd_color_balanced_csc", "gencd_get_colors", "gencd_set_colors",
           "gencd_permutation", "gencd_profile_enable", "gencd_profile_read", "gencd_profile_reset",
           "gencd_last_error", "gencd_stats", "gencd_stats_reset", "gencd_propose_all_noalloc",
           "gencd_propose_schedule", "gencd_set_propose_schedule", "gencd_block_pstar", "gencd_duality_gap",
           # include/gencd_batch.h
           "gencd_batch_create", "gencd_batch_destroy", "gencd_batch_slots", "gencd_batch_lambda_max",
           "gencd_batch_set_params", "gencd_batch_set_slot", "gencd_batch_copy_slot", "gencd_batch_clear_slot",
           "gencd_batch_get_w", "gencd_batch_iterate", "gencd_batch_objective", "gencd_batch_propose",
           "gencd_batch_path", "gencd_batch_schedule", "gencd_batch_set_schedule",
           # include/gencd_serve.h
           "gencd_serve", "gencd_serve_dry_run"]


class gencd_params(C.Structure):
    _fields_ = [("variant", C.c_int32), ("blocks", C.c_int32), ("P", C.c_int64), ("seed", C.c_uint64),
                ("max_iter", C.c_int64), ("tol_kkt", C.c_double), ("check_every", C.c_int32),
                ("beta_mode", C.c_int32), ("timeout_s", C.c_double), ("improve_steps", C.c_int32),
                ("reserved", C.c_int32), ("tol_gap", C.c_double)]


class gencd_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("reserved", C.c_int32), ("iters", C.c_int64),
                ("updates", C.c_int64), ("nnz_processed", C.c_int64), ("objective", C.c_double),
                ("kkt", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class gencd_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int64), ("nnz", C.c_int64), ("col_ptr", C.c_void_p),
                ("row_idx", C.c_void_p), ("val", C.c_void_p), ("val_dtype", C.c_int32), ("loss", C.c_int32),
                ("y", C.c_void_p), ("lambda_frac", C.c_double), ("arrival", C.c_double)]


class gencd_serve_params(C.Structure):
    _fields_ = [("workers", C.c_int32), ("precision", C.c_int32), ("hbm_fraction", C.c_double),
                ("params", gencd_params), ("tol_rel", C.c_double)]


class gencd_response(C.Structure):
    _fields_ = [("status", C.c_int32), ("worker", C.c_int32), ("iters", C.c_int64), ("lambda_", C.c_double),
                ("objective", C.c_double), ("kkt", C.c_double), ("arrival", C.c_double), ("start", C.c_double),
                ("end", C.c_double), ("bytes", C.c_int64)]


class gencd_path(C.Structure):
    _fields_ = [("nchains", C.c_int32), ("nlambda", C.c_int32), ("held_out", C.c_void_p), ("lambda_", C.c_void_p),
                ("handoff", C.c_double), ("warm", C.c_int32), ("reserved", C.c_int32), ("tol_rel", C.c_double)]


class gencd_path_solve(C.Structure):
    _fields_ = [("status", C.c_int32), ("slot", C.c_int32), ("iters", C.c_int64), ("objective", C.c_double),
                ("kkt", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double), ("group", C.c_int32),
                ("reserved", C.c_int32)]


class GencdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gencd error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Loads libgencd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        pp = C.POINTER(C.c_void_p)
        sig = {
            "gencd_create": (C.c_int, [pp, i64, i64, i64, vp, vp, vp, i32, vp, i32, i32, i32, vp]),
            "gencd_destroy": (None, [vp]),
            "gencd_set_lambda": (C.c_int, [vp, f64]),
            "gencd_set_loss": (C.c_int, [vp, i32]),
            "gencd_lambda_max": (C.c_int, [vp, C.POINTER(f64)]),
            "gencd_default_params": (C.c_int, [C.POINTER(gencd_params)]),
            "gencd_set_params": (C.c_int, [vp, C.POINTER(gencd_params)]),
            "gencd_get_params": (C.c_int, [vp, C.POINTER(gencd_params)]),
            "gencd_solve": (C.c_int, [vp, C.POINTER(gencd_result)]),
            "gencd_iterate": (C.c_int, [vp, i64, C.POINTER(gencd_result)]),
            "gencd_set_iteration": (C.c_int, [vp, i64]),
            "gencd_get_iteration": (C.c_int, [vp, C.POINTER(i64)]),
            "gencd_get_w": (C.c_int, [vp, vp, i64, i32]),
            "gencd_set_w": (C.c_int, [vp, vp, i64, i32]),
            "gencd_get_z": (C.c_int, [vp, vp, i64, i32]),
            "gencd_objective": (C.c_int, [vp, C.POINTER(f64), C.POINTER(f64)]),
            "gencd_duality_gap": (C.c_int, [vp, C.POINTER(f64), C.POINTER(f64), C.POINTER(f64)]),
            "gencd_propose_at": (C.c_int, [vp, vp, i64, vp, vp, i32]),
            "gencd_propose_all": (C.c_int, [vp, vp, vp, i32, C.POINTER(f64)]),
            "gencd_spectral_radius": (C.c_int, [vp, C.POINTER(f64), C.POINTER(i64), C.POINTER(i32)]),
            "gencd_color": (C.c_int, [vp, C.POINTER(i32)]),
            "gencd_block_pstar": (C.c_int, [vp, i32, vp, vp]),
            "gencd_color_balanced_csc": (C.c_int, [i64, i64, vp, vp, i64, vp, C.POINTER(i32)]),
            "gencd_get_colors": (C.c_int, [vp, vp, i64, i32]),
            "gencd_set_colors": (C.c_int, [vp, vp, i64, i32]),
            "gencd_permutation": (C.c_int, [vp, C.c_uint64, i64, i64, vp]),
            "gencd_profile_enable": (C.c_int, [vp, i32]),
            "gencd_profile_read": (C.c_int, [vp, i32, C.POINTER(f64), C.POINTER(i64), C.POINTER(i64)]),
            "gencd_profile_reset": (C.c_int, [vp]),
            "gencd_propose_schedule": (C.c_int, [vp, C.POINTER(i32), C.POINTER(f64), i32]),
            "gencd_set_propose_schedule": (C.c_int, [vp, i32]),
            "gencd_last_error": (C.c_char_p, []),
            "gencd_stats": (C.c_int, [vp, C.POINTER(gencd_result)]),
            "gencd_stats_reset": (C.c_int, [vp]),
            "gencd_propose_all_noalloc": (C.c_int, [i64, i64, i64, vp, vp, vp, vp, vp, vp, i32, f64, i32, vp, vp,
                                                    vp, vp]),
            # include/gencd_batch.h
            "gencd_batch_create": (C.c_int, [pp, i64, i64, i64, vp, vp, vp, i32, vp, i32, vp, i32, i32, i32, vp]),
            "gencd_batch_destroy": (None, [vp]),
            "gencd_batch_slots": (C.c_int, [vp, C.POINTER(i32)]),
            "gencd_batch_lambda_max": (C.c_int, [vp, i32, C.POINTER(f64)]),
            "gencd_batch_set_params": (C.c_int, [vp, C.POINTER(gencd_params)]),
            "gencd_batch_set_slot": (C.c_int, [vp, i32, i32, f64, vp, i32]),
            "gencd_batch_copy_slot": (C.c_int, [vp, i32, i32, i32, f64]),
            "gencd_batch_clear_slot": (C.c_int, [vp, i32]),
            "gencd_batch_get_w": (C.c_int, [vp, i32, vp, i64, i32]),
            "gencd_batch_iterate": (C.c_int, [vp, i64, i32]),
            "gencd_batch_objective": (C.c_int, [vp, vp, vp]),
            "gencd_batch_propose": (C.c_int, [vp, vp, vp, i32]),
            "gencd_batch_path": (C.c_int, [vp, C.POINTER(gencd_path), vp, vp, C.POINTER(gencd_result)]),
            "gencd_batch_schedule": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(f64), i32]),
            "gencd_batch_set_schedule": (C.c_int, [vp, i32, i32]),
            # include/gencd_serve.h
            "gencd_serve": (C.c_int, [vp, i64, C.POINTER(gencd_serve_params), vp, vp]),
            "gencd_serve_dry_run": (C.c_int, [vp, i64, C.POINTER(gencd_serve_params), f64, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def gencd_last_error() -> str:
    return lib().gencd_last_error().decode()


def _check(rc):
    if rc < 0:
        raise GencdError(rc, gencd_last_error())
    return rc


def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _buf(a, dtype):
    """(pointer, memory kind, keep-alive) of a numpy array or a CUDA tensor."""
    if a is None:
        return None, GENCD_HOST, None
    if _is_cuda_tensor(a):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), GENCD_DEVICE, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), GENCD_HOST, arr


def default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def gencd_create(n, k, nnz, col_ptr, row_idx, val, y, loss="logistic", precision="f64", stream=None):
    """Returns an opaque handle (c_void_p).  Inputs are all numpy arrays (host)
    or all CUDA tensors (device); the library copies them."""
    if _is_cuda_tensor(val):
        val_dtype = 0 if str(val.dtype) == "torch.float64" else 1
        vdt = None
    else:
        vdt = np.float32 if np.asarray(val).dtype == np.float32 else np.float64
        val_dtype = 0 if vdt == np.float64 else 1
    cp, m0, k0 = _buf(col_ptr, np.int64)
    ri, m1, k1 = _buf(row_idx, np.int32)
    va, m2, k2 = _buf(val, vdt)
    yy, m3, k3 = _buf(y, np.float64)
    mems = {m0, m1, m2, m3} if nnz > 0 else {m0, m3}
    if len(mems) != 1:
        raise ValueError("inputs must be all host arrays or all device tensors")
    handle = C.c_void_p()
    st = default_stream() if stream is None else int(stream)
    _check(lib().gencd_create(C.byref(handle), int(n), int(k), int(nnz), cp, ri, va, val_dtype, yy,
                              LOSSES.get(loss, loss), PRECISIONS.get(precision, precision), mems.pop(),
                              C.c_void_p(st)))
    del k0, k1, k2, k3
    return handle


def gencd_destroy(h):
    lib().gencd_destroy(h)


def gencd_set_lambda(h, lam):
    _check(lib().gencd_set_lambda(h, float(lam)))


def gencd_set_loss(h, loss):
    _check(lib().gencd_set_loss(h, LOSSES.get(loss, loss)))


def gencd_lambda_max(h) -> float:
    v = C.c_double()
    _check(lib().gencd_lambda_max(h, C.byref(v)))
    return v.value


def gencd_default_params() -> gencd_params:
    p = gencd_params()
    _check(lib().gencd_default_params(C.byref(p)))
    return p


def gencd_set_params(h, params: gencd_params):
    _check(lib().gencd_set_params(h, C.byref(params)))


def gencd_get_params(h) -> gencd_params:
    p = gencd_params()
    _check(lib().gencd_get_params(h, C.byref(p)))
    return p


def gencd_solve(h) -> gencd_result:
    """Runs to convergence; a diverged solve is reported in result.status
    (GENCD_EDIVERGED) rather than raised."""
    r = gencd_result()
    rc = lib().gencd_solve(h, C.byref(r))
    if rc < 0 and rc != GENCD_EDIVERGED:
        _check(rc)
    return r


def gencd_iterate(h, iters, sync=True):
    if not sync:
        _check(lib().gencd_iterate(h, int(iters), None))
        return None
    r = gencd_result()
    _check(lib().gencd_iterate(h, int(iters), C.byref(r)))
    return r


def gencd_stats(h) -> gencd_result:
    r = gencd_result()
    _check(lib().gencd_stats(h, C.byref(r)))
    return r


def gencd_stats_reset(h):
    _check(lib().gencd_stats_reset(h))


def gencd_set_iteration(h, t):
    _check(lib().gencd_set_iteration(h, int(t)))


def gencd_get_iteration(h) -> int:
    v = C.c_int64()
    _check(lib().gencd_get_iteration(h, C.byref(v)))
    return v.value


def gencd_get_w(h, k, out=None):
    """w as a numpy array (or into `out`, a CUDA float64 tensor)."""
    if out is not None and _is_cuda_tensor(out):
        _check(lib().gencd_get_w(h, C.c_void_p(out.data_ptr()), int(k), GENCD_DEVICE))
        return out
    w = np.empty(int(k))
    _check(lib().gencd_get_w(h, C.c_void_p(w.ctypes.data), int(k), GENCD_HOST))
    return w


def gencd_set_w(h, w):
    ptr, mem, keep = _buf(w, np.float64)
    n = keep.numel() if _is_cuda_tensor(keep) else keep.size
    _check(lib().gencd_set_w(h, ptr, int(n), mem))


def gencd_get_z(h, n):
    z = np.empty(int(n))
    _check(lib().gencd_get_z(h, C.c_void_p(z.ctypes.data), int(n), GENCD_HOST))
    return z


def gencd_objective(h):
    o, kk = C.c_double(), C.c_double()
    _check(lib().gencd_objective(h, C.byref(o), C.byref(kk)))
    return o.value, kk.value


def gencd_propose_at(h, J):
    J = np.ascontiguousarray(J, np.int32)
    d = np.empty(J.size)
    f = np.empty(J.size)
    _check(lib().gencd_propose_at(h, C.c_void_p(J.ctypes.data), J.size, C.c_void_p(d.ctypes.data),
                                  C.c_void_p(f.ctypes.data), GENCD_HOST))
    return d, f


def gencd_propose_all(h, k):
    d = np.empty(int(k))
    f = np.empty(int(k))
    kk = C.c_double()
    _check(lib().gencd_propose_all(h, C.c_void_p(d.ctypes.data), C.c_void_p(f.ctypes.data), GENCD_HOST,
                                   C.byref(kk)))
    return d, f, kk.value


def gencd_spectral_radius(h):
    rho, ps, it = C.c_double(), C.c_int64(), C.c_int32()
    _check(lib().gencd_spectral_radius(h, C.byref(rho), C.byref(ps), C.byref(it)))
    return rho.value, ps.value, it.value


def gencd_color(h) -> int:
    c = C.c_int32()
    _check(lib().gencd_color(h, C.byref(c)))
    return c.value


def gencd_color_balanced_csc(n, k, col_ptr, row_idx, cap=0):
    """Balanced distance-2 colouring of a host CSC (no GPU work); returns
    (colors int32[k], ncolors)."""
    cp = np.ascontiguousarray(col_ptr, np.int64)
    ri = np.ascontiguousarray(row_idx, np.int32)
    c = np.empty(int(k), np.int32)
    nc = C.c_int32()
    _check(lib().gencd_color_balanced_csc(int(n), int(k), C.c_void_p(cp.ctypes.data), C.c_void_p(ri.ctypes.data),
                                          int(cap), C.c_void_p(c.ctypes.data), C.byref(nc)))
    return c, nc.value


def gencd_get_colors(h, k):
    c = np.empty(int(k), np.int32)
    _check(lib().gencd_get_colors(h, C.c_void_p(c.ctypes.data), int(k), GENCD_HOST))
    return c


def gencd_set_colors(h, colors):
    c = np.ascontiguousarray(colors, np.int32)
    _check(lib().gencd_set_colors(h, C.c_void_p(c.ctypes.data), c.size, GENCD_HOST))


def gencd_permutation(h, seed, epoch, m):
    out = np.empty(int(m), np.int32)
    _check(lib().gencd_permutation(h, int(seed) & ((1 << 64) - 1), int(epoch), int(m),
                                   C.c_void_p(out.ctypes.data)))
    return out


def gencd_profile_enable(h, enable=True):
    _check(lib().gencd_profile_enable(h, 1 if enable else 0))


def gencd_duality_gap(h):
    """(gap, primal P(w), dual D) at the current state."""
    g, pr, du = C.c_double(), C.c_double(), C.c_double()
    _check(lib().gencd_duality_gap(h, C.byref(g), C.byref(pr), C.byref(du)))
    return g.value, pr.value, du.value


def gencd_block_pstar(h, B):
    """(P*_b int64[B], rho_b float64[B]) of block Shotgun's B column blocks."""
    P = np.zeros(int(B), np.int64)
    rho = np.zeros(int(B), np.float64)
    _check(lib().gencd_block_pstar(h, int(B), P.ctypes.data_as(C.c_void_p), rho.ctypes.data_as(C.c_void_p)))
    return P, rho


def gencd_propose_schedule(h):
    """(split, {form: mean ms}) of the streaming propose's autotuner: split 0
    is the two separate kernels, else the fused kernel's slab warps."""
    split = C.c_int32()
    ms = (C.c_double * 5)()
    _check(lib().gencd_propose_schedule(h, C.byref(split), ms, 5))
    forms = ["separate", "fused20", "fused24", "fused28", "fused31"]
    return int(split.value), {f: float(v) for f, v in zip(forms, ms) if v >= 0}


def gencd_set_propose_schedule(h, split):
    """0: two kernels; 20, 24, 28, 31: the fused kernel's slab warps; -1: autotune."""
    _check(lib().gencd_set_propose_schedule(h, int(split)))


def gencd_profile_read(h, kernel):
    """(summed ms, kernel launches, timed invocations) of a kernel family."""
    kid = KERNELS.index(kernel) if isinstance(kernel, str) else int(kernel)
    ms, n, calls = C.c_double(), C.c_int64(), C.c_int64()
    _check(lib().gencd_profile_read(h, kid, C.byref(ms), C.byref(n), C.byref(calls)))
    return ms.value, n.value, calls.value


def gencd_profile_reset(h):
    _check(lib().gencd_profile_reset(h))


def gencd_propose_all_noalloc(n, k, nnz, col_ptr, row_idx, val, y, z, w, loss, lam, beta_mode, delta, phi, kkt,
                              stream=None):
    """The allocation-free streaming Propose.  Every array argument is a
    contiguous CUDA tensor on the current device (inputs and the outputs
    delta, phi of k float64 and kkt of one float64); nothing is allocated and
    the call does not synchronise."""
    ts = [col_ptr, row_idx, val, y, z, w, delta, phi, kkt]
    if not all(_is_cuda_tensor(t) and t.is_contiguous() for t in ts):
        raise ValueError("gencd_propose_all_noalloc takes contiguous CUDA tensors only")
    ptr = [C.c_void_p(t.data_ptr()) for t in ts]
    st = default_stream() if stream is None else int(stream)
    _check(lib().gencd_propose_all_noalloc(int(n), int(k), int(nnz), *ptr[:6], LOSSES.get(loss, loss), float(lam),
                                           int(beta_mode), *ptr[6:], C.c_void_p(st)))


class Problem:
    """Owns one gencd handle; methods forward to the C calls above."""

    def __init__(self, prob=None, *, n=None, k=None, col_ptr=None, row_idx=None, val=None, y=None,
                 loss=None, precision="f64", stream=None):
        if prob is not None:
            n, k, col_ptr, row_idx, val, y = prob.n, prob.k, prob.col_ptr, prob.row_idx, prob.val, prob.y
            loss = loss or prob.loss
        nnz = int(col_ptr[-1]) if not _is_cuda_tensor(col_ptr) else int(col_ptr[-1].item())
        self.n, self.k, self.nnz = int(n), int(k), nnz
        self.h = gencd_create(n, k, nnz, col_ptr, row_idx, val, y, loss or "logistic", precision, stream)

    def close(self):
        if getattr(self, "h", None):
            gencd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_lambda(self, lam):
        gencd_set_lambda(self.h, lam)

    def lambda_max(self):
        return gencd_lambda_max(self.h)

    def set_loss(self, loss):
        gencd_set_loss(self.h, loss)

    def set_params(self, **kw):
        p = gencd_get_params(self.h)
        for key, v in kw.items():
            if key == "variant" and isinstance(v, str):
                v = VARIANTS[v]
            setattr(p, key, v)
        gencd_set_params(self.h, p)
        return p

    def solve(self):
        return gencd_solve(self.h)

    def iterate(self, iters, sync=True):
        return gencd_iterate(self.h, iters, sync)

    def w(self):
        return gencd_get_w(self.h, self.k)

    def z(self):
        return gencd_get_z(self.h, self.n)

    def set_w(self, w):
        gencd_set_w(self.h, w)

    def objective(self):
        return gencd_objective(self.h)

    def duality_gap(self):
        return gencd_duality_gap(self.h)

    def propose_at(self, J):
        return gencd_propose_at(self.h, J)

    def propose_all(self):
        return gencd_propose_all(self.h, self.k)

    def spectral_radius(self):
        return gencd_spectral_radius(self.h)

    def color(self):
        return gencd_color(self.h)

    def block_pstar(self, B):
        return gencd_block_pstar(self.h, B)

    def colors(self):
        return gencd_get_colors(self.h, self.k)

    def set_colors(self, c):
        gencd_set_colors(self.h, c)

    def permutation(self, seed, epoch, m):
        return gencd_permutation(self.h, seed, epoch, m)

    def set_iteration(self, t):
        gencd_set_iteration(self.h, t)

    def stats(self):
        return gencd_stats(self.h)

    def stats_reset(self):
        gencd_stats_reset(self.h)


# --- include/gencd_batch.h ----------------------------------------------------

def gencd_batch_create(n, k, nnz, col_ptr, row_idx, val, y, loss="logistic", fold=None, nfolds=0, slots=32,
                       stream=None):
    """Opaque batch handle over one X (host numpy arrays or CUDA tensors)."""
    if _is_cuda_tensor(val):
        val_dtype = 0 if str(val.dtype) == "torch.float64" else 1
        vdt = None
    else:
        vdt = np.float32 if np.asarray(val).dtype == np.float32 else np.float64
        val_dtype = 0 if vdt == np.float64 else 1
    cp, m0, k0 = _buf(col_ptr, np.int64)
    ri, m1, k1 = _buf(row_idx, np.int32)
    va, m2, k2 = _buf(val, vdt)
    yy, m3, k3 = _buf(y, np.float64)
    fo, m4, k4 = _buf(fold, np.uint8)
    mems = {m0, m1, m2, m3} if nnz > 0 else {m0, m3}
    if fold is not None:
        mems.add(m4)
    if len(mems) != 1:
        raise ValueError("inputs must be all host arrays or all device tensors")
    handle = C.c_void_p()
    st = default_stream() if stream is None else int(stream)
    _check(lib().gencd_batch_create(C.byref(handle), int(n), int(k), int(nnz), cp, ri, va, val_dtype, yy,
                                    LOSSES.get(loss, loss), fo, int(nfolds), int(slots), mems.pop(),
                                    C.c_void_p(st)))
    del k0, k1, k2, k3, k4
    return handle


def gencd_batch_destroy(h):
    lib().gencd_batch_destroy(h)


def gencd_batch_slots(h) -> int:
    v = C.c_int32()
    _check(lib().gencd_batch_slots(h, C.byref(v)))
    return v.value


def gencd_batch_lambda_max(h, held_out=-1) -> float:
    v = C.c_double()
    _check(lib().gencd_batch_lambda_max(h, int(held_out), C.byref(v)))
    return v.value


def gencd_batch_set_params(h, params: gencd_params):
    _check(lib().gencd_batch_set_params(h, C.byref(params)))


def gencd_batch_set_slot(h, slot, held_out, lam, w=None):
    ptr, mem, keep = _buf(w, np.float64)
    _check(lib().gencd_batch_set_slot(h, int(slot), int(held_out), float(lam), ptr, mem))
    del keep


def gencd_batch_copy_slot(h, dst, src, held_out, lam):
    _check(lib().gencd_batch_copy_slot(h, int(dst), int(src), int(held_out), float(lam)))


def gencd_batch_clear_slot(h, slot):
    _check(lib().gencd_batch_clear_slot(h, int(slot)))


def gencd_batch_get_w(h, slot, k):
    w = np.empty(int(k))
    _check(lib().gencd_batch_get_w(h, int(slot), C.c_void_p(w.ctypes.data), int(k), GENCD_HOST))
    return w


def gencd_batch_iterate(h, iters, sync=True):
    _check(lib().gencd_batch_iterate(h, int(iters), 1 if sync else 0))


def gencd_batch_objective(h, slots):
    o = np.empty(int(slots))
    kk = np.empty(int(slots))
    _check(lib().gencd_batch_objective(h, C.c_void_p(o.ctypes.data), C.c_void_p(kk.ctypes.data)))
    return o, kk


def gencd_batch_propose(h, slots, k):
    d = np.empty((int(slots), int(k)))
    f = np.empty((int(slots), int(k)))
    _check(lib().gencd_batch_propose(h, C.c_void_p(d.ctypes.data), C.c_void_p(f.ctypes.data), GENCD_HOST))
    return d, f


def gencd_batch_path(h, held_out, lambdas, k, handoff=0.0, warm=True, want_w=False, tol_rel=0.0):
    """Runs a path: held_out int[nchains], lambdas float[nchains, nlambda].
    Returns (per-solve records as a list of dicts, w array [nchains, nlambda, k]
    or None, totals gencd_result).  A solve that did not converge is reported
    in its record's status, not raised."""
    ho = np.ascontiguousarray(held_out, np.int32)
    lam = np.ascontiguousarray(lambdas, np.float64)
    C_, L = lam.shape
    if ho.size != C_:
        raise ValueError("one held-out fold per chain")
    spec = gencd_path(nchains=C_, nlambda=L, held_out=C.c_void_p(ho.ctypes.data),
                      lambda_=C.c_void_p(lam.ctypes.data), handoff=float(handoff), warm=1 if warm else 0,
                      tol_rel=float(tol_rel))
    recs = (gencd_path_solve * (C_ * L))()
    w = np.empty((C_, L, int(k))) if want_w else None
    r = gencd_result()
    rc = lib().gencd_batch_path(h, C.byref(spec), C.cast(recs, C.c_void_p),
                                C.c_void_p(w.ctypes.data) if want_w else None, C.byref(r))
    _check(rc)
    out = [{f: getattr(x, f) for f, _ in gencd_path_solve._fields_} for x in recs]
    return out, w, r


def gencd_batch_schedule(h):
    """(spmm_kind, update_kind, {form: mean ms}) of the batch's autotuner."""
    a, u = C.c_int32(), C.c_int32()
    ms = (C.c_double * 4)()
    _check(lib().gencd_batch_schedule(h, C.byref(a), C.byref(u), ms, 4))
    forms = ["spmm_entries", "spmm_slots", "step_update_pairs", "step_update_grouped"]
    return int(a.value), int(u.value), {f: float(v) for f, v in zip(forms, ms) if v >= 0}


def gencd_batch_set_schedule(h, spmm_kind=-1, update_kind=-1):
    _check(lib().gencd_batch_set_schedule(h, int(spmm_kind), int(update_kind)))


class Batch:
    """Owns one batch handle; methods forward to the calls above."""

    def __init__(self, prob, *, fold=None, nfolds=0, slots=32, loss=None, stream=None):
        self.n, self.k, self.nnz = int(prob.n), int(prob.k), int(prob.nnz)
        self.h = gencd_batch_create(prob.n, prob.k, prob.nnz, prob.col_ptr, prob.row_idx, prob.val, prob.y,
                                    loss or prob.loss, fold, nfolds, slots, stream)
        self.slots = gencd_batch_slots(self.h)

    def close(self):
        if getattr(self, "h", None):
            gencd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def schedule(self):
        return gencd_batch_schedule(self.h)

    def set_schedule(self, spmm_kind=-1, update_kind=-1):
        gencd_batch_set_schedule(self.h, spmm_kind, update_kind)

    def lambda_max(self, held_out=-1):
        return gencd_batch_lambda_max(self.h, held_out)

    def set_params(self, **kw):
        p = gencd_default_params()
        for key, v in kw.items():
            if key == "variant" and isinstance(v, str):
                v = VARIANTS[v]
            setattr(p, key, v)
        gencd_batch_set_params(self.h, p)
        return p

    def set_slot(self, slot, held_out, lam, w=None):
        gencd_batch_set_slot(self.h, slot, held_out, lam, w)

    def copy_slot(self, dst, src, held_out, lam):
        gencd_batch_copy_slot(self.h, dst, src, held_out, lam)

    def clear_slot(self, slot):
        gencd_batch_clear_slot(self.h, slot)

    def w(self, slot):
        return gencd_batch_get_w(self.h, slot, self.k)

    def iterate(self, iters, sync=True):
        gencd_batch_iterate(self.h, iters, sync)

    def objective(self):
        return gencd_batch_objective(self.h, self.slots)

    def propose(self):
        return gencd_batch_propose(self.h, self.slots, self.k)

    def path(self, held_out, lambdas, handoff=0.0, warm=True, want_w=False, tol_rel=0.0):
        return gencd_batch_path(self.h, held_out, lambdas, self.k, handoff, warm, want_w, tol_rel)


# --- include/gencd_serve.h ----------------------------------------------------

def gencd_serve(problems, lambda_fracs, arrivals, workers=4, precision="f32", hbm_fraction=0.5, want_w=False,
                tol_rel=0.0, **params):
    """Serves a stream of independent problems (workloads.Problem, host
    arrays) arriving at `arrivals` seconds in up to `workers` slots; lambda =
    lambda_frac * lambda_max per problem, and with tol_rel > 0 each solve
    stops at KKT <= tol_rel * lambda.  Returns (responses as dicts, list of w
    arrays or None)."""
    keep = []
    reqs = (gencd_request * len(problems))()
    for q, (p, lf, at) in enumerate(zip(problems, lambda_fracs, arrivals)):
        cp = np.ascontiguousarray(p.col_ptr, np.int64)
        ri = np.ascontiguousarray(p.row_idx, np.int32)
        va = np.ascontiguousarray(p.val)
        if va.dtype not in (np.float32, np.float64):
            va = va.astype(np.float64)
        yy = np.ascontiguousarray(p.y, np.float64)
        keep += [cp, ri, va, yy]
        reqs[q] = gencd_request(n=p.n, k=p.k, nnz=p.nnz, col_ptr=cp.ctypes.data, row_idx=ri.ctypes.data,
                                val=va.ctypes.data, val_dtype=0 if va.dtype == np.float64 else 1,
                                loss=LOSSES[p.loss], y=yy.ctypes.data, lambda_frac=float(lf), arrival=float(at))
    pr = gencd_default_params()
    for key, v in params.items():
        if key == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        setattr(pr, key, v)
    sp = gencd_serve_params(workers=int(workers), precision=PRECISIONS.get(precision, precision),
                            hbm_fraction=float(hbm_fraction), params=pr, tol_rel=float(tol_rel))
    out = (gencd_response * len(problems))()
    ws = [np.empty(p.k) for p in problems] if want_w else None
    wp = (C.c_void_p * len(problems))(*[w.ctypes.data for w in ws]) if want_w else None
    _check(lib().gencd_serve(C.cast(reqs, C.c_void_p), len(problems), C.byref(sp), C.cast(out, C.c_void_p),
                             C.cast(wp, C.c_void_p) if want_w else None))
    del keep
    return [{f: getattr(x, f) for f, _ in gencd_response._fields_} for x in out], ws


def gencd_serve_dry_run(sizes, arrivals, service_s, budget_bytes, workers=4, hbm_fraction=1.0):
    """The serving admission policy without a GPU: sizes are (n, k, nnz) per
    request, service_s the seconds each request holds its worker.  Returns the
    responses as dicts (worker, arrival, start, end, bytes)."""
    reqs = (gencd_request * len(sizes))()
    for q, ((n, k, nnz), at) in enumerate(zip(sizes, arrivals)):
        reqs[q] = gencd_request(n=int(n), k=int(k), nnz=int(nnz), lambda_frac=0.1, arrival=float(at))
    svc = np.ascontiguousarray(service_s, np.float64)
    sp = gencd_serve_params(workers=int(workers), precision=GENCD_F32, hbm_fraction=float(hbm_fraction),
                            params=gencd_default_params())
    out = (gencd_response * len(sizes))()
    _check(lib().gencd_serve_dry_run(C.cast(reqs, C.c_void_p), len(sizes), C.byref(sp), float(budget_bytes),
                                     C.c_void_p(svc.ctypes.data), C.cast(out, C.c_void_p)))
    return [{f: getattr(x, f) for f, _ in gencd_response._fields_} for x in out]
