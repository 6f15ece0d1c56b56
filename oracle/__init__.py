"""ctypes binding of the plain FP64 CPU oracle (oracle/gencd_oracle.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The CUDA library never
does, and this package never imports the CUDA library.

The functions mirror the C entry points; arrays are numpy arrays in the CSC
layout produced by ``workloads``.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

SQUARED, LOGISTIC = 0, 1
SHOTGUN, THREAD_GREEDY, GREEDY, COLORING, CCD, TOP_GREEDY, SHOTGUN_BLOCKS = 0, 1, 2, 3, 4, 5, 6
_LOSS = {"squared": SQUARED, "logistic": LOGISTIC, SQUARED: SQUARED, LOGISTIC: LOGISTIC}
_VARIANT = {"shotgun": SHOTGUN, "thread_greedy": THREAD_GREEDY, "greedy": GREEDY, "top_greedy": TOP_GREEDY,
            "shotgun_blocks": SHOTGUN_BLOCKS,
            "coloring": COLORING, "ccd": CCD}

_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int64), ("col_ptr", _i64p), ("row_idx", _i32p),
                ("val", _f64p), ("y", _f64p), ("loss", C.c_int32), ("beta_mode", C.c_int32),
                ("lam", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("variant", C.c_int32), ("B", C.c_int32), ("P", C.c_int64), ("seed", C.c_uint64),
                ("colors", _i32p), ("ncolors", C.c_int32), ("improve_steps", C.c_int32),
                ("block_P", _i64p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        sig = {
            "oracle_loss": (C.c_double, [C.c_int32, C.c_double, C.c_double]),
            "oracle_dloss": (C.c_double, [C.c_int32, C.c_double, C.c_double]),
            "oracle_beta": (C.c_double, [C.c_int32]),
            "oracle_fitted": (None, [vp, _f64p, _f64p]),
            "oracle_col_scale": (None, [vp, _f64p]),
            "oracle_gradient": (None, [vp, _f64p, _f64p]),
            "oracle_objective": (C.c_double, [vp, _f64p]),
            "oracle_objective_z": (C.c_double, [vp, _f64p, _f64p]),
            "oracle_kkt": (C.c_double, [vp, _f64p, _f64p]),
            "oracle_lambda_max": (C.c_double, [vp]),
            "oracle_conjugate": (C.c_double, [C.c_int32, C.c_double, C.c_double]),
            "oracle_duality_gap": (C.c_double, [vp, _f64p, _f64p]),
            "oracle_step": (None, [C.c_double, C.c_double, C.c_double, C.c_double, _f64p, _f64p]),
            "oracle_propose": (None, [vp, _f64p, _f64p, _i32p, C.c_int64, _f64p, _f64p]),
            "oracle_improve": (C.c_double, [vp, _f64p, _f64p, C.c_int64, C.c_double, C.c_int32]),
            "oracle_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
            "oracle_stored_values": (C.c_int64, [C.c_int32, C.c_int64, _i64p, _f64p, _f64p]),
            "oracle_permutation": (None, [C.c_uint64, C.c_int64, C.c_int64, _i32p]),
            "oracle_spectral_radius": (C.c_double, [vp, C.c_int32, C.c_double, _i32p]),
            "oracle_pstar": (C.c_int64, [C.c_int64, C.c_double]),
            "oracle_block_pstar": (None, [vp, C.c_int32, C.c_int32, C.c_double, _i64p]),
            "oracle_color": (C.c_int32, [vp, _i32p]),
            "oracle_color_balanced": (C.c_int32, [vp, C.c_int64, _i32p]),
            "oracle_run": (C.c_int, [vp, vp, C.c_int64, C.c_int64, _f64p, _f64p, _f64p, _i64p]),
            "oracle_solve": (C.c_int64, [vp, vp, C.c_double, C.c_int64, C.c_int64, _f64p, _f64p,
                                         _f64p, _i64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class Oracle:
    """One problem (X, y, loss, lambda) bound to the C oracle.

    Keeps references to contiguous copies of the arrays for the lifetime of
    the object, so the C side can hold raw pointers.
    """

    def __init__(self, prob, lam: float = 0.0, beta_mode: int = 0, loss=None):
        self.n, self.k = int(prob.n), int(prob.k)
        self.col_ptr = np.ascontiguousarray(prob.col_ptr, np.int64)
        self.row_idx = np.ascontiguousarray(prob.row_idx, np.int32)
        self.val = np.ascontiguousarray(prob.val, np.float64)
        self.y = np.ascontiguousarray(prob.y, np.float64)
        self.loss = _LOSS[loss if loss is not None else prob.loss]
        self.beta_mode = int(beta_mode)
        self.lam = float(lam)
        self._s = _Problem()
        self._refresh()

    def _refresh(self):
        s = self._s
        s.n, s.k = self.n, self.k
        s.col_ptr = _p(self.col_ptr, _i64p)
        s.row_idx = _p(self.row_idx, _i32p)
        s.val = _p(self.val, _f64p)
        s.y = _p(self.y, _f64p)
        s.loss, s.beta_mode, s.lam = self.loss, self.beta_mode, self.lam

    def set_lambda(self, lam: float):
        self.lam = float(lam)
        self._refresh()

    @property
    def _ptr(self):
        return C.byref(self._s)

    # --- plain definitions ---------------------------------------------------
    def fitted(self, w):
        w = np.ascontiguousarray(w, np.float64)
        z = np.empty(self.n)
        lib().oracle_fitted(self._ptr, _p(w, _f64p), _p(z, _f64p))
        return z

    def col_scale(self):
        c = np.empty(self.k)
        lib().oracle_col_scale(self._ptr, _p(c, _f64p))
        return c

    def gradient(self, z):
        z = np.ascontiguousarray(z, np.float64)
        g = np.empty(self.k)
        lib().oracle_gradient(self._ptr, _p(z, _f64p), _p(g, _f64p))
        return g

    def objective(self, w, z=None):
        w = np.ascontiguousarray(w, np.float64)
        if z is None:
            return lib().oracle_objective(self._ptr, _p(w, _f64p))
        z = np.ascontiguousarray(z, np.float64)
        return lib().oracle_objective_z(self._ptr, _p(w, _f64p), _p(z, _f64p))

    def kkt(self, w, z=None):
        w = np.ascontiguousarray(w, np.float64)
        z = self.fitted(w) if z is None else np.ascontiguousarray(z, np.float64)
        return lib().oracle_kkt(self._ptr, _p(w, _f64p), _p(z, _f64p))

    def lambda_max(self):
        return lib().oracle_lambda_max(self._ptr)

    def duality_gap(self, w, z=None):
        """P(w) - D(s u): an upper bound on P(w) - P* (Fenchel duality)."""
        w = np.ascontiguousarray(w, np.float64)
        z = self.fitted(w) if z is None else np.ascontiguousarray(z, np.float64)
        return lib().oracle_duality_gap(self._ptr, _p(w, _f64p), _p(z, _f64p))

    def propose(self, w, z, J):
        w = np.ascontiguousarray(w, np.float64)
        z = np.ascontiguousarray(z, np.float64)
        J = np.ascontiguousarray(J, np.int32)
        d = np.empty(J.size)
        f = np.empty(J.size)
        lib().oracle_propose(self._ptr, _p(w, _f64p), _p(z, _f64p), _p(J, _i32p), J.size,
                             _p(d, _f64p), _p(f, _f64p))
        return d, f

    def block_pstar(self, B, max_iter=100, rel_tol=1e-6):
        """R14: P*_b of each of B contiguous column blocks."""
        out = np.empty(int(B), np.int64)
        lib().oracle_block_pstar(self._ptr, int(B), int(max_iter), float(rel_tol), _p(out, _i64p))
        return out

    def improve(self, w, z, j, d, steps):
        """R11: the increment d of column j improved by up to `steps` Eq. 7
        steps on coordinate j alone (Algorithm 3's Improve)."""
        w = np.ascontiguousarray(w, np.float64)
        z = np.ascontiguousarray(z, np.float64)
        return lib().oracle_improve(self._ptr, _p(w, _f64p), _p(z, _f64p), int(j), float(d), int(steps))

    def spectral_radius(self, max_iter=100, rel_tol=1e-6):
        it = C.c_int32(0)
        rho = lib().oracle_spectral_radius(self._ptr, max_iter, rel_tol, C.byref(it))
        return rho, it.value

    def color(self):
        c = np.empty(self.k, np.int32)
        nc = lib().oracle_color(self._ptr, _p(c, _i32p))
        return c, nc

    def color_balanced(self, cap=0):
        """R13: balanced distance-2 colouring; returns (colors, ncolors)."""
        c = np.empty(self.k, np.int32)
        nc = lib().oracle_color_balanced(self._ptr, int(cap), _p(c, _i32p))
        return c, int(nc)

    # --- iterations ----------------------------------------------------------
    def _params(self, variant, B=1, P=1, seed=0, colors=None, improve_steps=0, block_P=None):
        pa = _Params()
        pa.variant = _VARIANT[variant] if isinstance(variant, str) else int(variant)
        pa.B, pa.P, pa.seed = int(B), int(P), int(seed) & ((1 << 64) - 1)
        pa.improve_steps = int(improve_steps)
        if colors is not None:
            colors = np.ascontiguousarray(colors, np.int32)
            pa.colors = _p(colors, _i32p)
            pa.ncolors = int(colors.max()) + 1 if colors.size else 0
        if block_P is not None:
            block_P = np.ascontiguousarray(block_P, np.int64)
            pa.block_P = _p(block_P, _i64p)
        return pa, (colors, block_P)

    def run(self, variant, iters, w=None, z=None, t0=0, B=1, P=1, seed=0, colors=None,
            trace=False, improve_steps=0, block_P=None):
        """Runs iterations t0..t0+iters-1; returns (w, z, trace, stats)."""
        w = np.zeros(self.k) if w is None else np.array(w, np.float64)
        z = self.fitted(w) if z is None else np.array(z, np.float64)
        pa, keep = self._params(variant, B, P, seed, colors, improve_steps, block_P)
        tr = np.empty(iters) if trace else None
        st = np.zeros(3, np.int64)
        rc = lib().oracle_run(self._ptr, C.byref(pa), t0, iters, _p(w, _f64p), _p(z, _f64p),
                              _p(tr, _f64p), _p(st, _i64p))
        if rc != 0:
            raise ValueError("oracle_run rejected its parameters")
        del keep
        return w, z, tr, st

    def solve(self, variant="ccd", tol_kkt=1e-10, max_iter=10**8, check_every=None, w=None,
              B=1, P=1, seed=0, colors=None, improve_steps=0, block_P=None):
        """Iterates until KKT <= tol_kkt; returns (w, z, iters, kkt, stats)."""
        w = np.zeros(self.k) if w is None else np.array(w, np.float64)
        z = self.fitted(w)
        if check_every is None:
            check_every = self.k if variant == "ccd" else 10
        pa, keep = self._params(variant, B, P, seed, colors, improve_steps, block_P)
        kkt = C.c_double(0.0)
        st = np.zeros(3, np.int64)
        it = lib().oracle_solve(self._ptr, C.byref(pa), tol_kkt, max_iter, check_every,
                                _p(w, _f64p), _p(z, _f64p), C.byref(kkt), _p(st, _i64p))
        del keep
        return w, z, int(it), kkt.value, st


def loss(loss_id, y, t):
    return lib().oracle_loss(_LOSS[loss_id], y, t)


def dloss(loss_id, y, t):
    return lib().oracle_dloss(_LOSS[loss_id], y, t)


def conjugate(loss_id, y, v):
    """l*(y, v) = sup_t (v t - l(y, t))."""
    return lib().oracle_conjugate(_LOSS[loss_id], y, v)


def beta(loss_id):
    return lib().oracle_beta(_LOSS[loss_id])


def step(g, w_j, lam, beta_j):
    d, f = C.c_double(), C.c_double()
    lib().oracle_step(g, w_j, lam, beta_j, C.byref(d), C.byref(f))
    return d.value, f.value


STORAGE = {"f64": 0, "f32": 1, "bf16": 2, "binary": 3}


def stored_values(prob, mode):
    """The values of X as storage mode ``mode`` holds them (R10), float64[nnz].

    Raises ValueError for a binary column whose values differ, or a value
    beyond the bfloat16 range."""
    col_ptr = np.ascontiguousarray(prob.col_ptr, np.int64)
    val = np.ascontiguousarray(prob.val, np.float64)
    out = np.empty(val.size)
    bad = lib().oracle_stored_values(STORAGE[mode], int(prob.k), _p(col_ptr, _i64p), _p(val, _f64p),
                                     _p(out, _f64p))
    if bad == -2:
        raise ValueError("a value of X is beyond the bfloat16 range")
    if bad >= 0:
        raise ValueError(f"column {bad} has non-zeros of different values")
    return out


def stored_problem(prob, mode):
    """``prob`` with X replaced by the values storage mode ``mode`` holds."""
    import dataclasses

    return dataclasses.replace(prob, val=stored_values(prob, mode))


_omp_lib = None


def omp_lib():
    """The OpenMP baseline library (Section 4.2's design), built on first use."""
    global _omp_lib
    if _omp_lib is None:
        L = C.CDLL(_build.build_omp())
        vp = C.c_void_p
        L.omp_solver_max_threads.restype = C.c_int32
        L.omp_solver_create.restype = vp
        L.omp_solver_create.argtypes = [vp, _f64p, _f64p, C.c_int32]
        L.omp_solver_iterate.restype = C.c_int
        L.omp_solver_iterate.argtypes = [vp, C.c_int32, C.c_int32, C.c_int64, _i64p]
        L.omp_solver_get.restype = None
        L.omp_solver_get.argtypes = [vp, _f64p, _f64p]
        L.omp_solver_destroy.restype = None
        L.omp_solver_destroy.argtypes = [vp]
        _omp_lib = L
    return _omp_lib


class OmpSolver:
    """Thread-Greedy / Greedy with OpenMP (static schedule, atomic z, critical
    section for Greedy) on an Oracle's problem, from (w, z = Xw)."""

    def __init__(self, orc: Oracle, w=None, threads=0):
        self.orc = orc  # keeps the problem arrays alive
        w = np.zeros(orc.k) if w is None else np.ascontiguousarray(w, np.float64)
        z = orc.fitted(w)
        self.threads = int(threads) if threads > 0 else int(omp_lib().omp_solver_max_threads())
        self.h = omp_lib().omp_solver_create(orc._ptr, _p(w, _f64p), _p(z, _f64p), self.threads)
        if not self.h:
            raise MemoryError("omp_solver_create failed")

    def iterate(self, iters, B=1024, greedy=False):
        """Runs iterations; returns (updates, nnz processed, iterations)."""
        st = np.zeros(3, np.int64)
        if omp_lib().omp_solver_iterate(self.h, int(B), int(bool(greedy)), int(iters), _p(st, _i64p)) != 0:
            raise ValueError("omp_solver_iterate rejected its parameters")
        return tuple(int(x) for x in st)

    def state(self):
        w, z = np.empty(self.orc.k), np.empty(self.orc.n)
        omp_lib().omp_solver_get(self.h, _p(w, _f64p), _p(z, _f64p))
        return w, z

    def close(self):
        if getattr(self, "h", None):
            omp_lib().omp_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def splitmix64(s, i):
    return lib().oracle_splitmix64(s & ((1 << 64) - 1), i)


def permutation(seed, epoch, m):
    out = np.empty(m, np.int32)
    lib().oracle_permutation(seed & ((1 << 64) - 1), epoch, m, _p(out, _i32p))
    return out


def pstar(k, rho):
    return lib().oracle_pstar(k, rho)


__all__ = ["Oracle", "OmpSolver", "loss", "dloss", "conjugate", "beta", "step", "splitmix64", "permutation", "pstar",
           "stored_values", "stored_problem", "STORAGE",
           "SQUARED", "LOGISTIC"]
