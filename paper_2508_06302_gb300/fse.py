"""Thin ctypes binding of the FSE-Shooting C ABI (include/fse.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names (``fse_setup``, ``fse_residual_jacobian``,
...); ``Context`` wraps one ``fse_ctx``.  Loading fails loudly when the
library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

from . import _build

FSE_OK = 0
FSE_EINVAL = -1
FSE_ENOMEM = -2
FSE_ENOCONV = -3
FSE_ENONPOS_PIVOT = -4
FSE_ENAN = -5
FSE_ECUDA = -6
FSE_ENOJAC = -7
FSE_FP64 = 0
FSE_MIXED_FP32 = 1
FSE_LIN_AUTO = 0
FSE_LIN_DENSE = 1
FSE_LIN_GMRES = 2
FSE_NL_VDP = 4
FSE_SOLVE_AUTO = 0
FSE_SOLVE_SIMT = 1
FSE_SOLVE_TC = 2

_PREC = {"fp64": FSE_FP64, "mixed_fp32": FSE_MIXED_FP32, "fp32": FSE_MIXED_FP32}


class fse_nl_elem(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("dof", ctypes.c_int * 6), ("p", ctypes.c_double * 6)]


class fse_model(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("M", ctypes.POINTER(ctypes.c_double)),
                ("D", ctypes.POINTER(ctypes.c_double)), ("K", ctypes.POINTER(ctypes.c_double)),
                ("n_nl", ctypes.c_int), ("nl", ctypes.POINTER(fse_nl_elem)),
                ("e", ctypes.c_int), ("F", ctypes.POINTER(ctypes.c_double))]


class fse_opts(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("S", ctypes.POINTER(ctypes.c_int)),
                ("H", ctypes.POINTER(ctypes.c_int)), ("rho", ctypes.POINTER(ctypes.c_double)),
                ("S1", ctypes.c_int), ("newton_tol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int), ("precision", ctypes.c_int)]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
_IP = ctypes.POINTER(ctypes.c_int)
_VP = ctypes.c_void_p


def header_symbols():
    """Names of the functions declared in include/fse.h."""
    hdr = os.path.join(os.path.dirname(_build.HERE), "include", "fse.h")
    src = open(hdr).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fse_[a-z0-9_]+)\s*\(", src)))


def load(path: Optional[str] = None):
    """Load the shared library (built by ``_build.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.lib_path()
    if not os.path.exists(p):
        raise RuntimeError("FSE CUDA library not built (%s); run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    sig = {
        "fse_setup": (ctypes.c_int, [ctypes.POINTER(fse_model), ctypes.POINTER(fse_opts), ctypes.c_int,
                                     ctypes.POINTER(_VP)]),
        "fse_destroy": (None, [_VP]),
        "fse_last_error": (ctypes.c_char_p, [_VP]),
        "fse_sizes": (ctypes.c_int, [_VP, _IP, _IP, _IP, _IP, _IP]),
        "fse_harmonics": (ctypes.c_int, [_VP, _IP]),
        "fse_residual_jacobian": (ctypes.c_int, [_VP, _DP, ctypes.c_double, _DP, ctypes.c_int, _IP, _IP]),
        "fse_residual_jacobian_dev": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP, ctypes.c_int, _VP]),
        "fse_status": (ctypes.c_int, [_VP, _IP, _IP]),
        "fse_jacobian_apply": (ctypes.c_int, [_VP, _DP, _DP, ctypes.c_int]),
        "fse_jacobian_domega": (ctypes.c_int, [_VP, _DP]),
        "fse_jacobian_dense": (ctypes.c_int, [_VP, _DP]),
        "fse_monodromy": (ctypes.c_int, [_VP, _DP, _DP]),
        "fse_monodromy_traj": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP]),
        "fse_newton_step": (ctypes.c_int, [_VP, _DP, ctypes.c_double, _DP]),
        "fse_lyapunov": (ctypes.c_int, [_VP, _DP, ctypes.c_double, ctypes.c_int, ctypes.c_int, _DP]),
        "fse_lyapunov_noalloc": (ctypes.c_int, [_VP, _DP, ctypes.c_double, ctypes.c_int, ctypes.c_int, _DP]),
        "fse_set_linear_solver": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
        "fse_linear_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "fse_set_tangent_solve": (ctypes.c_int, [_VP, ctypes.c_int]),
        "fse_set_fallback": (ctypes.c_int, [_VP, _VP]),
        "fse_residual_jacobian_hypertime": (ctypes.c_int, [_VP, _DP, ctypes.c_double, _DP, ctypes.c_int, _IP,
                                                           _IP]),
        "fse_jacobian_apply_hypertime": (ctypes.c_int, [_VP, _DP, _DP, ctypes.c_int]),
        "fse_newton_step_hypertime": (ctypes.c_int, [_VP, _DP, ctypes.c_double, _DP]),
        "fse_set_rho": (ctypes.c_int, [_VP, _DP]),
        "fse_setup_shard": (ctypes.c_int, [ctypes.POINTER(fse_model), ctypes.POINTER(fse_opts), ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
        "fse_set_reduce": (ctypes.c_int, [_VP, REDUCE_FN, _VP]),
        "fse_newton_step_unknown": (ctypes.c_int, [_VP, _DP, ctypes.c_double, _DP, _IP, _DP]),
        "fse_timings": (ctypes.c_int, [_VP, _DP, ctypes.c_int]),
        "fse_profile": (ctypes.c_int, [_VP, ctypes.c_int]),
        "fse_set_steps": (ctypes.c_int, [_VP, ctypes.c_int]),
        "fse_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_VP)]),
        "fse_mlp_destroy": (None, [_VP]),
        "fse_mlp_nparams": (ctypes.c_int, [_VP]),
        "fse_mlp_last_error": (ctypes.c_char_p, [_VP]),
        "fse_mlp_set_params": (ctypes.c_int, [_VP, _FP]),
        "fse_mlp_get_params": (ctypes.c_int, [_VP, _FP]),
        "fse_mlp_forward": (ctypes.c_int, [_VP, _FP, ctypes.c_int, _FP]),
        "fse_mlp_grad": (ctypes.c_int, [_VP, _FP, _FP, ctypes.c_int, _FP, _FP]),
        "fse_mlp_train": (ctypes.c_int, [_VP, _FP, _FP, ctypes.c_int, ctypes.c_int, ctypes.c_float, _FP]),
        "fse_pod_build": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP, _DP, _DP]),
        "fse_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
        "fse_batch_destroy": (None, [_VP]),
        "fse_batch_last_error": (ctypes.c_char_p, [_VP]),
        "fse_batch_residual_jacobian": (ctypes.c_int, [_VP, ctypes.POINTER(_DP), _DP, ctypes.POINTER(_DP),
                                                       ctypes.c_int, _IP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_IP)


def _f64_vector(a, size, what):
    """Contiguous float64 copy-or-view of `a` with exactly `size` entries (ValueError otherwise):
    the C side reads and writes whole vectors, so a short buffer must never reach it."""
    v = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if v.size != size:
        raise ValueError("%s: expected %d values, got %d" % (what, size, v.size))
    return v


# int (*fse_reduce_fn)(void* user, double* buf_dev, size_t count, void* stream)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class FSEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("FSE error %d: %s" % (code, msg))
        self.code = code


# ----------------------------------------------------------------------------
# C-named wrappers
# ----------------------------------------------------------------------------

def fse_setup(model, d, S, H, rho, S1, newton_tol=1e-10, newton_maxit=20, precision="fp64",
              device=-1, shard=None):
    """fse_setup() (fse_setup_shard() for shard = (s_begin, s_end)): returns an opaque context
    handle (int)."""
    lib = load()
    M = np.ascontiguousarray(model.M, dtype=np.float64)
    D = np.ascontiguousarray(model.D, dtype=np.float64)
    K = np.ascontiguousarray(model.K, dtype=np.float64)
    F = np.ascontiguousarray(model.F, dtype=np.float64)
    m = int(model.nl_type.shape[0])
    els = (fse_nl_elem * max(1, m))()
    for k in range(m):
        els[k].type = int(model.nl_type[k])
        for a in range(6):
            els[k].dof[a] = int(model.nl_dof[k, a])
            els[k].p[a] = float(model.nl_p[k, a])
    fm = fse_model(int(M.shape[0]), _dp(M), _dp(D), _dp(K), m, els, int(F.shape[0]), _dp(F))
    Sa = np.ascontiguousarray(S, dtype=np.int32)
    Ha = np.ascontiguousarray(H, dtype=np.int32)
    ra = np.ascontiguousarray(rho, dtype=np.float64)
    prec = _PREC[precision] if isinstance(precision, str) else int(precision)
    fo = fse_opts(int(d), _ip(Sa), _ip(Ha), _dp(ra), int(S1), float(newton_tol), int(newton_maxit), prec)
    h = _VP()
    if shard is None:
        rc = lib.fse_setup(ctypes.byref(fm), ctypes.byref(fo), int(device), ctypes.byref(h))
    else:
        rc = lib.fse_setup_shard(ctypes.byref(fm), ctypes.byref(fo), int(shard[0]), int(shard[1]), int(device),
                                 ctypes.byref(h))
    if rc != FSE_OK:
        raise FSEError(rc, lib.fse_last_error(None).decode())
    return h.value


def fse_destroy(ctx):
    load().fse_destroy(ctx)


def fse_last_error(ctx):
    return load().fse_last_error(ctx).decode()


def fse_sizes(ctx):
    v = [ctypes.c_int() for _ in range(5)]
    rc = load().fse_sizes(ctx, *[ctypes.byref(x) for x in v])
    if rc:
        raise FSEError(rc, "fse_sizes")
    return tuple(x.value for x in v)


class Context:
    """One FSE-Shooting problem on one GPU (owns an ``fse_ctx``)."""

    def __init__(self, model, d, S, H, rho, S1, newton_tol=1e-10, newton_maxit=20,
                 precision="fp64", device=-1, shard=None):
        self.h = fse_setup(model, d, S, H, rho, S1, newton_tol, newton_maxit, precision, device, shard)
        self.n_unknowns, self.U, self.N, self.n, self.band = fse_sizes(self.h)
        self.d = d
        self.precision = precision
        self.shard = shard
        self._reduce_cb = None     # keeps the ctypes callback alive while the library holds it

    def set_reduce(self, fn):
        """fse_set_reduce with a Python callable fn(ptr, count, stream) -> None that leaves the sum
        over all shards of the `count` doubles at device address ptr in place (None clears it)."""
        if fn is None:
            self._check(load().fse_set_reduce(self.h, None, None))
            self._reduce_cb = None
            return

        def _cb(user, ptr, count, stream):
            try:
                fn(int(ptr), int(count), int(stream or 0))
                return 0
            except Exception:
                return 1
        self._reduce_cb = REDUCE_FN(_cb)
        self._check(load().fse_set_reduce(self.h, self._reduce_cb, None))

    @classmethod
    def from_workload(cls, wl, precision="fp64", newton_tol=None, newton_maxit=None, device=-1):
        return cls(wl.model, wl.d, wl.S, wl.H, wl.rho, wl.S1,
                   wl.newton_tol if newton_tol is None else newton_tol,
                   wl.newton_maxit if newton_maxit is None else newton_maxit, precision, device)

    def close(self):
        if getattr(self, "h", None):
            fse_destroy(self.h)
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

    def _check(self, rc, allow=()):
        if rc != FSE_OK and rc not in allow:
            raise FSEError(rc, fse_last_error(self.h))
        return rc

    def harmonics(self):
        out = np.zeros(((self.U + 1) // 2) * (self.d - 1), np.int32)
        self._check(load().fse_harmonics(self.h, _ip(out)))
        return out.reshape(-1, self.d - 1)

    def residual_jacobian(self, Z0, omega1, want_jacobian=True, allow_status=(FSE_ENOCONV,)):
        """fse_residual_jacobian(): returns (R, traj_status, newton_iters, rc)."""
        Z = _f64_vector(Z0, self.n_unknowns, "Z0")
        R = np.zeros(self.n_unknowns)
        st = np.zeros(self.N, np.int32)
        it = np.zeros(self.N, np.int32)
        rc = load().fse_residual_jacobian(self.h, _dp(Z), float(omega1), _dp(R), int(want_jacobian),
                                          _ip(st), _ip(it))
        self._check(rc, allow_status)
        return R, st, it, rc

    def residual_jacobian_dev(self, Z0_ptr, omega1, R_ptr, want_jacobian=True, stream=0):
        """fse_residual_jacobian_dev() on device pointers (ints), async on ``stream``."""
        rc = load().fse_residual_jacobian_dev(self.h, ctypes.c_void_p(Z0_ptr), float(omega1),
                                              ctypes.c_void_p(R_ptr), int(want_jacobian),
                                              ctypes.c_void_p(stream))
        return self._check(rc)

    def status(self):
        st = np.zeros(self.N, np.int32)
        it = np.zeros(self.N, np.int32)
        rc = load().fse_status(self.h, _ip(st), _ip(it))
        return rc, st, it

    def jacobian_apply(self, V):
        V = np.ascontiguousarray(np.atleast_2d(V), dtype=np.float64)
        if V.ndim != 2 or V.shape[1] != self.n_unknowns:
            raise ValueError("V: expected rows of %d values, got shape %s" % (self.n_unknowns, V.shape))
        out = np.zeros_like(V)
        self._check(load().fse_jacobian_apply(self.h, _dp(V), _dp(out), V.shape[0]))
        return out

    def jacobian_domega(self):
        out = np.zeros(self.n_unknowns)
        self._check(load().fse_jacobian_domega(self.h, _dp(out)))
        return out

    def jacobian_dense(self):
        m = self.n_unknowns
        J = np.zeros((m, m))
        self._check(load().fse_jacobian_dense(self.h, _dp(J)))
        return J

    def monodromy(self):
        Phi = np.zeros((self.N, 2 * self.n, 2 * self.n))
        dz = np.zeros((self.N, 2 * self.n))
        self._check(load().fse_monodromy(self.h, _dp(Phi), _dp(dz)))
        return Phi, dz

    def monodromy_traj(self, s):
        """fse_monodromy_traj: (Phi_s, d zbar_s / d w_1) of trajectory s."""
        Phi = np.zeros((2 * self.n, 2 * self.n))
        dz = np.zeros(2 * self.n)
        self._check(load().fse_monodromy_traj(self.h, int(s), _dp(Phi), _dp(dz)))
        return Phi, dz

    def newton_step(self, Z0, omega1):
        Z = _f64_vector(Z0, self.n_unknowns, "Z0").copy()
        rn = ctypes.c_double()
        rc = load().fse_newton_step(self.h, _dp(Z), float(omega1), ctypes.byref(rn))
        self._check(rc, (FSE_ENOCONV,))
        return Z, rn.value, rc

    def set_linear_solver(self, kind="auto", rel_tol=1e-8, restart=40, max_iters=400):
        """fse_set_linear_solver: kind in {"auto", "dense", "gmres"}."""
        k = {"auto": FSE_LIN_AUTO, "dense": FSE_LIN_DENSE, "gmres": FSE_LIN_GMRES}[kind]
        self._check(load().fse_set_linear_solver(self.h, k, float(rel_tol), int(restart), int(max_iters)))

    def _samples(self, zb, what):
        """A sample-major (N, 2n) array of the hyper-time form, as a contiguous float64 copy."""
        a = np.ascontiguousarray(zb, dtype=np.float64)
        if a.size != self.N * 2 * self.n:
            raise ValueError("%s: expected %d x %d values, got %d" % (what, self.N, 2 * self.n, a.size))
        return a.reshape(self.N, 2 * self.n).copy()

    def residual_jacobian_hypertime(self, zbar0, omega1, want_jacobian=True, allow_status=(FSE_ENOCONV,)):
        """fse_residual_jacobian_hypertime(): returns (R_T (N x 2n), traj_status, newton_iters, rc)."""
        zb = self._samples(zbar0, "zbar0")
        RT = np.zeros_like(zb)
        st = np.zeros(self.N, np.int32)
        it = np.zeros(self.N, np.int32)
        rc = load().fse_residual_jacobian_hypertime(self.h, _dp(zb), float(omega1), _dp(RT), int(want_jacobian),
                                                    _ip(st), _ip(it))
        self._check(rc, allow_status)
        return RT, st, it, rc

    def jacobian_apply_hypertime(self, V):
        """fse_jacobian_apply_hypertime() for a stack of vectors (k, N, 2n) or one (N, 2n)."""
        a = np.ascontiguousarray(V, dtype=np.float64)
        m = self.N * 2 * self.n
        if a.size % m or a.size == 0:
            raise ValueError("V: size must be a positive multiple of N * 2n = %d" % m)
        k = a.size // m
        a = a.reshape(k, m)
        out = np.zeros_like(a)
        self._check(load().fse_jacobian_apply_hypertime(self.h, _dp(a), _dp(out), k))
        return out.reshape((self.N, 2 * self.n) if k == 1 else (k, self.N, 2 * self.n))

    def newton_step_hypertime(self, zbar0, omega1):
        """fse_newton_step_hypertime(): returns (updated zbar0, ||R_T||_2 before the update, rc)."""
        zb = self._samples(zbar0, "zbar0")
        rn = ctypes.c_double()
        rc = load().fse_newton_step_hypertime(self.h, _dp(zb), float(omega1), ctypes.byref(rn))
        self._check(rc, (FSE_ENOCONV,))
        return zb, rn.value, rc

    def set_rho(self, rho):
        """fse_set_rho: the d-1 frequency ratios rho_j = w_{j+1} / w_1."""
        r = _f64_vector(rho, self.d - 1, "rho")
        self._check(load().fse_set_rho(self.h, _dp(r)))

    def newton_step_unknown(self, Z0, omega1, rho, unknown):
        """fse_newton_step_unknown: one Newton update of (Z(0), the unknown frequencies) at fixed w_1.
        unknown: indices j (0-based, w_{j+2}) that are unknowns.  Returns (Z, rho, ||R||_2 before, rc)."""
        Z = _f64_vector(Z0, self.n_unknowns, "Z0").copy()
        r = _f64_vector(rho, self.d - 1, "rho").copy()
        mask = np.zeros(self.d - 1, np.int32)
        for j in unknown:
            mask[int(j)] = 1
        rn = ctypes.c_double()
        rc = load().fse_newton_step_unknown(self.h, _dp(Z), float(omega1), _dp(r), _ip(mask), ctypes.byref(rn))
        self._check(rc, (FSE_ENOCONV,))
        return Z, r, rn.value, rc

    def set_tangent_solve(self, kind="auto"):
        """fse_set_tangent_solve: kind in {"auto", "simt", "tc"} (banded tangent-solve kernels)."""
        k = {"auto": FSE_SOLVE_AUTO, "simt": FSE_SOLVE_SIMT, "tc": FSE_SOLVE_TC}[kind]
        self._check(load().fse_set_tangent_solve(self.h, k))

    def set_fallback(self, other):
        """fse_set_fallback: attach an FP64 Context of the same problem (None detaches); the
        continuation driver re-corrects the points this mixed-precision context rejects there.
        The caller keeps `other` alive while it is attached."""
        self._fallback = other
        self._check(load().fse_set_fallback(self.h, other.h if other is not None else None))

    def linear_stats(self):
        """fse_linear_stats: (Krylov iterations, relative residual) of the last outer solve."""
        it = ctypes.c_int()
        rr = ctypes.c_double()
        self._check(load().fse_linear_stats(self.h, ctypes.byref(it), ctypes.byref(rr)))
        return it.value, rr.value

    def lyapunov(self, Z0, omega1, N_Ly, h):
        Z = _f64_vector(Z0, self.n_unknowns, "Z0")
        if int(h) < 1:
            raise ValueError("h must be >= 1")
        out = np.zeros(int(h))
        rc = load().fse_lyapunov(self.h, _dp(Z), float(omega1), int(N_Ly), int(h), _dp(out))
        self._check(rc, (FSE_ENOCONV,))
        return out

    def lyapunov_noalloc(self, Z0, omega1, N_Ly, h):
        """fse_lyapunov_noalloc: the exponents of `lyapunov` with no device
        allocation (static library scratch shared by every call)."""
        Z = _f64_vector(Z0, self.n_unknowns, "Z0")
        if int(h) < 1:
            raise ValueError("h must be >= 1")
        out = np.zeros(int(h))
        rc = load().fse_lyapunov_noalloc(self.h, _dp(Z), float(omega1), int(N_Ly), int(h), _dp(out))
        self._check(rc, (FSE_ENOCONV,))
        return out

    def set_steps(self, n_steps):
        self._check(load().fse_set_steps(self.h, int(n_steps)))

    def profile(self, enable=True):
        self._check(load().fse_profile(self.h, int(enable)))

    def timings(self):
        out = np.zeros(6)
        load().fse_timings(self.h, _dp(out), 6)
        return out


def _fp(a: np.ndarray):
    return a.ctypes.data_as(_FP)


class Batch:
    """fse_batch_*: evaluate several contexts together (own streams, or one CUDA graph)."""

    def __init__(self, contexts, use_graph=False):
        self.ctx = list(contexts)
        arr = (_VP * len(self.ctx))(*[c.h for c in self.ctx])
        h = _VP()
        rc = load().fse_batch_create(arr, len(self.ctx), int(bool(use_graph)), ctypes.byref(h))
        if rc:
            raise FSEError(rc, fse_last_error(self.ctx[0].h))
        self.h = h.value

    def residual_jacobian(self, Z0s, omegas, want_jacobian=True):
        """Returns (list of R, status array, rc)."""
        if len(Z0s) != len(self.ctx):
            raise ValueError("Z0s: expected %d vectors, got %d" % (len(self.ctx), len(Z0s)))
        Zs = [_f64_vector(z, c.n_unknowns, "Z0s[%d]" % i) for i, (z, c) in enumerate(zip(Z0s, self.ctx))]
        Rs = [np.zeros(c.n_unknowns) for c in self.ctx]
        zp = (_DP * len(Zs))(*[_dp(z) for z in Zs])
        rp = (_DP * len(Rs))(*[_dp(r) for r in Rs])
        om = _f64_vector(omegas, len(self.ctx), "omegas")
        st = np.zeros(len(self.ctx), np.int32)
        rc = load().fse_batch_residual_jacobian(self.h, zp, _dp(om), rp, int(bool(want_jacobian)), _ip(st))
        if rc not in (FSE_OK, FSE_ENOCONV):
            raise FSEError(rc, load().fse_batch_last_error(self.h).decode())
        return Rs, st, rc

    def close(self):
        if getattr(self, "h", None):
            load().fse_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The BF16 predictor network (fse_mlp_*)."""

    ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")

    def __init__(self, n_in=3, n_hidden=256, n_out=64, max_batch=512, device=-1):
        lib = load()
        h = _VP()
        rc = lib.fse_mlp_create(n_in, n_hidden, n_out, max_batch, device, ctypes.byref(h))
        if rc:
            raise FSEError(rc, "fse_mlp_create")
        self.h = h.value
        self.dims = (n_in, n_hidden, n_out)
        self.np = lib.fse_mlp_nparams(self.h)

    def close(self):
        if getattr(self, "h", None):
            load().fse_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise FSEError(rc, load().fse_mlp_last_error(self.h).decode())

    def set_params(self, params):
        flat = np.ascontiguousarray(np.concatenate([np.asarray(params[k], np.float32).reshape(-1)
                                                    for k in self.ORDER]), dtype=np.float32)
        if flat.size != self.np:
            raise ValueError("params: expected %d values, got %d" % (self.np, flat.size))
        self._check(load().fse_mlp_set_params(self.h, _fp(flat)))

    def get_params(self):
        flat = np.zeros(self.np, np.float32)
        self._check(load().fse_mlp_get_params(self.h, _fp(flat)))
        return flat

    def _inputs(self, X, T=None):
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != self.dims[0]:
            raise ValueError("X: expected shape (B, %d), got %s" % (self.dims[0], X.shape))
        if T is None:
            return X
        T = np.ascontiguousarray(T, dtype=np.float32)
        if T.shape != (X.shape[0], self.dims[2]):
            raise ValueError("T: expected shape (%d, %d), got %s" % (X.shape[0], self.dims[2], T.shape))
        return X, T

    def forward(self, X):
        X = self._inputs(X)
        Y = np.zeros((X.shape[0], self.dims[2]), np.float32)
        self._check(load().fse_mlp_forward(self.h, _fp(X), X.shape[0], _fp(Y)))
        return Y

    def grad(self, X, T):
        X, T = self._inputs(X, T)
        loss = np.zeros(1, np.float32)
        g = np.zeros(self.np, np.float32)
        self._check(load().fse_mlp_grad(self.h, _fp(X), _fp(T), X.shape[0], _fp(loss), _fp(g)))
        return float(loss[0]), g

    def train(self, X, T, steps, lr):
        X, T = self._inputs(X, T)
        loss = np.zeros(1, np.float32)
        self._check(load().fse_mlp_train(self.h, _fp(X), _fp(T), X.shape[0], int(steps), float(lr), _fp(loss)))
        return float(loss[0])


def fse_pod_build(snaps, r):
    """POD of the rows of snaps (m x nu): mean, r modes (r x nu), singular values."""
    S = np.ascontiguousarray(snaps, dtype=np.float64)
    m, nu = S.shape
    mean = np.zeros(nu)
    basis = np.zeros((r, nu))
    sing = np.zeros(r)
    rc = load().fse_pod_build(_dp(S), nu, m, r, _dp(mean), _dp(basis), _dp(sing))
    if rc:
        raise FSEError(rc, "fse_pod_build")
    return mean, basis, sing


FSE_PRED_SECANT = 0
FSE_PRED_MLP = 1


class fse_cont_opts(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int), ("omega1", _DP), ("predictor", ctypes.c_int),
                ("rel_tol", ctypes.c_double), ("max_newton", ctypes.c_int), ("warmup", ctypes.c_int),
                ("pod_modes", ctypes.c_int), ("pod_every", ctypes.c_int), ("train_steps", ctypes.c_int),
                ("lr", ctypes.c_float), ("omega_lo", ctypes.c_double), ("omega_hi", ctypes.c_double),
                ("chord", ctypes.c_int)]


class fse_cont_point(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("evals", ctypes.c_int), ("res", ctypes.c_double),
                ("znorm", ctypes.c_double), ("pred_err", ctypes.c_double), ("ms", ctypes.c_double),
                ("status", ctypes.c_int), ("predictor", ctypes.c_int), ("fallback", ctypes.c_int)]


class fse_arc_opts(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int), ("omega_start", ctypes.c_double), ("ds", ctypes.c_double),
                ("ds_max", ctypes.c_double), ("omega_scale", ctypes.c_double), ("direction", ctypes.c_int), ("rel_tol", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("omega_min", ctypes.c_double), ("omega_max", ctypes.c_double)]


def fse_continue_arclength(ctx, Z_start, omega_start, ds, n_points, direction=1, omega_scale=0.0,
                           rel_tol=1e-10, max_newton=12, omega_min=0.0, omega_max=0.0, ds_max=0.0):
    """fse_continue_arclength(): returns (Z (n_done x nu), omegas (n_done), list of dicts, rc)."""
    lib = load()
    if not hasattr(lib, "_arc_sig"):
        lib.fse_continue_arclength.restype = ctypes.c_int
        lib.fse_continue_arclength.argtypes = [_VP, ctypes.POINTER(fse_arc_opts), _DP, _DP, _DP,
                                               ctypes.POINTER(fse_cont_point), _IP]
        lib._arc_sig = True
    if int(n_points) < 1:
        raise ValueError("n_points must be >= 1")
    Z0 = _f64_vector(Z_start, ctx.n_unknowns, "Z_start")
    o = fse_arc_opts(int(n_points), float(omega_start), float(ds), float(ds_max), float(omega_scale),
                     int(direction),
                     float(rel_tol), int(max_newton), float(omega_min), float(omega_max))
    Zout = np.zeros((n_points, Z0.size))
    om = np.zeros(n_points)
    info = (fse_cont_point * n_points)()
    nd = np.zeros(1, np.int32)
    rc = lib.fse_continue_arclength(ctx.h, ctypes.byref(o), _dp(Z0), _dp(Zout), _dp(om), info, _ip(nd))
    if rc not in (FSE_OK, FSE_ENOCONV):
        raise FSEError(rc, fse_last_error(ctx.h))
    k = int(nd[0])
    pts = [{f: getattr(info[j], f) for f, _ in fse_cont_point._fields_} for j in range(k)]
    return Zout[:k], om[:k], pts, rc


def fse_continue(ctx, omegas, Z_start, predictor="secant", mlp=None, rel_tol=1e-10, max_newton=10,
                 warmup=8, pod_modes=64, pod_every=8, train_steps=200, lr=1e-3, omega_range=None,
                 chord=False):
    """fse_continue(): returns (Z (n_points x nu), list of per-point dicts, rc)."""
    lib = load()
    if not hasattr(lib, "_cont_sig"):
        lib.fse_continue.restype = ctypes.c_int
        lib.fse_continue.argtypes = [_VP, _VP, ctypes.POINTER(fse_cont_opts), _DP, _DP,
                                     ctypes.POINTER(fse_cont_point)]
        lib.fse_mlp_nouts.restype = ctypes.c_int
        lib.fse_mlp_nouts.argtypes = [_VP]
        lib._cont_sig = True
    om = np.ascontiguousarray(omegas, dtype=np.float64).reshape(-1)
    P = om.size
    if P < 1:
        raise ValueError("omegas: at least one point")
    lo, hi = (float(om.min()), float(om.max())) if omega_range is None else omega_range
    o = fse_cont_opts(P, _dp(om), FSE_PRED_MLP if predictor == "mlp" else FSE_PRED_SECANT, rel_tol, max_newton,
                      warmup, pod_modes, pod_every, train_steps, lr, lo, hi, int(bool(chord)))
    Z0 = _f64_vector(Z_start, ctx.n_unknowns, "Z_start")
    Zout = np.zeros((P, Z0.size))
    info = (fse_cont_point * P)()
    rc = lib.fse_continue(ctx.h, mlp.h if mlp is not None else None, ctypes.byref(o), _dp(Z0), _dp(Zout), info)
    if rc not in (FSE_OK, FSE_ENOCONV):
        raise FSEError(rc, fse_last_error(ctx.h))
    pts = [{k: getattr(info[j], k) for k, _ in fse_cont_point._fields_} for j in range(P)]
    return Zout, pts, rc
