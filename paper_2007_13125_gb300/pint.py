"""ctypes binding of include/pint.h: argument marshalling only.

Every function keeps the C name (without the ``pint_`` prefix where it is a method of
``Plan``). Device arrays are passed as torch CUDA tensors (float64, contiguous), whose
``data_ptr()`` goes straight to the library; streams are torch.cuda.Stream objects or
raw handles. No arithmetic of the method happens in Python.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpint.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "pint.h")

PINT_OK, PINT_EINVAL, PINT_ENOMEM, PINT_ECUDA, PINT_ENOTCONV = 0, 1, 2, 3, 4
PINT_ETIMEOUT, PINT_EAGAIN, PINT_EBUDGET, PINT_ENOTFOUND = 5, 6, 7, 8
PINT_FP64, PINT_MIXED, PINT_FP32 = 0, 1, 2
PINT_EIG_TRUNC_DFT, PINT_EIG_CLOSED_FORM = 0, 1
PRECISIONS = {"fp64": PINT_FP64, "mixed": PINT_MIXED, "fp32": PINT_FP32}
PINT_SPACE_FD, PINT_SPACE_FEM_P1, PINT_SPACE_PERIODIC = 0, 1, 2
SPACES = {"fd": PINT_SPACE_FD, "fem": PINT_SPACE_FEM_P1, "periodic": PINT_SPACE_PERIODIC}


class PintError(RuntimeError):
    """A pint_status other than PINT_OK, with the library's message (pint_last_error)."""
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int), ("mz", ctypes.c_int)]


class _Desc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("alpha", ctypes.c_double), ("kappa", ctypes.c_double),
                ("tau", ctypes.c_double), ("N", ctypes.c_int), ("grid", _Grid),
                ("precision", ctypes.c_int), ("eig", ctypes.c_int), ("ysolve", ctypes.c_int),
                ("space", ctypes.c_int), ("xdst", ctypes.c_int)]


class _Req(ctypes.Structure):
    _fields_ = [("desc", _Desc), ("tol", ctypes.c_double), ("max_sweeps", ctypes.c_int),
                ("inputs_on_device", ctypes.c_int)]


class _Poly(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 4)]


PINT_NL_MAX_STEPS = 64


class _NlInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("sweeps", ctypes.c_int * PINT_NL_MAX_STEPS),
                ("upd", ctypes.c_double * PINT_NL_MAX_STEPS)]


def _poly(g):
    """pint_poly from 4 coefficients c_0..c_3 of g(u) = sum_i c_i u^i."""
    c = [float(x) for x in g]
    if len(c) != 4:
        raise ValueError("g: four coefficients c_0..c_3")
    return _Poly((ctypes.c_double * 4)(*c))


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps", ctypes.c_int), ("upd_rel", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def lib():
    """Load libpint.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "pint_plan_create": (_I, [_I, _D, _D, _D, _I, ctypes.POINTER(_Grid), _I, ctypes.POINTER(_P)]),
        "pint_plan_create_desc": (_I, [ctypes.POINTER(_Desc), ctypes.POINTER(_P)]),
        "pint_plan_destroy": (_I, [_P]),
        "pint_plan_workspace_bytes": (ctypes.c_size_t, [_P]),
        "pint_form_rhs": (_I, [_P, _P, _P, _P, _P, _P]),
        "pint_initial_guess": (_I, [_P, _P, _P, _P]),
        "pint_wr_sweep": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D), _P]),
        "pint_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
        "pint_solve_async": (_I, [_P, _P, _P, _D, _I, _P]),
        "pint_solve_v": (_I, [_P, _P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
        "pint_solve_fv": (_I, [_P, _P, _P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
        "pint_solve_v_async": (_I, [_P, _P, _P, _P, _D, _I, _P]),
        "pint_solve_result": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
        "pint_solve_host": (_I, [_P, _P, _P, _P, _P, _D, _I, _P]),
        "pint_solve_resume": (_I, [_P, _P, _P, _I, _D, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
        "pint_solve_host_join": (_I, [_P, _P]),
        "pint_plan_tuning": (_I, [_P, ctypes.POINTER(_I), _I]),
        "pint_time_weights": (_I, [_I, _D, _I, ctypes.POINTER(_D)]),
        "pint_correction_coefficients": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
        "pint_circulant_eigenvalues": (_I, [_I, _D, _D, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
        "pint_last_error": (ctypes.c_char_p, []),
        "pint_status_string": (ctypes.c_char_p, [_I]),
        "pint_version": (ctypes.c_char_p, []),
        "pint_set_profiling": (_I, [_I]),
        "pint_kappa_solve_noalloc": (_I, [_I, _D, _D, _I, _I, _P, _P, _P]),
        "pint_device_bytes_held": (ctypes.c_longlong, []),
        "pint_debug_fail_allocation": (_I, [_I]),
        "pint_batch_solve": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I,
                                  ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
        "pint_batch_solve_v": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                    _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _P]),
        "pint_kernel_stats": (_I, [_I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_I),
                                   ctypes.POINTER(_D), _I]),
        "pint_set_reaction": (_I, [_P, _P, _P]),
        "pint_form_rhs_window": (_I, [_P, _P, _P, _P, _P]),
        "pint_nl_form_rhs": (_I, [_P, ctypes.POINTER(_Poly), _P, _P, _P, _P, _P]),
        "pint_nl_solve": (_I, [_P, ctypes.POINTER(_Poly), _P, _P, _D, _I, _D, _I, ctypes.POINTER(_NlInfo), _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    for name, (res, args) in _server_sig().items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
    _LIB = L
    return L


def _server_sig():
    return {
        "pint_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
        "pint_server_destroy": (_I, [_P]),
        "pint_submit": (_I, [_P, ctypes.POINTER(_Req), _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
        "pint_poll": (_I, [_P, ctypes.c_uint64, _I, _P, ctypes.POINTER(_Info)]),
        "pint_server_stats": (_I, [_P, ctypes.POINTER(_D)]),
    }


def header_functions() -> list[str]:
    """Names of the functions declared in include/pint.h."""
    text = open(HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pint_[a-z0-9_]+)\s*\(", text)))


def status_string(s: int) -> str:
    """Name of a pint_status (pint_status_string)."""
    try:
        return lib().pint_status_string(s).decode()
    except Exception:  # library not loadable: still format the number
        return f"status {s}"


def last_error() -> str:
    """Message of the calling thread's last failed call (pint_last_error)."""
    return lib().pint_last_error().decode()


def check(status: int):
    """Raise PintError for a status other than PINT_OK."""
    if status != PINT_OK:
        raise PintError(status, last_error())


def _ptr(t):
    """data_ptr of a CUDA float64 contiguous tensor (or None)."""
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---- host-only queries ----
def time_weights(k: int, alpha: float, n: int) -> np.ndarray:
    """omega_0..omega_{n-1} of BDF-k (alpha = 1) or CQ-BDF-k (pint_time_weights)."""
    out = np.zeros(n)
    check(lib().pint_time_weights(k, alpha, n, out.ctypes.data_as(ctypes.POINTER(_D))))
    return out


def correction_coefficients(k: int):
    """Table 1 for BDF-k: (a_n [5], b_{l,n} [4][5]) (pint_correction_coefficients)."""
    a = np.zeros(5)
    b = np.zeros(20)
    check(lib().pint_correction_coefficients(k, a.ctypes.data_as(ctypes.POINTER(_D)),
                                             b.ctypes.data_as(ctypes.POINTER(_D))))
    return a, b.reshape(4, 5)


def circulant_eigenvalues(k: int, alpha: float, kappa: float, N: int, eig: int = PINT_EIG_TRUNC_DFT):
    """Eigenvalues g_0..g_{N-1} of B_k(kappa) (pint_circulant_eigenvalues), complex."""
    re_, im_ = np.zeros(N), np.zeros(N)
    check(lib().pint_circulant_eigenvalues(k, alpha, kappa, N, eig,
                                           re_.ctypes.data_as(ctypes.POINTER(_D)),
                                           im_.ctypes.data_as(ctypes.POINTER(_D))))
    return re_ + 1j * im_


def kappa_solve_noalloc(k, kappa, tau, N, mx, R, Q, stream=None):
    """Q = P_kappa^{-1} R (1D heat, FP64) with no device allocation (pint_kappa_solve_noalloc).

    R and Q must each hold N * mx elements, be distinct tensors, and live on the current CUDA
    device (the library uses that device's static scratch array); ValueError otherwise, before
    anything reaches the library."""
    n = int(N) * int(mx)
    if R.numel() != n or Q.numel() != n:
        raise ValueError(f"R and Q must hold N * mx = {n} elements (got {R.numel()} and {Q.numel()})")
    if R.data_ptr() == Q.data_ptr():
        raise ValueError("Q may not alias R")
    pr, pq = _ptr(R), _ptr(Q)
    import torch
    cur = torch.cuda.current_device()
    if R.device.index != cur or Q.device.index != cur:
        raise ValueError(f"R and Q must be on the current CUDA device (cuda:{cur})")
    check(lib().pint_kappa_solve_noalloc(int(k), float(kappa), float(tau), int(N), int(mx), pr, pq,
                                         _stream(stream)))


def device_bytes_held() -> int:
    """Device bytes held by live plans and servers (pint_device_bytes_held)."""
    return int(lib().pint_device_bytes_held())


def debug_fail_allocation(n: int) -> int:
    """Make the n-th next allocation of the library fail (n < 0 disarms; pint_debug_fail_allocation)."""
    return int(lib().pint_debug_fail_allocation(int(n)))


def set_profiling(on: bool):
    """Launch sweeps one by one with per-kernel CUDA-event timing (pint_set_profiling)."""
    check(lib().pint_set_profiling(1 if on else 0))


def kernel_stats(reset: bool = True) -> dict:
    """{kernel: (launches, total ms)} timed while profiling is on (pint_kernel_stats)."""
    n = 64
    names = (ctypes.c_char_p * n)()
    launches = (_I * n)()
    tot = (_D * n)()
    k = lib().pint_kernel_stats(n, names, launches, tot, 1 if reset else 0)
    return {names[i].decode(): (launches[i], tot[i]) for i in range(min(k, n))}


class Plan:
    """Owns a pint_plan handle."""

    def __init__(self, k, alpha, kappa, tau, N, dim, mx, my=1, precision="mixed",
                 eig=PINT_EIG_TRUNC_DFT, ysolve=0, space="fd", mz=1, xdst=0):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        spc = SPACES[space] if isinstance(space, str) else int(space)
        d = _Desc(k, float(alpha), float(kappa), float(tau), int(N),
                  _Grid(dim, mx, my if dim >= 2 else 1, mz if dim == 3 else 1), prec, eig, int(ysolve), spc,
                  int(xdst))
        h = _P()
        check(lib().pint_plan_create_desc(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.k, self.alpha, self.kappa, self.tau, self.N = k, alpha, kappa, tau, N
        self.dim, self.mx, self.my = dim, mx, (my if dim >= 2 else 1)
        self.mz = mz if dim == 3 else 1
        self.M = self.mx * self.my * self.mz
        self.precision = prec

    @classmethod
    def for_problem(cls, p, precision="mixed", eig=PINT_EIG_TRUNC_DFT, ysolve=0, xdst=0):
        """Plan for a workloads.Problem (its k, alpha, kappa, tau, N, grid and space)."""
        return cls(p.k, p.alpha, p.kappa, p.tau, p.N, p.dim, p.mx, p.my, precision, eig, ysolve,
                   getattr(p, "space", "fd"), getattr(p, "mz", 1), xdst)

    def close(self):
        """Destroy the plan (pint_plan_destroy); idempotent."""
        if self.handle:
            lib().pint_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tuning(self) -> dict:
        """The plan's tuned choices (pint_plan_tuning): tile widths, y solver, FFT radix bounds,
        x sine transform, y sine transform and z solve of 3D plans."""
        out = (_I * 10)()
        if lib().pint_plan_tuning(self.handle, out, 10) < 0:
            raise PintError(PINT_EINVAL, last_error())
        keys = ["resid_width", "update_width", "history_width", "ysolve", "resid_max_radix",
                "update_max_radix", "one_cta", "xdst", "ydst", "zsolve"]
        return {k: int(out[i]) for i, k in enumerate(keys)}

    def workspace_bytes(self) -> int:
        """Device bytes the plan owns (pint_plan_workspace_bytes)."""
        return int(lib().pint_plan_workspace_bytes(self.handle))

    def form_rhs(self, v, f, fderiv, Fhat, stream=None):
        """F_hat [N][M] from v [M], f [N][M] and the derivatives of f at 0 (pint_form_rhs)."""
        check(lib().pint_form_rhs(self.handle, _ptr(v), _ptr(f), _ptr(fderiv) if fderiv is not None and fderiv.numel() else None,
                                  _ptr(Fhat), _stream(stream)))

    def form_rhs_window(self, f, U_prev, Fhat, stream=None):
        """F_hat of a time window after the first (pint_form_rhs_window)."""
        check(lib().pint_form_rhs_window(self.handle, _ptr(f), _ptr(U_prev), _ptr(Fhat), _stream(stream)))

    def initial_guess(self, v, U, stream=None):
        """U_0^n = v for every level (pint_initial_guess)."""
        check(lib().pint_initial_guess(self.handle, _ptr(v), _ptr(U), _stream(stream)))

    def wr_sweep(self, Fhat, U_prev, U_next, stream=None, want_update=True) -> float | None:
        """One WR sweep U_prev -> U_next (pint_wr_sweep); returns ||U_next - U_prev|| / ||U_next||."""
        upd = _D(0.0)
        check(lib().pint_wr_sweep(self.handle, _ptr(Fhat), _ptr(U_prev), _ptr(U_next),
                                  ctypes.byref(upd) if want_update else None, _stream(stream)))
        return upd.value if want_update else None

    def solve(self, Fhat, U, tol=1e-10, max_sweeps=50, stream=None, raise_on_notconv=True):
        """Sweeps from the guess in U until the stopping rule meets tol (pint_solve): (status, sweeps, update)."""
        sweeps = _I(0)
        upd = _D(0.0)
        st = lib().pint_solve(self.handle, _ptr(Fhat), _ptr(U), float(tol), int(max_sweeps),
                              ctypes.byref(sweeps), ctypes.byref(upd), _stream(stream))
        if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
            raise PintError(st, last_error())
        return st, sweeps.value, upd.value

    def solve_resume(self, Fhat, U, sweeps_done, upd_last, tol=1e-10, max_sweeps=50, stream=None,
                     raise_on_notconv=True):
        """Resume a preempted solve from the iterate in U (pint_solve_resume): (status, total sweeps, update)."""
        sweeps = _I(0)
        upd = _D(0.0)
        st = lib().pint_solve_resume(self.handle, _ptr(Fhat), _ptr(U), int(sweeps_done), float(upd_last), float(tol),
                                     int(max_sweeps), ctypes.byref(sweeps), ctypes.byref(upd), _stream(stream))
        if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
            raise PintError(st, last_error())
        return st, sweeps.value, upd.value

    def solve_v(self, Fhat, v, U, tol=1e-10, max_sweeps=50, stream=None, raise_on_notconv=True):
        """pint_solve from U_0^n = v without materialising it (pint_solve_v); U is output only."""
        sweeps = _I(0)
        upd = _D(0.0)
        st = lib().pint_solve_v(self.handle, _ptr(Fhat), _ptr(v), _ptr(U), float(tol), int(max_sweeps),
                                ctypes.byref(sweeps), ctypes.byref(upd), _stream(stream))
        if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
            raise PintError(st, last_error())
        return st, sweeps.value, upd.value

    def solve_fv(self, v, f, fderiv, U, tol=1e-10, max_sweeps=50, stream=None, raise_on_notconv=True):
        """From the problem data to U (pint_solve_fv): pint_form_rhs + pint_solve_v, with F_hat
        never materialised for MIXED BDF plans; (status, sweeps, update)."""
        sweeps = _I(0)
        upd = _D(0.0)
        fd = _ptr(fderiv) if fderiv is not None and fderiv.numel() else None
        st = lib().pint_solve_fv(self.handle, _ptr(v), _ptr(f), fd, _ptr(U), float(tol), int(max_sweeps),
                                 ctypes.byref(sweeps), ctypes.byref(upd), _stream(stream))
        if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
            raise PintError(st, last_error())
        return st, sweeps.value, upd.value

    def solve_v_async(self, Fhat, v, U, tol=1e-10, max_sweeps=50, stream=None):
        """pint_solve_v enqueued on `stream` without waiting (pint_solve_v_async); see solve_result."""
        check(lib().pint_solve_v_async(self.handle, _ptr(Fhat), _ptr(v), _ptr(U), float(tol), int(max_sweeps),
                                       _stream(stream)))

    def solve_async(self, Fhat, U, tol=1e-10, max_sweeps=50, stream=None):
        """Enqueue the whole solve on `stream` without waiting (pint_solve_async)."""
        check(lib().pint_solve_async(self.handle, _ptr(Fhat), _ptr(U), float(tol), int(max_sweeps),
                                     _stream(stream)))

    def set_reaction(self, c, stream=None):
        """Reaction term A + w diag(c) for the linear solves (pint_set_reaction); None removes it."""
        check(lib().pint_set_reaction(self.handle, _ptr(c) if c is not None else None, _stream(stream)))

    def nl_form_rhs(self, g, v, f, fderiv, Fhat, stream=None):
        """F_hat of the semilinear scheme (pint_nl_form_rhs); g = (c_0, c_1, c_2, c_3)."""
        q = _poly(g)
        check(lib().pint_nl_form_rhs(self.handle, ctypes.byref(q), _ptr(v), _ptr(f),
                                     _ptr(fderiv) if fderiv is not None and fderiv.numel() else None,
                                     _ptr(Fhat), _stream(stream)))

    def nl_solve(self, g, Fhat, U, newton_tol=1e-8, max_steps=20, tol=1e-10, max_sweeps=50, stream=None,
                 raise_on_notconv=True):
        """Algorithm 3 (pint_nl_solve): (status, [inner sweeps per outer step], [outer updates])."""
        q = _poly(g)
        info = _NlInfo()
        st = lib().pint_nl_solve(self.handle, ctypes.byref(q), _ptr(Fhat), _ptr(U), float(newton_tol),
                                 int(max_steps), float(tol), int(max_sweeps), ctypes.byref(info),
                                 _stream(stream))
        if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
            raise PintError(st, last_error())
        n = info.steps
        return st, list(info.sweeps[:n]), list(info.upd[:n])

    def solve_host(self, v, f, fderiv, U_out, tol=1e-10, max_sweeps=50, stream=None):
        """End-to-end solve through host buffers (pint_solve_host): v [M], f [N][M], fderiv [k-1][M]
        and U_out [N][M] are host float64 arrays (numpy, or CPU tensors, preferably pinned) that
        must stay alive until the work is complete (solve_host_join, then a sync of the stream)."""
        def hp(x, n):
            if x is None:
                return None
            if hasattr(x, "is_cuda"):
                if x.is_cuda or x.dtype.itemsize != 8 or not x.dtype.is_floating_point or not x.is_contiguous():
                    raise ValueError("expected a contiguous float64 host tensor")
                if x.numel() != n:
                    raise ValueError(f"expected {n} elements, got {x.numel()}")
                return ctypes.c_void_p(x.data_ptr())
            if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size != n:
                raise ValueError(f"expected a C-contiguous float64 array of {n} elements")
            return ctypes.c_void_p(x.ctypes.data)
        NM, M = self.N * self.M, self.M
        fdp = hp(fderiv, (self.k - 1) * M) if self.k > 1 else None
        check(lib().pint_solve_host(self.handle, hp(v, M), hp(f, NM), fdp, hp(U_out, NM), float(tol),
                                    int(max_sweeps), _stream(stream)))

    def solve_host_join(self, stream=None):
        """Make `stream` wait for every copy-out of solve_host issued so far (pint_solve_host_join)."""
        check(lib().pint_solve_host_join(self.handle, _stream(stream)))

    def solve_result(self, raise_on_notconv=True):
        """(status, sweeps, update) of the last graph-launched solve, once its stream completed it."""
        sweeps = _I(0)
        upd = _D(0.0)
        st = lib().pint_solve_result(self.handle, ctypes.byref(sweeps), ctypes.byref(upd))
        if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
            raise PintError(st, last_error())
        return st, sweeps.value, upd.value


def batch_solve(plans, Fhats, Us, tol=1e-8, max_sweeps=50, stream=None, raise_on_notconv=True):
    """Solve independent problems with one graph launch (pint_batch_solve)."""
    n = len(plans)
    ph = (_P * n)(*[pl.handle for pl in plans])
    fh = (_P * n)(*[_ptr(F) for F in Fhats])
    uh = (_P * n)(*[_ptr(U) for U in Us])
    sw = (_I * n)()
    up = (_D * n)()
    st = lib().pint_batch_solve(ph, n, fh, uh, float(tol), int(max_sweeps), sw, up, _stream(stream))
    if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
        raise PintError(st, last_error())
    return st, list(sw), list(up)


def batch_solve_v(plans, Fhats, vs, Us, tol=1e-8, max_sweeps=50, stream=None, raise_on_notconv=True):
    """pint_batch_solve_v: every problem from U_0^n = v (U output only)."""
    n = len(plans)
    ph = (_P * n)(*[pl.handle for pl in plans])
    fh = (_P * n)(*[_ptr(F) for F in Fhats])
    vh = (_P * n)(*[_ptr(v) for v in vs])
    uh = (_P * n)(*[_ptr(U) for U in Us])
    sw = (_I * n)()
    up = (_D * n)()
    st = lib().pint_batch_solve_v(ph, n, fh, vh, uh, float(tol), int(max_sweeps), sw, up, _stream(stream))
    if st != PINT_OK and not (st == PINT_ENOTCONV and not raise_on_notconv):
        raise PintError(st, last_error())
    return st, list(sw), list(up)


class Server:
    """Owns a pint_server handle (continuous-batching solve server)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 16):
        h = _P()
        check(lib().pint_server_create(ctypes.c_size_t(int(hbm_budget_bytes)), int(max_active),
                                       ctypes.byref(h)))
        self.handle = h

    def close(self):
        """Destroy the server, cancelling queued requests (pint_server_destroy); idempotent."""
        if self.handle:
            lib().pint_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, p, v, f, fderiv, tol=1e-8, max_sweeps=50, precision="mixed"):
        """v, f, fderiv: host float64 numpy arrays (copied at submit), or CUDA float64 tensors
        (read at admission; the caller keeps them alive until the request is polled)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        d = _Desc(p.k, float(p.alpha), float(p.kappa), float(p.tau), int(p.N),
                  _Grid(p.dim, p.mx, p.my if p.dim >= 2 else 1, getattr(p, "mz", 1) if p.dim == 3 else 1),
                  prec, PINT_EIG_TRUNC_DFT, 0,
                  SPACES[getattr(p, "space", "fd")])
        t = ctypes.c_uint64(0)
        if hasattr(v, "is_cuda"):
            req = _Req(d, float(tol), int(max_sweeps), 1)
            check(lib().pint_submit(self.handle, ctypes.byref(req), _ptr(v), _ptr(f),
                                    _ptr(fderiv) if fderiv is not None and fderiv.numel() else None,
                                    ctypes.byref(t)))
            return int(t.value)
        req = _Req(d, float(tol), int(max_sweeps), 0)
        v = np.ascontiguousarray(v, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        fd = np.ascontiguousarray(fderiv, dtype=np.float64)
        check(lib().pint_submit(self.handle, ctypes.byref(req), v.ctypes.data_as(_P),
                                f.ctypes.data_as(_P), fd.ctypes.data_as(_P) if fd.size else None,
                                ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, out: np.ndarray | None, timeout_us: int = 0):
        """Wait up to timeout_us for a request (pint_poll): (status, info); on PINT_OK the solution
        is copied into `out` (host float64 [N][M]) and the request is released."""
        info = _Info()
        st = lib().pint_poll(self.handle, ctypes.c_uint64(ticket), int(timeout_us),
                             out.ctypes.data_as(_P) if out is not None else None, ctypes.byref(info))
        return st, info

    def stats(self) -> dict:
        """Server counters (pint_server_stats)."""
        v = (_D * 8)()
        check(lib().pint_server_stats(self.handle, v))
        keys = ["completed", "active", "queued", "hbm_in_use", "dof_done", "sweeps_done", "busy_s", "peak_hbm"]
        return {k: v[i] for i, k in enumerate(keys)}
