"""Thin ctypes binding of the S-ADI C ABI (include/sadi.h).

Argument marshalling only: every numerical step runs inside libsadi.so.  The
library is loaded from this package directory; if it is missing the import of
this module fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsadi.so")

SADI_OK, SADI_EINVAL, SADI_ENOMEM, SADI_ECUDA, SADI_ENOTSPD, SADI_ESTATE, SADI_ETIMEOUT, \
    SADI_ENONFINITE, SADI_EUNSUPPORTED = range(9)
STATUS_NAMES = {0: "SADI_OK", 1: "SADI_EINVAL", 2: "SADI_ENOMEM", 3: "SADI_ECUDA", 4: "SADI_ENOTSPD",
                5: "SADI_ESTATE", 6: "SADI_ETIMEOUT", 7: "SADI_ENONFINITE", 8: "SADI_EUNSUPPORTED"}
SADI_G_ZERO, SADI_G_NEG_CUBE, SADI_G_NEG_SIN, SADI_G_GENERAL = 0, 1, 2, 3
SADI_PREC_FP64, SADI_PREC_FP32, SADI_PREC_FP32_DENSE = 0, 1, 2
SADI_PREC_AUTO = -1

# every symbol include/sadi.h declares, with its ctypes signature
_SIGS = {
    "sadi_create": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                              C.POINTER(C.c_void_p)]),
    "sadi_create_diffusion": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                        C.POINTER(C.c_void_p)]),
    "sadi_get_equation": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "sadi_set_options": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "sadi_get_options": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sadi_set_source": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
    "sadi_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sadi_set_initial": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sadi_step": (C.c_int, [C.c_void_p, C.c_int]),
    "sadi_batch_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "sadi_get": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_longlong)]),
    "sadi_get_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sadi_wait": (C.c_int, [C.c_void_p]),
    "sadi_get_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sadi_get_setup": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "sadi_get_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sadi_set_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "sadi_get_tiles": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "sadi_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "sadi_get_phase_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "sadi_last_error": (C.c_char_p, [C.c_void_p]),
    "sadi_destroy": (None, [C.c_void_p]),
    "sadi_gemm_split_bf16": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                        C.c_void_p]),
    "sadi_save_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "sadi_load_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sadi_graph_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "sadi_graph_launch": (C.c_int, [C.c_void_p, C.c_int]),
    "sadi_graph_destroy": (None, [C.c_void_p]),
    "sadi_graph_kernels": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "sadi_autotune": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int]),
    "sadi_tuning_log": (C.c_char_p, [C.c_void_p]),
    "sadi_step_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong]),
    "sadi_set_watchdog": (C.c_int, [C.c_void_p, C.c_int]),
    "sadi_set_nonlinearity": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
    "sadi_step_source": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sadi_get_watchdog": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "sadi_debug_expire_waits": (C.c_int, [C.c_void_p, C.c_longlong]),
    "sadi_batch_create": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "sadi_batch_set_initial": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "sadi_batch_run": (C.c_int, [C.c_void_p, C.c_int]),
    "sadi_batch_get": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_longlong)]),
    "sadi_batch_member": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "sadi_batch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "sadi_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sadi_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "sadi_batch_destroy": (None, [C.c_void_p]),
}


class SadiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libsadi.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None
_lib_lock = threading.Lock()


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        with _lib_lock:
            if _lib is None:
                _lib = load_library()
    return _lib


def _check(st: int, ctx=None):
    if st != SADI_OK:
        msg = lib().sadi_last_error(ctx)
        raise SadiError(st, msg.decode() if msg else "")


def _f64(a, N):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (N, N):
        raise ValueError(f"expected shape {(N, N)}, got {a.shape}")
    return a


def sadi_gemm_split_bf16(A_ptr: int, B_ptr: int, C_ptr: int, M: int, N: int, K: int, stream: int = 0):
    """C = A B^T in split BF16 on the tensor cores (device FP32 pointers); see sadi.h."""
    st = lib().sadi_gemm_split_bf16(C.c_void_p(A_ptr), C.c_void_p(B_ptr), C.c_void_p(C_ptr), int(M), int(N),
                                    int(K), C.c_void_p(stream or 0))
    if st != SADI_OK:
        raise SadiError(st, "sadi_gemm_split_bf16 failed")


def _batch_error(st, instances, what):
    msgs = [s.sadi_last_error() for s in instances]
    raise SadiError(st, "; ".join(m for m in msgs if m) or what)


class SadiGraph:
    """A captured batched step (sadi_graph_create); launch() replays it."""

    def __init__(self, instances, nsteps: int = 1):
        self.instances = list(instances)
        arr = (C.c_void_p * len(self.instances))(*[s.ctx for s in self.instances])
        out = C.c_void_p()
        st = lib().sadi_graph_create(arr, len(self.instances), int(nsteps), C.byref(out))
        if st != SADI_OK:
            _batch_error(st, self.instances, "sadi_graph_create failed")
        self.handle = out.value
        self.nsteps = int(nsteps)

    def sadi_graph_launch(self, reps: int = 1):
        st = lib().sadi_graph_launch(self.handle, int(reps))
        if st != SADI_OK:
            _batch_error(st, self.instances, "sadi_graph_launch failed")

    launch = sadi_graph_launch

    def sadi_graph_kernels(self) -> int:
        k = C.c_int()
        st = lib().sadi_graph_kernels(self.handle, C.byref(k))
        if st != SADI_OK:
            _batch_error(st, self.instances, "sadi_graph_kernels failed")
        return k.value

    def sadi_graph_destroy(self):
        if getattr(self, "handle", None):
            lib().sadi_graph_destroy(self.handle)
            self.handle = None

    close = sadi_graph_destroy

    def __del__(self):
        try:
            self.sadi_graph_destroy()
        except Exception:
            pass


def sadi_autotune(instances, g: int, flags: int = 0):
    """Pick the step form and tiles per N for these (uninitialised) instances."""
    arr = (C.c_void_p * len(instances))(*[s.ctx for s in instances])
    st = lib().sadi_autotune(arr, len(instances), int(g), int(flags))
    if st != SADI_OK:
        _batch_error(st, instances, "sadi_autotune failed")


def sadi_batch_step(instances, nsteps: int = 1):
    """Advance several Sadi instances together (same stream); see sadi.h."""
    arr = (C.c_void_p * len(instances))(*[s.ctx for s in instances])
    st = lib().sadi_batch_step(arr, len(instances), int(nsteps))
    if st != SADI_OK:
        msgs = [s.sadi_last_error() for s in instances]
        raise SadiError(st, "; ".join(m for m in msgs if m) or "invalid batch")


class SadiBatch:
    """Independent instances behind one sadi_batch* handle (sadi_batch_create)."""

    def __init__(self, Ns, alphas, kappas, taus, domains=None, g: int = SADI_G_ZERO, prec: int = SADI_PREC_AUTO):
        n = len(Ns)
        self.Ns = [int(x) for x in Ns]
        arr_i = (C.c_int * n)(*self.Ns)
        arr = [(C.c_double * n)(*[float(x) for x in v]) for v in (alphas, kappas, taus)]
        dom = None if domains is None else (C.c_double * (2 * n))(*[float(x) for d in domains for x in d])
        out = C.c_void_p()
        st = lib().sadi_batch_create(n, arr_i, arr[0], arr[1], arr[2], dom, int(g), int(prec), C.byref(out))
        if st != SADI_OK:
            msg = lib().sadi_batch_last_error(None)
            raise SadiError(st, msg.decode() if msg else "sadi_batch_create failed")
        self.handle = out.value

    def _check(self, st):
        if st != SADI_OK:
            msg = lib().sadi_batch_last_error(self.handle)
            raise SadiError(st, msg.decode() if msg else "")

    def _n_of(self, k, arr=None):
        # an out-of-range k goes to the library, which rejects it
        if 0 <= k < len(self.Ns):
            return self.Ns[k]
        return np.asarray(arr).shape[0] if arr is not None else 1

    def sadi_batch_set_initial(self, k: int, phi1, phi2=None):
        N = self._n_of(k, phi1)
        p1 = _f64(phi1, N)
        p2 = None if phi2 is None else _f64(phi2, N)
        self._check(lib().sadi_batch_set_initial(self.handle, int(k), p1.ctypes.data,
                                                 None if p2 is None else p2.ctypes.data))

    def sadi_batch_run(self, nsteps: int = 1):
        self._check(lib().sadi_batch_run(self.handle, int(nsteps)))

    def sadi_batch_get(self, k: int):
        N = self._n_of(k)
        out = np.empty((N, N), dtype=np.float64)
        n = C.c_longlong()
        self._check(lib().sadi_batch_get(self.handle, int(k), out.ctypes.data, C.byref(n)))
        return out, n.value

    def sadi_batch_member(self, k: int) -> int:
        out = C.c_void_p()
        self._check(lib().sadi_batch_member(self.handle, int(k), C.byref(out)))
        return out.value

    def sadi_batch_count(self) -> int:
        c = C.c_int()
        self._check(lib().sadi_batch_count(self.handle, C.byref(c)))
        return c.value

    def sadi_batch_set_stream(self, stream_handle):
        self._check(lib().sadi_batch_set_stream(self.handle, C.c_void_p(stream_handle or 0)))

    def sadi_batch_destroy(self):
        if getattr(self, "handle", None):
            lib().sadi_batch_destroy(self.handle)
            self.handle = None

    set_initial = sadi_batch_set_initial
    run = sadi_batch_run
    get = sadi_batch_get
    close = sadi_batch_destroy

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.sadi_batch_destroy()

    def __del__(self):
        try:
            self.sadi_batch_destroy()
        except Exception:
            pass


class Sadi:
    """One S-ADI instance (wraps a sadi_ctx*)."""

    def __init__(self, N: int, alpha: float, kappa: float, tau: float, domain=(-1.0, 1.0),
                 equation: str = "wave"):
        """equation: "wave" (sadi_create) or "diffusion" (sadi_create_diffusion)."""
        self.N = int(N)
        dom = (C.c_double * 2)(float(domain[0]), float(domain[1]))
        out = C.c_void_p()
        if equation not in ("wave", "diffusion"):
            raise ValueError(f"unknown equation {equation!r}")
        create = lib().sadi_create if equation == "wave" else lib().sadi_create_diffusion
        st = create(self.N, float(alpha), float(kappa), float(tau), dom, C.byref(out))
        _check(st, None)
        self.ctx = out.value

    # -- C ABI calls, same names -------------------------------------------
    def sadi_set_options(self, g: int = SADI_G_ZERO, prec: int = SADI_PREC_FP64):
        _check(lib().sadi_set_options(self.ctx, int(g), int(prec)), self.ctx)

    def sadi_get_equation(self) -> int:
        e = C.c_int()
        _check(lib().sadi_get_equation(self.ctx, C.byref(e)), self.ctx)
        return e.value

    def sadi_get_options(self):
        g, p = C.c_int(), C.c_int()
        _check(lib().sadi_get_options(self.ctx, C.byref(g), C.byref(p)), self.ctx)
        return g.value, p.value

    def sadi_set_source(self, F=None, omega: float = 0.0, phase: float = 0.0):
        f = None if F is None else _f64(F, self.N)
        _check(lib().sadi_set_source(self.ctx, None if f is None else f.ctypes.data, float(omega),
                                     float(phase)), self.ctx)

    def sadi_set_stream(self, stream_handle: int | None):
        _check(lib().sadi_set_stream(self.ctx, C.c_void_p(stream_handle or 0)), self.ctx)

    def sadi_set_initial(self, phi1, phi2=None):
        p1 = _f64(phi1, self.N)
        p2 = None if phi2 is None else _f64(phi2, self.N)
        _check(lib().sadi_set_initial(self.ctx, p1.ctypes.data,
                                      None if p2 is None else p2.ctypes.data), self.ctx)

    def sadi_step(self, nsteps: int = 1):
        _check(lib().sadi_step(self.ctx, int(nsteps)), self.ctx)

    def sadi_get(self):
        u = np.empty((self.N, self.N), dtype=np.float64)
        n = C.c_longlong()
        _check(lib().sadi_get(self.ctx, u.ctypes.data, C.byref(n)), self.ctx)
        return u, int(n.value)

    def sadi_get_async(self, host_ptr: int):
        """Queue the copy of u^n into host memory at host_ptr (N*N doubles,
        pinned); valid after sadi_wait()."""
        _check(lib().sadi_get_async(self.ctx, C.c_void_p(host_ptr)), self.ctx)

    def sadi_wait(self):
        _check(lib().sadi_wait(self.ctx), self.ctx)

    def sadi_get_device(self, dst_ptr: int, dtype: int):
        _check(lib().sadi_get_device(self.ctx, C.c_void_p(dst_ptr), int(dtype)), self.ctx)

    def sadi_get_setup(self, which: int):
        Np, _ = self.sadi_get_info()
        n = {0: self.N, 1: self.N * self.N, 2: Np, 3: (Np + 1) ** 2, 4: self.N * self.N}[which]
        out = np.empty(n, dtype=np.float64)
        _check(lib().sadi_get_setup(self.ctx, int(which), out.ctypes.data, n), self.ctx)
        if which in (1, 4):
            return out.reshape(self.N, self.N)
        if which == 3:
            return out.reshape(Np + 1, Np + 1)
        return out

    def sadi_get_info(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().sadi_get_info(self.ctx, C.byref(a), C.byref(b)), self.ctx)
        return a.value, b.value

    def sadi_set_tiles(self, rows: int = 0, conv_cols: int = 0, solve_cols: int = 0):
        _check(lib().sadi_set_tiles(self.ctx, int(rows), int(conv_cols), int(solve_cols)), self.ctx)

    def sadi_get_tiles(self):
        t = (C.c_int * 3)()
        _check(lib().sadi_get_tiles(self.ctx, t), self.ctx)
        return tuple(t)

    def sadi_profile(self, enable: bool):
        _check(lib().sadi_profile(self.ctx, 1 if enable else 0), self.ctx)

    def sadi_get_phase_times(self):
        ms = (C.c_double * 4)()
        n = C.c_longlong()
        _check(lib().sadi_get_phase_times(self.ctx, ms, C.byref(n)), self.ctx)
        return list(ms), int(n.value)

    def sadi_step_noalloc(self, u_prev_ptr: int, u_cur_ptr: int, u_next_ptr: int, n: int):
        """One step on caller-owned device buffers (N*N doubles each); no allocation."""
        _check(lib().sadi_step_noalloc(self.ctx, C.c_void_p(u_prev_ptr), C.c_void_p(u_cur_ptr),
                                       C.c_void_p(u_next_ptr), int(n)), self.ctx)

    def sadi_set_nonlinearity(self, c1: float, c3: float, cs: float):
        _check(lib().sadi_set_nonlinearity(self.ctx, float(c1), float(c3), float(cs)), self.ctx)

    def sadi_step_source(self, f_ptr: int, dtype: int = 0):
        """One step with the source field at device address f_ptr (N*N of dtype 0 double / 1 float)."""
        _check(lib().sadi_step_source(self.ctx, C.c_void_p(f_ptr), int(dtype)), self.ctx)

    def sadi_set_watchdog(self, every: int):
        _check(lib().sadi_set_watchdog(self.ctx, int(every)), self.ctx)

    def sadi_get_watchdog(self):
        """(discrete L2 norm of u^n at the last check, its step n)."""
        v, n = C.c_double(), C.c_longlong()
        _check(lib().sadi_get_watchdog(self.ctx, C.byref(v), C.byref(n)), self.ctx)
        return v.value, n.value

    def sadi_debug_expire_waits(self, wait_limit_ns: int):
        _check(lib().sadi_debug_expire_waits(self.ctx, int(wait_limit_ns)), self.ctx)

    def sadi_save_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(lib().sadi_save_state(self.ctx, None, C.byref(n)), self.ctx)
        buf = C.create_string_buffer(n.value)
        _check(lib().sadi_save_state(self.ctx, buf, C.byref(n)), self.ctx)
        return buf.raw[:n.value]

    def sadi_load_state(self, blob: bytes):
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _check(lib().sadi_load_state(self.ctx, buf, len(blob)), self.ctx)

    def sadi_tuning_log(self) -> str:
        return lib().sadi_tuning_log(self.ctx).decode()

    def sadi_last_error(self) -> str:
        return lib().sadi_last_error(self.ctx).decode()

    def sadi_destroy(self):
        if getattr(self, "ctx", None):
            lib().sadi_destroy(self.ctx)
            self.ctx = None

    # -- conveniences ------------------------------------------------------
    set_options = sadi_set_options
    set_stream = sadi_set_stream
    set_initial = sadi_set_initial
    step = sadi_step
    get = sadi_get
    close = sadi_destroy

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.sadi_destroy()

    def __del__(self):
        try:
            self.sadi_destroy()
        except Exception:
            pass
