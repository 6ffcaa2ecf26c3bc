"""GB300 (sm_103a) implementation of the method-of-lines right-hand side of the
FFT-based 3D bulk-magnetization method (Prigozhin & Sokolovsky, §2) and of its
Bogacki-Shampine time integrator.

All arithmetic runs in the CUDA library libscfft.so behind the C ABI of
include/scfft.h.  This module only marshals arguments (ctypes): device arrays
are torch CUDA tensors (float64, contiguous) passed by pointer, host arrays are
numpy arrays.  There is no CPU fallback: importing works without a GPU, but
every call that reaches the library fails loudly if the library is missing or
no GPU is present.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

__all__ = ["ScfftError", "Context", "load_library", "library_path", "PREC_F64", "PREC_F32", "PREC_DF64", "FAULT_TMA_WAIT",
           "EXPORTS", "rhs_autograd", "integrate_autograd", "batch_step", "curl_noalloc"]

PREC_F64 = 0
PREC_F32 = 1
PREC_DF64 = 2  # double-float FFT passes (FP64-equivalent accuracy on the FP32 pipes)
FAULT_TMA_WAIT = 1  # scfft_inject_fault: the next directly launched TMA-fed y pass times out (tests)
CURL_SPECTRAL = 0   # scfft_set_curl: smoothed spectral derivatives (§2)
CURL_FD = 1         # scfft_set_curl: second-order central differences

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBNAME = "libscfft.so"

# every entry point declared in include/scfft.h
EXPORTS = ("scfft_create", "scfft_set_geometry", "scfft_set_jc_map", "scfft_set_field_path",
           "scfft_precompute_kernel", "scfft_rhs", "scfft_curl", "scfft_phi", "scfft_integrate",
           "scfft_step", "scfft_profile", "scfft_profile_read", "scfft_kind_name",
           "scfft_rhs_vjp", "scfft_adjoint_integrate", "scfft_batch_step", "scfft_sync", "scfft_get_stats", "scfft_status_string", "scfft_destroy",
           "scfft_curl_noalloc", "scfft_last_cuda_error", "scfft_inject_fault", "scfft_checkpoint_save",
           "scfft_checkpoint_load", "scfft_step_host", "scfft_adjoint_record", "scfft_adjoint_step", "scfft_set_ej_law", "scfft_set_curl",
           "scfft_autotune", "scfft_get_schedule", "scfft_set_schedule",
           "scfft_advance")

NKINDS = 15


def library_path() -> str:
    return os.path.join(_HERE, _LIBNAME)


class ScfftError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        if code == 3 and _lib is not None:
            msg = f"{msg}: {_lib.scfft_last_cuda_error().decode()}"
        super().__init__(f"{what}: {msg} (status {code})")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double)]


class _Material(ctypes.Structure):
    _fields_ = [("n", ctypes.c_double), ("e0", ctypes.c_double), ("jc", ctypes.c_double),
                ("rho_out", ctypes.c_double), ("mu0", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("delta_it", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("sigma_scale", ctypes.c_double), ("rtol", ctypes.c_double), ("atol", ctypes.c_double)]


class _FieldPath(ctypes.Structure):
    _fields_ = [("nknots", ctypes.c_int), ("t", ctypes.POINTER(ctypes.c_double)),
                ("he", ctypes.POINTER(ctypes.c_double)), ("sin_amp", ctypes.c_double),
                ("sin_period", ctypes.c_double), ("sin_t0", ctypes.c_double), ("sin_t1", ctypes.c_double),
                ("sin_dir", ctypes.c_double * 3)]


class _EjLaw(ctypes.Structure):
    _fields_ = [("kim_h0", ctypes.c_double), ("aniso", ctypes.c_double * 3)]


class _Schedule(ctypes.Structure):
    _fields_ = [("z_kernel_tile", ctypes.c_int), ("z_curl_tile", ctypes.c_int), ("y_unpadded_tile", ctypes.c_int),
                ("y_padded_tma", ctypes.c_int), ("z_kernel_tmem", ctypes.c_int), ("box_fused", ctypes.c_int),
                ("x_update_split", ctypes.c_int), ("us", ctypes.c_double * 15)]


class _Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("rhs_calls", ctypes.c_longlong),
                ("iterations", ctypes.c_longlong),
                ("accepted", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("last_iters", ctypes.c_int), ("last_residual", ctypes.c_double),
                ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("h2d_bytes", ctypes.c_longlong), ("d2h_bytes", ctypes.c_longlong)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libscfft.so (build it first with paper_1803_01346_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run `python -m paper_1803_01346_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(p)
    P, D, I, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, None
    sig = {
        "scfft_create": (I, [ctypes.POINTER(_Grid), ctypes.POINTER(_Material), ctypes.POINTER(_Options), P,
                             ctypes.POINTER(P)]),
        "scfft_set_geometry": (I, [P, P]),
        "scfft_set_jc_map": (I, [P, P]),
        "scfft_set_field_path": (I, [P, ctypes.POINTER(_FieldPath)]),
        "scfft_precompute_kernel": (I, [P]),
        "scfft_rhs": (I, [P, D, I, P, P, P, ctypes.POINTER(I)]),
        "scfft_curl": (I, [P, P, P]),
        "scfft_phi": (I, [P, P, P]),
        "scfft_integrate": (I, [P, D, D, D, I, P, P, P, P, P, I, ctypes.POINTER(_Stats)]),
        "scfft_step": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), D, P, P, ctypes.POINTER(I)]),
        "scfft_step_host": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), D, P, P, P, P, ctypes.POINTER(I)]),
        "scfft_profile": (I, [P, I]),
        "scfft_profile_read": (I, [P, P, P]),
        "scfft_kind_name": (ctypes.c_char_p, [I]),
        "scfft_sync": (I, [P]),
        "scfft_get_stats": (I, [P, ctypes.POINTER(_Stats)]),
        "scfft_status_string": (ctypes.c_char_p, [I]),
        "scfft_destroy": (V, [P]),
        "scfft_curl_noalloc": (I, [ctypes.POINTER(_Grid), D, P, P, P]),
        "scfft_rhs_vjp": (I, [P, P, P, P, P, P, ctypes.POINTER(D)]),
        "scfft_last_cuda_error": (ctypes.c_char_p, []),
        "scfft_inject_fault": (I, [P, I]),
        "scfft_checkpoint_save": (I, [P, D, D, P, P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "scfft_checkpoint_load": (I, [P, P, ctypes.c_size_t, ctypes.POINTER(D), ctypes.POINTER(D), P, P]),
        "scfft_adjoint_integrate": (I, [P, D, P, I, P, P, P, P, P, ctypes.POINTER(D), I]),
        "scfft_adjoint_record": (I, [P, P, I, P, P, I, P]),
        "scfft_adjoint_step": (I, [P, I, P, P, P]),
        "scfft_set_ej_law": (I, [P, ctypes.POINTER(_EjLaw)]),
        "scfft_set_curl": (I, [P, I]),
        "scfft_autotune": (I, [P, I, P]),
        "scfft_get_schedule": (I, [P, P]),
        "scfft_set_schedule": (I, [P, P]),
        "scfft_advance": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), D, I, P, P, ctypes.POINTER(I)]),
        "scfft_batch_step": (I, [P, I, P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(x) -> int:
    """Device pointer of a contiguous float64 CUDA tensor (or None -> 0)."""
    if x is None:
        return None
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return x.data_ptr()


def curl_noalloc(n: Sequence[int], L: Sequence[float], f, out, sigma_scale: float = 1.0, stream=None):
    """curl_S f into out without any allocation (FP64, grids up to 64^3 nodes).

    For callers that cannot allocate device memory when they need the curl;
    it uses one static device array per GPU, so calls that overlap on the GPU
    race.  Raises ScfftError (status 9) for grids beyond the fixed maximum."""
    lib = load_library()
    g = _Grid(int(n[0]), int(n[1]), int(n[2]), float(L[0]), float(L[1]), float(L[2]))
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    code = lib.scfft_curl_noalloc(ctypes.byref(g), float(sigma_scale), _ptr(f), _ptr(out),
                                  ctypes.c_void_p(int(stream) if stream else 0))
    if code != 0:
        raise ScfftError(code, "scfft_curl_noalloc", lib.scfft_status_string(code).decode())


class Context:
    """One grid, material, option set and CUDA stream (§2 of the paper).

    grid: (nx, ny, nz), L: half extents (Lx, Ly, Lz)."""

    def __init__(self, n: Sequence[int], L: Sequence[float], n_power: float = 20.0, rho_out: float = 20.0,
                 e0: float = 1.0, jc: float = 1.0, mu0: float = 1.0, precision: int = PREC_F64,
                 delta_it: float = 2e-5, max_iter: int = 100, sigma_scale: float = 1.0,
                 rtol: float = 2e-4, atol: float = 1e-6, stream=None):
        self._lib = load_library()
        self.n = tuple(int(v) for v in n)
        self.N = self.n[0] * self.n[1] * self.n[2]
        g = _Grid(self.n[0], self.n[1], self.n[2], float(L[0]), float(L[1]), float(L[2]))
        m = _Material(float(n_power), float(e0), float(jc), float(rho_out), float(mu0))
        o = _Options(int(precision), float(delta_it), int(max_iter), float(sigma_scale), float(rtol), float(atol))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._h = ctypes.c_void_p()
        self._check(self._lib.scfft_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(o),
                                           ctypes.c_void_p(int(stream) if stream else 0), ctypes.byref(self._h)),
                    "scfft_create")

    def _check(self, code: int, what: str, ok=(0,)):
        if code not in ok:
            raise ScfftError(code, what, self._lib.scfft_status_string(code).decode())
        return code

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.scfft_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, mask: np.ndarray):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        if m.size != self.N:
            raise ValueError("mask must have nx*ny*nz entries")
        self._check(self._lib.scfft_set_geometry(self._h, m.ctypes.data), "scfft_set_geometry")

    def set_jc_map(self, jc=None):
        self._check(self._lib.scfft_set_jc_map(self._h, _ptr(jc)), "scfft_set_jc_map")

    def set_field_path(self, t, he, sin_amp=0.0, sin_period=1.0, sin_t0=0.0, sin_t1=0.0, sin_dir=(0.0, 0.0, 1.0)):
        tt = np.ascontiguousarray(t, dtype=np.float64)
        hh = np.ascontiguousarray(he, dtype=np.float64).reshape(-1)
        self._keep = (tt, hh)
        self._nknots = len(tt)
        fp = _FieldPath(len(tt), tt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        hh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(sin_amp), float(sin_period),
                        float(sin_t0), float(sin_t1), (ctypes.c_double * 3)(*[float(v) for v in sin_dir]))
        self._check(self._lib.scfft_set_field_path(self._h, ctypes.byref(fp)), "scfft_set_field_path")

    def set_curl(self, kind: int):
        """CURL_SPECTRAL (§2) or CURL_FD (central differences) for the curls of the rhs."""
        self._check(self._lib.scfft_set_curl(self._h, int(kind)), "scfft_set_curl")

    _SCHED_KEYS = ("z_kernel_tile", "z_curl_tile", "y_unpadded_tile", "y_padded_tma", "z_kernel_tmem", "box_fused",
                  "x_update_split")

    def autotune(self, retune: bool = False):
        """Time the launch schedules of the FP32 passes on this context's grid and keep the
        fastest (cached per device and grid); returns the schedule and the candidates' times."""
        o = _Schedule()
        self._check(self._lib.scfft_autotune(self._h, 1 if retune else 0, ctypes.byref(o)), "scfft_autotune")
        d = {k: getattr(o, k) for k in self._SCHED_KEYS}
        d["us"] = list(o.us)
        return d

    def get_schedule(self):
        o = _Schedule()
        self._check(self._lib.scfft_get_schedule(self._h, ctypes.byref(o)), "scfft_get_schedule")
        return {k: getattr(o, k) for k in self._SCHED_KEYS}

    def set_schedule(self, **kw):
        cur = self.get_schedule()
        cur.update(kw)
        o = _Schedule(*(int(cur[k]) for k in self._SCHED_KEYS))
        self._check(self._lib.scfft_set_schedule(self._h, ctypes.byref(o)), "scfft_set_schedule")

    def set_ej_law(self, kim_h0: float = 0.0, aniso=(1.0, 1.0, 1.0)):
        """The e(j, h) law in Omega (see scfft_set_ej_law): Kim's jc(|h|) = jc/(1 + |h|/kim_h0)
        and/or the anisotropic norm |j|_A = |diag(aniso) j|; the defaults are Eq. 1."""
        law = _EjLaw(float(kim_h0), (ctypes.c_double * 3)(*[float(v) for v in aniso]))
        self._check(self._lib.scfft_set_ej_law(self._h, ctypes.byref(law)), "scfft_set_ej_law")

    def precompute_kernel(self):
        self._check(self._lib.scfft_precompute_kernel(self._h), "scfft_precompute_kernel")

    def rhs(self, t: float, h, warm, hdot, left: bool = False, sync: bool = True):
        """dh/dt into hdot; warm is the Eq. 5 warm start (overwritten with hdot).
        Returns the iteration count when sync is True."""
        it = ctypes.c_int(0)
        code = self._lib.scfft_rhs(self._h, float(t), 1 if left else 0, _ptr(h), _ptr(warm), _ptr(hdot),
                                   ctypes.byref(it) if sync else None)
        self._check(code, "scfft_rhs", ok=(0, 4))
        return it.value if sync else None

    def curl(self, f, out):
        self._check(self._lib.scfft_curl(self._h, _ptr(f), _ptr(out)), "scfft_curl")

    def phi(self, j, out):
        self._check(self._lib.scfft_phi(self._h, _ptr(j), _ptr(out)), "scfft_phi")

    def integrate(self, t0, t1, dt0, h, tsnap=(), snaps=None, warm=None, dt_fixed=None):
        ts = np.ascontiguousarray(tsnap, dtype=np.float64)
        df = None if dt_fixed is None else np.ascontiguousarray(dt_fixed, dtype=np.float64)
        st = _Stats()
        self._check(self._lib.scfft_integrate(self._h, float(t0), float(t1), float(dt0), len(ts),
                                              ts.ctypes.data if len(ts) else None, _ptr(h), _ptr(snaps),
                                              _ptr(warm), df.ctypes.data if df is not None else None,
                                              0 if df is None else len(df), ctypes.byref(st)),
                    "scfft_integrate")
        return {k: getattr(st, k) for k, _ in _Stats._fields_}

    def step(self, t: float, dt: float, tstop: float, h, warm):
        """One accepted BS23 step; returns (t_new, dt_next, rejected_trials)."""
        tt, dd, rj = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_int(0)
        self._check(self._lib.scfft_step(self._h, ctypes.byref(tt), ctypes.byref(dd), float(tstop), _ptr(h),
                                         _ptr(warm), ctypes.byref(rj)), "scfft_step")
        return tt.value, dd.value, rj.value

    def advance(self, t: float, dt: float, tstop: float, nsteps: int, h, warm):
        """Up to nsteps accepted BS23 steps without the host between steps (one CUDA graph
        launch on the FP32 path); returns (t_new, dt_next, steps_taken)."""
        tt, dd, nd = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_int(0)
        self._check(self._lib.scfft_advance(self._h, ctypes.byref(tt), ctypes.byref(dd), float(tstop), int(nsteps),
                                            _ptr(h), _ptr(warm), ctypes.byref(nd)), "scfft_advance")
        return tt.value, dd.value, nd.value

    def step_host(self, t: float, dt: float, tstop: float, h_host, warm_host, h, warm):
        """One accepted BS23 step with the state in host memory (h_host, warm_host: CPU
        tensors, pinned for speed; warm_host may be None: the warm start then stays in the
        device buffer warm), run on the device buffers h, warm; returns
        (t_new, dt_next, rejected_trials)."""
        import torch
        for a in (h_host, warm_host):
            if a is None and a is warm_host:
                continue
            if a.device.type != "cpu" or a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("h_host, warm_host: contiguous float64 CPU tensors")
        tt, dd, rj = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_int(0)
        self._check(self._lib.scfft_step_host(self._h, ctypes.byref(tt), ctypes.byref(dd), float(tstop),
                                              ctypes.c_void_p(h_host.data_ptr()),
                                              ctypes.c_void_p(None if warm_host is None else warm_host.data_ptr()),
                                              _ptr(h), _ptr(warm), ctypes.byref(rj)), "scfft_step_host")
        return tt.value, dd.value, rj.value

    def profile(self, enable: bool = True):
        self._check(self._lib.scfft_profile(self._h, 1 if enable else 0), "scfft_profile")

    def profile_read(self):
        """{pass name: (launches, total ms)} since profiling was enabled."""
        cnt = (ctypes.c_longlong * NKINDS)()
        ms = (ctypes.c_double * NKINDS)()
        self._check(self._lib.scfft_profile_read(self._h, cnt, ms), "scfft_profile_read")
        return {self._lib.scfft_kind_name(k).decode(): (cnt[k], ms[k]) for k in range(NKINDS)}

    def rhs_vjp(self, h, lam, mu_h, mu_g=None, mu_jc=None):
        """Reverse-mode derivative of the fixed-iteration rhs; returns mu_a (3 floats)."""
        mu_a = (ctypes.c_double * 3)()
        self._check(self._lib.scfft_rhs_vjp(self._h, _ptr(h), _ptr(lam), _ptr(mu_h), _ptr(mu_g), _ptr(mu_jc),
                                            mu_a), "scfft_rhs_vjp")
        return [mu_a[0], mu_a[1], mu_a[2]]

    def adjoint_integrate(self, t0, dts, y0, lam_T, mu_y0, y_end=None, mu_jc=None, checkpoint_every=50):
        """Discrete adjoint of fixed-step BS23 (see scfft.h); returns mu_a."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        mu_a = (ctypes.c_double * 3)()
        self._check(self._lib.scfft_adjoint_integrate(self._h, float(t0), d.ctypes.data, len(d), _ptr(y0),
                                                      _ptr(lam_T), _ptr(y_end), _ptr(mu_y0), _ptr(mu_jc), mu_a,
                                                      int(checkpoint_every)), "scfft_adjoint_integrate")
        return [mu_a[0], mu_a[1], mu_a[2]]

    def adjoint_record(self, ts, y0, warm0=None, y_end=None, checkpoint_every=50):
        """Record the frozen forward map over the step times ts (host, nsteps + 1 values) from
        y0 for the per-step reverse mode (see scfft.h); y_end receives the end state."""
        tt = np.ascontiguousarray(ts, dtype=np.float64)
        self._check(self._lib.scfft_adjoint_record(self._h, tt.ctypes.data, len(tt) - 1, _ptr(y0), _ptr(warm0),
                                                   int(checkpoint_every), _ptr(y_end)), "scfft_adjoint_record")
        return len(tt) - 1

    def adjoint_step(self, n: int, lam, grad_jc=None, grad_path=None):
        """Reverse of step n (n = nsteps-1 down to 0): lam (device) goes from the cotangent of
        y_{n+1} to that of y_n; grad_jc (device) and grad_path (numpy float64 array of
        3 * nknots + 1) are accumulated."""
        gp = None
        if grad_path is not None:
            if grad_path.dtype != np.float64 or not grad_path.flags.c_contiguous:
                raise TypeError("grad_path: contiguous float64 numpy array")
            gp = grad_path.ctypes.data
        self._check(self._lib.scfft_adjoint_step(self._h, int(n), _ptr(lam), _ptr(grad_jc), gp),
                    "scfft_adjoint_step")

    def sync(self):
        self._check(self._lib.scfft_sync(self._h), "scfft_sync")

    def checkpoint_save(self, t: float, dt: float, h, warm) -> bytes:
        """Snapshot of the trajectory at (t, dt) on the device buffers h, warm (see scfft.h)."""
        n = ctypes.c_size_t(0)
        self._check(self._lib.scfft_checkpoint_save(self._h, float(t), float(dt), _ptr(h), _ptr(warm), None,
                                                    ctypes.byref(n)), "scfft_checkpoint_save")
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._lib.scfft_checkpoint_save(self._h, float(t), float(dt), _ptr(h), _ptr(warm), buf,
                                                    ctypes.byref(n)), "scfft_checkpoint_save")
        return buf.raw[:n.value]

    def checkpoint_load(self, data: bytes, h, warm):
        """Restore a snapshot into h, warm (device) and this context; returns (t, dt)."""
        t, dt = ctypes.c_double(0.0), ctypes.c_double(0.0)
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(self._lib.scfft_checkpoint_load(self._h, buf, len(data), ctypes.byref(t), ctypes.byref(dt),
                                                    _ptr(h), _ptr(warm)), "scfft_checkpoint_load")
        return t.value, dt.value

    def inject_fault(self, kind: int):
        """Arm (kind = FAULT_TMA_WAIT) or disarm (0) the one-shot timeout fault; for tests of
        the device-side timeout path only."""
        self._check(self._lib.scfft_inject_fault(self._h, int(kind)), "scfft_inject_fault")

    def stats(self):
        st = _Stats()
        self._check(self._lib.scfft_get_stats(self._h, ctypes.byref(st)), "scfft_get_stats")
        return {k: getattr(st, k) for k, _ in _Stats._fields_}


def _autograd():
    import torch

    class RhsFunction(torch.autograd.Function):
        """dh/dt = rhs(t, h, warm[, jc]) as a differentiable torch op; the backward
        pass is the library's hand-written reverse mode (scfft_rhs_vjp).  The
        context must iterate Eq. 5 a fixed number of times (delta_it = 0), so that
        forward and backward describe the same map."""

        @staticmethod
        def forward(fctx, sc, t, h, warm, jc=None):
            if jc is not None:
                sc.set_jc_map(jc.detach().contiguous())
            out = torch.empty_like(h)
            w = warm.detach().clone()
            sc.rhs(float(t), h.detach().contiguous(), w, out)
            fctx.sc = sc
            fctx.has_jc = jc is not None
            fctx.save_for_backward(h.detach())
            return out

        @staticmethod
        def backward(fctx, lam):
            (h,) = fctx.saved_tensors
            mu_h = torch.empty_like(h)
            mu_g = torch.empty_like(h)
            mu_jc = torch.empty(h.numel() // 3, dtype=h.dtype, device=h.device) if fctx.has_jc else None
            fctx.sc.rhs_vjp(h, lam.contiguous(), mu_h, mu_g, mu_jc)
            return None, None, mu_h, mu_g, mu_jc

    return RhsFunction


def _integrate_autograd():
    import torch

    class IntegrateFunction(torch.autograd.Function):
        """y(ts[-1]) of the frozen BS23 map over the step times ts from y0 (every rhs with
        max_iter Eq. 5 iterations), as a differentiable op of y0, the jc map and the knot
        amplitudes of the applied-field path; the backward pass is the library's
        checkpointed reverse sweep (scfft_adjoint_record / scfft_adjoint_step)."""

        @staticmethod
        def forward(fctx, sc, ts, y0, jc, knots_t, knots_he, checkpoint_every):
            sc.set_jc_map(jc.detach().contiguous())
            sc.set_field_path(list(knots_t), knots_he.detach().cpu().numpy().reshape(-1, 3))
            y_end = torch.empty_like(y0)
            sc.adjoint_record(ts, y0.detach().contiguous(), y_end=y_end, checkpoint_every=checkpoint_every)
            fctx.sc, fctx.S = sc, len(ts) - 1
            fctx.shapes = (jc.shape, knots_he.shape, knots_he.dtype, knots_he.device)
            return y_end

        @staticmethod
        def backward(fctx, lam):
            sc = fctx.sc
            jc_shape, he_shape, he_dtype, he_dev = fctx.shapes
            lam_h = lam.detach().clone().contiguous()
            gjc = torch.zeros(jc_shape, dtype=torch.float64, device=lam.device).reshape(-1)
            gp = np.zeros(3 * (he_shape[0]) + 1)
            for n in range(fctx.S - 1, -1, -1):
                sc.adjoint_step(n, lam_h, gjc, gp)
            ghe = torch.from_numpy(gp[:-1].reshape(he_shape)).to(device=he_dev, dtype=he_dtype)
            return None, None, lam_h, gjc.reshape(jc_shape), None, ghe, None

    return IntegrateFunction


def integrate_autograd(sc: "Context", ts, y0, jc, knots_t, knots_he, checkpoint_every: int = 50):
    """Differentiable end state of the frozen fixed-step BS23 map over the step times ts (the
    accepted step end times of an adaptive run reproduce it, kinks included): gradients flow
    to y0 (device), jc (device, per node) and knots_he (a (K, 3) tensor of the path's knot
    amplitudes at times knots_t).  The context must use delta_it = 0 semantics for the
    forward to equal the map (the record runs with exactly max_iter iterations per rhs)."""
    return _integrate_autograd().apply(sc, ts, y0, jc, knots_t, knots_he, checkpoint_every)


def rhs_autograd(sc: "Context", t: float, h, warm, jc=None):
    """Differentiable dh/dt (see RhsFunction): gradients flow to h, warm and jc."""
    return _autograd().apply(sc, t, h, warm, jc)


def batch_step(ctxs, t, dt, tstop, h, warm):
    """One accepted BS23 step for each of several independent contexts,
    concurrently (scfft_batch_step).  t, dt, tstop: sequences of floats; h, warm:
    sequences of float64 CUDA tensors.  Returns (t_new, dt_new, statuses)."""
    lib = load_library()
    nb = len(ctxs)
    C = ctypes.c_void_p * nb
    Dn = ctypes.c_double * nb
    cs = C(*[c._h.value for c in ctxs])
    tt, dd, ts = Dn(*t), Dn(*dt), Dn(*tstop)
    hp = C(*[_ptr(x) for x in h])
    wp = C(*[_ptr(x) for x in warm])
    st = (ctypes.c_int * nb)()
    code = lib.scfft_batch_step(cs, nb, tt, dd, ts, hp, wp, st)
    if code not in (0,):
        raise ScfftError(code, "scfft_batch_step", lib.scfft_status_string(code).decode())
    return list(tt), list(dd), list(st)
