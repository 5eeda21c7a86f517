"""ctypes binding of include/etd.h: argument marshalling only.

Every computation happens in libetd.so.  Tensors are passed as raw device pointers; the
binding checks dtype, device and contiguity and nothing else.  A missing library raises
immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes as ct

import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libetd.so")

ETD_STATUS = {0: "ETD_OK", 1: "ETD_EINVAL", 2: "ETD_ENOMEM", 3: "ETD_ECUDA", 4: "ETD_ENONFINITE",
              5: "ETD_ENOTCONV", 6: "ETD_ETIMEOUT", 7: "ETD_EMBP"}


class EtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ETD_STATUS.get(code, code)}: {msg}")
        self.code = code


class etd_params(ct.Structure):
    _fields_ = [
        ("dim", ct.c_int), ("n", ct.c_int * 3), ("half_len", ct.c_double * 3),
        ("scheme", ct.c_int), ("model", ct.c_int), ("precision", ct.c_int),
        ("tau", ct.c_double), ("eps_phi", ct.c_double), ("eps_u", ct.c_double),
        ("mu", ct.c_double), ("lambda_surf", ct.c_double), ("kappa", ct.c_double),
        ("lambda_line", ct.c_double), ("M_area", ct.c_double), ("A0", ct.c_double),
        ("alpha", ct.c_double), ("u0", ct.c_double),
        ("gamma", ct.c_double), ("M", ct.c_double), ("ubar", ct.c_double),
        ("A1", ct.c_double), ("A2", ct.c_double), ("B1", ct.c_double), ("B2", ct.c_double),
        ("band_mask_hi", ct.c_double), ("recover_delta", ct.c_double),
        ("cg_rtol", ct.c_double), ("cg_maxit", ct.c_int), ("linear_only", ct.c_int),
        ("cg_rtol_pred", ct.c_double), ("krylov_tol", ct.c_double),
    ]


class etd_diag(ct.Structure):
    _fields_ = [
        ("energy", ct.c_double), ("mass", ct.c_double), ("max_bound", ct.c_double),
        ("umin", ct.c_double), ("umax", ct.c_double), ("volume", ct.c_double),
        ("band_size", ct.c_long), ("cg_iters_last", ct.c_int), ("cg_resid_last", ct.c_double),
        ("krylov_dim_last", ct.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None

SIGNATURES = {
    "etd_plan": (ct.c_int, [ct.POINTER(etd_params), ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "etd_step": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, ct.POINTER(etd_diag)]),
    "etd_energy": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(etd_diag)]),
    "etd_free": (ct.c_int, [ct.c_void_p]),
    "etd_last_error": (ct.c_char_p, []),
    "etd_fft_forward": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "etd_fft_inverse": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "etd_band": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_long)]),
    "etd_nonlocal": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                ct.POINTER(ct.c_int), ct.POINTER(ct.c_double)]),
    "etd_remainder": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                 ct.c_void_p]),
    "etd_timing": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "etd_timing_read": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_long),
                                   ct.POINTER(ct.c_double)]),
}

SIGNATURES.update({
    "etd_plan_batch": (ct.c_int, [ct.POINTER(etd_params), ct.c_int, ct.c_void_p, ct.c_int, ct.POINTER(ct.c_void_p)]),
    "etd_batch_step": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_void_p), ct.c_int]),
    "etd_batch_check": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_void_p),
                                   ct.POINTER(etd_diag)]),
    "etd_batch_info": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int),
                                  ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "etd_batch_free": (ct.c_int, [ct.c_void_p]),
})

SIGNATURES["etd_krylov_coeffs"] = (ct.c_int, [ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.c_double,
                                               ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)])
SIGNATURES["etd_fft_forward_noalloc"] = (ct.c_int, [ct.c_int, ct.POINTER(ct.c_int), ct.c_int, ct.c_void_p,
                                                  ct.c_void_p, ct.c_void_p])

KERNEL_KINDS = ["fft_a_fwd", "fft_a_inv", "fft_b", "cg", "pointwise", "band", "reduce", "krylov"]


def load_library(path: str = LIB_PATH):
    """Load libetd.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2606_04347_gb300/build.py")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(code):
    if code != 0:
        raise EtdError(code, load_library().etd_last_error().decode())


def params_struct(p) -> etd_params:
    """etd_params from a workloads.ModelParams (or any object with the same fields)."""
    s = etd_params()
    s.dim = p.dim
    for i in range(3):
        s.n[i] = int(p.n[i])
        s.half_len[i] = float(p.half_len[i])
    for name, _ in etd_params._fields_:
        if name in ("dim", "n", "half_len"):
            continue
        v = getattr(p, name)
        setattr(s, name, int(v) if name in ("scheme", "model", "precision", "cg_maxit", "linear_only") else float(v))
    return s


def _ptr(t, dtype=None):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if t.device.type != "cuda":
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr()


class Plan:
    """Owns one etd_plan_t.  Field arguments are CUDA tensors of the plan's dtype."""

    def __init__(self, params, stream=None):
        import torch
        self.lib = load_library()
        self.params = params
        self.dtype = torch.float64 if params.precision == 0 else torch.float32
        self.cdtype = torch.complex128 if params.precision == 0 else torch.complex64
        self._s = params_struct(params)
        h = ct.c_void_p()
        st = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
        _check(self.lib.etd_plan(ct.byref(self._s), st, ct.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.etd_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, phi, u, nsteps=1, diag=False):
        d = etd_diag() if diag else None
        _check(self.lib.etd_step(self.h, _ptr(phi, self.dtype), _ptr(u, self.dtype), int(nsteps),
                                 ct.byref(d) if diag else None))
        return d.as_dict() if diag else None

    def energy(self, phi, u):
        d = etd_diag()
        _check(self.lib.etd_energy(self.h, _ptr(phi, self.dtype), _ptr(u, self.dtype), ct.byref(d)))
        return d.as_dict()

    def fft_forward(self, field, out):
        _check(self.lib.etd_fft_forward(self.h, _ptr(field, self.dtype), _ptr(out, self.cdtype)))

    def fft_inverse(self, half, out):
        _check(self.lib.etd_fft_inverse(self.h, _ptr(half, self.cdtype), _ptr(out, self.dtype)))

    def band(self, phi, idx_out):
        import torch
        c = ct.c_long()
        _check(self.lib.etd_band(self.h, _ptr(phi, self.dtype), _ptr(idx_out, torch.int32), ct.byref(c)))
        return c.value

    def nonlocal_solve(self, phi, f, w):
        it, rs = ct.c_int(), ct.c_double()
        _check(self.lib.etd_nonlocal(self.h, _ptr(phi, self.dtype), _ptr(f, self.dtype), _ptr(w, self.dtype),
                                     ct.byref(it), ct.byref(rs)))
        return it.value, rs.value

    def timing(self, enable):
        _check(self.lib.etd_timing(self.h, 1 if enable else 0))

    def timing_read(self):
        """{kind: (total_ms, launches, algorithmic_bytes)} since timing(True)."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            ms, n, b = ct.c_double(), ct.c_long(), ct.c_double()
            _check(self.lib.etd_timing_read(self.h, k, ct.byref(ms), ct.byref(n), ct.byref(b)))
            out[name] = (ms.value, n.value, b.value)
        return out

    def remainder(self, which, phi, phi_old, u, out):
        _check(self.lib.etd_remainder(self.h, int(which), _ptr(phi, self.dtype), _ptr(phi_old, self.dtype),
                                      _ptr(u, self.dtype), _ptr(out, self.dtype)))




class Batch:
    """Owns one etd_batch_t: independent runs, each with its own plan and stream."""

    def __init__(self, params_list, stream=None, autotune=True):
        import torch
        self.lib = load_library()
        self.params = list(params_list)
        n = len(self.params)
        self._arr = (etd_params * n)(*[params_struct(p) for p in self.params])
        self.dtypes = [torch.float64 if p.precision == 0 else torch.float32 for p in self.params]
        h = ct.c_void_p()
        st = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
        _check(self.lib.etd_plan_batch(self._arr, n, st, 1 if autotune else 0, ct.byref(h)))
        self.h = h

    def _ptrs(self, tensors):
        n = len(self.params)
        if tensors is None:
            return None
        vals = [None if t is None else _ptr(t, self.dtypes[i]) for i, t in enumerate(tensors)]
        return (ct.c_void_p * n)(*vals)

    def step(self, phis, us, nsteps):
        _check(self.lib.etd_batch_step(self.h, self._ptrs(phis), self._ptrs(us), int(nsteps)))

    def check(self, phis, us):
        n = len(self.params)
        d = (etd_diag * n)()
        _check(self.lib.etd_batch_check(self.h, self._ptrs(phis), self._ptrs(us), d))
        return [d[i].as_dict() for i in range(n)]

    def info(self, run):
        zb, kb, tma, graph = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        _check(self.lib.etd_batch_info(self.h, int(run), ct.byref(zb), ct.byref(kb), ct.byref(tma), ct.byref(graph)))
        out = {"zb": zb.value, "kb": kb.value, "tma": tma.value, "graph": graph.value}
        if graph.value == 0:
            out["graph_error"] = self.lib.etd_last_error().decode()
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.etd_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def krylov_coeffs(alpha, beta, tau, j):
    """(y, tail) of etd_krylov_coeffs: y = phi_j(tau T) e_1 and |e_m^T phi_{j+1}(tau T) e_1| for the
    tridiagonal T with diagonal alpha and off-diagonal beta (host computation, no GPU)."""
    import numpy as np
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    m = a.size
    b = np.ascontiguousarray(beta if m > 1 else [0.0], dtype=np.float64)
    y = np.zeros(m)
    tail = ct.c_double()
    dp = ct.POINTER(ct.c_double)
    _check(load_library().etd_krylov_coeffs(m, a.ctypes.data_as(dp), b.ctypes.data_as(dp), float(tau), int(j),
                                            y.ctypes.data_as(dp), ct.byref(tail)))
    return y, tail.value
