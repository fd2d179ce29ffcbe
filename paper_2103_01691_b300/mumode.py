"""Thin Python binding of libmumode.so (include/mumode.h): argument
marshalling only.  Every step of the hot path runs in the library's CUDA
kernels; torch supplies device memory and the current stream.  There is no
fallback: if the library is missing or a call fails, an exception is
raised.

Tensors follow the paper's layout (i_1 fastest): a tensor with sizes
(n_1, ..., n_d) is a contiguous torch tensor of shape (n_d, ..., n_1).
Matrices are numpy arrays (FP64, real or complex) indexed [row, column].
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmumode.so")

MM_R64, MM_C64, MM_C128, MM_R32 = 0, 1, 2, 3
PREC = {"fp64": 0, "fp32": 1, "bf16x6": 2, "bf16x3": 3, "bf16": 4, "f16x6": 5, "fp64dmma": 6, "auto": 7, "tf32x3": 8}
STATUS = {0: "MM_OK", 1: "MM_ERR_INVALID_ARG", 2: "MM_ERR_SHAPE", 3: "MM_ERR_DTYPE", 4: "MM_ERR_ALIGN",
          5: "MM_ERR_OOM", 6: "MM_ERR_CUDA", 7: "MM_ERR_TIMEOUT", 8: "MM_ERR_UNSUPPORTED", 9: "MM_ERR_RANGE"}

# Every symbol include/mumode.h declares, with its ctypes signature.
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "mm_ctx_create": (_i, [_i, ctypes.POINTER(_vp)]),
    "mm_ctx_destroy": (None, [_vp]),
    "mm_last_error": (ctypes.c_char_p, []),
    "mm_device_status": (_i, [_vp, _vp]),
    "mm_launch_count": (_i64, []),
    "mm_kernel_timing": (_i, [_vp, _i]),
    "mm_kernel_timing_read": (_i, [_vp, _dp, ctypes.POINTER(_i64)]),
    "mm_fd_laplacian_dirichlet": (_i, [_i, _dp]),
    "mm_expm": (_i, [_i, _dp, _dp, _d, _d, _dp]),
    "mm_gauss_hermite": (_i, [_i, _dp, _dp]),
    "mm_hermite_matrices": (_i, [_i, _dp, _dp]),
    "mumode_product": (_i, [_vp, _i, _i64p, _i, _dp, _i64, _i, _i, _i, _vp, _vp, _vp]),
    "mumode_product_noalloc": (_i, [_i, _i64p, _i, _dp, _i64, _i, _vp, _vp, _vp]),
    "mumode_plan_create": (_i, [_vp, _i, _i64p, ctypes.POINTER(_dp), _i, _i, _i, ctypes.POINTER(_i),
                                ctypes.POINTER(_vp)]),
    "mumode_step": (_i, [_vp, _vp, _i64, _vp]),
    "mumode_step_host": (_i, [_vp, _vp, _i64, _vp]),
    "mm_plan_destroy": (None, [_vp]),
    "mm_plan_set_graphs": (_i, [_vp, _i]),
    "mm_plan_get_fold": (_i, [_vp, ctypes.POINTER(_i)]),
    "mm_plan_set_fold": (_i, [_vp, _i]),
    "mm_plan_issued_flops": (_i, [_vp, _dp]),
    "mumode_batch_create": (_i, [_vp, ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "mumode_batch_step": (_i, [_vp, ctypes.POINTER(_vp), _i64, _vp]),
    "mm_batch_destroy": (None, [_vp]),
    "mumode_step_batched": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i64, _vp]),
    "mm_plan_autotune": (_i, [_vp, _vp, _i64, _vp]),
    "split_step_gpe_autotune": (_i, [_vp, _vp, ctypes.c_double, ctypes.c_double, _i64, _vp]),
    "mumode_batch_autotune": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i64, ctypes.POINTER(_i), _vp]),
    "mm_plan_get_config": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "mm_plan_set_config": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "hermite_plan_create": (_i, [_vp, _i, _i64p, _i, _i, ctypes.POINTER(_vp)]),
    "mm_hermite_hamiltonian": (_i, [_i, _dp, _dp]),
    "mm_expm_device": (_i, [_vp, _i, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            _vp, _vp]),
    "mm_plan_set_matrix_device": (_i, [_vp, _i, _vp, ctypes.c_double, _vp]),
    "hkmp_plan_create": (_i, [_vp, _i, _i64p, ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.c_double, _i, _i,
                              ctypes.POINTER(_vp)]),
    "hkmp_evolve": (_i, [_vp, _vp, _i64, _dp, _vp]),
    "hkmp_set_f_range": (_i, [_vp, ctypes.c_double, ctypes.c_double, _vp]),
    "mm_pipe_operators": (_i, [_i, _i, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp,
                               _dp]),
    "pipe_plan_create": (_i, [_vp, _i, _i, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp,
                              ctypes.c_double, _i, ctypes.POINTER(_vp)]),
    "hkp_plan_create": (_i, [_vp, _i, _i64p, ctypes.POINTER(_dp), ctypes.c_double, _i, _i, ctypes.POINTER(_i),
                             ctypes.POINTER(_vp)]),
    "hermite_nodes": (_i, [_vp, _i, _dp, _dp]),
    "hermite_forward": (_i, [_vp, _vp, _vp, _vp]),
    "hermite_backward": (_i, [_vp, _vp, _vp, _vp]),
    "hermite_ho_step": (_i, [_vp, _vp, _d, _i64, _vp]),
    "split_step_gpe": (_i, [_vp, _vp, _d, _d, _i64, _vp]),
    "split_step_gpe_norm2": (_i, [_vp, _vp, _d, _d, _i64, ctypes.POINTER(ctypes.c_double), _vp]),
    "split_step_gpe_adjoint": (_i, [_vp, _vp, _vp, _vp, _d, _d, _i64, _i64, _vp]),
    "mm_norm2": (_i, [_vp, _vp, _i, _dp, _vp]),
}

_lib = None


class MumodeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libmumode.so (built by ``python -m paper_2103_01691_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2103_01691_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise MumodeError(status, lib().mm_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _complex_interleaved(M) -> tuple[np.ndarray, int]:
    M = np.asarray(M)
    if np.iscomplexobj(M):
        return np.ascontiguousarray(M, dtype=np.complex128).view(np.float64), 1
    return np.ascontiguousarray(M, dtype=np.float64), 0


def _stream(stream=None):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch

    codes = {torch.complex64: MM_C64, torch.complex128: MM_C128, torch.float64: MM_R64, torch.float32: MM_R32}
    if t.dtype not in codes:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return codes[t.dtype]


def _dims(shape) -> np.ndarray:
    return np.array(list(shape)[::-1], dtype=np.int64)


def _need_cuda(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")


# --------------------------------------------------------------------- context

class Context:
    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(lib().mm_ctx_create(device, ctypes.byref(h)))
        self.handle = h
        self.device = device

    def status(self, stream=None):
        _check(lib().mm_device_status(self.handle, _stream(stream)))

    def kernel_timing(self, enable: bool = True):
        _check(lib().mm_kernel_timing(self.handle, int(enable)))

    def kernel_timing_read(self):
        """(total milliseconds, launches) of the mode-product kernels timed since enabling."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        _check(lib().mm_kernel_timing_read(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if self.handle:
            lib().mm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    return int(lib().mm_launch_count())


# ------------------------------------------------------------ host set-up (FP64)

def fd_laplacian_dirichlet(n: int) -> np.ndarray:
    A = np.empty((n, n))
    _check(lib().mm_fd_laplacian_dirichlet(n, _dptr(A)))
    return A


def expm(A, z: complex = 1.0) -> np.ndarray:
    A = np.asarray(A)
    n = A.shape[0]
    Are = np.ascontiguousarray(A.real, dtype=np.float64)
    Aim = np.ascontiguousarray(A.imag, dtype=np.float64) if np.iscomplexobj(A) else None
    E = np.empty((n, n), dtype=np.complex128)
    z = complex(z)
    _check(lib().mm_expm(n, _dptr(Are), _dptr(Aim) if Aim is not None else None, z.real, z.imag,
                         E.view(np.float64).ctypes.data_as(_dp)))
    return E


def gauss_hermite(m: int):
    x, W = np.empty(m), np.empty(m)
    _check(lib().mm_gauss_hermite(m, _dptr(x), _dptr(W)))
    return x, W


def hermite_matrices(m: int):
    F, B = np.empty((m, m)), np.empty((m, m))
    _check(lib().mm_hermite_matrices(m, _dptr(F), _dptr(B)))
    return F, B


def hermite_hamiltonian(m: int, V=None):
    """mm_hermite_hamiltonian: one direction's Hamiltonian in the m Hermite
    functions for the potential values V at the nodes (None: harmonic)."""
    H = np.empty((m, m))
    Vc = None if V is None else np.ascontiguousarray(V, dtype=np.float64)
    _check(lib().mm_hermite_hamiltonian(m, _dptr(Vc) if Vc is not None else None, _dptr(H)))
    return H


def expm_device(ctx: Context, A, B=None, f: float = 0.0, z: complex = 1.0, norm_bound: float = 0.0, out=None,
                stream=None):
    """mm_expm_device: exp(z (A + f B)) in FP64 on the GPU for real CUDA
    float64 matrices A, B (n x n); returns (or fills) a complex128 CUDA tensor."""
    import torch

    _need_cuda(A)
    n = A.shape[0]
    if A.dtype != torch.float64 or A.shape != (n, n) or not A.is_contiguous():
        raise ValueError("A must be a contiguous square float64 tensor")
    if B is not None:
        _need_cuda(B)
        if B.dtype != torch.float64 or B.shape != (n, n) or not B.is_contiguous():
            raise ValueError("B must match A")
    if out is None:
        out = torch.empty((n, n), dtype=torch.complex128, device=A.device)
    z = complex(z)
    _check(lib().mm_expm_device(ctx.handle, n, ctypes.c_void_p(A.data_ptr()),
                                ctypes.c_void_p(B.data_ptr()) if B is not None else None, float(f), z.real, z.imag,
                                float(norm_bound), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


# ------------------------------------------------------------- mu-mode product

def mumode_product(ctx: Context, u, mu: int, L, prec: str = "f16x6", out=None, stream=None):
    """S = U x_mu L (Definition 2.1) on a CUDA tensor u."""
    import torch

    _need_cuda(u)
    Lf, Lc = _complex_interleaved(L)
    m = int(np.asarray(L).shape[0])
    dims = _dims(u.shape)
    d = len(dims)
    out_shape = list(u.shape)
    out_shape[d - mu] = m
    if out is None:
        out = torch.empty(out_shape, dtype=u.dtype, device=u.device)
    _check(lib().mumode_product(ctx.handle, d, dims.ctypes.data_as(_i64p), mu, _dptr(Lf), m, Lc,
                                _dtype_code(u), PREC[prec], ctypes.c_void_p(u.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def mumode_product_noalloc(u, mu: int, L, out=None, stream=None):
    """S = U x_mu L with MM_PREC_F16X6, using only the library's static
    device scratch (no device allocation inside the call; `out` may be
    passed preallocated).  See mumode_product_noalloc in include/mumode.h."""
    import torch

    _need_cuda(u)
    if u.dtype != torch.complex64:
        raise TypeError("mumode_product_noalloc takes complex64 data")
    dims = _dims(u.shape)
    d = len(dims)
    if not 1 <= mu <= d:
        raise ValueError(f"mu = {mu} outside 1..{d}")
    La = np.asarray(L)
    if La.ndim != 2 or La.shape[1] != u.shape[d - mu]:
        raise ValueError(f"L must be 2-D with {u.shape[d - mu]} columns (n_mu), got shape {La.shape}")
    Lf, Lc = _complex_interleaved(La)
    m = int(La.shape[0])
    out_shape = list(u.shape)
    out_shape[d - mu] = m
    if out is None:
        out = torch.empty(out_shape, dtype=u.dtype, device=u.device)
    elif (out.dtype != torch.complex64 or out.device != u.device or not out.is_contiguous()
          or list(out.shape) != out_shape):
        raise ValueError(f"out must be a contiguous complex64 tensor of shape {out_shape} on {u.device}")
    # the library works on the current device: make it u's
    with torch.cuda.device(u.device):
        _check(lib().mumode_product_noalloc(d, dims.ctypes.data_as(_i64p), mu, _dptr(Lf), m, Lc,
                                            ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            _stream(stream)))
    return out


# tensor-core kernels, mm_plan_set_config codes 0..3; "chain" runs all products of a Tucker step
# call in one persistent launch of the pair64 kernel (F16X6), elsewhere it launches like pair64
VARIANTS = ("pair64", "pair128", "one_sm", "chain")


class _Tunable:
    """Kernel variant and mode order of a plan, and the autotuner."""

    def autotune(self, u, nsteps: int = 3, stream=None):
        """mm_plan_autotune: time the variants and mode orders on a copy of u
        (left unchanged) and keep the fastest; returns (variant, order)."""
        _need_cuda(u)
        _check(lib().mm_plan_autotune(self.handle, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream(stream)))
        return self.config()

    def config(self):
        v = _i()
        order = (_i * len(self.dims))()
        _check(lib().mm_plan_get_config(self.handle, ctypes.byref(v), order))
        return VARIANTS[v.value], tuple(order)

    def set_graphs(self, enable: bool):
        _check(lib().mm_plan_set_graphs(self.handle, int(enable)))

    def fold(self) -> int:
        """mm_plan_get_fold: the directions the steps run folded (bit v: direction v + 1)."""
        m = _i()
        _check(lib().mm_plan_get_fold(self.handle, ctypes.byref(m)))
        return m.value

    def set_fold(self, enable: bool):
        _check(lib().mm_plan_set_fold(self.handle, int(enable)))

    def set_config(self, variant: str, order=None):
        optr = (_i * len(order))(*order) if order is not None else None
        _check(lib().mm_plan_set_config(self.handle, VARIANTS.index(variant), optr))


class TuckerPlan(_Tunable):
    """U <- U x_1 E_1 ... x_d E_d repeated (eq. (dd-tensor))."""

    def __init__(self, ctx: Context, dims, Es, prec: str = "f16x6", dtype=None, order=None):
        import torch

        self.ctx = ctx
        self.dims = np.array(dims, dtype=np.int64)
        d = len(self.dims)
        cplx = any(np.iscomplexobj(E) for E in Es)
        self._mats = [(np.ascontiguousarray(E, dtype=np.complex128).view(np.float64) if cplx
                       else np.ascontiguousarray(E, dtype=np.float64)) for E in Es]
        ptrs = (_dp * d)(*[_dptr(M) for M in self._mats])
        if dtype is None:
            dtype = torch.complex128 if prec in ("fp64", "fp64dmma") else torch.complex64
        self.dtype = dtype
        code = {torch.complex64: MM_C64, torch.complex128: MM_C128, torch.float64: MM_R64, torch.float32: MM_R32}[dtype]
        optr = (_i * d)(*order) if order is not None else None
        h = ctypes.c_void_p()
        _check(lib().mumode_plan_create(ctx.handle, d, self.dims.ctypes.data_as(_i64p), ptrs, int(cplx), code,
                                        PREC[prec], optr, ctypes.byref(h)))
        self.handle = h

    def set_matrix_device(self, mu: int, E, row_norm_bound: float = 0.0, stream=None):
        """mm_plan_set_matrix_device: direction mu's matrix from a CUDA
        complex128 tensor (n_mu x n_mu), used by the following steps."""
        _need_cuda(E)
        _check(lib().mm_plan_set_matrix_device(self.handle, int(mu), ctypes.c_void_p(E.data_ptr()),
                                               float(row_norm_bound), _stream(stream)))

    def issued_flops(self) -> float:
        """Tensor-core flops issued per step (see mm_plan_issued_flops)."""
        f = ctypes.c_double()
        _check(lib().mm_plan_issued_flops(self.handle, ctypes.byref(f)))
        return f.value

    def step(self, u, nsteps: int = 1, stream=None):
        _need_cuda(u)
        _check(lib().mumode_step(self.handle, ctypes.c_void_p(u.data_ptr()), int(nsteps), _stream(stream)))
        return u

    def norm2(self, u, stream=None) -> float:
        _need_cuda(u)
        out = ctypes.c_double()
        _check(lib().mm_norm2(self.handle, ctypes.c_void_p(u.data_ptr()), 0, ctypes.byref(out), _stream(stream)))
        return out.value

    def step_host(self, u_host, nsteps: int = 1, stream=None):
        """u_host: a CPU torch tensor (pinned for speed), stepped in place."""
        if u_host.is_cuda or not u_host.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        _check(lib().mumode_step_host(self.handle, ctypes.c_void_p(u_host.data_ptr()), int(nsteps),
                                      _stream(stream)))
        return u_host

    def close(self):
        if self.handle:
            lib().mm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_batched(ctx: Context, plans, us, nsteps: int = 1, stream=None):
    """mumode_step_batched: plans stepped together in one call (the batch is
    made and released inside; keep a Batch for repeated calls)."""
    for u in us:
        _need_cuda(u)
    parr = (_vp * len(plans))(*[p.handle.value for p in plans])
    uarr = (_vp * len(us))(*[u.data_ptr() for u in us])
    _check(lib().mumode_step_batched(ctx.handle, parr, uarr, len(plans), int(nsteps), _stream(stream)))
    return us


def batch_autotune(ctx: Context, plans, us, nsteps: int = 3, stream=None):
    """mumode_batch_autotune: the fastest common mode order of a batch over
    plans, timed on copies of us (left unchanged) and set on every plan."""
    for u in us:
        _need_cuda(u)
    parr = (_vp * len(plans))(*[p.handle.value for p in plans])
    uarr = (_vp * len(us))(*[u.data_ptr() for u in us])
    order = (_i * len(plans[0].dims))()
    _check(lib().mumode_batch_autotune(ctx.handle, parr, uarr, len(plans), int(nsteps), order, _stream(stream)))
    return tuple(order)


class Batch:
    """Independent Tucker plans stepped together, one launch per direction."""

    def __init__(self, ctx: Context, plans):
        self.ctx = ctx
        self.plans = list(plans)  # keeps the plans alive
        arr = (_vp * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib().mumode_batch_create(ctx.handle, arr, len(self.plans), ctypes.byref(h)))
        self.handle = h

    def step(self, us, nsteps: int = 1, stream=None):
        for u in us:
            _need_cuda(u)
        arr = (_vp * len(us))(*[u.data_ptr() for u in us])
        _check(lib().mumode_batch_step(self.handle, arr, int(nsteps), _stream(stream)))
        return us

    def close(self):
        if self.handle:
            lib().mm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HKPPlan(TuckerPlan):
    """hkp_plan_create: Tucker plan of the values-space propagators
    Psi_mu exp(-i tau H_mu) Phi_mu^W of a Kronecker potential (section 4.3).
    Vs[mu-1] holds V_mu at the Gauss-Hermite nodes of direction mu (see
    gauss_hermite), or None for the harmonic x^2/2.  step() advances the
    values at the nodes by nsteps * tau."""

    def __init__(self, ctx: Context, dims, Vs, tau: float, prec: str = "f16x6", dtype=None, order=None):
        import torch

        self.ctx = ctx
        self.dims = np.array(dims, dtype=np.int64)
        d = len(self.dims)
        self._mats = [None if V is None else np.ascontiguousarray(V, dtype=np.float64) for V in Vs]
        ptrs = (_dp * d)(*[_dptr(V) if V is not None else None for V in self._mats])
        if dtype is None:
            dtype = torch.complex128 if prec in ("fp64", "fp64dmma") else torch.complex64
        self.dtype = dtype
        code = {torch.complex64: MM_C64, torch.complex128: MM_C128}[dtype]
        optr = (_i * d)(*order) if order is not None else None
        h = ctypes.c_void_p()
        _check(lib().hkp_plan_create(ctx.handle, d, self.dims.ctypes.data_as(_i64p), ptrs, float(tau), code,
                                     PREC[prec], optr, ctypes.byref(h)))
        self.handle = h


def pipe_operators(n_r: int, n_z: int, rmin: float, rmax: float, zmax: float, alpha: float, s=None):
    """mm_pipe_operators: the radial and axial operators of the pipe flow (section 4.2)."""
    Ar, Az = np.empty((n_r, n_r)), np.empty((n_z, n_z))
    sc = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
    _check(lib().mm_pipe_operators(n_r, n_z, float(rmin), float(rmax), float(zmax), float(alpha),
                                   _dptr(sc) if sc is not None else None, _dptr(Ar), _dptr(Az)))
    return Ar, Az


class PipePlan(TuckerPlan):
    """pipe_plan_create: the pipe-flow solution operator over T as a d = 2
    real FP64 Tucker plan (direction 1 = r).  step(c) advances c, a CUDA
    float64 tensor of shape (n_z, n_r), by T."""

    def __init__(self, ctx: Context, n_r: int, n_z: int, rmin: float, rmax: float, zmax: float, alpha: float, s,
                 T: float, prec: str = "fp64dmma"):
        import torch

        self.ctx = ctx
        self.dims = np.array([n_r, n_z], dtype=np.int64)
        self.dtype = torch.float64
        self._s = np.ascontiguousarray(s, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib().pipe_plan_create(ctx.handle, n_r, n_z, float(rmin), float(rmax), float(zmax), float(alpha),
                                      _dptr(self._s), float(T), PREC[prec], ctypes.byref(h)))
        self.handle = h


class HKMPPlan:
    """hkmp_plan_create / hkmp_evolve (section 4.4): Magnus steps for the
    potential V_mu(x_mu) + f(t) U_mu(x_mu).  Vs, Us: values at the
    Gauss-Hermite nodes per direction (None: harmonic / no time dependence)."""

    def __init__(self, ctx: Context, dims, Vs, Us, tau: float, prec: str = "f16x6", dtype=None):
        import torch

        self.ctx = ctx
        self.dims = np.array(dims, dtype=np.int64)
        d = len(self.dims)
        self._v = [None if V is None else np.ascontiguousarray(V, dtype=np.float64) for V in Vs]
        self._u = [None if U is None else np.ascontiguousarray(U, dtype=np.float64) for U in Us]
        vp = (_dp * d)(*[_dptr(V) if V is not None else None for V in self._v])
        up = (_dp * d)(*[_dptr(U) if U is not None else None for U in self._u])
        if dtype is None:
            dtype = torch.complex128 if prec in ("fp64", "fp64dmma") else torch.complex64
        self.dtype = dtype
        code = {torch.complex64: MM_C64, torch.complex128: MM_C128}[dtype]
        h = ctypes.c_void_p()
        _check(lib().hkmp_plan_create(ctx.handle, d, self.dims.ctypes.data_as(_i64p), vp, up, float(tau), code,
                                      PREC[prec], ctypes.byref(h)))
        self.handle = h

    def set_f_range(self, f_lo: float, f_hi: float, stream=None):
        """hkmp_set_f_range: the exponentials at the Chebyshev nodes of [f_lo, f_hi], computed
        once and used by every later chunk of steps whose f values lie in the range."""
        _check(lib().hkmp_set_f_range(self.handle, float(f_lo), float(f_hi), _stream(stream)))

    def evolve(self, psi, f_mid, stream=None):
        """len(f_mid) Magnus steps on the values psi (in place); f_mid[k] = f(t_k + tau/2)."""
        _need_cuda(psi)
        f = np.ascontiguousarray(f_mid, dtype=np.float64)
        _check(lib().hkmp_evolve(self.handle, ctypes.c_void_p(psi.data_ptr()), int(f.size), _dptr(f),
                                 _stream(stream)))
        return psi

    def close(self):
        if self.handle:
            lib().mm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HermitePlan(_Tunable):
    """Hermite spectral transforms and the HKP / GPE steps (sections 3, 4.3, 4.5)."""

    def __init__(self, ctx: Context, dims, prec: str = "f16x6", dtype=None):
        import torch

        self.ctx = ctx
        self.dims = np.array(dims, dtype=np.int64)
        if dtype is None:
            dtype = torch.complex128 if prec in ("fp64", "fp64dmma") else torch.complex64
        self.dtype = dtype
        code = MM_C128 if dtype == torch.complex128 else MM_C64
        h = ctypes.c_void_p()
        _check(lib().hermite_plan_create(ctx.handle, len(self.dims), self.dims.ctypes.data_as(_i64p), code,
                                         PREC[prec], ctypes.byref(h)))
        self.handle = h

    def nodes(self, mu: int):
        m = int(self.dims[mu - 1])
        x, W = np.empty(m), np.empty(m)
        _check(lib().hermite_nodes(self.handle, mu, _dptr(x), _dptr(W)))
        return x, W

    def forward(self, vals, out=None, stream=None):
        import torch

        _need_cuda(vals)
        out = torch.empty_like(vals) if out is None else out
        _check(lib().hermite_forward(self.handle, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     _stream(stream)))
        return out

    def backward(self, coef, out=None, stream=None):
        import torch

        _need_cuda(coef)
        out = torch.empty_like(coef) if out is None else out
        _check(lib().hermite_backward(self.handle, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      _stream(stream)))
        return out

    def ho_step(self, psi, tau: float, nsteps: int = 1, stream=None):
        _need_cuda(psi)
        _check(lib().hermite_ho_step(self.handle, ctypes.c_void_p(psi.data_ptr()), float(tau), int(nsteps),
                                     _stream(stream)))
        return psi

    def gpe_step(self, psi, beta: float, tau: float, nsteps: int = 1, stream=None):
        _need_cuda(psi)
        _check(lib().split_step_gpe(self.handle, ctypes.c_void_p(psi.data_ptr()), float(beta), float(tau),
                                    int(nsteps), _stream(stream)))
        return psi

    def gpe_step_norm2(self, psi, beta: float, tau: float, nsteps: int = 1, stream=None) -> float:
        """gpe_step, returning the weighted norm sum |psi|^2 W of the result (taken in the last
        product's epilogue, or in the unfold of folded steps, where the plan allows)."""
        _need_cuda(psi)
        out = ctypes.c_double()
        _check(lib().split_step_gpe_norm2(self.handle, ctypes.c_void_p(psi.data_ptr()), float(beta), float(tau),
                                          int(nsteps), ctypes.byref(out), _stream(stream)))
        return out.value

    def gpe_autotune(self, psi, beta: float, tau: float, nsteps: int = 3, stream=None):
        """split_step_gpe_autotune: the kernel variant timed on GPE steps (on a copy of psi)."""
        _need_cuda(psi)
        _check(lib().split_step_gpe_autotune(self.handle, ctypes.c_void_p(psi.data_ptr()), float(beta), float(tau),
                                             int(nsteps), _stream(stream)))
        return self.config()

    def gpe_adjoint(self, psi0, gT, beta: float, tau: float, nsteps: int, ckpt_every: int = 50, out=None,
                    stream=None):
        """Gradient at psi0 of a real loss whose gradient at psi_T is gT."""
        import torch

        _need_cuda(psi0)
        _need_cuda(gT)
        out = torch.empty_like(psi0) if out is None else out
        _check(lib().split_step_gpe_adjoint(self.handle, ctypes.c_void_p(psi0.data_ptr()),
                                            ctypes.c_void_p(gT.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            float(beta), float(tau), int(nsteps), int(ckpt_every),
                                            _stream(stream)))
        return out

    def norm2(self, u, weighted: bool = True, stream=None) -> float:
        _need_cuda(u)
        out = ctypes.c_double()
        _check(lib().mm_norm2(self.handle, ctypes.c_void_p(u.data_ptr()), int(weighted), ctypes.byref(out),
                              _stream(stream)))
        return out.value

    def close(self):
        if self.handle:
            lib().mm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gpe_evolve(plan: HermitePlan, psi0, beta: float, tau: float, nsteps: int, ckpt_every: int = 50):
    """psi_T = nsteps Strang steps of psi0, differentiable with respect to psi0
    (torch.autograd); the backward pass runs split_step_gpe_adjoint."""
    import torch

    class _GPE(torch.autograd.Function):
        @staticmethod
        def forward(ctx, psi):
            out = psi.detach().clone()
            plan.gpe_step(out, beta, tau, nsteps)
            ctx.save_for_backward(psi.detach())
            return out

        @staticmethod
        def backward(ctx, g):
            (psi,) = ctx.saved_tensors
            return plan.gpe_adjoint(psi, g.contiguous(), beta, tau, nsteps, ckpt_every)

    return _GPE.apply(psi0)
