"""Python face of the FP64 CPU oracle (``mumode_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The product package never imports this module.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

Arrays follow the paper's layout (section 4.1: i_1 fastest): a d-way tensor
with sizes (n_1, ..., n_d) is a C-contiguous numpy array of shape
(n_d, ..., n_1).  Matrices are numpy arrays indexed [row, column].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mumode_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_c128 = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_f64 = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i, d, i64, vp = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        L.or_fd_dirichlet.argtypes = [i, _f64]
        L.or_fd_periodic.argtypes = [i, d, _f64]
        L.or_expm_dirichlet_fd.argtypes = [i, d, d, _c128]
        L.or_expm_taylor.argtypes = [i, _f64, vp, d, d, _c128]
        L.or_mode_product.argtypes = [i, _i64, i, i64, _c128, _c128, _c128]
        L.or_tucker.argtypes = [i, _i64, ctypes.POINTER(vp), vp, i64, _c128, _c128]
        L.or_tucker3_entries.argtypes = [_i64, _c128, _c128, _c128, _c128, i64, _i64, _c128]
        L.or_hermite_functions.argtypes = [i, i, _f64, _f64]
        L.or_gauss_hermite.argtypes = [i, _f64, _f64, _f64]
        L.or_gauss_hermite.restype = i
        L.or_hermite_forward.argtypes = [i, _f64, _f64, _c128, _c128]
        L.or_hermite_backward.argtypes = [i, _f64, _f64, _c128, _c128]
        L.or_ho_steps.argtypes = [i, _f64, _f64, d, i64, _c128]
        L.or_gpe_steps.argtypes = [i, _f64, _f64, d, d, i64, _c128]
        L.or_gpe_adjoint.argtypes = [i, _f64, _f64, d, d, i64, _c128, _c128, _c128]
        L.or_hkp_hamiltonian.argtypes = [i, _f64, _f64, _f64, _f64]
        L.or_hermite_galerkin.argtypes = [i, _f64, _f64, _f64, _f64]
        L.or_pipe_radial.argtypes = [i, d, d, d, i, _f64]
        L.or_pipe_axial.argtypes = [i, d, d, vp, _f64]
        L.or_hkmp_steps.argtypes = [_i64, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), d, i64, _f64, _c128]
        L.or_hkp_steps.argtypes = [_i64, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), d, i64,
                                   _c128]
        _lib = L
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims(U):
    """Sizes (n_1, ..., n_d) of a tensor stored with shape (n_d, ..., n_1)."""
    return np.array(U.shape[::-1], dtype=np.int64)


# --- 1D operators and exponentials (section 2; section 4.1) ---------------

def fd_dirichlet(n: int) -> np.ndarray:
    A = np.empty((n, n))
    lib().or_fd_dirichlet(n, A)
    return A


def fd_periodic(n: int, length: float) -> np.ndarray:
    A = np.empty((n, n))
    lib().or_fd_periodic(n, float(length), A)
    return A


def expm_dirichlet_fd(n: int, z: complex) -> np.ndarray:
    """exp(z A) for the Dirichlet FD Laplacian, closed form (sine basis)."""
    E = np.empty((n, n), dtype=np.complex128)
    z = complex(z)
    lib().or_expm_dirichlet_fd(n, z.real, z.imag, E)
    return E


def expm_taylor(A: np.ndarray, z: complex = 1.0) -> np.ndarray:
    """exp(z A), Taylor series with scaling and squaring."""
    n = A.shape[0]
    Are = np.ascontiguousarray(A.real, dtype=np.float64)
    keep = None
    aim = None
    if np.iscomplexobj(A):
        keep = np.ascontiguousarray(A.imag, dtype=np.float64)
        aim = keep.ctypes.data
    E = np.empty((n, n), dtype=np.complex128)
    z = complex(z)
    lib().or_expm_taylor(n, Are, aim, z.real, z.imag, E)
    del keep
    return E


# --- mu-mode product and Tucker operator (Definition 2.1; eq. (dd-tensor)) -

def mode_product(U: np.ndarray, mu: int, L: np.ndarray) -> np.ndarray:
    """S = U x_mu L (mu is 1-based, L is m x n_mu)."""
    U = _c(U)
    L = _c(L)
    n = _dims(U)
    d = len(n)
    m = L.shape[0]
    assert L.shape[1] == n[mu - 1]
    out_dims = n.copy()
    out_dims[mu - 1] = m
    S = np.empty(tuple(out_dims[::-1]), dtype=np.complex128)
    lib().or_mode_product(d, n, mu, m, L, U, S)
    return S


def tucker(U: np.ndarray, E, order=None, nsteps: int = 1) -> np.ndarray:
    """nsteps applications of U x_{o_1} E_{o_1} ... x_{o_d} E_{o_d}."""
    U = _c(U)
    n = _dims(U)
    d = len(n)
    Es = [_c(e) for e in E]
    ptrs = (ctypes.c_void_p * d)(*[e.ctypes.data for e in Es])
    keep = None
    optr = None
    if order is not None:
        keep = np.array(order, dtype=np.int32)
        optr = keep.ctypes.data
    out = np.empty_like(U)
    lib().or_tucker(d, n, ptrs, optr, int(nsteps), U, out)
    del keep
    return out


def tucker3_entries(U: np.ndarray, E1, E2, E3, idx: np.ndarray) -> np.ndarray:
    """Entries S(i1,i2,i3) of U x_1 E1 x_2 E2 x_3 E3; idx is (P,3) 0-based."""
    U = _c(U)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.shape[0], dtype=np.complex128)
    lib().or_tucker3_entries(_dims(U), _c(E1), _c(E2), _c(E3), U, idx.shape[0], idx, out)
    return out


# --- Hermite functions, quadrature, HKP and GPE (sections 3, 4.3, 4.5) ----

def gauss_hermite(m: int):
    """Nodes x, weights w for exp(-x^2), and W = w exp(x^2)."""
    x, w, W = np.empty(m), np.empty(m), np.empty(m)
    st = lib().or_gauss_hermite(m, x, w, W)
    if st != 0:
        raise RuntimeError("oracle Gauss-Hermite Newton iteration did not converge")
    return x, w, W


def hermite_functions(nfun: int, x: np.ndarray) -> np.ndarray:
    """H[k, l] = phi_k(x_l)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    H = np.empty((nfun, x.size))
    lib().or_hermite_functions(nfun, x.size, x, H)
    return H


def hermite_forward(vals, x, W):
    vals = _c(vals)
    out = np.empty_like(vals)
    lib().or_hermite_forward(vals.shape[0], _f(x), _f(W), vals, out)
    return out


def hermite_backward(coef, x, W):
    coef = _c(coef)
    out = np.empty_like(coef)
    lib().or_hermite_backward(coef.shape[0], _f(x), _f(W), coef, out)
    return out


def ho_steps(psi, x, W, tau: float, nsteps: int):
    psi = _c(psi).copy()
    lib().or_ho_steps(psi.shape[0], _f(x), _f(W), float(tau), int(nsteps), psi)
    return psi


def gpe_steps(psi, x, W, beta: float, tau: float, nsteps: int):
    psi = _c(psi).copy()
    lib().or_gpe_steps(psi.shape[0], _f(x), _f(W), float(beta), float(tau), int(nsteps), psi)
    return psi


def gpe_adjoint(psi0, gT, x, W, beta: float, tau: float, nsteps: int):
    psi0 = _c(psi0)
    gT = _c(gT)
    g0 = np.empty_like(psi0)
    lib().or_gpe_adjoint(psi0.shape[0], _f(x), _f(W), float(beta), float(tau), int(nsteps),
                         psi0, gT, g0)
    return g0


def hkp_hamiltonian(x, W, V):
    """H[j, k] = (k + 1/2) delta_jk + sum_l W_l phi_j(x_l) (V_l - x_l^2/2) phi_k(x_l)
    (section 4.3: one direction's Hamiltonian in the Hermite basis)."""
    x, W, V = _f(x), _f(W), _f(V)
    H = np.empty((x.size, x.size))
    lib().or_hkp_hamiltonian(x.size, x, W, V, H)
    return H


def hkp_steps(psi, xs, Ws, Vs, tau: float, nsteps: int = 1):
    """nsteps HKP steps (section 4.3) for the Kronecker potential whose
    direction-mu values at the nodes xs[mu-1] are Vs[mu-1]; psi has shape
    (n_3, n_2, n_1)."""
    psi = _c(psi).copy()
    n = _dims(psi)
    keep = [_f(a) for a in (*xs, *Ws, *Vs)]
    for v in range(3):
        assert keep[v].size == keep[3 + v].size == keep[6 + v].size == n[v]
    ptr = [a.ctypes.data_as(ctypes.c_void_p) for a in keep]
    arr = lambda k: (ctypes.c_void_p * 3)(*ptr[3 * k:3 * k + 3])
    lib().or_hkp_steps(n, arr(0), arr(1), arr(2), float(tau), int(nsteps), psi)
    return psi


def hermite_galerkin(x, W, U):
    """G[j, k] = sum_l W_l phi_j(x_l) U_l phi_k(x_l): the Galerkin matrix of
    the multiplication by U under the Gauss-Hermite rule."""
    x, W, U = _f(x), _f(W), _f(U)
    G = np.empty((x.size, x.size))
    lib().or_hermite_galerkin(x.size, x, W, U, G)
    return G


def hkmp_steps(psi, xs, Ws, Vs, Us, tau: float, f_mid):
    """len(f_mid) Magnus steps (section 4.4, eq. (mag2)) for the potential
    V_mu(x_mu) + f(t) U_mu(x_mu); Us[mu-1] may be None; f_mid[s] = f(t_s + tau/2)."""
    psi = _c(psi).copy()
    n = _dims(psi)
    f_mid = _f(f_mid)
    keep = [_f(a) for a in (*xs, *Ws, *Vs)]
    ukeep = [None if u is None else _f(u) for u in Us]
    for v in range(3):
        assert keep[v].size == keep[3 + v].size == keep[6 + v].size == n[v]
        assert ukeep[v] is None or ukeep[v].size == n[v]
    ptr = [a.ctypes.data_as(ctypes.c_void_p) for a in keep]
    arr = lambda k: (ctypes.c_void_p * 3)(*ptr[3 * k:3 * k + 3])
    uarr = (ctypes.c_void_p * 3)(*[None if u is None else u.ctypes.data_as(ctypes.c_void_p) for u in ukeep])
    lib().or_hkmp_steps(n, arr(0), arr(1), arr(2), uarr, float(tau), int(f_mid.size), f_mid, psi)
    return psi


# --- pipe flow (section 4.2) ---------------------------------------------

def pipe_radial(n: int, rmin: float, rmax: float, alpha: float, first: bool = True) -> np.ndarray:
    """alpha (D2 + diag(1/r) D1), Neumann at both ends, nodes r_min..r_max."""
    A = np.empty((n, n))
    lib().or_pipe_radial(n, float(rmin), float(rmax), float(alpha), int(first), A)
    return A


def pipe_axial(n: int, zmax: float, alpha: float, s=None) -> np.ndarray:
    """alpha D2 - diag(s) D1 on z_j = j z_max / n, j = 1..n (Dirichlet at 0, Neumann at z_max)."""
    A = np.empty((n, n))
    keep = None if s is None else _f(s)
    lib().or_pipe_axial(n, float(zmax), float(alpha), None if keep is None else keep.ctypes.data, A)
    return A


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --- metrics (relative L2 error, weighted norms) ---------------------------

def rel_l2(u, ref, weight=None) -> float:
    """||u - ref|| / ||ref|| over all points (optionally weighted)."""
    u = np.asarray(u, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    e = np.abs(u - ref) ** 2
    r = np.abs(ref) ** 2
    if weight is not None:
        e = e * weight
        r = r * weight
    return float(np.sqrt(e.sum() / r.sum()))


def weight3(W: np.ndarray) -> np.ndarray:
    """w_l = W_{l1} W_{l2} W_{l3} as a (m, m, m) array (section 3, eq. (quadrature))."""
    return W[:, None, None] * W[None, :, None] * W[None, None, :]
