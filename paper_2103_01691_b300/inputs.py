"""Seeded synthetic inputs for the five workloads (shared by tests, the
oracle checks and the benchmark).

This module holds random draws and their shaping only; none of the
method's arithmetic lives here.  Quantities the method computes (grid
nodes, quadrature weights) are passed in by the caller, so each side uses
its own.  Every tensor follows the paper's layout (section 4.1: i_1
fastest): a numpy array of shape (n_d, ..., n_1).

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64),
drawn in float64 on the host.
"""
from __future__ import annotations

import numpy as np


def heat_u0(n: int = 32, seed: int = 0) -> np.ndarray:
    """Real FP64 heat initial datum, i.i.d. uniform on [-1, 1]."""
    rng = np.random.default_rng(seed)
    return 2.0 * rng.random((n, n, n)) - 1.0


def complex_normal(shape, seed: int) -> np.ndarray:
    """Complex normal tensor: real and imaginary parts i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def free_schrodinger_u0(n: int = 256, seed: int = 2) -> np.ndarray:
    """Random complex normal datum for the free Schroedinger precision sweep."""
    return complex_normal((n, n, n), seed)


def gaussian_at_nodes(x: np.ndarray) -> np.ndarray:
    """pi^{-3/4} exp(-|x|^2 / 2) on the tensor grid of 1D nodes x (m^3 values)."""
    g = np.exp(-0.5 * x * x)
    return (np.pi ** -0.75) * g[:, None, None] * g[None, :, None] * g[None, None, :]


def _normalise(psi: np.ndarray, W: np.ndarray) -> np.ndarray:
    w3 = W[:, None, None] * W[None, :, None] * W[None, None, :]
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2 * w3))


def harmonic_psi0(x: np.ndarray, W: np.ndarray, seed: int = 1, sigma: float = 0.1) -> np.ndarray:
    """Normalised Gaussian times (1 + sigma (xi_r + i xi_i)), xi i.i.d. N(0,1)
    at the nodes, renormalised in the discrete weighted norm."""
    m = x.size
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((m, m, m)) + 1j * rng.standard_normal((m, m, m))
    return _normalise(gaussian_at_nodes(x) * (1.0 + sigma * xi), W)


def gpe_psi0(x: np.ndarray, W: np.ndarray, seed: int = 4, noise: float = 0.05) -> np.ndarray:
    """Normalised Gaussian ground-state guess with a random phase
    exp(i noise xi), xi i.i.d. N(0,1), renormalised."""
    m = x.size
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((m, m, m))
    return _normalise(gaussian_at_nodes(x) * np.exp(1j * noise * xi), W)


def gpe_psi0_dims(xs, Ws, seed: int = 4, noise: float = 0.05) -> np.ndarray:
    """gpe_psi0 on a grid with its own nodes xs[v] and weights Ws[v] per
    direction v = 0, 1, 2 (shape (n3, n2, n1)); equal to gpe_psi0 when all
    three are the same."""
    g = [np.exp(-0.5 * np.asarray(x) * np.asarray(x)) for x in xs]
    gauss = (np.pi ** -0.75) * g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]
    rng = np.random.default_rng(seed)
    psi = gauss * np.exp(1j * noise * rng.standard_normal(gauss.shape))
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2 * w3))


def gpe_target(x: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Noise-free normalised Gaussian, the target state of the adjoint loss."""
    return _normalise(gaussian_at_nodes(x).astype(np.complex128), W)


def batched_dims(count: int = 64, seed: int = 3) -> np.ndarray:
    """Per-direction sizes of the uneven batch: uniform on {48, 64, ..., 160}."""
    rng = np.random.default_rng(seed)
    return 48 + 16 * rng.integers(0, 8, size=(count, 3))


def batched_u0(dims: np.ndarray, seed: int = 3) -> list:
    """One complex normal datum per problem, drawn after the sizes."""
    rng = np.random.default_rng(seed)
    rng.integers(0, 8, size=(dims.shape[0], 3))  # the size draw comes first
    out = []
    for n1, n2, n3 in dims:
        shape = (int(n3), int(n2), int(n1))
        out.append(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return out


def direction(shape, seed: int = 5) -> np.ndarray:
    """Random complex direction for finite-difference checks."""
    return complex_normal(shape, seed)


def hkp_potentials(x1: np.ndarray, x2: np.ndarray, x3: np.ndarray):
    """Values at the nodes of the Kronecker potential of section 4.3:
    V_1 = cos(2 pi x_1), V_2 = x_2^2/2, V_3 = x_3^2/2."""
    return np.cos(2.0 * np.pi * x1), 0.5 * x2 * x2, 0.5 * x3 * x3


def hkp_psi0(x1: np.ndarray, x2: np.ndarray, x3: np.ndarray) -> np.ndarray:
    """Initial datum of section 4.3 on the tensor grid of the nodes,
    2^{-5/2} pi^{-3/4} (x_1 + i x_2) exp(-|x|^2/4), shape (n_3, n_2, n_1)."""
    g1, g2, g3 = np.exp(-0.25 * x1 * x1), np.exp(-0.25 * x2 * x2), np.exp(-0.25 * x3 * x3)
    lin = x1[None, None, :] + 1j * x2[None, :, None]
    return 2.0 ** -2.5 * np.pi ** -0.75 * lin * g3[:, None, None] * g2[None, :, None] * g1[None, None, :]


def hkmp_potentials(x1: np.ndarray, x2: np.ndarray, x3: np.ndarray):
    """Potential of section 4.4 split as V_mu + f(t) U_mu at the nodes: the
    Hamiltonian (i/2)(Lap - |x|^2 - 2 x_3 sin^2 t) of the equation
    psi_t = H psi is i psi_t = -1/2 Lap psi + (|x|^2/2 + x_3 sin^2 t) psi,
    so V_mu = x_mu^2/2, U_3 = x_3, U_1 = U_2 = None, f(t) = sin^2 t."""
    return (0.5 * x1 * x1, 0.5 * x2 * x2, 0.5 * x3 * x3), (None, None, np.array(x3, dtype=np.float64))


def hkmp_f_mid(tau: float, nsteps: int, t0: float = 0.0) -> np.ndarray:
    """f(t) = sin^2 t at the step midpoints t0 + (s + 1/2) tau (eq. (mag2))."""
    return np.sin(t0 + (np.arange(nsteps) + 0.5) * tau) ** 2


# pipe flow (section 4.2): parameters and data as the paper states them
PIPE = {"rmin": 0.1, "rmax": 5.0, "zmax": 8.0, "alpha": 1.0 / 90.0, "z0": 1.5, "T": 4.0}
PIPE["r0"] = 0.5 * (PIPE["rmin"] + PIPE["rmax"])


def pipe_velocity(z: np.ndarray) -> np.ndarray:
    """Advection velocity s(z) = 2 + tanh(4 (z - 5/2)) - tanh(4 (z - 5))."""
    return 2.0 + np.tanh(4.0 * (z - 2.5)) - np.tanh(4.0 * (z - 5.0))


def pipe_c0(r: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Initial concentration exp(-8 (r - r0)^2 - 8 (z - z0)^2) on the tensor
    grid, shape (n_z, n_r) (r is direction 1, fastest)."""
    return np.exp(-8.0 * (z[:, None] - PIPE["z0"]) ** 2 - 8.0 * (r[None, :] - PIPE["r0"]) ** 2)
