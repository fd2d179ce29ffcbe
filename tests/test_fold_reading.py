"""Pins for the even/odd folding the tensor-core path runs on (a change of basis, not from the
paper): the propagators it folds are centrosymmetric, their folded form is block-diagonal, and
steps taken in the folded basis (the GPE's nonlinear phase applied between unfold and refold)
give the oracle's results (FP64 numpy around the oracle); and the phase pass's short series for
sine and cosine holds FP32 accuracy.  CPU only."""
import math

import numpy as np
import pytest

from paper_2103_01691_b300 import inputs


def fold_matrix(n: int) -> np.ndarray:
    """F: row k < n/2 takes x_k + x_(n-1-k), row c + k takes x_k - x_(n-1-k) (c = ceil(n/2)),
    row n/2 of an odd n takes the middle entry."""
    c, h = (n + 1) // 2, n // 2
    F = np.zeros((n, n))
    for k in range(h):
        F[k, k] = F[k, n - 1 - k] = 1.0
        F[c + k, k], F[c + k, n - 1 - k] = 1.0, -1.0
    if n % 2:
        F[h, h] = 1.0
    return F


def reverse(E: np.ndarray) -> np.ndarray:
    return E[::-1, ::-1]


def hermite_propagator(orc, m: int, s: float) -> np.ndarray:
    """Values-space harmonic-oscillator flow over time s in one direction: backward transform,
    exp(-i s (k + 1/2)) per coefficient, forward transform with the weights (section 3)."""
    x, _, W = orc.gauss_hermite(m)
    H = orc.hermite_functions(m, x)  # H[k, l] = phi_k(x_l)
    ph = np.exp(-1j * s * (np.arange(m) + 0.5))
    return H.T @ np.diag(ph) @ H @ np.diag(W)


def apply_all(U: np.ndarray, mats) -> np.ndarray:
    """U (shape (n3, n2, n1)) times mats[v] in direction v + 1, v = 0, 1, 2."""
    U = np.einsum("ij,abj->abi", mats[0], U)
    U = np.einsum("ij,ajb->aib", mats[1], U)
    return np.einsum("ij,jab->iab", mats[2], U)


@pytest.mark.parametrize("n", [8, 9])
def test_dirichlet_propagator_is_centrosymmetric_and_folds_block_diagonal(orc, n):
    E = orc.expm_dirichlet_fd(n, 3e-3j)
    assert np.max(np.abs(E - reverse(E))) <= 1e-14 * np.max(np.abs(E))
    F = fold_matrix(n)
    D = F @ E @ np.linalg.inv(F)
    c = (n + 1) // 2
    assert np.max(np.abs(D[:c, c:])) <= 1e-14 and np.max(np.abs(D[c:, :c])) <= 1e-14
    # a matrix that is not centrosymmetric (one off-diagonal entry doubled) does not fold
    A = orc.fd_dirichlet(n)
    A[0, 1] *= 2.0
    Dn = F @ A @ np.linalg.inv(F)
    assert np.max(np.abs(Dn[:c, c:])) > 1e-3 * np.max(np.abs(A))


@pytest.mark.parametrize("m", [8, 9])
def test_hermite_propagator_is_centrosymmetric(orc, m):
    """Symmetric nodes and weights and phi_k(-x) = (-1)^k phi_k(x) make the values-space flow of
    an even potential centrosymmetric."""
    P = hermite_propagator(orc, m, 0.05)
    assert np.max(np.abs(P - reverse(P))) <= 1e-13 * np.max(np.abs(P))


def test_folded_tucker_step_equals_oracle(orc):
    """fold(u x E) = D x fold(u) with D's off-diagonal blocks zeroed, on odd, even and mixed
    directions, against the oracle's Tucker step."""
    dims = (8, 9, 7)  # n1, n2, n3
    Es = [orc.expm_dirichlet_fd(n, z) for n, z in zip(dims, (2e-3j, 5e-3j, 1e-3j))]
    U = inputs.complex_normal(dims[::-1], seed=5)
    ref = orc.tucker(U, Es)
    Fs = [fold_matrix(n) for n in dims]
    Ds = []
    for F, E, n in zip(Fs, Es, dims):
        D = F @ E @ np.linalg.inv(F)
        c = (n + 1) // 2
        D[:c, c:] = 0.0
        D[c:, :c] = 0.0
        Ds.append(D)
    got = apply_all(apply_all(apply_all(U, Fs), Ds), [np.linalg.inv(F) for F in Fs])
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("m", [8, 9])
def test_folded_gpe_steps_equal_oracle(orc, m):
    """The folded GPE scheme: fold once, half-step flow D_(tau/2), then per step unfold, nonlinear
    phase psi exp(-i tau beta |psi|^2) at each node, refold and the full-step flow D_tau (the last
    one D_(tau/2)), unfold once; equal to the oracle's Strang steps (section 4.5)."""
    beta, tau, nsteps = 100.0, 1e-3, 4
    x, _, W = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(x, W, seed=4)
    ref = orc.gpe_steps(psi0, x, W, beta, tau, nsteps)
    F = fold_matrix(m)
    Fi = np.linalg.inv(F)
    c = (m + 1) // 2

    def folded(P):
        D = F @ P @ Fi
        D[:c, c:] = 0.0
        D[c:, :c] = 0.0
        return [D] * 3

    Dh, Df = folded(hermite_propagator(orc, m, 0.5 * tau)), folded(hermite_propagator(orc, m, tau))
    u = apply_all(psi0, [F] * 3)
    for k in range(nsteps):
        u = apply_all(u, Dh if k == 0 else Df)
        v = apply_all(u, [Fi] * 3)
        v = v * np.exp(-1j * tau * beta * np.abs(v) ** 2)
        u = apply_all(v, [F] * 3)
    u = apply_all(u, Dh)
    got = apply_all(u, [Fi] * 3)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the phase's sign matters here as in the oracle: the opposite sign is far off
    v = apply_all(psi0, [hermite_propagator(orc, m, 0.5 * tau)] * 3)
    v = v * np.exp(+1j * tau * beta * np.abs(v) ** 2)
    wrong = apply_all(v, [hermite_propagator(orc, m, 0.5 * tau)] * 3)
    one = orc.gpe_steps(psi0, x, W, beta, tau, 1)
    assert np.max(np.abs(wrong - one)) > 1e-6 * np.max(np.abs(one))


def test_phase_series_error_bound():
    """The folded GPE's phase pass takes sin a and cos a for |a| <= 1/4 from their Taylor series
    (through a^9 and a^8, Horner form, FP32).  Evaluated the same way in FP32 here, both stay
    within 2 units in the last place of FP32 of the FP64 library values over the whole range:
    the truncation (below 3e-13) is far under FP32 rounding."""
    a = np.linspace(-0.25, 0.25, 200001, dtype=np.float32)
    a2 = a * a
    f = np.float32
    sn = a * (f(1) + a2 * (f(-1 / 6) + a2 * (f(1 / 120) + a2 * (f(-1 / 5040) + a2 * f(1 / 362880)))))
    cs = f(1) + a2 * (f(-0.5) + a2 * (f(1 / 24) + a2 * (f(-1 / 720) + a2 * f(1 / 40320))))
    ad = a.astype(np.float64)
    ulp_s = np.spacing(np.abs(np.sin(ad)).astype(np.float32)).astype(np.float64)
    ulp_c = np.spacing(np.cos(ad).astype(np.float32)).astype(np.float64)
    nz = ad != 0
    assert np.all(np.abs(sn[nz] - np.sin(ad[nz])) <= 2 * ulp_s[nz])
    assert np.all(np.abs(cs - np.cos(ad)) <= 2 * ulp_c)
    # the first omitted terms, at the end of the range
    assert 0.25 ** 11 / math.factorial(11) < 3e-13 and 0.25 ** 10 / math.factorial(10) < 3e-13
