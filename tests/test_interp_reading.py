"""The HKMP exponentials of tensor-core plans come from Chebyshev interpolation in f (not from the
paper, whose Magnus steps take one exponential each): E(f) = exp(-i tau (H0 + f G)) at K
Chebyshev points of [f_lo, f_hi], combined by the barycentric formula, with K the fewest (4..12)
whose bound 2 (tau ||G||_1 (f_hi - f_lo) / 4)^K / K! is below 1e-14.  Here, in FP64 on the CPU,
against scipy's expm at every f: the Hamiltonian and the Galerkin matrix of x_3 are the oracle's
(section 4.4), the interpolation is written out.  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg

from paper_2103_01691_b300 import inputs


def fewest_nodes(tau, gnorm, width, kmax=12):
    x = abs(tau) * gnorm * width / 4.0
    for k in range(4, kmax + 1):
        if 2.0 * x ** k / math.factorial(k) <= 1e-14:
            return k
    return kmax + 1


def cheb_interp(fs, nodes_f, mats):
    """Barycentric interpolation (Chebyshev points of the first kind) of mats[j] = E(nodes_f[j])."""
    K = len(nodes_f)
    bw = np.array([(-1.0) ** j * math.sin((2 * j + 1) * math.pi / (2 * K)) for j in range(K)])
    out = []
    for f in fs:
        d = f - nodes_f
        if np.any(d == 0):
            out.append(mats[int(np.argmin(np.abs(d)))])
            continue
        w = bw / d
        out.append(np.tensordot(w / w.sum(), mats, axes=1))
    return out


@pytest.mark.parametrize("m,tau,lo,hi", [(24, 0.02, 0.0, 1.0), (31, 0.05, 0.1, 0.6), (40, 0.025, 0.0, 0.3)])
def test_chebyshev_interpolation_of_the_magnus_exponential(orc, m, tau, lo, hi):
    x, _, W = orc.gauss_hermite(m)
    V, U = inputs.hkmp_potentials(x, x, x)
    H0 = orc.hkp_hamiltonian(x, W, V[2])
    G = orc.hermite_galerkin(x, W, U[2])
    gnorm = np.max(np.sum(np.abs(G), axis=0))
    K = fewest_nodes(tau, gnorm, hi - lo)
    assert 4 <= K <= 12
    th = (2 * np.arange(K) + 1) * np.pi / (2 * K)
    nodes_f = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(th)
    mats = np.array([scipy.linalg.expm(-1j * tau * (H0 + f * G)) for f in nodes_f])
    fs = np.linspace(lo, hi, 41)
    approx = cheb_interp(fs, nodes_f, mats)
    err = max(np.max(np.abs(a - scipy.linalg.expm(-1j * tau * (H0 + f * G)))) for a, f in zip(approx, fs))
    bound = 2.0 * (abs(tau) * gnorm * (hi - lo) / 4.0) ** K / math.factorial(K)
    # the interpolation error bound, plus the rounding of the FP64 combination (unitary: entries <= 1)
    assert err <= bound + 1e-13, (K, err, bound)
    # one node fewer than the rule asks for is measurably worse whenever the bound is tight
    if K > 4:
        nodes2 = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2 * np.arange(K - 1) + 1) * np.pi / (2 * (K - 1)))
        mats2 = np.array([scipy.linalg.expm(-1j * tau * (H0 + f * G)) for f in nodes2])
        err2 = max(np.max(np.abs(a - scipy.linalg.expm(-1j * tau * (H0 + f * G))))
                   for a, f in zip(cheb_interp(fs, nodes2, mats2), fs))
        assert err2 > err


def test_declared_range_for_sin_squared_needs_at_most_twelve_nodes(orc):
    """f = sin^2 t lies in [0, 1]: at the paper's tau = 0.02 the range needs at most 12 nodes up to
    n = 511, since ||G||_1 of x_3 under the n-point rule stays below sqrt(2 n) + 1 (the rule is
    exact for phi_j x phi_k, so G is the tridiagonal matrix of x in the Hermite basis)."""
    for n in (31, 127):
        x, _, W = orc.gauss_hermite(n)
        G = orc.hermite_galerkin(x, W, np.array(x))
        assert np.max(np.sum(np.abs(G), axis=0)) <= math.sqrt(2 * n) + 1.0
    for n in (127, 255, 511):
        assert fewest_nodes(0.02, math.sqrt(2 * n) + 1.0, 1.0) <= 12
