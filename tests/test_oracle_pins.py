"""Pins for the FP64 CPU oracle, against facts fixed independently of it:
library routines in special cases (scipy expm, numpy hermgauss, scipy
Hermite polynomials), the Kronecker-sum identity, closed forms, invariants
and the values the paper prints.  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special

from paper_2103_01691_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kron_operator(mats, mu):
    """I_d x ... x L_mu x ... x I_1 for vectorisation with i_1 fastest
    (section 2, eq. (tensor-structure))."""
    d = len(mats)
    out = np.array([[1.0]])
    for v in range(d, 0, -1):  # leftmost factor is direction d
        f = mats[v - 1] if v == mu else np.eye(mats[v - 1].shape[1])
        out = np.kron(out, f)
    return out


# ---------------------------------------------------------------- operators

def test_fd_dirichlet_special_case(orc):
    A = orc.fd_dirichlet(3)  # h = 1/4
    assert np.array_equal(A, 16.0 * np.array([[-2, 1, 0], [1, -2, 1], [0, 1, -2]]))


def test_fd_periodic_special_case(orc):
    A = orc.fd_periodic(4, 4.0)  # h = 1
    expect = np.array([[-2, 1, 0, 1], [1, -2, 1, 0], [0, 1, -2, 1], [1, 0, 1, -2]], float)
    assert np.array_equal(A, expect)


@pytest.mark.parametrize("n", [4, 7, 16, 33])
@pytest.mark.parametrize("z", [1e-3, -2e-3, 1e-4j, 0.05j, 1e-3 + 2e-3j])
def test_expm_closed_form_vs_scipy(orc, n, z):
    ref = scipy.linalg.expm(z * orc.fd_dirichlet(n))
    got = orc.expm_dirichlet_fd(n, z)
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("scale", [0.1, 3.0, 40.0])
def test_expm_taylor_vs_scipy(orc, scale):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9))
    A *= scale / np.linalg.norm(A, 1)
    ref = scipy.linalg.expm(A)
    got = orc.expm_taylor(A, 1.0)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_expm_taylor_matches_closed_form(orc):
    n = 40
    A = orc.fd_dirichlet(n)
    for z in (1e-4j * 10, 2e-3):
        assert np.max(np.abs(orc.expm_taylor(A, z) - orc.expm_dirichlet_fd(n, z))) < 1e-12


# ------------------------------------------------------------ mode products

@pytest.mark.parametrize("dims", [(4, 5), (5, 4), (4, 5, 6), (6, 5, 4), (3, 4, 2, 5)])
def test_mode_product_is_kronecker_matvec(orc, dims):
    """vec(U x_mu L) = (I x .. x L x .. x I) vec(U), L rectangular (Def. 2.1)."""
    rng = np.random.default_rng(3)
    U = rng.standard_normal(dims[::-1]) + 1j * rng.standard_normal(dims[::-1])
    for mu in range(1, len(dims) + 1):
        m = dims[mu - 1] + 2
        L = rng.standard_normal((m, dims[mu - 1])) + 1j * rng.standard_normal((m, dims[mu - 1]))
        mats = [np.eye(n) for n in dims]
        mats[mu - 1] = L
        ref = kron_operator(mats, mu) @ U.reshape(-1)
        got = orc.mode_product(U, mu, L)
        out_dims = list(dims)
        out_dims[mu - 1] = m
        assert got.shape == tuple(out_dims[::-1])
        assert np.max(np.abs(got.reshape(-1) - ref)) < 1e-12


@pytest.mark.parametrize("dims", [(4, 5), (4, 5, 6), (8, 7, 6), (5, 5, 5)])
def test_tucker_equals_expm_of_kronecker_sum(orc, dims):
    """Section 2: exp(t M) u0 with M = A_d (+) ... (+) A_1 equals the Tucker
    operator with the 1D exponentials; A_mu arbitrary (non-symmetric)."""
    rng = np.random.default_rng(7)
    As = [rng.standard_normal((n, n)) for n in dims]
    t = 0.3
    M = sum(kron_operator(As, mu) for mu in range(1, len(dims) + 1))
    U = rng.standard_normal(dims[::-1]) + 1j * rng.standard_normal(dims[::-1])
    ref = scipy.linalg.expm(t * M) @ U.reshape(-1)
    Es = [orc.expm_taylor(A, t) for A in As]
    got = orc.tucker(U, Es)
    assert np.linalg.norm(got.reshape(-1) - ref) <= 1e-13 * np.linalg.norm(ref)


def test_mode_order_independence(orc):
    import itertools

    rng = np.random.default_rng(8)
    dims = (6, 7, 5)
    Es = [orc.expm_taylor(rng.standard_normal((n, n)), 0.2) for n in dims]
    U = rng.standard_normal(dims[::-1]) + 1j * rng.standard_normal(dims[::-1])
    base = orc.tucker(U, Es)
    for order in itertools.permutations([1, 2, 3]):
        got = orc.tucker(U, Es, order=order)
        assert np.linalg.norm(got - base) <= 1e-14 * np.linalg.norm(base) * 10


@pytest.mark.parametrize("z", [1e-3, 1e-4j])
def test_sine_modes_decay_in_closed_form(orc, z):
    """A product of discrete sine modes is an eigenvector of the Dirichlet FD
    Kronecker sum: one step multiplies it by exp(z sum lambda_k)."""
    n = 32
    h = 1.0 / (n + 1)
    j = np.arange(1, n + 1)
    ks = (1, 5, 17)
    vec = [np.sin(k * j * np.pi / (n + 1)) for k in ks]
    U = vec[2][:, None, None] * vec[1][None, :, None] * vec[0][None, None, :]
    lam = sum(-4.0 / h**2 * np.sin(k * np.pi / (2 * (n + 1))) ** 2 for k in ks)
    E = orc.expm_dirichlet_fd(n, z)
    got = orc.tucker(U.astype(complex), [E, E, E], nsteps=3)
    ref = np.exp(3 * z * lam) * U
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(U)


def test_unitary_flow_conserves_norm_and_one_shot(orc):
    """i Lap flow: E = exp(i tau A) is unitary, so the l2 norm is conserved
    (section 2, "conserved quantities ... are preserved"); and 10 steps of
    exp(i tau A) equal one step of exp(10 i tau A)."""
    n = 24
    U = inputs.complex_normal((n, n, n), seed=2)
    E1 = orc.expm_dirichlet_fd(n, 1e-4j)
    E10 = orc.expm_dirichlet_fd(n, 1e-3j)
    many = orc.tucker(U, [E1] * 3, nsteps=10)
    once = orc.tucker(U, [E10] * 3)
    assert abs(np.linalg.norm(many) / np.linalg.norm(U) - 1) < 1e-13
    assert np.linalg.norm(many - once) <= 1e-12 * np.linalg.norm(once)


def test_tucker3_entries_match_full(orc):
    rng = np.random.default_rng(9)
    dims = (7, 6, 5)
    Es = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for n in dims]
    U = rng.standard_normal(dims[::-1]) + 1j * rng.standard_normal(dims[::-1])
    full = orc.tucker(U, Es)
    idx = np.array([[0, 0, 0], [6, 5, 4], [3, 2, 1], [1, 4, 2]])
    got = orc.tucker3_entries(U, *Es, idx)
    ref = full[idx[:, 2], idx[:, 1], idx[:, 0]]
    assert np.max(np.abs(got - ref)) < 1e-12


# ------------------------------------------------- printed heat errors (4.1, 5.1)

def _golden_heat():
    rows = []
    with open(os.path.join(GOLDEN, "heat_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, err, use = line.split()
            if int(use):
                rows.append((int(n), float(err)))
    return rows


@pytest.mark.parametrize("n,printed", [r for r in _golden_heat() if r[0] <= 100])
def test_printed_heat_errors_3d(orc, n, printed):
    """3D periodic heat, FD2, T = 1 (section 4.1, Test 1): the relative error
    of the mu-mode solution equals the printed value to 3 digits."""
    L = 2 * np.pi
    x = np.arange(n) * (L / n)
    c = np.cos(x)
    U0 = c[:, None, None] + c[None, :, None] + c[None, None, :]
    E = orc.expm_taylor(orc.fd_periodic(n, L), 1.0)
    U = orc.tucker(U0.astype(complex), [E, E, E]).real
    err = np.linalg.norm(U - np.exp(-1.0) * U0) / np.linalg.norm(np.exp(-1.0) * U0)
    assert float(f"{err:.2e}") == printed


@pytest.mark.parametrize("n,printed", [r for r in _golden_heat() if r[0] > 100])
def test_printed_heat_errors_large_n(orc, n, printed):
    """Section 5.1 errors (n = 200..400).  u0 is a sum of 1D cosines, so the
    3D error equals the error of one direction's 1D problem."""
    L = 2 * np.pi
    x = np.arange(n) * (L / n)
    E = orc.expm_taylor(orc.fd_periodic(n, L), 1.0)
    u = (E @ np.cos(x)).real
    err = np.linalg.norm(u - np.exp(-1.0) * np.cos(x)) / np.linalg.norm(np.exp(-1.0) * np.cos(x))
    assert float(f"{err:.2e}") == printed


# ------------------------------------------------------------------ Hermite

@pytest.mark.parametrize("m", [1, 2, 5, 16, 64, 128, 150])
def test_gauss_hermite_vs_numpy(orc, m):
    x, w, W = orc.gauss_hermite(m)
    xr, wr = np.polynomial.hermite.hermgauss(m)
    assert np.max(np.abs(x - xr)) < 1e-13 * max(1.0, np.max(np.abs(xr)))
    big = wr > 1e-280
    assert np.max(np.abs(w[big] - wr[big]) / wr[big]) < 1e-11
    assert abs(w.sum() - math.sqrt(math.pi)) < 1e-14 * 10


def test_hermite_functions_vs_scipy(orc):
    x = np.linspace(-6, 6, 41)
    H = orc.hermite_functions(21, x)
    for k in range(21):
        norm = math.sqrt(2.0**k * math.factorial(k) * math.sqrt(math.pi))
        ref = scipy.special.eval_hermite(k, x) * np.exp(-x * x / 2) / norm
        assert np.max(np.abs(H[k] - ref)) < 1e-13


@pytest.mark.parametrize("m", [16, 64, 128, 192, 256])
def test_discrete_orthonormality(orc, m):
    """Section 3: with m = k Gauss-Hermite nodes the Hermite functions are
    orthonormal at the discrete level as well."""
    x, _, W = orc.gauss_hermite(m)
    H = orc.hermite_functions(m, x)
    G = (H * W) @ H.T
    assert np.max(np.abs(G - np.eye(m))) < 1e-12


def test_hermite_round_trip(orc):
    m = 12
    x, _, W = orc.gauss_hermite(m)
    v = inputs.complex_normal((m, m, m), seed=6)
    c = orc.hermite_forward(v, x, W)
    back = orc.hermite_backward(c, x, W)
    assert np.linalg.norm(back - v) <= 1e-12 * np.linalg.norm(v)


def test_harmonic_oscillator_exact_phase(orc):
    """phi_k1 phi_k2 phi_k3 is an eigenfunction with lambda = k1+k2+k3+3/2
    (section 3); after t it picks up exp(-i lambda t); after t = 2 pi it is
    -psi0."""
    m = 16
    x, _, W = orc.gauss_hermite(m)
    H = orc.hermite_functions(m, x)
    k1, k2, k3 = 3, 0, 7
    psi0 = (H[k3][:, None, None] * H[k2][None, :, None] * H[k1][None, None, :]).astype(complex)
    lam = k1 + k2 + k3 + 1.5
    tau, steps = 0.01, 25
    got = orc.ho_steps(psi0, x, W, tau, steps)
    assert np.max(np.abs(got - np.exp(-1j * lam * tau * steps) * psi0)) < 1e-12
    period = orc.ho_steps(psi0, x, W, 2 * np.pi / 8, 8)
    assert np.max(np.abs(period + psi0)) < 1e-12


# ---------------------------------------------------------------------- GPE

def test_gpe_beta_zero_is_linear_flow(orc):
    m = 10
    x, _, W = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(x, W)
    a = orc.gpe_steps(psi0, x, W, 0.0, 0.01, 5)
    b = orc.ho_steps(psi0, x, W, 0.01, 5)
    assert np.linalg.norm(a - b) < 1e-13


def test_gpe_norm_and_reversibility(orc):
    m = 12
    x, _, W = orc.gauss_hermite(m)
    w3 = orc.weight3(W)
    psi0 = inputs.gpe_psi0(x, W)
    fwd = orc.gpe_steps(psi0, x, W, 100.0, 1e-3, 20)
    n0 = np.sum(np.abs(psi0) ** 2 * w3)
    assert abs(np.sum(np.abs(fwd) ** 2 * w3) / n0 - 1) < 1e-12
    back = orc.gpe_steps(fwd, x, W, 100.0, -1e-3, 20)
    assert orc.rel_l2(back, psi0, w3) < 1e-11


def test_gpe_second_order_in_tau(orc):
    m = 10
    x, _, W = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(x, W)
    T = 0.08
    ref = orc.gpe_steps(psi0, x, W, 100.0, T / 64, 64)
    e1 = np.linalg.norm(orc.gpe_steps(psi0, x, W, 100.0, T / 4, 4) - ref)
    e2 = np.linalg.norm(orc.gpe_steps(psi0, x, W, 100.0, T / 8, 8) - ref)
    assert 3.0 < e1 / e2 < 5.0


def _gpe_energy(orc, psi, x, W, beta):
    """Discrete GPE energy <psi, H psi>_W + (beta/2) sum_l W_l |psi_l|^4, H the harmonic
    Hamiltonian (eigenvalues k1 + k2 + k3 + 3/2 on the Hermite coefficients, section 3), applied
    through the oracle's forward and backward transforms."""
    m = x.size
    k = np.arange(m, dtype=np.float64)
    lam = k[:, None, None] + k[None, :, None] + k[None, None, :] + 1.5
    w3 = orc.weight3(W)
    h_psi = orc.hermite_backward(lam * orc.hermite_forward(psi, x, W), x, W)
    return float(np.real(np.sum(w3 * np.conj(psi) * h_psi)) + 0.5 * beta * np.sum(w3 * np.abs(psi) ** 4))


def test_gpe_energy_pins_the_nonlinear_direction(orc):
    """The nodal system i psi' = H psi + beta |psi|^2 psi (section 4.5) is Hamiltonian in the
    W-weighted inner product and conserves the energy above with the same beta.  Strang splitting
    with exact subflows keeps it to O(tau^2) over a fixed time, so its drift falls fourfold per
    halving of tau.  A nonlinear subflow of the wrong direction, psi exp(+i tau beta |psi|^2),
    is the scheme of -beta: it conserves the energy of -beta instead and leaves that of +beta
    off by O(1) however small tau is."""
    m = 10
    x, _, W = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(x, W)
    T = 0.2
    for beta in (100.0, -100.0):
        e0 = _gpe_energy(orc, psi0, x, W, beta)
        e0_other = _gpe_energy(orc, psi0, x, W, -beta)
        drift, other = [], []
        for n in (8, 16, 32):
            p = orc.gpe_steps(psi0, x, W, beta, T / n, n)
            drift.append(abs(_gpe_energy(orc, p, x, W, beta) - e0) / abs(e0))
            other.append(abs(_gpe_energy(orc, p, x, W, -beta) - e0_other) / abs(e0_other))
        assert 3.5 < drift[0] / drift[1] < 4.5 and 3.5 < drift[1] / drift[2] < 4.5, drift
        assert drift[2] < 5e-4, drift
        assert min(other) > 0.05, other


def test_gpe_adjoint_finite_differences(orc):
    m = 8
    x, _, W = orc.gauss_hermite(m)
    w3 = orc.weight3(W)
    beta, tau, steps = 100.0, 1e-3, 6
    psi0 = inputs.gpe_psi0(x, W)
    target = inputs.gpe_target(x, W)

    def J(p):
        pT = orc.gpe_steps(p, x, W, beta, tau, steps)
        return float(np.sum(np.abs(pT - target) ** 2 * w3))

    pT = orc.gpe_steps(psi0, x, W, beta, tau, steps)
    gT = 2.0 * w3 * (pT - target)
    g0 = orc.gpe_adjoint(psi0, gT, x, W, beta, tau, steps)
    delta = inputs.direction(psi0.shape)
    delta /= np.linalg.norm(delta)
    eps = 1e-6
    fd = (J(psi0 + eps * delta) - J(psi0 - eps * delta)) / (2 * eps)
    an = float(np.real(np.vdot(g0, delta)))
    assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12) + 1e-12


# ---------------------------------------------------------------------- HKP

def _cos_matrix_closed_form(nmax: int, q: float) -> np.ndarray:
    """<j| cos(q x) |k> in the Hermite functions, from the matrix elements of
    the displacement operator D(a), a = i q / sqrt(2), between number
    states: for j >= k, sqrt(k!/j!) a^(j-k) e^{-|a|^2/2} L_k^(j-k)(|a|^2);
    the cosine keeps the even differences j - k = 2p, with a^(2p) =
    (-1)^p (q^2/2)^p."""
    r = q * q / 2.0
    C = np.zeros((nmax, nmax))
    for j in range(nmax):
        for k in range(j + 1):
            if (j - k) % 2:
                continue
            p = (j - k) // 2
            lg = 0.5 * (math.lgamma(k + 1) - math.lgamma(j + 1))
            C[j, k] = C[k, j] = ((-1) ** p * math.exp(lg + p * math.log(r) - r / 2)
                                 * scipy.special.eval_genlaguerre(k, j - k, r))
    return C


def test_hkp_hamiltonian_closed_form(orc):
    """Section 4.3 Hamiltonian of direction 1 (V_1 = cos(2 pi x)) in the
    Hermite basis against closed forms for the leading block: the kinetic
    part -1/2 d^2/dx^2 = p^2/2 from the ladder operators (diagonal
    (2k+1)/4, second off-diagonals -sqrt((k+1)(k+2))/4) plus the cosine's
    matrix elements from the displacement operator."""
    m, nmax = 80, 14
    x, _, W = orc.gauss_hermite(m)
    H = orc.hkp_hamiltonian(x, W, np.cos(2 * np.pi * x))[:nmax, :nmax]
    k = np.arange(nmax, dtype=float)
    T = np.diag((2 * k + 1) / 4)
    off = -np.sqrt((k[:-2] + 1) * (k[:-2] + 2)) / 4
    T += np.diag(off, 2) + np.diag(off, -2)
    ref = T + _cos_matrix_closed_form(nmax, 2 * np.pi)
    assert np.max(np.abs(H - ref)) < 1e-11
    assert np.max(np.abs(H - H.T)) < 1e-13


def test_hkp_harmonic_potential_is_ho(orc):
    """With V_mu = x^2/2 in every direction the HKP step is the harmonic
    oscillator step (the Hamiltonian is diagonal, section 3)."""
    m = 10
    x, _, W = orc.gauss_hermite(m)
    psi0 = inputs.harmonic_psi0(x, W, seed=1)
    V = 0.5 * x * x
    got = orc.hkp_steps(psi0, [x] * 3, [W] * 3, [V] * 3, 0.3, 2)
    ref = orc.ho_steps(psi0, x, W, 0.3, 2)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_hkp_eigenstate_phase(orc):
    """An eigenvector v of H_1 (numpy eigh) times phi_2(x_2) phi_1(x_3) is an
    eigenstate with energy lambda + 5/2 + 3/2; one HKP step of any length
    multiplies it by exp(-i E tau) (the method is exact in time)."""
    n = (24, 20, 16)
    xs, Ws = [], []
    for v in n:
        x, _, W = orc.gauss_hermite(v)
        xs.append(x)
        Ws.append(W)
    Vs = inputs.hkp_potentials(*xs)
    lam, vec = np.linalg.eigh(orc.hkp_hamiltonian(xs[0], Ws[0], Vs[0]))
    f1 = orc.hermite_functions(n[0], xs[0]).T @ vec[:, 3]
    f2 = orc.hermite_functions(n[1], xs[1])[2]
    f3 = orc.hermite_functions(n[2], xs[2])[1]
    psi0 = (f3[:, None, None] * f2[None, :, None] * f1[None, None, :]).astype(complex)
    E, tau = lam[3] + 2.5 + 1.5, 0.8
    got = orc.hkp_steps(psi0, xs, Ws, Vs, tau, 1)
    assert np.max(np.abs(got - np.exp(-1j * E * tau) * psi0)) < 1e-11 * np.max(np.abs(psi0))


def test_hkp_norm_and_group_property(orc):
    """The paper's initial datum: its discrete weighted norm is 2^{-5/2}
    (closed form of the Gaussian integral), the flow conserves it, and one
    step to T = 1 equals two steps of 1/2."""
    n = (40, 36, 32)
    xs, Ws = [], []
    for v in n:
        x, _, W = orc.gauss_hermite(v)
        xs.append(x)
        Ws.append(W)
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    psi0 = inputs.hkp_psi0(*xs)
    nrm0 = np.sum(np.abs(psi0) ** 2 * w3)
    assert abs(nrm0 - 2 ** -2.5) < 1e-10
    Vs = inputs.hkp_potentials(*xs)
    one = orc.hkp_steps(psi0, xs, Ws, Vs, 1.0, 1)
    two = orc.hkp_steps(psi0, xs, Ws, Vs, 0.5, 2)
    assert abs(np.sum(np.abs(one) ** 2 * w3) / nrm0 - 1) < 1e-12
    assert np.linalg.norm(one - two) <= 1e-11 * np.linalg.norm(one)


# --------------------------------------------------------------------- HKMP

def test_hermite_galerkin_closed_form(orc):
    """Galerkin matrices of x and x^2 in the Hermite functions: x is exactly
    tridiagonal with sqrt((k+1)/2) (ladder operators; the quadrature is exact
    for every entry), x^2 has (2k+1)/2 on the diagonal and
    sqrt((k+1)(k+2))/2 two off (exact away from the last row)."""
    m = 12
    x, _, W = orc.gauss_hermite(m)
    k = np.arange(m, dtype=float)
    X = orc.hermite_galerkin(x, W, x)
    ref = np.diag(np.sqrt((k[:-1] + 1) / 2), 1)
    ref = ref + ref.T
    assert np.max(np.abs(X - ref)) < 1e-13
    X2 = orc.hermite_galerkin(x, W, x * x)[: m - 1, : m - 1]
    k = k[: m - 1]
    ref2 = np.diag((2 * k + 1) / 2) + np.diag(np.sqrt((k[:-2] + 1) * (k[:-2] + 2)) / 2, 2)
    ref2 = ref2 + np.triu(ref2, 1).T
    assert np.max(np.abs(X2 - ref2)) < 1e-13


def _hkmp_grid(orc, n):
    xs, Ws = [], []
    for v in n:
        x, _, W = orc.gauss_hermite(v)
        xs.append(x)
        Ws.append(W)
    return xs, Ws


def test_hkmp_reduces_to_hkp(orc):
    """With f = 0 the Magnus steps are HKP steps of V; with a constant f = c
    the midpoint rule is exact and equals HKP with V + c U."""
    n = (10, 12, 14)
    xs, Ws = _hkmp_grid(orc, n)
    Vs, Us = inputs.hkmp_potentials(*xs)
    psi0 = inputs.hkp_psi0(*xs)
    tau, steps = 0.3, 3
    got0 = orc.hkmp_steps(psi0, xs, Ws, Vs, Us, tau, np.zeros(steps))
    ref0 = orc.hkp_steps(psi0, xs, Ws, Vs, tau, steps)
    assert np.max(np.abs(got0 - ref0)) < 1e-12
    c = 0.7
    gotc = orc.hkmp_steps(psi0, xs, Ws, Vs, Us, tau, np.full(steps, c))
    Vc = (Vs[0], Vs[1], Vs[2] + c * Us[2])
    refc = orc.hkp_steps(psi0, xs, Ws, Vc, tau * steps, 1)
    assert np.max(np.abs(gotc - refc)) < 1e-12


def test_hkmp_second_order_and_norm(orc):
    """f = sin^2 t: the error at T = 1 against a run with tau = 1/128 falls by
    ~4 when tau halves (order two, eq. (mag2)); the weighted norm is
    conserved (unitary exponentials)."""
    n = (12, 10, 14)
    xs, Ws = _hkmp_grid(orc, n)
    Vs, Us = inputs.hkmp_potentials(*xs)
    psi0 = inputs.hkp_psi0(*xs)
    run = lambda k: orc.hkmp_steps(psi0, xs, Ws, Vs, Us, 1.0 / k, inputs.hkmp_f_mid(1.0 / k, k))
    ref = run(128)
    e8, e16 = np.linalg.norm(run(8) - ref), np.linalg.norm(run(16) - ref)
    assert 3.5 < e8 / e16 < 4.5
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    nrm = lambda p: np.sum(np.abs(p) ** 2 * w3)
    assert abs(nrm(ref) / nrm(psi0) - 1) < 1e-12


# ---------------------------------------------------------------- pipe flow

def test_pipe_second_differences_closed_form(orc):
    """Without first-derivative terms the two operators have closed-form
    eigenvectors: Neumann-Neumann (reflection) D2 on n nodes, cos(k pi j/(n-1))
    with -4 sin^2(k pi/(2(n-1)))/h^2; Dirichlet-Neumann D2 on z_j = j h,
    sin((2k-1) pi j/(2n)) with -4 sin^2((2k-1) pi/(4n))/h^2."""
    n, rmin, rmax, zmax = 17, 0.1, 5.0, 8.0
    A = orc.pipe_radial(n, rmin, rmax, 1.0, first=False)
    h = (rmax - rmin) / (n - 1)
    j = np.arange(n)
    for k in (0, 1, 5, 16):
        v = np.cos(k * np.pi * j / (n - 1))
        lam = -4.0 * np.sin(k * np.pi / (2 * (n - 1))) ** 2 / h ** 2
        assert np.max(np.abs(A @ v - lam * v)) < 1e-10
    B = orc.pipe_axial(n, zmax, 1.0)
    h = zmax / n
    j = np.arange(1, n + 1)
    for k in (1, 2, 9, n):
        th = (2 * k - 1) * np.pi / (2 * n)
        v = np.sin(th * j)
        lam = -4.0 * np.sin(th / 2) ** 2 / h ** 2
        assert np.max(np.abs(B @ v - lam * v)) < 1e-10


def test_pipe_first_derivative_terms_on_quadratics(orc):
    """Centred differences are exact on quadratics at interior nodes:
    alpha (c_rr + c_r / r) of r^2 is 4 alpha; alpha c_zz - s c_z of z^2 is
    2 alpha - 2 s z.  Constants are steady under the radial operator (both
    ends Neumann), so exp(t A_r) 1 = 1."""
    from paper_2103_01691_b300 import inputs as inp

    n, rmin, rmax, zmax, alpha = 23, 0.1, 5.0, 8.0, 1.0 / 90.0
    r = rmin + (rmax - rmin) / (n - 1) * np.arange(n)
    A = orc.pipe_radial(n, rmin, rmax, alpha)
    assert np.max(np.abs((A @ r ** 2)[1:-1] - 4 * alpha)) < 1e-11
    assert np.max(np.abs(A @ np.ones(n))) < 1e-12
    E = orc.expm_taylor(A, 4.0)
    assert np.max(np.abs(E @ np.ones(n) - 1)) < 1e-12
    z = zmax / n * np.arange(1, n + 1)
    s = inp.pipe_velocity(z)
    B = orc.pipe_axial(n, zmax, alpha, s)
    assert np.max(np.abs((B @ z ** 2)[1:-1] - (2 * alpha - 2 * s * z)[1:-1])) < 1e-11
