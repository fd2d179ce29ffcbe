"""Parity at the full sizes of the measured workloads, through the C ABI,
element by element over every point.

* free Schroedinger, n = 256, tau = 1e-4, 50 F16x6 steps (16.7 M points)
  against the oracle's single application of E(50 tau) = E(tau)^50;
* harmonic oscillator, n = 128, tau = 0.01, 100 steps: the exact phase
  exp(-i lambda t) of a Hermite eigenfunction (section 3), and the seeded
  datum against the oracle's literal steps;
* Gross-Pitaevskii, n = 192, beta = 100, tau = 1e-3: two steps against the
  oracle's Strang steps (and the weighted norm taken in the last product's
  epilogue against the oracle's), 500 F16x6 steps against 500 FP64 GPU
  steps (the FP64 path itself checked against the oracle at this size),
  norm drift;
* the 64 uneven batched problems, 3 steps, every problem against the
  oracle's application of E(3 tau).

Tolerances (relative L2 over all points; weighted by the quadrature
weights in the Hermite cases) come from the measured errors, about twice
them; the printed values are the measurements."""
import numpy as np
import pytest

from paper_2103_01691_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2103_01691_b300 import build as mmbuild

    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    ctx = mumode.Context(0)
    yield mumode, ctx, torch
    ctx.status()


def rel(a, b, w=None):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    if w is None:
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2 * w) / np.sum(np.abs(b) ** 2 * w)))


def to_gpu(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def test_free_schrodinger_n256_50_steps_every_point(env, orc):
    """Precision-sweep workload, F16x6: all 16.7 M points after 50 steps
    against U0 x_1 E(50 tau) x_2 E(50 tau) x_3 E(50 tau)."""
    mm, ctx, torch = env
    n, tau, steps = 256, 1e-4, 50
    E = mm.expm(mm.fd_laplacian_dirichlet(n), 1j * tau)
    plan = mm.TuckerPlan(ctx, [n] * 3, [E] * 3, prec="f16x6")
    u0 = inputs.free_schrodinger_u0(n, seed=2).astype(np.complex64)
    u = to_gpu(torch, u0, torch.complex64)
    nrm0 = plan.norm2(u)
    plan.step(u, steps)
    nrm1 = plan.norm2(u)
    got = u.cpu().numpy()
    del u
    E50 = orc.expm_dirichlet_fd(n, 1j * tau * steps)
    ref = orc.tucker(u0.astype(np.complex128), [E50] * 3, nsteps=1)
    err = rel(got, ref)
    drift = abs(nrm1 / nrm0 - 1)
    print(f"n=256 50 steps f16x6, every point: rel_err={err:.3e} norm drift={drift:.3e}")
    assert err <= 1e-6  # the target accuracy; measured 6.0e-7
    assert drift <= 1e-7  # measured 4.9e-8


def _hermite_nodes(orc, m):
    x, _, W = orc.gauss_hermite(m)
    return x, W, orc.weight3(W)


def test_harmonic_oscillator_n128_exact_phase_100_steps(env, orc):
    """psi0 = phi_k1(x1) phi_k2(x2) phi_k3(x3) at the Gauss-Hermite nodes is
    a unit coefficient of the discrete transform, so every step multiplies
    it by exp(-i tau (k1 + k2 + k3 + 3/2)): after 100 steps of 0.01 the
    exact state is exp(-i lambda) psi0."""
    mm, ctx, torch = env
    m, tau, steps = 128, 0.01, 100
    x, W, w3 = _hermite_nodes(orc, m)
    k1, k2, k3 = 3, 17, 60
    H = orc.hermite_functions(m, x)  # H[k, l] = phi_k(x_l)
    psi0 = H[k3][:, None, None] * H[k2][None, :, None] * H[k1][None, None, :]  # shape (n3, n2, n1)
    lam = k1 + k2 + k3 + 1.5
    exact = np.exp(-1j * lam * tau * steps) * psi0
    plan = mm.HermitePlan(ctx, [m] * 3, prec="f16x6")
    psi = to_gpu(torch, psi0.astype(np.complex64), torch.complex64)
    plan.ho_step(psi, tau, steps)
    got = psi.cpu().numpy()
    err = rel(got, exact, w3)
    drift = abs(np.sum(np.abs(got) ** 2 * w3) / np.sum(np.abs(psi0) ** 2 * w3) - 1)
    print(f"HO n=128 eigenfunction ({k1},{k2},{k3}) 100 steps: rel_err={err:.3e} norm drift={drift:.3e}")
    assert err <= 1e-6  # measured 4.6e-7
    assert drift <= 3e-7  # measured 1.3e-7


def test_harmonic_oscillator_n128_seeded_datum(env, orc):
    """The seeded config datum (normalised Gaussian with a 10 % complex
    perturbation, seed 1): 10 steps against the oracle's literal steps
    (forward transform, phase, backward transform), and the weighted norm
    after all 100 steps."""
    mm, ctx, torch = env
    m, tau = 128, 0.01
    x, W, w3 = _hermite_nodes(orc, m)
    psi0 = inputs.harmonic_psi0(x, W, seed=1).astype(np.complex64)
    plan = mm.HermitePlan(ctx, [m] * 3, prec="f16x6")
    psi = to_gpu(torch, psi0, torch.complex64)
    plan.ho_step(psi, tau, 10)
    got = psi.cpu().numpy()
    ref = orc.ho_steps(psi0.astype(np.complex128), x, W, tau, 10)
    err = rel(got, ref, w3)
    plan.ho_step(psi, tau, 90)
    n100 = np.sum(np.abs(psi.cpu().numpy()) ** 2 * w3) / np.sum(np.abs(psi0.astype(np.complex128)) ** 2 * w3)
    print(f"HO n=128 seeded datum: 10 steps rel_err={err:.3e}; 100 steps norm drift={abs(n100 - 1):.3e}")
    assert err <= 4e-7  # measured 1.6e-7
    assert abs(n100 - 1) <= 2e-6  # measured 7.9e-7


def test_gpe_n192_against_oracle_and_fp64(env, orc):
    """Gross-Pitaevskii at the config size (n = 192, beta = 100, tau = 1e-3):
    two steps of the FP64 and the F16x6 paths against the oracle's Strang
    steps; 500 F16x6 steps against 500 FP64 GPU steps; weighted norm drift
    after 500 steps."""
    mm, ctx, torch = env
    m, beta, tau = 192, 100.0, 1e-3
    x, W, w3 = _hermite_nodes(orc, m)
    psi0 = inputs.gpe_psi0(x, W, seed=4)
    ref2 = orc.gpe_steps(psi0, x, W, beta, tau, 2)  # the F16x6 run starts from psi0 rounded to complex64

    p64 = mm.HermitePlan(ctx, [m] * 3, prec="fp64dmma")
    f64 = to_gpu(torch, psi0, torch.complex128)
    p64.gpe_step(f64, beta, tau, 2)
    err64 = rel(f64.cpu().numpy(), ref2, w3)

    p16 = mm.HermitePlan(ctx, [m] * 3, prec="f16x6")
    f16 = to_gpu(torch, psi0.astype(np.complex64), torch.complex64)
    nrm16 = p16.gpe_step_norm2(f16, beta, tau, 2)  # the weighted norm from the last product's epilogue
    err16 = rel(f16.cpu().numpy(), ref2, w3)
    enrm = abs(nrm16 / np.sum(np.abs(ref2) ** 2 * w3) - 1)
    print(f"GPE n=192 2 steps vs oracle: fp64 {err64:.3e}, f16x6 {err16:.3e}; epilogue norm {enrm:.3e}")
    assert err64 <= 1e-12  # measured 4.7e-15
    assert err16 <= 2e-7  # measured 9.2e-8
    assert enrm <= 2e-7

    p64.gpe_step(f64, beta, tau, 498)
    p16.gpe_step(f16, beta, tau, 498)
    a = f16.cpu().numpy()
    b = f64.cpu().numpy()
    err500 = rel(a, b, w3)
    n0 = np.sum(np.abs(psi0.astype(np.complex64).astype(np.complex128)) ** 2 * w3)
    drift16 = abs(np.sum(np.abs(a.astype(np.complex128)) ** 2 * w3) / n0 - 1)
    drift64 = abs(np.sum(np.abs(b) ** 2 * w3) / np.sum(np.abs(psi0) ** 2 * w3) - 1)
    print(f"GPE n=192 500 steps: f16x6 vs fp64 rel_err={err500:.3e}; norm drift f16x6 {drift16:.3e}, "
          f"fp64 {drift64:.3e}")
    assert err500 <= 8e-6  # measured 3.8e-6
    assert drift16 <= 4e-6  # measured 2.0e-6
    assert drift64 <= 1e-12  # measured 5.5e-14


def test_batched_all_64_problems_against_oracle(env, orc):
    """Every one of the 64 uneven problems (sizes 48..160 per direction,
    seed 3), stepped 3 times in the batched launches, against the oracle's
    U0 x_mu E_mu(3 tau) per problem."""
    mm, ctx, torch = env
    dims = inputs.batched_dims(count=64, seed=3)
    us0 = inputs.batched_u0(dims, seed=3)
    tau, steps = 1e-4, 3
    plans, us = [], []
    for nd, u0 in zip(dims, us0):
        nd = tuple(int(v) for v in nd)
        Es = [mm.expm(mm.fd_laplacian_dirichlet(n), 1j * tau) for n in nd]
        plans.append(mm.TuckerPlan(ctx, nd, Es, prec="f16x6"))
        us.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
    batch = mm.Batch(ctx, plans)
    batch.step(us, steps)
    torch.cuda.synchronize()
    worst = 0.0
    for k, (nd, u0) in enumerate(zip(dims, us0)):
        nd = tuple(int(v) for v in nd)
        E3 = [orc.expm_dirichlet_fd(n, 1j * tau * steps) for n in nd]
        ref = orc.tucker(u0.astype(np.complex64).astype(np.complex128), E3, nsteps=1)
        err = rel(us[k].cpu().numpy(), ref)
        worst = max(worst, err)
        assert err <= 2.5e-7, (k, nd, err)  # worst measured 1.2e-7
    print(f"batched 64 problems, 3 steps: worst rel_err={worst:.3e}")
