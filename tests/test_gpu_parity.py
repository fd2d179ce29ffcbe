"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over all compared points):
  FP64 SIMT                      1e-12
  FP32 SIMT                      2e-5 per run of a few steps
  F16x6 (fixed-point leading     1.5e-7 per mode product, 1e-6 after the
  piece, 6 products)             50-step n=256 run (the target accuracy)
  BF16x6 (floating pieces)       3e-7 per mode product; its truncation bias
                                 grows linearly, so it fails the 50-step bound
  BF16x3                         2e-4 per run
  3xTF32 (two TF32 pieces,       4e-6 per run of two steps (measured up to 1.6e-6 at 511),
  three products)                2e-6 per mode product; its truncation bias grows like
                                 BF16x6's (3.9e-5 after 50 steps at n = 256)
  BF16 (1 piece)                 3e-2 per run (reported only)
"""
import numpy as np
import pytest

from paper_2103_01691_b300 import inputs

pytestmark = pytest.mark.gpu

TOL_STEP = {"fp64": 1e-12, "fp32": 2e-5, "f16x6": 1e-6, "bf16x6": 1e-6, "bf16x3": 2e-4, "bf16": 3e-2, "tf32x3": 4e-6}
TOL_MODE = {"f16x6": 1.5e-7, "bf16x6": 3e-7}


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2103_01691_b300 import build as mmbuild

    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    ctx = mumode.Context(0)
    yield mumode, ctx, torch
    ctx.status()


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fd_schrodinger_E(mm, n, tau):
    return mm.expm(mm.fd_laplacian_dirichlet(n), 1j * tau)


def to_gpu(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


# ------------------------------------------------------------------ FP64 paths

@pytest.mark.parametrize("prec", ["fp64", "fp64dmma"])
def test_heat_fp64_n32(env, orc, prec):
    """Real FP64 heat equation, n = 32, tau = 1e-3, 10 steps, on the CUDA
    cores and on the tensor cores (warp MMA m8n8k4)."""
    mm, ctx, torch = env
    n, tau = 32, 1e-3
    u0 = inputs.heat_u0(n, seed=0)
    E = mm.expm(mm.fd_laplacian_dirichlet(n), tau).real
    plan = mm.TuckerPlan(ctx, [n] * 3, [E] * 3, prec=prec, dtype=torch.float64)
    u = to_gpu(torch, u0, torch.float64)
    plan.step(u, 10)
    Eo = orc.expm_dirichlet_fd(n, tau)
    ref = orc.tucker(u0.astype(complex), [Eo] * 3, nsteps=10).real
    assert rel(u.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp64dmma"])
@pytest.mark.parametrize("dims,order", [((20, 24, 17), None), ((20, 24, 17), (3, 1, 2)), ((7, 5), None),
                                        ((9,), None), ((5, 6, 4, 3), (2, 4, 1, 3)), ((70, 33, 66), None)])
def test_complex_fp64_ragged(env, orc, dims, order, prec):
    mm, ctx, torch = env
    tau = 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2)
    plan = mm.TuckerPlan(ctx, dims, Es, prec=prec, order=order)
    u = to_gpu(torch, u0, torch.complex128)
    plan.step(u, 3)
    Eo = [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims]
    ref = orc.tucker(u0, Eo, order=order, nsteps=3)
    assert rel(u.cpu().numpy(), ref) <= 1e-12


def test_fp32_simt(env, orc):
    mm, ctx, torch = env
    dims, tau = (33, 16, 20), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="fp32")
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, 3)
    ref = orc.tucker(u0.astype(np.complex64).astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=3)
    assert rel(u.cpu().numpy(), ref) <= TOL_STEP["fp32"]


# ------------------------------------------------------------ tensor-core paths

TC_DIMS = [(16, 16, 16), (32, 48, 16), (17, 33, 20), (64, 64, 64), (100, 37, 48), (128, 128, 64), (256, 16, 16),
           (16, 256, 16), (16, 16, 256), (160, 48, 80), (9,), (40, 24), (241, 20, 16), (16, 20, 255),
           (20, 16, 24, 18), (9, 12, 7, 10, 8), (300, 20, 16), (16, 20, 511), (400, 33, 24)]


@pytest.mark.parametrize("dims", TC_DIMS)
@pytest.mark.parametrize("prec", ["f16x6", "bf16x6", "bf16x3", "bf16", "tf32x3"])
def test_tc_tucker_steps(env, orc, dims, prec):
    mm, ctx, torch = env
    tau, steps = 1e-4, 2
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec=prec)
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, steps)
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=steps)
    err = rel(u.cpu().numpy(), ref)
    print(f"{prec} dims={dims} steps={steps} rel_err={err:.3e}")
    tol = {"f16x6": TOL_MODE["f16x6"] * steps * len(dims), "bf16x6": TOL_MODE["bf16x6"] * steps * len(dims),
           "bf16x3": TOL_STEP["bf16x3"], "bf16": TOL_STEP["bf16"], "tf32x3": TOL_STEP["tf32x3"]}[prec]
    assert err <= tol


@pytest.mark.parametrize("prec", ["f16x6", "bf16x6", "fp64", "fp64dmma", "fp32", "tf32x3"])
@pytest.mark.parametrize("dims", [(40, 24, 18), (17, 64, 9)])
def test_mumode_product_rectangular(env, orc, prec, dims):
    """Definition 2.1 with a rectangular complex (and a real) L."""
    mm, ctx, torch = env
    rng = np.random.default_rng(12)
    u0 = inputs.complex_normal(dims[::-1], seed=3)
    dt = torch.complex128 if prec in ("fp64", "fp64dmma") else torch.complex64
    tol = {"fp64": 1e-13, "fp64dmma": 1e-13, "fp32": 1e-5, "bf16x6": 3e-7, "f16x6": 1.5e-7, "tf32x3": 8e-7}[prec]
    for mu in range(1, 4):
        for m in (dims[mu - 1] + 8, max(1, dims[mu - 1] - 5)):
            for cplx in (True, False):
                L = rng.standard_normal((m, dims[mu - 1]))
                if cplx:
                    L = L + 1j * rng.standard_normal(L.shape)
                uin = u0 if prec in ("fp64", "fp64dmma") else u0.astype(np.complex64)
                s = mm.mumode_product(ctx, to_gpu(torch, uin, dt), mu, L, prec=prec)
                ref = orc.mode_product(uin.astype(complex), mu, L.astype(complex))
                err = rel(s.cpu().numpy(), ref)
                if prec == "tf32x3":
                    print(f"tf32x3 product dims={dims} mu={mu} m={m} complex={cplx}: rel_err={err:.3e}")
                assert err <= tol, (mu, m, cplx, err)


def test_mode_order_independence_tc(env, orc):
    mm, ctx, torch = env
    dims, tau = (48, 32, 64), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=2)
    for order in [(1, 2, 3), (3, 2, 1), (2, 3, 1)]:
        plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6", order=order)
        u = to_gpu(torch, u0, torch.complex64)
        plan.step(u, 2)
        assert rel(u.cpu().numpy(), ref) <= TOL_MODE["f16x6"] * 6


# ------------------------------------------------------------------ Hermite / GPE

@pytest.mark.parametrize("prec", ["f16x6", "bf16x6", "fp64"])
def test_hermite_transforms(env, orc, prec):
    mm, ctx, torch = env
    m = 32
    plan = mm.HermitePlan(ctx, [m] * 3, prec=prec)
    x, W = plan.nodes(1)
    xo, _, Wo = orc.gauss_hermite(m)
    v = inputs.complex_normal((m, m, m), seed=6)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    vin = v if prec == "fp64" else v.astype(np.complex64)
    c = plan.forward(to_gpu(torch, vin, dt))
    ref_c = orc.hermite_forward(vin.astype(complex), xo, Wo)
    tol = {"fp64": 1e-12, "f16x6": 5e-7, "bf16x6": 1e-6}[prec]
    assert rel(c.cpu().numpy(), ref_c) <= tol
    back = plan.backward(c)
    ref_b = orc.hermite_backward(c.cpu().numpy().astype(complex), xo, Wo)
    assert rel(back.cpu().numpy(), ref_b) <= tol


@pytest.mark.parametrize("prec", ["f16x6", "fp64"])
def test_harmonic_oscillator_steps(env, orc, prec):
    mm, ctx, torch = env
    m, tau, steps = 24, 0.01, 20
    plan = mm.HermitePlan(ctx, [m] * 3, prec=prec)
    xo, _, Wo = orc.gauss_hermite(m)
    psi0 = inputs.harmonic_psi0(xo, Wo, seed=1)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    pin = psi0 if prec == "fp64" else psi0.astype(np.complex64)
    psi = to_gpu(torch, pin, dt)
    plan.ho_step(psi, tau, steps)
    ref = orc.ho_steps(pin.astype(complex), xo, Wo, tau, steps)
    w3 = orc.weight3(Wo)
    tol = 1e-12 if prec == "fp64" else 1e-6
    err = orc.rel_l2(psi.cpu().numpy(), ref, w3)
    print(f"HO {prec} m={m} steps={steps} rel_err={err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("prec", ["f16x6", "fp64", "fp64dmma"])
def test_gpe_strang_steps(env, orc, prec):
    mm, ctx, torch = env
    m, beta, tau, steps = 16, 100.0, 1e-3, 20
    plan = mm.HermitePlan(ctx, [m] * 3, prec=prec)
    xo, _, Wo = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(xo, Wo, seed=4)
    f64 = prec in ("fp64", "fp64dmma")
    dt = torch.complex128 if f64 else torch.complex64
    pin = psi0 if f64 else psi0.astype(np.complex64)
    psi = to_gpu(torch, pin, dt)
    plan.gpe_step(psi, beta, tau, steps)
    ref = orc.gpe_steps(pin.astype(complex), xo, Wo, beta, tau, steps)
    w3 = orc.weight3(Wo)
    tol = 1e-11 if f64 else 1e-6
    err = orc.rel_l2(psi.cpu().numpy(), ref, w3)
    print(f"GPE {prec} m={m} steps={steps} rel_err={err:.3e}")
    assert err <= tol
    n0 = plan.norm2(to_gpu(torch, pin, dt))
    n1 = plan.norm2(psi)
    assert abs(n1 / n0 - 1) <= (1e-12 if f64 else 1e-6)


# ------------------------------------------- CTA-pair kernel vs one-SM kernel

@pytest.mark.parametrize("tile", [64, 128])
@pytest.mark.parametrize("dims", [(256, 64, 32), (32, 256, 96), (64, 32, 256)])
@pytest.mark.parametrize("prec", ["f16x6", "bf16x3"])
def test_pair_kernel_matches_one_sm_kernel(env, monkeypatch, dims, prec, tile):
    """The CTA-pair kernel (M = 256 over the two SMs of a cluster) issues the
    same piece products as the one-SM kernel, in the same order for every
    output (the real plane's product, then the imaginary plane's, with -S
    stored negated instead of the MMA's negate bit; k-blocks outside a row
    tile's band only add exact zeros): the results agree bit for bit, for
    row tiles of 64 (two accumulator sets) and of 128 (MM_PAIR_TILE=128).
    MM_TC_1SM=1 selects the one-SM kernel."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_PAIR_TILE", str(tile))
    tau = 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=6).astype(np.complex64)

    def run():
        plan = mm.TuckerPlan(ctx, dims, Es, prec=prec)
        plan.set_graphs(False)
        u = to_gpu(torch, u0, torch.complex64)
        plan.step(u, 2)
        torch.cuda.synchronize()
        return u.cpu().numpy()

    monkeypatch.delenv("MM_TC_1SM", raising=False)
    pair = run()
    monkeypatch.setenv("MM_TC_1SM", "1")
    one = run()
    monkeypatch.delenv("MM_TC_1SM")
    print(f"pair (tile {tile}) vs one-SM {prec} dims={dims}: max |diff| = {np.abs(pair - one).max():.3e}, "
          f"rel = {rel(pair, one):.3e}")
    assert np.array_equal(pair.view(np.uint32), one.view(np.uint32))


@pytest.mark.parametrize("dims,steps", [((64, 64, 64), 3), ((128, 128, 128), 2), ((256, 64, 48), 2),
                                         ((100, 37, 48), 2), ((40, 24), 4), ((256, 256, 256), 1),
                                         ((64, 64, 64), 9), ((192, 192, 192), 3), ((32, 24, 40, 16), 3),
                                         ((48, 40, 512), 2), ((300,), 5)])
def test_chained_launch_matches_single_launches(env, orc, dims, steps):
    """The chained variant (every product of a step call in one persistent launch, each item's
    loads waiting for the slab groups it reads through counters, so that products overlap) runs
    the same items with the same kernel code as one launch per product: the results agree bit
    for bit, from plain launches and from a replayed graph, over d = 1 .. 4 and padded directions.
    Shapes whose directions have row tiles of different sizes fall back to one launch per
    product."""
    mm, ctx, torch = env
    tau = 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=6).astype(np.complex64)
    out = {}
    for variant in ("pair64", "chain"):
        for graphs in (False, True):
            plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
            plan.set_config(variant)
            plan.set_graphs(graphs)
            u = to_gpu(torch, u0, torch.complex64)
            plan.step(u, steps)
            if graphs:
                u = to_gpu(torch, u0, torch.complex64)
                plan.step(u, steps)  # replayed
            torch.cuda.synchronize()
            out[(variant, graphs)] = u.cpu().numpy()
            ctx.status()
    ref = out[("pair64", False)]
    for key, got in out.items():
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), key
    if max(dims) <= 128:
        ora = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=steps)
        assert rel(out[("chain", True)], ora) <= TOL_MODE["f16x6"] * steps * len(dims)


@pytest.mark.parametrize("m,tile", [(32, 64), (96, 128)])
def test_pair_kernel_gpe_epilogue(env, orc, monkeypatch, m, tile):
    """The nonlinear-phase epilogue in the CTA-pair kernel (m = 32 quadrature
    points: one row tile of 32; m = 96 with MM_PAIR_TILE=128: one row tile of
    96, two chunks of 16 rows per epilogue warp): against the oracle and bit
    for bit against the one-SM kernel."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_PAIR_TILE", str(tile))
    beta, tau, steps = 100.0, 1e-3, 6
    xo, _, Wo = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(xo, Wo, seed=4).astype(np.complex64)

    def run():
        plan = mm.HermitePlan(ctx, [m] * 3, prec="f16x6")
        psi = to_gpu(torch, psi0, torch.complex64)
        plan.gpe_step(psi, beta, tau, steps)
        torch.cuda.synchronize()
        return psi.cpu().numpy()

    monkeypatch.delenv("MM_TC_1SM", raising=False)
    pair = run()
    monkeypatch.setenv("MM_TC_1SM", "1")
    one = run()
    monkeypatch.delenv("MM_TC_1SM")
    ref = orc.gpe_steps(psi0.astype(complex), xo, Wo, beta, tau, steps)
    err = orc.rel_l2(pair, ref, orc.weight3(Wo))
    print(f"GPE pair m={m} rel_err={err:.3e}, pair vs one-SM max |diff| = {np.abs(pair - one).max():.3e}")
    assert err <= 1e-6
    assert np.array_equal(pair.view(np.uint32), one.view(np.uint32))


# ------------------------------------------------- full size, sampled (n = 256)

def test_free_schrodinger_n256_50_steps_sampled(env, orc):
    """The precision-sweep workload at full size: n = 256, tau = 1e-4, 50
    steps of F16x6.  The oracle evaluates sampled entries of the exact
    50-step result U0 x_mu E(50 tau) (E(tau)^50 = E(50 tau))."""
    mm, ctx, torch = env
    n, tau, steps = 256, 1e-4, 50
    E = fd_schrodinger_E(mm, n, tau)
    plan = mm.TuckerPlan(ctx, [n] * 3, [E] * 3, prec="f16x6")
    u0 = inputs.free_schrodinger_u0(n, seed=2).astype(np.complex64)
    u = to_gpu(torch, u0, torch.complex64)
    nrm0 = plan.norm2(u)
    plan.step(u, steps)
    nrm1 = plan.norm2(u)
    got = u.cpu().numpy()
    rng = np.random.default_rng(21)
    idx = rng.integers(0, n, size=(48, 3))
    idx[0] = (0, 0, 0)
    idx[1] = (n - 1, n - 1, n - 1)
    E50 = orc.expm_dirichlet_fd(n, 1j * tau * steps)
    ref = orc.tucker3_entries(u0.astype(complex), E50, E50, E50, idx)
    err = rel(got[idx[:, 2], idx[:, 1], idx[:, 0]], ref)
    print(f"n=256 50 steps f16x6 sampled rel_err={err:.3e} norm drift={abs(nrm1 / nrm0 - 1):.3e}")
    assert err <= 1e-6
    assert abs(nrm1 / nrm0 - 1) <= 1e-6


# ------------------------------------------------------------- HKP (section 4.3)

def _hkp_nodes(orc, n):
    xs, Ws = [], []
    for v in n:
        x, _, W = orc.gauss_hermite(v)
        xs.append(x)
        Ws.append(W)
    return xs, Ws


@pytest.mark.parametrize("prec,tau,steps", [("f16x6", 1.0, 1), ("f16x6", 0.5, 2), ("bf16x6", 1.0, 1),
                                            ("fp64", 1.0, 1), ("fp64dmma", 0.5, 2)])
def test_hkp_kronecker_potential(env, orc, prec, tau, steps):
    """HKP plan (V_1 = cos(2 pi x_1), V_2 = V_3 = x^2/2; direction 2 passed
    as harmonic, direction 3 by its values) against the oracle's literal
    forward / exp(-i tau H) / backward steps, to T = 1 on ragged sizes."""
    mm, ctx, torch = env
    n = (72, 48, 40)
    xs, Ws = _hkp_nodes(orc, n)
    psi0 = inputs.hkp_psi0(*xs)
    f64 = prec in ("fp64", "fp64dmma")
    pin = psi0 if f64 else psi0.astype(np.complex64)
    ref = orc.hkp_steps(pin.astype(complex), xs, Ws, inputs.hkp_potentials(*xs), tau, steps)
    xl = [mm.gauss_hermite(v)[0] for v in n]
    Vl = inputs.hkp_potentials(*xl)
    plan = mm.HKPPlan(ctx, n, [Vl[0], None, Vl[2]], tau, prec=prec)
    psi = to_gpu(torch, pin, torch.complex128 if f64 else torch.complex64)
    plan.step(psi, steps)
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    err = orc.rel_l2(psi.cpu().numpy(), ref, w3)
    print(f"HKP {prec} n={n} tau={tau} steps={steps} rel_err={err:.3e}")
    assert err <= (1e-12 if f64 else 1e-6)


def test_hkp_above_256(env, orc):
    """HKP on the tensor cores with a direction of more than 256 nodes."""
    mm, ctx, torch = env
    n = (300, 24, 20)
    xs, Ws = _hkp_nodes(orc, n)
    psi0 = inputs.hkp_psi0(*xs).astype(np.complex64)
    ref = orc.hkp_steps(psi0.astype(complex), xs, Ws, inputs.hkp_potentials(*xs), 1.0, 1)
    xl = [mm.gauss_hermite(v)[0] for v in n]
    plan = mm.HKPPlan(ctx, n, [inputs.hkp_potentials(*xl)[0], None, None], 1.0, prec="f16x6")
    psi = to_gpu(torch, psi0, torch.complex64)
    plan.step(psi, 1)
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    err = orc.rel_l2(psi.cpu().numpy(), ref, w3)
    print(f"HKP f16x6 n={n} rel_err={err:.3e}")
    assert err <= 1e-6


def test_hkp_hamiltonian_matches_oracle(env, orc):
    """mm_hermite_hamiltonian (library, FP64 host) equals the oracle's."""
    mm, ctx, torch = env
    for m in (1, 17, 64):
        xl, _ = mm.gauss_hermite(m)
        xo, _, Wo = orc.gauss_hermite(m)
        H = mm.hermite_hamiltonian(m, np.cos(2 * np.pi * xl))
        ref = orc.hkp_hamiltonian(xo, Wo, np.cos(2 * np.pi * xo))
        assert np.max(np.abs(H - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
        assert np.array_equal(mm.hermite_hamiltonian(m, None), np.diag(np.arange(m) + 0.5))
    with pytest.raises(mm.MumodeError):
        mm.HKPPlan(ctx, (8, 8, 8), [None] * 3, float("nan"))


def test_hkp_full_size_sampled(env, orc):
    """The paper's largest single-GPU HKP size that the tensor-core path
    takes, n = 255 per direction, one step to T = 1 in F16x6: sampled
    entries against the oracle's Tucker operator with each direction's
    forward transform, exp(-i H) (oracle Taylor) and backward transform
    multiplied out, and the weighted norm against its initial value."""
    mm, ctx, torch = env
    n = (255, 255, 255)
    xs, Ws = _hkp_nodes(orc, n)
    Vs = inputs.hkp_potentials(*xs)
    psi0 = inputs.hkp_psi0(*xs).astype(np.complex64)
    xl = mm.gauss_hermite(255)[0]
    Vl = inputs.hkp_potentials(xl, xl, xl)
    plan = mm.HKPPlan(ctx, n, list(Vl), 1.0, prec="f16x6")
    psi = to_gpu(torch, psi0, torch.complex64)
    plan.step(psi, 1)
    got = psi.cpu().numpy()
    P = orc.hermite_functions(255, xs[0])
    E1 = orc.expm_taylor(orc.hkp_hamiltonian(xs[0], Ws[0], Vs[0]), -1j)
    M1 = P.T @ E1 @ (P * Ws[0][None, :])
    M2 = P.T @ np.diag(np.exp(-1j * (np.arange(255) + 0.5))) @ (P * Ws[0][None, :])
    # the packet lives at |x| < ~5 (node indices 127 +- 35); the grid reaches
    # |x| ~ 22, where the values are tiny and the fixed-point pieces (whose
    # error is relative to the maximum) bound the absolute error only
    # samples: three full grid lines through the packet, one along each
    # direction, and 40 points of its bulk, so that the sample's norm is
    # carried by the large values like the norm of the whole tensor
    rng = np.random.default_rng(22)
    a = np.arange(255)
    c = np.full(255, 127)
    lines = [np.stack([a, c + 4, c - 3], 1), np.stack([c - 2, a, c + 5], 1), np.stack([c + 3, c - 4, a], 1)]
    near = np.concatenate(lines + [127 + rng.integers(-35, 36, size=(40, 3))])
    far = rng.integers(0, 255, size=(24, 3))
    far[0] = (254, 0, 254)
    ref_n = orc.tucker3_entries(psi0.astype(complex), M1, M2, M2, near)
    ref_f = orc.tucker3_entries(psi0.astype(complex), M1, M2, M2, far)
    err = rel(got[near[:, 2], near[:, 1], near[:, 0]], ref_n)
    far_err = np.max(np.abs(got[far[:, 2], far[:, 1], far[:, 0]] - ref_f)) / np.max(np.abs(got))
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    drift = abs(np.sum(np.abs(got) ** 2 * w3) / np.sum(np.abs(psi0.astype(complex)) ** 2 * w3) - 1)
    print(f"HKP n=255 f16x6 sampled rel_err={err:.3e} far abs/max={far_err:.3e} norm drift={drift:.3e}")
    assert err <= 1e-5
    assert far_err <= 1e-6
    assert drift <= 1e-6


# ------------------------------------------- device exponentials, HKMP (section 4.4)

@pytest.mark.parametrize("n", [1, 40, 97, 200])
def test_expm_device(env, orc, n):
    """mm_expm_device, exp(z (A + f B)) in FP64 on the GPU, against the
    oracle's Taylor exponential, for an imaginary and a real z, with the
    norm bound given and computed by the call."""
    mm, ctx, torch = env
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) * 3.0
    A = A + A.T  # symmetric: exp(-i s A) is unitary, as in the Magnus steps
    B = rng.standard_normal((n, n))
    B = B + B.T
    f = 0.3
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    for z in (-0.05j, 0.01):
        ref = orc.expm_taylor(A + f * B, z)
        bound = np.abs(A + f * B).sum(axis=0).max()
        for nb in (bound, 0.0):
            E = mm.expm_device(ctx, Ad, Bd, f, z, norm_bound=nb).cpu().numpy()
            err = np.linalg.norm(E - ref) / np.linalg.norm(ref)
            print(f"expm_device n={n} z={z} bound={nb:.1f} rel_err={err:.2e}")
            assert err <= 1e-11, (z, nb)
    E0 = mm.expm_device(ctx, Ad, None, 0.0, 0.01).cpu().numpy()
    ref0 = orc.expm_taylor(A, 0.01)
    assert np.linalg.norm(E0 - ref0) <= 1e-11 * np.linalg.norm(ref0)


@pytest.mark.parametrize("prec,variant", [("f16x6", "pair64"), ("f16x6", "pair128"), ("f16x6", "one_sm"),
                                          ("bf16x3", "pair64"), ("fp64", None)])
def test_set_matrix_device_matches_host_matrix(env, monkeypatch, prec, variant):
    """A matrix split on the device (mm_plan_set_matrix_device) gives the same
    bits as the host-built one: a plan created with other matrices and then
    given E on the device steps exactly like a plan created with E (both
    unfolded: a matrix set on the device is used as it is)."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_NO_FOLD", "1")
    dims, tau = (72, 40, 33), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    other = [fd_schrodinger_E(mm, n, 3 * tau) for n in dims]
    f64 = prec == "fp64"
    u0 = inputs.complex_normal(dims[::-1], seed=4)
    if not f64:
        u0 = u0.astype(np.complex64)
    a = mm.TuckerPlan(ctx, dims, Es, prec=prec)
    b = mm.TuckerPlan(ctx, dims, other, prec=prec)
    if variant:
        a.set_config(variant, (1, 2, 3))
        b.set_config(variant, (1, 2, 3))
    for mu, E in enumerate(Es, start=1):
        b.set_matrix_device(mu, torch.from_numpy(np.ascontiguousarray(E)).cuda(), row_norm_bound=0.0)
    dt = torch.complex128 if f64 else torch.complex64
    ua, ub = to_gpu(torch, u0, dt), to_gpu(torch, u0, dt)
    a.step(ua, 3)
    b.step(ub, 3)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)


def _hkmp_case(orc, n):
    xs, Ws = [], []
    for v in n:
        x, _, W = orc.gauss_hermite(v)
        xs.append(x)
        Ws.append(W)
    return xs, Ws


@pytest.mark.parametrize("prec,tdir,variant", [("f16x6", 3, None), ("f16x6", 1, None), ("f16x6", 2, None),
                                               ("f16x6", 3, "one_sm"), ("f16x6", 3, "pair128"),
                                               ("f16x6", 1, "pair128"), ("fp64", 3, None), ("fp64dmma", 1, None)])
def test_hkmp_vs_oracle(env, orc, prec, tdir, variant):
    """HKMP (the section 4.4 potential |x|^2/2 + x_3 sin^2 t, or with the
    time dependence moved to direction 1) against the oracle's literal
    Magnus steps: 12 steps of 0.05 on ragged sizes."""
    mm, ctx, torch = env
    n = (72, 40, 48)
    xs, Ws = _hkmp_case(orc, n)
    Vs, Us = inputs.hkmp_potentials(*xs)
    if tdir != 3:  # move the time dependence: U = x in direction tdir
        Us = tuple(np.array(xs[v]) if v == tdir - 1 else None for v in range(3))
    tau, steps = 0.05, 12
    f_mid = inputs.hkmp_f_mid(tau, steps)
    f64 = prec in ("fp64", "fp64dmma")
    psi0 = inputs.hkp_psi0(*xs)
    pin = psi0 if f64 else psi0.astype(np.complex64)
    ref = orc.hkmp_steps(pin.astype(complex), xs, Ws, Vs, Us, tau, f_mid)
    xl = [mm.gauss_hermite(v)[0] for v in n]
    Vl, Ul = inputs.hkmp_potentials(*xl)
    if tdir != 3:
        Ul = tuple(np.array(xl[v]) if v == tdir - 1 else None for v in range(3))
    # harmonic directions passed as None: the tensor-core plan then fuses their phases into the
    # time-dependent direction's product (one product per step); one_sm runs the three products
    plan = mm.HKMPPlan(ctx, n, [None, None, None], list(Ul), tau, prec=prec)
    if variant:
        assert mm.lib().mm_plan_set_config(plan.handle, mm.VARIANTS.index(variant), None) == 0
    psi = to_gpu(torch, pin, torch.complex128 if f64 else torch.complex64)
    plan.evolve(psi, f_mid)
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    err = orc.rel_l2(psi.cpu().numpy(), ref, w3)
    print(f"HKMP {prec} dir {tdir} {variant or 'default'} n={n} steps={steps} rel_err={err:.3e}")
    assert err <= (1e-12 if f64 else 5e-6)
    ctx.status()


# ---------------------------------------------------------- pipe flow (section 4.2)


def test_hkmp_declared_f_range(env, orc):
    """hkmp_set_f_range(0, 1) for f = sin^2 t: the node exponentials are computed once and every
    chunk combines from them.  Against the oracle's literal Magnus steps and the plan without a
    range (the two exponentials differ below the pieces' resolution); a range that does not hold
    the values, and a dropped range, give the plan's own per-chunk nodes bit for bit; a range too
    wide for 12 nodes and an FP64 plan are refused."""
    mm, ctx, torch = env
    n = (40, 24, 36)
    xs, Ws = _hkmp_case(orc, n)
    Vs, Us = inputs.hkmp_potentials(*xs)
    tau, steps = 0.025, 40
    f_mid = inputs.hkmp_f_mid(tau, steps)
    psi0 = inputs.hkp_psi0(*xs).astype(np.complex64)
    ref = orc.hkmp_steps(psi0.astype(complex), xs, Ws, Vs, Us, tau, f_mid)
    xl = [mm.gauss_hermite(v)[0] for v in n]
    _, Ul = inputs.hkmp_potentials(*xl)

    def run(rng):
        plan = mm.HKMPPlan(ctx, n, [None, None, None], list(Ul), tau, prec="f16x6")
        if rng is not None:
            plan.set_f_range(*rng)
        psi = to_gpu(torch, psi0, torch.complex64)
        plan.evolve(psi, f_mid)
        torch.cuda.synchronize()
        ctx.status()
        return psi.cpu().numpy()

    base, ranged = run(None), run((0.0, 1.0))
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    e_base, e_rng = orc.rel_l2(base, ref, w3), orc.rel_l2(ranged, ref, w3)
    print(f"HKMP declared f range: {e_rng:.3e} against the oracle (per-chunk nodes {e_base:.3e}), "
          f"{rel(ranged, base):.2e} between them")
    assert e_rng <= 5e-6 and rel(ranged, base) <= 1e-6
    assert f_mid.min() < 0.5  # the next range misses some values: every chunk takes its own nodes
    assert np.array_equal(run((0.5, 1.0)).view(np.uint32), base.view(np.uint32))
    assert np.array_equal(run((1.0, 0.0)).view(np.uint32), base.view(np.uint32))  # dropped
    plan = mm.HKMPPlan(ctx, n, [None, None, None], list(Ul), tau, prec="f16x6")
    with pytest.raises(mm.MumodeError, match="MM_ERR_INVALID_ARG"):
        plan.set_f_range(0.0, 1e7)
    p64 = mm.HKMPPlan(ctx, n, [None, None, None], list(Ul), tau, prec="fp64dmma")
    with pytest.raises(mm.MumodeError, match="MM_ERR_UNSUPPORTED"):
        p64.set_f_range(0.0, 1.0)


@pytest.mark.parametrize("tdir,variant", [(3, None), (1, "one_sm")])
def test_hkmp_interpolated_exponentials(env, orc, tdir, variant):
    """Tensor-core HKMP with more than 12 steps in a chunk takes the chunk's
    exponentials from 12 Chebyshev nodes in f (interpolation error far below
    the pieces' resolution).  Against the oracle's literal Magnus steps, and
    against the same evolution in calls of at most 12 steps (each chunk then
    takes one exponential per step).  The two runs differ mostly by the
    short calls' extra transforms to and from coefficient space (about 1e-7
    relative each)."""
    mm, ctx, torch = env
    n = (40, 24, 36)
    xs, Ws = _hkmp_case(orc, n)
    Vs, Us = inputs.hkmp_potentials(*xs)
    if tdir != 3:
        Us = tuple(np.array(xs[v]) if v == tdir - 1 else None for v in range(3))
    tau, steps = 0.025, 40
    f_mid = inputs.hkmp_f_mid(tau, steps)
    psi0 = inputs.hkp_psi0(*xs).astype(np.complex64)
    ref = orc.hkmp_steps(psi0.astype(complex), xs, Ws, Vs, Us, tau, f_mid)
    xl = [mm.gauss_hermite(v)[0] for v in n]
    _, Ul = inputs.hkmp_potentials(*xl)
    if tdir != 3:
        Ul = tuple(np.array(xl[v]) if v == tdir - 1 else None for v in range(3))
    plan = mm.HKMPPlan(ctx, n, [None, None, None], list(Ul), tau, prec="f16x6")
    if variant:
        assert mm.lib().mm_plan_set_config(plan.handle, mm.VARIANTS.index(variant), None) == 0
    psi = to_gpu(torch, psi0, torch.complex64)
    plan.evolve(psi, f_mid)
    short = to_gpu(torch, psi0, torch.complex64)
    for k0 in range(0, steps, 10):
        plan.evolve(short, f_mid[k0:k0 + 10])
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    got, direct = psi.cpu().numpy(), short.cpu().numpy()
    err, err_direct = orc.rel_l2(got, ref, w3), orc.rel_l2(direct, ref, w3)
    diff = orc.rel_l2(got, direct, w3)
    print(f"HKMP interpolated dir {tdir} {variant or 'default'}: rel_err={err:.3e}, "
          f"direct={err_direct:.3e}, interpolated vs direct={diff:.3e}")
    assert err <= 5e-6 and err_direct <= 5e-6
    assert diff <= 2e-6
    ctx.status()

@pytest.mark.parametrize("prec,n_r,n_z,T", [("fp64dmma", 40, 56, 4.0), ("fp64", 40, 56, 4.0),
                                             ("fp64dmma", 257, 301, 1.0), ("fp64", 257, 301, 4.0)])
def test_pipe_flow_vs_oracle(env, orc, prec, n_r, n_z, T):
    """pipe_plan_create (operators on the host, exp(T A) on the device) and
    one step to T against the oracle's operators, Taylor exponentials and
    Tucker operator.  The pulse crosses the pipe (speed 2 to 4) and leaves
    through z_max by t ~ 3, so at T = 4 on a fine grid only small tails
    remain; T = 1 compares the pulse inside the pipe."""
    mm, ctx, torch = env
    P = dict(inputs.PIPE)
    P["T"] = T
    r = P["rmin"] + (P["rmax"] - P["rmin"]) / (n_r - 1) * np.arange(n_r)
    z = P["zmax"] / n_z * np.arange(1, n_z + 1)
    s = inputs.pipe_velocity(z)
    c0 = inputs.pipe_c0(r, z)
    plan = mm.PipePlan(ctx, n_r, n_z, P["rmin"], P["rmax"], P["zmax"], P["alpha"], s, P["T"], prec=prec)
    c = torch.from_numpy(c0).cuda()
    plan.step(c, 1)
    Er = orc.expm_taylor(orc.pipe_radial(n_r, P["rmin"], P["rmax"], P["alpha"]), P["T"])
    Ez = orc.expm_taylor(orc.pipe_axial(n_z, P["zmax"], P["alpha"], s), P["T"])
    ref = orc.tucker(c0.astype(complex), [Er, Ez]).real
    err = rel(c.cpu().numpy(), ref)
    print(f"pipe {prec} n=({n_r},{n_z}) rel_err={err:.3e} max c(T)={ref.max():.4f}")
    assert err <= 1e-12


def test_hkp_511_sampled(env, orc):
    """The paper's largest HKP size, n = 511 per direction (133 M points, 6.4 GB
    of split state), one step to T = 1 in F16x6: three full grid lines through
    the packet and 40 bulk points against the oracle's Tucker operator with
    each direction's transforms and exp(-i H) multiplied out."""
    mm, ctx, torch = env
    m = 511
    x, _, W = orc.gauss_hermite(m)
    V1 = inputs.hkp_potentials(x, x, x)[0]
    psi0 = inputs.hkp_psi0(x, x, x).astype(np.complex64)
    xl = mm.gauss_hermite(m)[0]
    plan = mm.HKPPlan(ctx, (m, m, m), [inputs.hkp_potentials(xl, xl, xl)[0], None, None], 1.0, prec="f16x6")
    psi = to_gpu(torch, psi0, torch.complex64)
    del psi0
    plan.step(psi, 1)
    P = orc.hermite_functions(m, x)
    M1 = P.T @ orc.expm_taylor(orc.hkp_hamiltonian(x, W, V1), -1j) @ (P * W[None, :])
    M2 = P.T @ np.diag(np.exp(-1j * (np.arange(m) + 0.5))) @ (P * W[None, :])
    rng = np.random.default_rng(23)
    a = np.arange(m)
    c = np.full(m, m // 2)
    near = np.concatenate([np.stack([a, c + 7, c - 5], 1), np.stack([c - 3, a, c + 9], 1),
                           np.stack([c + 6, c - 8, a], 1), m // 2 + rng.integers(-60, 61, size=(40, 3))])
    # the oracle's entries from the initial datum (recomputed in FP64 from its complex64 values)
    u0 = inputs.hkp_psi0(x, x, x).astype(np.complex64).astype(complex)
    ref = orc.tucker3_entries(u0, M1, M2, M2, near)
    del u0
    ix = [torch.from_numpy(np.ascontiguousarray(near[:, k])).cuda() for k in (2, 1, 0)]
    got = psi[ix[0], ix[1], ix[2]].cpu().numpy()
    err = rel(got, ref)
    print(f"HKP n=511 f16x6 sampled rel_err={err:.3e}")
    assert err <= 1e-5
    ctx.status()


@pytest.mark.parametrize("dims", [(200,), (72, 40)])
def test_fixed_point_scale_changes_every_sweep(env, orc, dims):
    """A growing flow (E = 2.5 x the Schroedinger propagator in every
    direction) moves the fixed-point state scale to a new power of two at
    every sweep; the result still matches the oracle (also for d = 1, where
    one launch both reads the input scale and sets the output scale)."""
    mm, ctx, torch = env
    tau, steps = 1e-4, 7
    Es = [2.5 * fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=9).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, steps)
    ref = orc.tucker(u0.astype(complex), [2.5 * orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=steps)
    assert rel(u.cpu().numpy(), ref) <= TOL_MODE["f16x6"] * steps * len(dims) * 2
    ctx.status()


def test_fixed_point_wide_dynamic_range(env, orc):
    """F16x6 keeps a relative L2 accuracy when magnitudes span 1e-6 .. 1:
    the fixed-point leading piece is relative to the maximum, the FP16
    remainders carry the small values."""
    mm, ctx, torch = env
    dims, tau = (32, 40, 24), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=8)
    scale = np.exp(np.linspace(np.log(1e-6), 0.0, dims[2]))[:, None, None]
    u0 = (u0 * scale).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, 3)
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=3)
    assert rel(u.cpu().numpy(), ref) <= TOL_MODE["f16x6"] * 9


def test_graph_replay_matches_plain_launches(env, monkeypatch):
    """Steps replayed from a captured CUDA graph give the same bits as the
    same steps launched one by one (plans without folding, so that the
    launch count is the products')."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_NO_FOLD", "1")
    dims, tau = (48, 40, 32), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plain = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
        plain.set_graphs(False)
        ref = to_gpu(torch, u0, torch.complex64)
        plain.step(ref, 3)
        plain.step(ref, 3)
        graphed = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
        u = to_gpu(torch, u0, torch.complex64)
        n0 = mm.launch_count()
        graphed.step(u, 3)   # captured, then replayed
        graphed.step(u, 3)   # replayed
        n1 = mm.launch_count()
    torch.cuda.synchronize()
    assert torch.equal(u, ref)
    assert n1 - n0 == 2 * (2 + 3 * 3 + 1)  # max + split, 3 sweeps x 3 products, merge; counted per replay


@pytest.mark.parametrize("dims", [(16, 16, 16), (20, 24, 40)])
def test_gpe_norm_in_epilogue(env, orc, dims):
    """split_step_gpe_norm2: the weighted norm sum |psi|^2 W1 W2 W3 taken in
    the last product's epilogue (F16X6, CTA pair) against the same quadrature
    of the oracle's Strang steps, against mm_norm2 of the returned state, and
    the state itself bit for bit against split_step_gpe.  Sizes padded in
    every direction (20, 24, 40 -> 32, 32, 48) check the weights' index
    decomposition; the one-SM variant takes the unfused form (one more
    launch: the norm pass)."""
    mm, ctx, torch = env
    beta, tau, steps = 100.0, 1e-3, 5
    plan = mm.HermitePlan(ctx, list(dims), prec="f16x6")
    grids = [orc.gauss_hermite(m) for m in dims]
    w3 = np.einsum("k,j,i->kji", grids[2][2], grids[1][2], grids[0][2])
    psi0 = inputs.gpe_psi0_dims([g[0] for g in grids], [g[2] for g in grids], seed=4).astype(np.complex64)
    cubic = len(set(dims)) == 1
    if cubic:  # the oracle's Strang steps (cubic grids)
        ref = orc.gpe_steps(psi0.astype(complex), grids[0][0], grids[0][2], beta, tau, steps)
        nref = float(np.sum(np.abs(ref) ** 2 * w3))
    a = to_gpu(torch, psi0, torch.complex64)
    b = to_gpu(torch, psi0, torch.complex64)
    plan.gpe_step(a, beta, tau, steps)
    torch.cuda.synchronize()
    l0 = mm.launch_count()
    plan.gpe_step(to_gpu(torch, psi0, torch.complex64), beta, tau, steps)
    torch.cuda.synchronize()
    l1 = mm.launch_count()
    nf = plan.gpe_step_norm2(b, beta, tau, steps)
    l2 = mm.launch_count()
    assert l2 - l1 == l1 - l0, "the fused norm adds no launch"
    assert torch.equal(a, b)
    n_pass = plan.norm2(b)
    n_np = float(np.sum(np.abs(b.cpu().numpy().astype(np.complex128)) ** 2 * w3))  # the quadrature, written out
    if not cubic:
        nref = n_np
    e_orc, e_pass, e_np = abs(nf / nref - 1), abs(nf / n_pass - 1), abs(nf / n_np - 1)
    print(f"GPE norm in epilogue {dims}: vs oracle {e_orc:.3e}, vs mm_norm2 {e_pass:.3e}, vs numpy {e_np:.3e}")
    assert e_orc <= 1e-6
    assert e_pass <= 2e-7 and e_np <= 2e-7
    # unfused form: the same result through split_step_gpe + mm_norm2
    plan.set_config("one_sm")
    c = to_gpu(torch, psi0, torch.complex64)
    l3 = mm.launch_count()
    nu = plan.gpe_step_norm2(c, beta, tau, steps)
    l4 = mm.launch_count()
    assert l4 - l3 >= 1
    if cubic:
        assert abs(nu / nref - 1) <= 1e-6
    assert abs(nu / plan.norm2(c) - 1) <= 1e-14  # the norm pass's FP64 atomics: order of additions
    assert abs(plan.gpe_step_norm2(c, beta, tau, 0) / nu - 1) <= 1e-14  # nsteps = 0: the norm of psi


def test_device_status_clean(env):
    mm, ctx, torch = env
    ctx.status()


# ---------------------------------------------------------------- GPE adjoint

@pytest.mark.parametrize("prec,ckpt", [("fp64", 4), ("fp64", 100), ("f16x6", 4)])
def test_gpe_adjoint_matches_oracle(env, orc, prec, ckpt):
    """split_step_gpe_adjoint (checkpointed reverse sweep) against the
    oracle's adjoint, itself pinned by finite differences."""
    mm, ctx, torch = env
    m, beta, tau, steps = 12, 100.0, 1e-3, 10
    plan = mm.HermitePlan(ctx, [m] * 3, prec=prec)
    xo, _, Wo = orc.gauss_hermite(m)
    w3 = orc.weight3(Wo)
    psi0 = inputs.gpe_psi0(xo, Wo, seed=4)
    target = inputs.gpe_target(xo, Wo)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    p0 = psi0 if prec == "fp64" else psi0.astype(np.complex64)
    pT = orc.gpe_steps(p0.astype(complex), xo, Wo, beta, tau, steps)
    gT = 2.0 * w3 * (pT - target)
    ref = orc.gpe_adjoint(p0.astype(complex), gT, xo, Wo, beta, tau, steps)
    g0 = plan.gpe_adjoint(to_gpu(torch, p0, dt), to_gpu(torch, gT, dt), beta, tau, steps, ckpt_every=ckpt)
    err = rel(g0.cpu().numpy(), ref)
    print(f"adjoint {prec} ckpt={ckpt} rel_err={err:.3e}")
    assert err <= (1e-10 if prec == "fp64" else 5e-7)


@pytest.mark.parametrize("prec", ["f16x6", "fp64"])
def test_gpe_adjoint_repeated_calls(env, orc, prec):
    """The adjoint keeps its matrices and checkpoint buffers with the plan:
    a second call with the same tau gives the same gradient bit for bit, a
    call with another tau rebuilds the matrices and matches the oracle, and
    uneven segments (10 steps, checkpoints every 3) are handled."""
    mm, ctx, torch = env
    m, beta, steps = 14, 100.0, 10
    plan = mm.HermitePlan(ctx, [m] * 3, prec=prec)
    xo, _, Wo = orc.gauss_hermite(m)
    w3 = orc.weight3(Wo)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    p0 = inputs.gpe_psi0(xo, Wo, seed=4)
    p0 = p0 if prec == "fp64" else p0.astype(np.complex64)
    target = inputs.gpe_target(xo, Wo)

    def case(tau):
        pT = orc.gpe_steps(p0.astype(complex), xo, Wo, beta, tau, steps)
        gT = 2.0 * w3 * (pT - target)
        g0 = plan.gpe_adjoint(to_gpu(torch, p0, dt), to_gpu(torch, gT, dt), beta, tau, steps, ckpt_every=3)
        ref = orc.gpe_adjoint(p0.astype(complex), gT, xo, Wo, beta, tau, steps)
        return g0.cpu().numpy(), ref

    tol = 1e-10 if prec == "fp64" else 5e-7  # F16X6 measured 2.3e-7 and 2.5e-7
    ga, ref_a = case(1e-3)
    gb, _ = case(1e-3)
    assert np.array_equal(ga.view(np.float64 if prec == "fp64" else np.float32),
                          gb.view(np.float64 if prec == "fp64" else np.float32))
    gc, ref_c = case(2e-3)
    gd, _ = case(1e-3)
    print(f"adjoint repeated {prec}: rel_err tau=1e-3 {rel(ga, ref_a):.3e}, tau=2e-3 {rel(gc, ref_c):.3e}")
    assert rel(ga, ref_a) <= tol and rel(gc, ref_c) <= tol
    assert np.array_equal(ga.view(np.float64 if prec == "fp64" else np.float32),
                          gd.view(np.float64 if prec == "fp64" else np.float32))
    ctx.status()


def test_gpe_autograd_gradient(env, orc):
    """torch.autograd through gpe_evolve gives the oracle's gradient of
    J = sum |psi_T - target|^2 W."""
    mm, ctx, torch = env
    m, beta, tau, steps = 10, 100.0, 1e-3, 6
    plan = mm.HermitePlan(ctx, [m] * 3, prec="fp64")
    xo, _, Wo = orc.gauss_hermite(m)
    w3 = torch.from_numpy(orc.weight3(Wo)).cuda()
    psi0 = inputs.gpe_psi0(xo, Wo, seed=4)
    target = torch.from_numpy(inputs.gpe_target(xo, Wo)).cuda()
    p = torch.from_numpy(psi0).cuda().requires_grad_(True)
    pT = mm.gpe_evolve(plan, p, beta, tau, steps, ckpt_every=4)
    J = (torch.abs(pT - target) ** 2 * w3).sum()
    J.backward()
    pTo = orc.gpe_steps(psi0, xo, Wo, beta, tau, steps)
    ref = orc.gpe_adjoint(psi0, 2.0 * orc.weight3(Wo) * (pTo - inputs.gpe_target(xo, Wo)), xo, Wo, beta, tau, steps)
    assert rel(p.grad.cpu().numpy(), ref) <= 1e-10


# ------------------------------------------------------- batched uneven problems

def test_batched_uneven_problems(env, orc, monkeypatch):
    """Independent problems of uneven sizes (48..160 per direction) stepped
    in one launch per direction: identical to stepping each plan alone, and
    within tolerance of the oracle.  (A batch folds wherever its plans can;
    the plans alone fold every call here too.)"""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_FOLD_ALWAYS", "1")
    dims = inputs.batched_dims(count=64, seed=3)[:6]
    us0 = inputs.batched_u0(inputs.batched_dims(count=64, seed=3), seed=3)[:6]
    tau, steps = 1e-4, 3
    plans, us, alone = [], [], []
    for (n1, n2, n3), u0 in zip(dims, us0):
        nd = (int(n1), int(n2), int(n3))
        Es = [fd_schrodinger_E(mm, n, tau) for n in nd]
        plans.append(mm.TuckerPlan(ctx, nd, Es, prec="f16x6"))
        us.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
        alone.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
    batch = mm.Batch(ctx, plans)
    batch.step(us, steps)
    for p, u in zip(plans, alone):
        p.step(u, steps)
    torch.cuda.synchronize()
    for k in range(len(plans)):
        assert torch.equal(us[k], alone[k]), k
    for k in (0, len(plans) - 1):
        nd = tuple(int(v) for v in dims[k])
        ref = orc.tucker(us0[k].astype(np.complex64).astype(complex),
                         [orc.expm_dirichlet_fd(n, 1j * tau) for n in nd], nsteps=steps)
        assert rel(us[k].cpu().numpy(), ref) <= TOL_MODE["f16x6"] * 3 * steps


# ------------------------------------------------------- AUTO precision, one-call batch

def test_auto_precision_resolves(env):
    """MM_PREC_AUTO picks F16X6 for complex64 data within the tensor-core
    sizes and FP64 on the tensor cores for complex128: the results equal
    those precisions bit for bit."""
    mm, ctx, torch = env
    dims, tau = (48, 40, 32), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2)
    for dt, concrete in ((torch.complex64, "f16x6"), (torch.complex128, "fp64dmma")):
        out = []
        for prec in ("auto", concrete):
            plan = mm.TuckerPlan(ctx, dims, Es, prec=prec, dtype=dt)
            plan.set_graphs(False)
            u = to_gpu(torch, u0, dt)
            plan.step(u, 2)
            out.append(u)
        torch.cuda.synchronize()
        assert torch.equal(out[0], out[1]), concrete



def test_tensor_core_size_limit(env, orc):
    """n_mu = 513 is past the tensor-core range (row tiles cover at most 512
    rows): an explicit tensor-core precision is refused with MM_ERR_SHAPE
    before any launch, and MM_PREC_AUTO falls back to FP32 on CUDA cores,
    which still agrees with the oracle."""
    mm, ctx, torch = env
    dims, tau = (513, 3, 2), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    with pytest.raises(RuntimeError, match="512"):
        mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="auto")
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, 2)
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=2)
    assert rel(u.cpu().numpy(), ref) <= TOL_STEP["fp32"]
    ctx.status()


@pytest.mark.parametrize("prec", ["f16x6", "fp64"])
def test_degenerate_inputs(env, orc, prec):
    """Degenerate cases of the Tucker step: zero steps leave u untouched (bit
    for bit); size-1 directions (the product is a scalar factor there) agree
    with the oracle; an all-zero state stays exactly zero with a clean device
    status (the fixed-point scale of a zero maximum); a direction of size 0
    is refused with MM_ERR_SHAPE."""
    mm, ctx, torch = env
    tau = 1e-4
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    tol = 1e-12 if prec == "fp64" else TOL_STEP["f16x6"]
    for dims in ((1, 40, 24), (40, 1, 24), (33, 20, 1), (1, 1, 1)):
        Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
        u0 = inputs.complex_normal(dims[::-1], seed=7)
        u0 = u0 if prec == "fp64" else u0.astype(np.complex64)
        plan = mm.TuckerPlan(ctx, dims, Es, prec=prec, dtype=dt)
        u = to_gpu(torch, u0, dt)
        plan.step(u, 0)
        torch.cuda.synchronize()
        assert np.array_equal(u.cpu().numpy(), u0), dims
        plan.step(u, 3)
        ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=3)
        err = rel(u.cpu().numpy(), ref)
        print(f"degenerate {prec} dims={dims}: rel_err={err:.3e}")
        assert err <= tol, dims
        z = torch.zeros_like(u)
        plan.step(z, 2)
        torch.cuda.synchronize()
        assert not torch.any(z != 0), dims
        ctx.status()
    Es = [fd_schrodinger_E(mm, n, tau) for n in (4, 4)]
    with pytest.raises(RuntimeError, match="MM_ERR_SHAPE"):
        mm.TuckerPlan(ctx, (0, 4, 4), [np.zeros((0, 0))] + Es, prec=prec, dtype=dt)


@pytest.mark.parametrize("dims", [(37,), (21, 9), (13, 10, 7)])
def test_state_not_16_byte_aligned(env, dims):
    """The ABI requires 16-byte aligned states: one that starts 8 bytes past
    a boundary (a contiguous slice one element into a buffer) is refused with
    MM_ERR_ALIGN before any launch, and the buffer is left as it was; an
    aligned copy steps normally."""
    mm, ctx, torch = env
    tau = 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    count = int(np.prod(dims))
    u0 = inputs.complex_normal(dims[::-1], seed=11).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    buf = torch.zeros(count + 1, dtype=torch.complex64, device="cuda")
    off = buf[1:].view(*dims[::-1])
    assert off.data_ptr() % 16 == 8 and off.is_contiguous()
    off.copy_(torch.from_numpy(u0).cuda())
    with pytest.raises(RuntimeError, match="MM_ERR_ALIGN"):
        plan.step(off, 3)
    torch.cuda.synchronize()
    assert np.array_equal(off.cpu().numpy(), u0) and buf[0].item() == 0
    ali = torch.from_numpy(u0).cuda()
    plan.step(ali, 3)
    torch.cuda.synchronize()
    assert not np.array_equal(ali.cpu().numpy(), u0)
    ctx.status()

def test_batched_pair_kernel_matches_one_sm_batch(env, monkeypatch):
    """Batched launches run the CTA-pair kernel over the problem records; the
    older one-SM-style batched kernel (forced with MM_TC_1SM=1 at batch
    creation) gives the same bits."""
    mm, ctx, torch = env
    dims = inputs.batched_dims(count=64, seed=3)[:6]
    us0 = inputs.batched_u0(inputs.batched_dims(count=64, seed=3), seed=3)[:6]
    tau, steps = 1e-4, 3
    plans, a, b = [], [], []
    for (n1, n2, n3), u0 in zip(dims, us0):
        nd = (int(n1), int(n2), int(n3))
        plans.append(mm.TuckerPlan(ctx, nd, [fd_schrodinger_E(mm, n, tau) for n in nd], prec="f16x6"))
        a.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
        b.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
    mm.Batch(ctx, plans).step(a, steps)
    monkeypatch.setenv("MM_TC_1SM", "1")
    mm.Batch(ctx, plans).step(b, steps)
    monkeypatch.delenv("MM_TC_1SM")
    torch.cuda.synchronize()
    for k in range(len(plans)):
        assert torch.equal(a[k], b[k]), k


def test_step_batched_one_call(env):
    """mumode_step_batched (the batch made and released in the call) equals
    a kept batch object."""
    mm, ctx, torch = env
    dims = inputs.batched_dims(count=64, seed=3)[:4]
    us0 = inputs.batched_u0(inputs.batched_dims(count=64, seed=3), seed=3)[:4]
    tau, steps = 1e-4, 2
    plans, a, b = [], [], []
    for (n1, n2, n3), u0 in zip(dims, us0):
        nd = (int(n1), int(n2), int(n3))
        plans.append(mm.TuckerPlan(ctx, nd, [fd_schrodinger_E(mm, n, tau) for n in nd], prec="f16x6"))
        a.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
        b.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
    mm.step_batched(ctx, plans, a, steps)
    mm.Batch(ctx, plans).step(b, steps)
    torch.cuda.synchronize()
    for k in range(len(plans)):
        assert torch.equal(a[k], b[k]), k


# ------------------------------------------------------------------ autotuner

def test_batch_autotune(env, orc):
    """mumode_batch_autotune sets one mode order on every plan of a batch,
    leaves the states unchanged, and the tuned batch matches the oracle in
    that order."""
    mm, ctx, torch = env
    dims = inputs.batched_dims(count=64, seed=3)[:3]
    us0 = inputs.batched_u0(inputs.batched_dims(count=64, seed=3), seed=3)[:3]
    tau, steps = 1e-4, 2
    plans, us = [], []
    for (n1, n2, n3), u0 in zip(dims, us0):
        nd = (int(n1), int(n2), int(n3))
        plans.append(mm.TuckerPlan(ctx, nd, [fd_schrodinger_E(mm, n, tau) for n in nd], prec="f16x6"))
        us.append(to_gpu(torch, u0.astype(np.complex64), torch.complex64))
    before = [u.clone() for u in us]
    order = mm.batch_autotune(ctx, plans, us, nsteps=2)
    torch.cuda.synchronize()
    assert sorted(order) == [1, 2, 3]
    for p, u, b in zip(plans, us, before):
        assert p.config()[1] == order
        assert torch.equal(u, b)
    mm.Batch(ctx, plans).step(us, steps)
    for (n1, n2, n3), u0, u in zip(dims, us0, us):
        nd = (int(n1), int(n2), int(n3))
        ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in nd], order=order,
                         nsteps=steps)
        assert rel(u.cpu().numpy(), ref) <= TOL_MODE["f16x6"] * 6
    hp = mm.HermitePlan(ctx, [32] * 3, prec="f16x6")
    with pytest.raises(mm.MumodeError):
        mm.batch_autotune(ctx, [plans[0], hp], us[:2], nsteps=1)
    ctx.status()


def test_autotune_tucker(env, orc):
    """mm_plan_autotune times the kernel variants and the mode orders on a
    copy of the state and keeps the fastest: the given state is unchanged,
    the chosen configuration is valid, and the tuned plan matches the
    oracle in its order."""
    mm, ctx, torch = env
    dims, tau = (64, 96, 32), 1e-4
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    assert plan.config() == ("pair64", (1, 2, 3))
    u = to_gpu(torch, u0, torch.complex64)
    before = u.clone()
    variant, order = plan.autotune(u, nsteps=2)
    torch.cuda.synchronize()
    assert torch.equal(u, before)
    assert variant in mm.VARIANTS and sorted(order) == [1, 2, 3]
    plan.step(u, 2)
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], order=order, nsteps=2)
    assert rel(u.cpu().numpy(), ref) <= TOL_MODE["f16x6"] * 6
    plan.set_config("one_sm", (3, 1, 2))
    assert plan.config() == ("one_sm", (3, 1, 2))
    L = mm.lib()
    assert L.mm_plan_set_config(plan.handle, 5, None) == 1  # MM_ERR_INVALID_ARG
    bad = (mm._i * 3)(1, 1, 2)
    assert L.mm_plan_set_config(plan.handle, 0, bad) == 1
    ctx.status()


def test_gpe_autotune(env, orc):
    """split_step_gpe_autotune keeps psi, picks a variant, and the tuned plan
    still matches the oracle's Strang steps."""
    mm, ctx, torch = env
    m, beta, tau, steps = 16, 100.0, 1e-3, 6
    plan = mm.HermitePlan(ctx, [m] * 3, prec="f16x6")
    xo, _, Wo = orc.gauss_hermite(m)
    psi0 = inputs.gpe_psi0(xo, Wo, seed=4).astype(np.complex64)
    psi = to_gpu(torch, psi0, torch.complex64)
    before = psi.clone()
    variant, _ = plan.gpe_autotune(psi, beta, tau, nsteps=2)
    torch.cuda.synchronize()
    assert torch.equal(psi, before) and variant in mm.VARIANTS
    plan.gpe_step(psi, beta, tau, steps)
    ref = orc.gpe_steps(psi0.astype(complex), xo, Wo, beta, tau, steps)
    assert orc.rel_l2(psi.cpu().numpy(), ref, orc.weight3(Wo)) <= 1e-5


@pytest.mark.parametrize("dims,mixed", [((64, 48, 40), False), ((33, 40, 17), False), ((33, 40, 17), True),
                                         ((300,), False), ((24, 20, 18, 16), False), ((256, 32, 31), True)])
def test_fold_matches_unfolded(env, orc, monkeypatch, dims, mixed):
    """Even/odd folding of a Tucker plan (centrosymmetric matrices run as block-diagonal products on
    the folded state, folded and unfolded once per call) gives the unfolded plan's result to the
    precision's tolerance, and the oracle's: even and odd sizes, d = 1 to 4, and plans where one
    direction's matrix is not centrosymmetric (that direction stays unfolded)."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_FOLD_ALWAYS", "1")  # fold every call, also where it would not pay
    tau, steps = 1e-4, 3
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    if mixed:  # the last direction: a random unitary matrix, not centrosymmetric
        rng = np.random.default_rng(11)
        n = dims[-1]
        Es[-1] = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    u0 = inputs.complex_normal(dims[::-1], seed=6).astype(np.complex64)
    out = {}
    for fold in (True, False):
        if fold:
            monkeypatch.delenv("MM_NO_FOLD", raising=False)
        else:
            monkeypatch.setenv("MM_NO_FOLD", "1")
        plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
        u = to_gpu(torch, u0, torch.complex64)
        plan.step(u, steps)
        torch.cuda.synchronize()
        ctx.status()
        out[fold] = u.cpu().numpy()
    monkeypatch.delenv("MM_NO_FOLD", raising=False)
    # the folded directions, and folding turned off on the plan: the unfolded plan's bits
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    want = sum(1 << v for v, n in enumerate(dims) if n > 1 and not (mixed and v == len(dims) - 1))
    assert plan.fold() == want
    plan.set_fold(False)
    assert plan.fold() == 0
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, steps)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy().view(np.uint32), out[False].view(np.uint32))
    plan.set_fold(True)
    assert plan.fold() == want
    d = rel(out[True], out[False])
    ora = orc.tucker(u0.astype(complex), [np.asarray(E, dtype=complex) for E in Es], nsteps=steps)
    print(f"fold vs unfolded dims={dims} mixed={mixed}: {d:.3e}; vs oracle {rel(out[True], ora):.3e}")
    assert d <= TOL_MODE["f16x6"] * steps * len(dims)
    assert rel(out[True], ora) <= TOL_MODE["f16x6"] * steps * len(dims)


@pytest.mark.parametrize("dims", [(64, 48, 40), (33, 40, 17)])
@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16", "tf32x3"])
def test_fold_other_precisions(env, orc, monkeypatch, dims, prec):
    """Folded steps in the other tensor-core precisions (floating BF16 pieces, TF32 pieces) match
    the oracle to the precision's tolerance, as the unfolded ones do."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_FOLD_ALWAYS", "1")
    tau, steps = 1e-4, 2
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec=prec)
    assert plan.fold() == 7
    u = to_gpu(torch, u0, torch.complex64)
    plan.step(u, steps)
    torch.cuda.synchronize()
    ctx.status()
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=steps)
    err = rel(u.cpu().numpy(), ref)
    print(f"folded {prec} dims={dims}: {err:.3e}")
    tol = {"bf16x6": TOL_MODE["bf16x6"] * steps * len(dims), "bf16x3": TOL_STEP["bf16x3"], "bf16": TOL_STEP["bf16"],
           "tf32x3": TOL_STEP["tf32x3"]}[prec]
    assert err <= tol


@pytest.mark.parametrize("m", [24, 25])
def test_ho_fold_matches_unfolded(env, orc, monkeypatch, m):
    """Harmonic-oscillator steps of a Hermite plan run folded (the values-space propagators at
    the symmetric Gauss-Hermite nodes are centrosymmetric): the result equals the unfolded
    plan's to the precision's tolerance, for an even and an odd number of nodes.  GPE steps on
    the same plan run folded too, with the nonlinear phase as a pass on the folded pieces between
    the sweeps: they match the unfolded plan and the oracle; the steps that also return the
    weighted norm sum it in the final unfold, and it equals the norm of the state they return."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_FOLD_ALWAYS", "1")
    tau, steps = 0.05, 4
    beta, gtau, gsteps = 100.0, 1e-3, 6
    psi0 = inputs.complex_normal((m, m, m), seed=9).astype(np.complex64)
    xo, _, Wo = orc.gauss_hermite(m)
    g0 = inputs.gpe_psi0(xo, Wo, seed=4).astype(np.complex64)
    out, gpe, gnorm, nret, nsep = {}, {}, {}, {}, {}
    for fold in (True, False):
        if fold:
            monkeypatch.delenv("MM_NO_FOLD", raising=False)
        else:
            monkeypatch.setenv("MM_NO_FOLD", "1")
        hp = mm.HermitePlan(ctx, [m] * 3, prec="f16x6")
        u = to_gpu(torch, psi0, torch.complex64)
        hp.ho_step(u, tau, steps)
        g = to_gpu(torch, g0, torch.complex64)
        hp.gpe_step(g, beta, gtau, gsteps)
        gn = to_gpu(torch, g0, torch.complex64)
        nret[fold] = hp.gpe_step_norm2(gn, beta, gtau, gsteps)
        nsep[fold] = hp.norm2(gn)
        torch.cuda.synchronize()
        ctx.status()
        out[fold], gpe[fold], gnorm[fold] = u.cpu().numpy(), g.cpu().numpy(), gn.cpu().numpy()
    monkeypatch.delenv("MM_NO_FOLD", raising=False)
    d = rel(out[True], out[False])
    print(f"HO fold vs unfolded m={m}: {d:.3e}")
    assert d <= TOL_MODE["f16x6"] * steps * 3
    ref = orc.gpe_steps(g0.astype(complex), xo, Wo, beta, gtau, gsteps)
    w3 = orc.weight3(Wo)
    e_fold, e_unf = orc.rel_l2(gpe[True], ref, w3), orc.rel_l2(gpe[False], ref, w3)
    print(f"GPE fold m={m}: {e_fold:.3e} against the oracle (unfolded {e_unf:.3e})")
    assert e_fold <= 1e-6 and rel(gpe[True], gpe[False]) <= 2e-6
    assert not np.array_equal(gpe[True].view(np.uint32), gpe[False].view(np.uint32)), "the GPE steps ran folded"
    assert np.array_equal(gnorm[True].view(np.uint32), gpe[True].view(np.uint32))
    assert np.array_equal(gnorm[False].view(np.uint32), gpe[False].view(np.uint32))
    # the unfold sums the complex64 values it writes (|psi|^2 in FP32, times the FP64 weight, the
    # sum in FP64: 2e-9 here); the unfolded epilogue sums the FP32 values before their split, which
    # the merge rounds (the tolerance of test_gpe_norm_in_epilogue)
    assert abs(nret[True] / nsep[True] - 1) <= 1e-8, (nret[True], nsep[True])
    assert abs(nret[False] / nsep[False] - 1) <= 2e-7, (nret[False], nsep[False])


def _hermite_flow(orc, x, W, s):
    """Values-space harmonic-oscillator flow over time s in one direction, from the oracle's nodes,
    weights and Hermite functions: backward transform, exp(-i s (k + 1/2)), forward transform."""
    H = orc.hermite_functions(x.size, x)
    return H.T @ np.diag(np.exp(-1j * s * (np.arange(x.size) + 0.5))) @ H @ np.diag(W)


def _strang_fp64(orc, psi, xs, Ws, beta, tau, nsteps):
    """FP64 Strang steps of the GPE on a grid of its own size per direction (the oracle's scheme,
    section 4.5, written with per-direction flows; shape (n3, n2, n1))."""
    def flow(u, s):
        P = [_hermite_flow(orc, x, W, s) for x, W in zip(xs, Ws)]
        u = np.einsum("ij,abj->abi", P[0], u)
        u = np.einsum("ij,ajb->aib", P[1], u)
        return np.einsum("ij,jab->iab", P[2], u)

    u = psi.astype(complex)
    for _ in range(nsteps):
        u = flow(u, 0.5 * tau)
        u = u * np.exp(-1j * tau * beta * np.abs(u) ** 2)
        u = flow(u, 0.5 * tau)
    return u


@pytest.mark.parametrize("dims", [(24, 25, 21), (25, 22, 24)])
def test_gpe_fold_mixed_sizes(env, orc, monkeypatch, dims):
    """Folded GPE steps on grids of different, even and odd, sizes per direction: the phase pass
    takes two points a thread when direction 1 has even length (24, 25, 21) and one otherwise
    (25, 22, 24); the result matches an FP64 Strang reference built from the oracle's Hermite
    functions (equal to the oracle's own GPE steps on a cube grid, checked first) and the
    unfolded plan."""
    mm, ctx, torch = env
    monkeypatch.setenv("MM_FOLD_ALWAYS", "1")
    beta, tau, nsteps = 100.0, 1e-3, 5
    x9, _, W9 = orc.gauss_hermite(9)
    p9 = inputs.gpe_psi0(x9, W9, seed=4)
    r9 = orc.gpe_steps(p9, x9, W9, beta, tau, nsteps)
    assert np.max(np.abs(_strang_fp64(orc, p9, [x9] * 3, [W9] * 3, beta, tau, nsteps) - r9)) <= 1e-12
    xs, Ws = [], []
    for n in dims:
        x, _, W = orc.gauss_hermite(n)
        xs.append(x)
        Ws.append(W)
    psi0 = inputs.gpe_psi0_dims(xs, Ws, seed=4).astype(np.complex64)
    out = {}
    for fold in (True, False):
        if fold:
            monkeypatch.delenv("MM_NO_FOLD", raising=False)
        else:
            monkeypatch.setenv("MM_NO_FOLD", "1")
        hp = mm.HermitePlan(ctx, list(dims), prec="f16x6")
        g = to_gpu(torch, psi0, torch.complex64)
        hp.gpe_step(g, beta, tau, nsteps)
        torch.cuda.synchronize()
        ctx.status()
        assert hp.fold() == (7 if fold else 0)  # the propagators (and their folded forms) exist now
        out[fold] = g.cpu().numpy()
    monkeypatch.delenv("MM_NO_FOLD", raising=False)
    ref = _strang_fp64(orc, psi0, xs, Ws, beta, tau, nsteps)
    w3 = Ws[2][:, None, None] * Ws[1][None, :, None] * Ws[0][None, None, :]
    e_fold, e_unf = orc.rel_l2(out[True], ref, w3), orc.rel_l2(out[False], ref, w3)
    print(f"GPE fold dims={dims}: {e_fold:.3e} against FP64 (unfolded {e_unf:.3e})")
    assert e_fold <= 1e-6 and e_unf <= 1e-6
    assert rel(out[True], out[False]) <= 2e-6


def test_autotune_cache(env, orc, tmp_path, monkeypatch):
    """With MM_AUTOTUNE_CACHE set, the first tuning of a plan appends one JSON
    line; a second plan with the same key takes that configuration without
    tuning (no new line; a line edited by hand is taken as written), and a
    plan whose matrices have other k-block bands gets a key of its own."""
    import json

    mm, ctx, torch = env
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("MM_AUTOTUNE_CACHE", str(path))
    dims, tau = (256, 48, 40), 1e-4  # direction 1: a banded propagator (6 to 8 of 16 k-blocks per row tile)
    Es = [fd_schrodinger_E(mm, n, tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    u = to_gpu(torch, u0, torch.complex64)
    cfg = mm.TuckerPlan(ctx, dims, Es, prec="f16x6").autotune(u, nsteps=1)
    lines = path.read_text().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["variant"] == mm.VARIANTS.index(cfg[0]) and tuple(rec["order"]) == cfg[1]
    assert "|tucker|d=256x48x40|" in rec["key"]
    assert mm.TuckerPlan(ctx, dims, Es, prec="f16x6").autotune(u, nsteps=1) == cfg
    assert len(path.read_text().splitlines()) == 1
    # a stored configuration is applied as written
    rec["variant"], rec["order"] = mm.VARIANTS.index("one_sm"), [2, 3, 1]
    path.write_text(json.dumps(rec) + "\n")
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    assert plan.autotune(u, nsteps=1) == ("one_sm", (2, 3, 1))
    plan.step(u, 2)
    ref = orc.tucker(u0.astype(complex), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], order=(2, 3, 1),
                     nsteps=2)
    assert rel(u.cpu().numpy(), ref) <= TOL_MODE["f16x6"] * 6
    # dense matrices of the same sizes: other bands, another key, tuned and appended
    rng = np.random.default_rng(7)
    dense = [np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0] for n in dims]
    mm.TuckerPlan(ctx, dims, dense, prec="f16x6").autotune(u, nsteps=1)
    keys = [json.loads(ln)["key"] for ln in path.read_text().splitlines()]
    assert len(keys) == 2 and keys[0] != keys[1]


def test_autotune_hermite_and_fp64(env):
    """Hermite plans tune the kernel variant only; FP64 plans the mode order."""
    mm, ctx, torch = env
    hp = mm.HermitePlan(ctx, [32] * 3, prec="f16x6")
    psi = torch.randn(32, 32, 32, dtype=torch.complex64, device="cuda")
    v, order = hp.autotune(psi, nsteps=2)
    assert v in mm.VARIANTS and order == (1, 2, 3)
    with pytest.raises(mm.MumodeError):
        hp.set_config("pair64", (2, 1, 3))
    dims = (24, 20, 16)
    p64 = mm.TuckerPlan(ctx, dims, [fd_schrodinger_E(mm, n, 1e-4) for n in dims], prec="fp64dmma")
    u = torch.randn(16, 20, 24, dtype=torch.complex128, device="cuda")
    _, order = p64.autotune(u, nsteps=1)
    assert sorted(order) == [1, 2, 3]
