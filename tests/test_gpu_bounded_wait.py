"""Bounded device waits: a wait that runs out ends the launch with
MM_ERR_TIMEOUT in the context's error word, and the context stays usable.

Every mbarrier wait in the tensor-core kernels gives up after a limit of SM
clocks.  MM_WAIT_LIMIT_CYCLES shortens that limit to 1e5 clocks (about 50
microseconds) and MM_WITHHOLD_STAGE makes the producers of every CTA skip the
loads of one stage (and the arrival that announces them), so the MMA issuer's
wait for that stage can never be satisfied.  The launch must end by itself,
report MM_ERR_TIMEOUT, and a following product on the same context and plan
must match the oracle.  No kernel is made to fault: the failure is a wait
that nothing satisfies, with a limit."""
import numpy as np
import pytest

from paper_2103_01691_b300 import inputs

pytestmark = pytest.mark.gpu

MM_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2103_01691_b300 import build as mmbuild

    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    ctx = mumode.Context(0)
    yield mumode, ctx, torch
    ctx.status()


@pytest.mark.parametrize("variant", ["pair64", "one_sm"])
def test_wait_that_runs_out_reports_timeout(env, orc, monkeypatch, variant):
    mm, ctx, torch = env
    dims, tau = (64, 48, 40), 1e-4
    Es = [mm.expm(mm.fd_laplacian_dirichlet(n), 1j * tau) for n in dims]
    u0 = inputs.complex_normal(dims[::-1], seed=2).astype(np.complex64)
    plan = mm.TuckerPlan(ctx, dims, Es, prec="f16x6")
    plan.set_graphs(False)
    plan.set_config(variant)
    ctx.status()  # nothing pending from earlier tests

    monkeypatch.setenv("MM_WAIT_LIMIT_CYCLES", "100000")
    monkeypatch.setenv("MM_WITHHOLD_STAGE", "1")
    u = torch.from_numpy(u0).cuda()
    plan.step(u, 1)
    with pytest.raises(mm.MumodeError) as info:
        ctx.status()
    assert info.value.status == MM_ERR_TIMEOUT
    monkeypatch.delenv("MM_WITHHOLD_STAGE")
    monkeypatch.delenv("MM_WAIT_LIMIT_CYCLES")
    ctx.status()  # the error word was cleared by the read above

    # the same plan and context, normal waits: a correct step
    u = torch.from_numpy(u0).cuda()
    plan.step(u, 2)
    ctx.status()
    ref = orc.tucker(u0.astype(np.complex128), [orc.expm_dirichlet_fd(n, 1j * tau) for n in dims], nsteps=2)
    got = u.cpu().numpy().astype(np.complex128)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print(f"{variant}: timeout reported; next step rel_err={err:.3e}")
    assert err <= 1.5e-7 * 2 * len(dims)
