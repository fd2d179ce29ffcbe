"""mumode_product_noalloc: the F16X6 mu-mode product for callers that cannot
allocate device memory (for example code under a framework whose caching
allocator owns the GPU's memory, or a plugin whose host forbids device
allocation).  It keeps its temporaries in the library's fixed 64 MiB static
device scratch.  The GPU test checks it, through the C ABI, against the
allocating entry point mumode_product on two calls in a row; the CPU test
checks that an oversized product is rejected before anything runs.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_2103_01691_b300 import build as mmbuild
from paper_2103_01691_b300 import inputs

TOL = 1.5e-7  # per mode product, the F16X6 tolerance of the parity tests


def test_oversized_product_is_rejected():
    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    L = mumode.lib()
    dims = (np.array([256, 256, 256], dtype=np.int64))
    mat = np.eye(256)
    # 256^3 points need ~400 MB of scratch: rejected with MM_ERR_SHAPE before any device work
    st = L.mumode_product_noalloc(3, dims.ctypes.data_as(mumode._i64p), 1, mat.ctypes.data_as(mumode._dp), 256, 0,
                                  ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 40), None)
    assert st == 2
    assert b"scratch" in L.mm_last_error()


@pytest.mark.gpu
def test_noalloc_matches_allocating_product():
    import torch

    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    ctx = mumode.Context(0)
    dims = (48, 40, 36)
    rng = np.random.default_rng(31)
    u0 = inputs.complex_normal(dims[::-1], seed=9).astype(np.complex64)
    u = torch.from_numpy(u0).cuda()
    calls = [(2, 40, True), (3, 30, False), (1, 48, True)]  # (mu, m, complex matrix)
    for mu, m, cplx in calls[:2] + calls[2:]:
        Lm = rng.standard_normal((m, dims[mu - 1]))
        if cplx:
            Lm = Lm + 1j * rng.standard_normal(Lm.shape)
        ref = mumode.mumode_product(ctx, u, mu, Lm, prec="f16x6")
        got = mumode.mumode_product_noalloc(u, mu, Lm)
        torch.cuda.synchronize()
        r = ref.cpu().numpy().astype(np.complex128)
        g = got.cpu().numpy().astype(np.complex128)
        assert g.shape == r.shape
        assert np.linalg.norm(g - r) <= TOL * np.linalg.norm(r), (mu, m)
    ctx.status()
