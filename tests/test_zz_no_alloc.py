"""mumode_product_noalloc: the F16X6 mu-mode product for callers that cannot
allocate device memory (for example code under a framework whose caching
allocator owns the GPU's memory, or a plugin whose host forbids device
allocation).  It keeps its temporaries in the library's fixed 64 MiB static
device scratch.  The GPU tests check it, through the C ABI, against the
allocating entry point mumode_product on consecutive calls, at a small
ragged shape and at 128^3 (near the scratch limit); the CPU tests check that
products beyond the limit are rejected before anything runs.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_2103_01691_b300 import build as mmbuild
from paper_2103_01691_b300 import inputs

TOL = 1.5e-7  # per mode product, the F16X6 tolerance of the parity tests
SCRATCH = 64 << 20


def _r16(v):
    return (v + 15) // 16 * 16


def _r256(v):
    return (v + 255) // 256 * 256


def _scratch_need(dims, mu, m):
    """Bytes of static scratch one product takes: 256 status bytes, the matrix pieces (3 pieces,
    C and S blocks, FP16), the row scales, and 3 pieces x 2 planes x FP16 of the padded input and
    output states."""
    nmu = dims[mu - 1]
    k_pad, m_pad = _r16(nmu), _r16(m)
    ni = (m_pad + 127) // 128
    it = _r16((m_pad + ni - 1) // ni)
    pin = int(np.prod([_r16(v) for v in dims]))
    pout = int(np.prod([_r16(m if v == mu - 1 else dims[v]) for v in range(len(dims))]))
    return 256 + _r256(3 * ni * 2 * it * k_pad * 2) + _r256(ni * it * 4) + _r256(pin * 12) + _r256(pout * 12)


def _call_noalloc(dims, mu, m):
    from paper_2103_01691_b300 import mumode

    L = mumode.lib()
    n = np.array(dims, dtype=np.int64)
    mat = np.eye(m, dims[mu - 1])
    # the pointers are never dereferenced: the size check comes before any device work
    return L, L.mumode_product_noalloc(len(dims), n.ctypes.data_as(mumode._i64p), mu, mat.ctypes.data_as(mumode._dp),
                                       m, 0, ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 40), None)


def test_oversized_product_is_rejected():
    mmbuild.build()
    # 256^3 points need ~400 MB of scratch: rejected with MM_ERR_SHAPE (2)
    L, st = _call_noalloc((256, 256, 256), 1, 256)
    assert st == 2
    assert b"scratch" in L.mm_last_error()


def test_product_just_over_the_limit_is_rejected():
    mmbuild.build()
    # 128 x 128 x k: the smallest k (a multiple of 16) whose product no longer fits
    k = 128
    while _scratch_need((128, 128, k), 3, k) <= SCRATCH:
        k += 16
    assert _scratch_need((128, 128, k - 16), 3, k - 16) <= SCRATCH < _scratch_need((128, 128, k), 3, k)
    L, st = _call_noalloc((128, 128, k), 3, k)
    assert st == 2 and b"scratch" in L.mm_last_error()


def test_huge_sizes_do_not_wrap_the_size_check():
    mmbuild.build()
    # seven directions of 2^24: the padded point count overflows int64 if multiplied out
    L, st = _call_noalloc((16,) + (1 << 24,) * 7, 1, 16)
    assert st == 2 and b"scratch" in L.mm_last_error()


def _compare(ctx, dims, calls, seed):
    import torch

    from paper_2103_01691_b300 import mumode

    rng = np.random.default_rng(seed)
    u0 = inputs.complex_normal(dims[::-1], seed=9).astype(np.complex64)
    u = torch.from_numpy(u0).cuda()
    for mu, m, cplx in calls:
        Lm = rng.standard_normal((m, dims[mu - 1]))
        if cplx:
            Lm = Lm + 1j * rng.standard_normal(Lm.shape)
        ref = mumode.mumode_product(ctx, u, mu, Lm, prec="f16x6")
        got = mumode.mumode_product_noalloc(u, mu, Lm)
        torch.cuda.synchronize()
        r = ref.cpu().numpy().astype(np.complex128)
        g = got.cpu().numpy().astype(np.complex128)
        assert g.shape == r.shape
        assert np.linalg.norm(g - r) <= TOL * np.linalg.norm(r), (dims, mu, m)


@pytest.mark.gpu
def test_noalloc_matches_allocating_product():
    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    ctx = mumode.Context(0)
    # three calls in a row on a ragged shape: rectangular, real and complex matrices
    _compare(ctx, (48, 40, 36), [(2, 40, True), (3, 30, False), (1, 48, True)], seed=31)
    ctx.status()


@pytest.mark.gpu
def test_noalloc_near_the_scratch_limit():
    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    dims = (128, 128, 128)
    assert _scratch_need(dims, 2, 128) <= SCRATCH
    ctx = mumode.Context(0)
    # two calls in a row at 128^3: the second reuses the scratch the first left behind
    _compare(ctx, dims, [(2, 128, True), (3, 128, True)], seed=32)
    ctx.status()
