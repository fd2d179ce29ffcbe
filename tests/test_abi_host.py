"""CPU-only checks of the C-ABI library: it loads, exports every symbol the
header declares, validates arguments without a GPU, and its FP64 host
set-up (FD operator, expm, Gauss-Hermite, Hermite matrices) agrees with the
oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2103_01691_b300 import build as mmbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mm():
    mmbuild.build()
    from paper_2103_01691_b300 import mumode

    mumode.lib()
    return mumode


def header_functions():
    text = open(os.path.join(ROOT, "include", "mumode.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_\w+|mumode_\w+|hermite_\w+|hkp_\w+|hkmp_\w+|pipe_\w+|split_step_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(mm):
    names = header_functions()
    assert len(names) >= 20
    L = ctypes.CDLL(mm.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(mm.SIGNATURES)


def test_argument_errors_without_gpu(mm):
    L = mm.lib()
    assert L.mm_fd_laplacian_dirichlet(0, None) == 2          # MM_ERR_SHAPE
    assert L.mm_fd_laplacian_dirichlet(4, None) == 1          # MM_ERR_INVALID_ARG
    assert L.mm_expm(3, None, None, 1.0, 0.0, None) == 1
    assert L.mm_gauss_hermite(0, None, None) == 2
    assert b"NULL" in L.mm_last_error() or len(L.mm_last_error()) > 0
    assert L.mumode_step(None, None, 1, None) == 1
    assert L.mm_norm2(None, None, 0, None, None) == 1
    assert L.mumode_plan_create(None, 3, None, None, 0, 1, 2, None, None) == 1
    h = ctypes.c_void_p()
    st = L.mm_ctx_create(0, ctypes.byref(h))
    assert st in (0, 1, 6)  # no device here: invalid device or CUDA error, never a crash


def test_fd_laplacian_matches_oracle(mm, orc):
    for n in (1, 5, 32):
        assert np.allclose(mm.fd_laplacian_dirichlet(n), orc.fd_dirichlet(n), rtol=1e-14, atol=0)


@pytest.mark.parametrize("n,z", [(32, 1e-3), (64, 1e-4j), (256, 1e-4j), (257, 1e-4j), (48, 5e-2j), (16, -3e-3)])
def test_expm_pade_matches_oracle_closed_form(mm, orc, n, z):
    E = mm.expm(mm.fd_laplacian_dirichlet(n), z)
    ref = orc.expm_dirichlet_fd(n, z)
    assert np.max(np.abs(E - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_expm_complex_matrix_matches_oracle_taylor(mm, orc):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    assert np.max(np.abs(mm.expm(A, 0.7 + 0.2j) - orc.expm_taylor(A, 0.7 + 0.2j))) < 1e-11


@pytest.mark.parametrize("m", [1, 2, 7, 64, 128, 192, 256])
def test_gauss_hermite_matches_oracle(mm, orc, m):
    x, W = mm.gauss_hermite(m)
    xo, _, Wo = orc.gauss_hermite(m)
    assert np.max(np.abs(x - xo)) < 1e-12 * max(1.0, np.max(np.abs(xo)))
    assert np.max(np.abs(W - Wo) / Wo) < 1e-10


@pytest.mark.parametrize("m", [8, 128, 192])
def test_hermite_matrices_match_oracle(mm, orc, m):
    F, B = mm.hermite_matrices(m)
    xo, _, Wo = orc.gauss_hermite(m)
    H = orc.hermite_functions(m, xo)
    assert np.max(np.abs(B - H.T)) < 1e-11
    assert np.max(np.abs(F - H * Wo)) < 1e-11 * np.max(np.abs(H * Wo))


@pytest.mark.parametrize("m", [1, 16, 96])
def test_hermite_hamiltonian_and_galerkin_match_oracle(mm, orc, m):
    """Host set-up of HKP / HKMP: mm_hermite_hamiltonian against the oracle's."""
    x, _ = mm.gauss_hermite(m)
    xo, _, Wo = orc.gauss_hermite(m)
    H = mm.hermite_hamiltonian(m, np.cos(2 * np.pi * x))
    ref = orc.hkp_hamiltonian(xo, Wo, np.cos(2 * np.pi * xo))
    assert np.max(np.abs(H - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n_r,n_z", [(2, 3), (17, 40), (128, 96)])
def test_pipe_operators_match_oracle(mm, orc, n_r, n_z):
    from paper_2103_01691_b300 import inputs

    P = inputs.PIPE
    z = P["zmax"] / n_z * np.arange(1, n_z + 1)
    s = inputs.pipe_velocity(z)
    Ar, Az = mm.pipe_operators(n_r, n_z, P["rmin"], P["rmax"], P["zmax"], P["alpha"], s)
    ref_r = orc.pipe_radial(n_r, P["rmin"], P["rmax"], P["alpha"])
    ref_z = orc.pipe_axial(n_z, P["zmax"], P["alpha"], s)
    assert np.max(np.abs(Ar - ref_r)) <= 1e-13 * np.max(np.abs(ref_r))
    assert np.max(np.abs(Az - ref_z)) <= 1e-13 * np.max(np.abs(ref_z))
    L = mm.lib()
    assert L.mm_pipe_operators(1, 4, 0.1, 5.0, 8.0, 0.01, None, None, None) == 2  # MM_ERR_SHAPE
    assert L.mm_pipe_operators(4, 4, 0.0, 5.0, 8.0, 0.01, None, None, None) == 1  # r_min must be > 0


def test_new_entry_points_reject_bad_arguments_without_gpu(mm):
    """HKP, HKMP, pipe flow, device exponentials and device matrices validate
    their arguments before touching the device."""
    L = mm.lib()
    n3 = (ctypes.c_int64 * 3)(8, 8, 8)
    out = ctypes.c_void_p()
    assert L.hkp_plan_create(None, 3, n3, None, 1.0, 1, 5, None, ctypes.byref(out)) == 1
    assert L.hkmp_plan_create(None, 3, n3, None, None, 0.1, 1, 5, ctypes.byref(out)) == 1
    assert L.hkmp_evolve(None, None, 1, None, None) == 1
    assert L.pipe_plan_create(None, 8, 8, 0.1, 5.0, 8.0, 0.01, None, 4.0, 6, ctypes.byref(out)) == 1
    assert L.mm_expm_device(None, 4, None, None, 0.0, 1.0, 0.0, 0.0, None, None) == 1
    assert L.mm_plan_set_matrix_device(None, 1, None, 0.0, None) == 1
    assert L.mm_hermite_hamiltonian(0, None, None) == 2
    assert L.mm_hermite_hamiltonian(4, None, None) == 1
    assert L.mumode_batch_autotune(None, None, None, 0, 1, None, None) == 1
    H = np.empty((5, 5))
    assert L.mm_hermite_hamiltonian(5, None, H.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
    assert np.array_equal(H, np.diag(np.arange(5) + 0.5))
