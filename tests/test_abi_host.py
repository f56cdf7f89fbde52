"""CPU-only checks of the C ABI: the library builds, loads, exports every symbol
that include/sbsolve.h declares, and rejects bad arguments on the host before
touching a GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sb():
    from paper_2107_05395_gb300 import build
    build.build()
    import paper_2107_05395_gb300 as pkg
    return pkg


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(sb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sb_factor_shared_tri", "sb_factor_shared_penta", "sb_solve_batched",
                 "sb_solve_batched_adjoint", "sb_factor_destroy", "sb_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(sb):
    L = ctypes.CDLL(sb._lib.LIB_PATH)
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol(sb):
    assert set(sb.SIGNATURES) == declared_functions()


def test_version_string(sb):
    assert "sm_103a" in sb.sb_version()


def test_factor_rejects_bad_sizes(sb):
    L = sb.lib()
    h = ctypes.c_void_p()
    z = np.zeros(1)
    p = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.sb_factor_shared_tri(0, p, p, p, ctypes.byref(h)) == sb.SB_ERR_INVALID_ARG
    assert "N must be >= 1" in sb.sb_last_error()
    assert L.sb_factor_shared_tri(1, None, p, p, ctypes.byref(h)) == sb.SB_ERR_INVALID_ARG
    assert L.sb_factor_shared_tri(1, p, p, p, None) == sb.SB_ERR_INVALID_ARG


def test_factor_rejects_non_finite_entries(sb):
    a = np.array([0.0, 1.0, 1.0])
    b = np.array([4.0, np.nan, 4.0])
    c = np.array([1.0, 1.0, 0.0])
    with pytest.raises(sb.SbError) as ei:
        sb.sb_factor_shared_tri(a, b, c)
    assert ei.value.code == sb.SB_ERR_INVALID_ARG


def test_factor_reports_singular_pivot_row(sb):
    # [[1, 1, 0], [1, 1, 1], [0, 1, 3]]: the second pivot is 1 - 1*1 = 0
    with pytest.raises(sb.SbError) as ei:
        sb.sb_factor_shared_tri([0.0, 1.0, 1.0], [1.0, 1.0, 3.0], [1.0, 1.0, 0.0])
    assert ei.value.code == sb.SB_ERR_SINGULAR and "row 1" in str(ei.value)
    z = np.zeros(4)
    with pytest.raises(sb.SbError) as ei:
        sb.sb_factor_shared_penta(z, z, np.array([2.0, 0.0, 1.0, 1.0]), z, z)
    assert ei.value.code == sb.SB_ERR_SINGULAR and "row 1" in str(ei.value)


def test_solve_rejects_null_factor(sb):
    L = sb.lib()
    assert L.sb_solve_batched(None, None, None, 1, 1, 0, None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_solve_batched_adjoint(None, None, None, 1, 1, 0, None) == sb.SB_ERR_INVALID_ARG


def test_no_device_fails_loudly_without_fallback(sb):
    """On a machine with no GPU a valid factorisation must fail with SB_ERR_CUDA
    (nothing is computed on the CPU instead)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sb.SbError) as ei:
        sb.sb_factor_shared_tri([0.0, -1.0], [2.0, 2.0], [-1.0, 0.0])
    assert ei.value.code in (sb.SB_ERR_CUDA, sb.SB_ERR_ALLOC)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 17, 256])
@pytest.mark.parametrize("kind", ["diffusion", "hinged", "truncated", "ch_noflux"])
def test_product_matrix_builder_matches_oracle(sb, kind, N):
    """The library builds its workload matrices itself (host code, no GPU); they must
    equal the oracle's independently assembled matrices."""
    from oracle import matrices
    coef = 0.37
    mine = sb.sb_build_matrix(kind, N, coef)
    ref = {"diffusion": lambda: matrices.diffusion_matrix(N, coef),
           "hinged": lambda: matrices.hyperdiffusion_matrix(N, coef, "hinged"),
           "truncated": lambda: matrices.hyperdiffusion_matrix(N, coef, "truncated"),
           "ch_noflux": lambda: matrices.ch_matrix(N, coef)}[kind]()
    P = len(ref) // 2
    for k, (u, v) in enumerate(zip(mine, ref)):
        off = k - P
        rows = [i for i in range(N) if 0 <= i + off < N]
        assert np.allclose(u[rows], v[rows], rtol=0, atol=1e-15), (kind, off)
        assert np.all(u[[i for i in range(N) if i not in rows]] == 0.0)


@pytest.mark.parametrize("N", [3, 4, 17, 256])
def test_product_periodic_matrix_builder_matches_oracle(sb, N):
    """The periodic diffusion matrix: all three diagonals equal the oracle's,
    corners included (a[0] couples x[N-1], c[N-1] couples x[0])."""
    from oracle import matrices
    mine = sb.sb_build_matrix("diffusion_periodic", N, 0.37)
    ref = matrices.diffusion_matrix_periodic(N, 0.37)
    for u, v in zip(mine, ref):
        assert np.allclose(u, v, rtol=0, atol=1e-15)
    with pytest.raises(sb.SbError):
        sb.sb_build_matrix("diffusion_periodic", 2, 0.37)


@pytest.mark.parametrize("N", [5, 6, 17, 256])
def test_product_periodic_ch_matrix_builder_matches_oracle(sb, N):
    from oracle import matrices
    mine = sb.sb_build_matrix("ch_periodic", N, 0.21)
    ref = matrices.ch_matrix_periodic(N, 0.21)
    for u, v in zip(mine, ref):
        assert np.allclose(u, v, rtol=0, atol=1e-15)
    with pytest.raises(sb.SbError):
        sb.sb_build_matrix("ch_periodic", 4, 0.21)


def test_product_matrix_builder_rejects_bad_input(sb):
    with pytest.raises(sb.SbError):
        sb.sb_build_matrix(99, 8, 0.1)
    with pytest.raises(sb.SbError):
        sb.sb_build_matrix("hinged", 8, float("inf"))


def test_stepper_entry_points_reject_null_handles(sb):
    """The stepper entry points added for the forced scheme, the refined steps and the
    coarsening run refuse a NULL stepper (or NULL outputs) on the host."""
    L = sb.lib()
    z = np.zeros(8)
    p = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = ctypes.c_size_t()
    assert L.sb_stepper_set_forcing(None, 0.1, p) == sb.SB_ERR_INVALID_ARG
    assert L.sb_stepper_run_forced(None, None, None, 8, 8, 1, 0, None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_stepper_refined_workspace_bytes(None, 8, 8, ctypes.byref(n)) == sb.SB_ERR_INVALID_ARG
    assert L.sb_stepper_run_refined(None, None, 8, 8, 2, 0, 1, 0, None, 0, None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_stepper_run_coarsening(None, None, 8, 8, 0, 1, None, None, 0, None) == sb.SB_ERR_INVALID_ARG
    assert L.sb_factor_shared_penta_periodic(3, p, p, p, p, p, ctypes.byref(ctypes.c_void_p())) \
        == sb.SB_ERR_INVALID_ARG  # N < 5
    assert sb.sb_last_error()
