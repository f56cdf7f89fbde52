"""CPU tests of the double-float arithmetic used by the SB_ARITH_DF32 sweeps and of
the integer FP64 -> FP32 truncation of the refinement residuals.

The library's own headers (paper_2107_05395_gb300/csrc/arith.cuh, narrow.cuh) are compiled for
the host (tests/native/arith_harness.cpp, -ffp-contract=off) and checked against
exact rational arithmetic: the FP64 -> pair split, the pair -> FP64 rounding, the
sweep step, and whole sweeps against the FP64 oracle."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import banded, matrices

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("arith") / "arith_h.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", out,
                    os.path.join(HERE, "native", "arith_harness.cpp")], check=True)
    L = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    L.h_double_to_df.argtypes = [dp, fp, fp, ctypes.c_long]
    L.h_df_to_double.argtypes = [fp, fp, dp, ctypes.c_long]
    L.h_df_step.argtypes = [ctypes.c_int, ctypes.c_int, fp, fp, fp, fp, fp]
    L.h_df_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, dp, dp]
    L.h_dmul_int.argtypes = [dp, dp, dp, ctypes.c_long]
    L.h_f64_to_f32_trunc.argtypes = [dp, fp, ctypes.c_long]
    return L


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def split(H, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    h = np.empty(v.shape, np.float32)
    l = np.empty(v.shape, np.float32)
    H.h_double_to_df(_p(v, ctypes.c_double), _p(h, ctypes.c_float), _p(l, ctypes.c_float), v.size)
    return h, l


def join(H, h, l):
    h = np.ascontiguousarray(h, dtype=np.float32)
    l = np.ascontiguousarray(l, dtype=np.float32)
    out = np.empty(h.shape, np.float64)
    H.h_df_to_double(_p(h, ctypes.c_float), _p(l, ctypes.c_float), _p(out, ctypes.c_double), h.size)
    return out


def ulp32(h):
    return np.spacing(np.abs(np.float32(h))).astype(np.float64)


def test_residual_truncation_to_fp32(H):
    """f64_to_f32_trunc (the refinement residual's FP64 -> FP32 step, integer
    operations only): truncation toward zero over FP32's normal range, a signed zero
    below 2^-126 (exact zeros included), an infinity from 2^128 up, NaNs kept.  The reference
    rounds to nearest with NumPy and steps back toward zero where that went past
    |v|."""
    rng = np.random.default_rng(5)
    n = 200000
    v = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-140, 135, n).astype(np.float64))
    v *= np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    v = np.concatenate([v, [0.0, -0.0, np.inf, -np.inf, np.nan, 2.0 ** -126, -(2.0 ** -126),
                            np.nextafter(2.0 ** -126, 0.0), np.nextafter(2.0 ** 128, 0.0),
                            float(np.finfo(np.float32).max), 1.0, -1.0 - 2.0 ** -40]])
    out = np.empty(v.shape, np.float32)
    H.h_f64_to_f32_trunc(_p(v, ctypes.c_double), _p(out, ctypes.c_float), v.size)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32)
    past = np.abs(ref.astype(np.float64)) > np.abs(v)
    ref[past] = np.nextafter(ref[past], np.float32(0.0))
    tiny = np.abs(v) < 2.0 ** -126
    ref[tiny] = np.copysign(np.float32(0.0), v[tiny]).astype(np.float32)
    huge = np.abs(v) >= 2.0 ** 128  # beyond FP32's range: rounded, i.e. infinite
    ref[huge] = np.copysign(np.float32(np.inf), v[huge]).astype(np.float32)
    assert np.array_equal(out.view(np.uint32)[~np.isnan(v)], ref.view(np.uint32)[~np.isnan(v)])
    assert np.all(np.isnan(out[np.isnan(v)]))


def test_split_is_accurate_and_normalised(H):
    rng = np.random.default_rng(0)
    mant = rng.uniform(1.0, 2.0, 20000)
    expo = rng.integers(-70, 110, 20000)
    sign = np.where(rng.uniform(size=20000) < 0.5, -1.0, 1.0)
    v = sign * np.ldexp(mant, expo)
    v = np.concatenate([v, [0.0, -0.0, 1.0, -1.0, 2.0 ** -60, 2.0 ** 99, 3.0, 1 / 3, -1e-30, 5e-324,
                            np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 2.0 ** 100, 2.0 ** -61]])
    h, l = split(H, v)
    for vi, hi, li in zip(v, h, l):
        exact = Fraction(float(hi)) + Fraction(float(li))
        err = abs(exact - Fraction(float(vi)))
        # relative 2^-46, plus FP32's underflow level for doubles below FP32's range
        assert err <= Fraction(abs(float(vi))) * Fraction(1, 2 ** 46) + Fraction(1, 2 ** 140), (vi, hi, li)
        assert abs(float(li)) <= float(np.spacing(np.abs(hi))) or hi == 0.0


def nearest_double_ok(result, exact):
    """|result - exact| <= ulp(result)/2 (ties may go either way)."""
    return abs(Fraction(float(result)) - exact) <= Fraction(float(np.spacing(abs(result)))) / 2


def test_join_rounds_to_nearest(H):
    rng = np.random.default_rng(1)
    n = 20000
    h = (np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
         * np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-59, 98, n))).astype(np.float32)
    frac = rng.uniform(-0.5, 0.5, n)
    l = (frac * ulp32(h)).astype(np.float32)
    # edge cases: zero low part, powers of two with a low part pointing down or up
    extra_h = np.array([1.0, 1.0, -1.0, 2.0 ** 20, 0.75, -3.0, 0.0, 2.0 ** -59], np.float32)
    extra_l = np.array([0.0, -2.0 ** -26, 2.0 ** -26, -1.0 / 64, 2.0 ** -30, -2.0 ** -23, 1e-20,
                        2.0 ** -90], np.float32)
    h = np.concatenate([h, extra_h])
    l = np.concatenate([l, extra_l])
    out = join(H, h, l)
    for hi, li, oi in zip(h, l, out):
        exact = Fraction(float(hi)) + Fraction(float(li))
        assert nearest_double_ok(oi, exact), (hi, li, oi)


def test_split_join_round_trip(H):
    v = synth.rhs_normal(seed=9, N=1, M=50000)[0] * 1e3
    h, l = split(H, v)
    back = join(H, h, l)
    assert np.max(np.abs(back - v) / np.abs(v)) <= 2.0 ** -46


@pytest.mark.parametrize("P,c0one", [(1, 0), (1, 1), (2, 0), (2, 1)])
def test_step_matches_exact_arithmetic(H, P, c0one):
    rng = np.random.default_rng(10 + 2 * P + c0one)
    worst = 0.0
    for _ in range(3000):
        vals = rng.standard_normal(4) * np.ldexp(1.0, rng.integers(-8, 8, 4))
        coefs = rng.uniform(-1.5, 1.5, 3)
        ch, cl = split(H, coefs)
        vh, vl = split(H, vals)
        c = np.array([ch[0], cl[0], ch[1], cl[1], ch[2], cl[2]], np.float32)
        ins = [np.array([vh[k], vl[k]], np.float32) for k in range(3)]
        out = np.empty(2, np.float32)
        H.h_df_step(P, c0one, _p(c, ctypes.c_float), _p(ins[0], ctypes.c_float),
                    _p(ins[1], ctypes.c_float), _p(ins[2], ctypes.c_float), _p(out, ctypes.c_float))
        F = lambda a, b: Fraction(float(a)) + Fraction(float(b))
        C = [F(ch[k], cl[k]) for k in range(3)]
        X = [F(vh[k], vl[k]) for k in range(3)]
        terms = [X[0] if c0one else C[0] * X[0], C[1] * X[1]] + ([C[2] * X[2]] if P == 2 else [])
        exact = terms[0] - sum(terms[1:])
        scale = sum(abs(t) for t in terms)
        err = abs(F(out[0], out[1]) - exact) / scale
        worst = max(worst, float(err))
    assert worst <= 2.0 ** -44, worst


def prescaled_rows(P, fac, adjoint):
    """Forward/backward rows in the kernel's prescaled layout, from oracle factors."""
    if P == 1:
        a, bh, ch = fac
        N = len(bh)
        W = 2
        fw = np.zeros((N, W))
        bw = np.zeros((N, W))
        for i in range(N):
            if not adjoint:
                fw[i] = [1 / bh[i], a[i] / bh[i] if i > 0 else 0.0]
                bw[i] = [1.0, ch[i] if i + 1 < N else 0.0]
            else:
                fw[i] = [1.0, ch[i - 1] if i > 0 else 0.0]
                bw[i] = [1 / bh[i], a[i + 1] / bh[i] if i + 1 < N else 0.0]
    else:
        eps, beta, alpha, gamma, delta = fac
        N = len(alpha)
        W = 3
        fw = np.zeros((N, W))
        bw = np.zeros((N, W))
        for i in range(N):
            if not adjoint:
                fw[i] = [1 / alpha[i], beta[i] / alpha[i], eps[i] / alpha[i]]
                bw[i] = [1.0, gamma[i], delta[i]]
            else:
                fw[i] = [1.0, gamma[i - 1] if i >= 1 else 0.0, delta[i - 2] if i >= 2 else 0.0]
                bw[i] = [1 / alpha[i], beta[i + 1] / alpha[i] if i + 1 < N else 0.0,
                         eps[i + 2] / alpha[i] if i + 2 < N else 0.0]
    return np.concatenate([fw.ravel(), bw.ravel()])


def df_sweep(H, P, rows, rhs, adjoint):
    N = rhs.shape[0]
    out = np.empty_like(rhs)
    for m in range(rhs.shape[1]):
        r = np.ascontiguousarray(rhs[:, m])
        x = np.empty(N)
        H.h_df_sweep(P, 1 if adjoint else 0, 0 if adjoint else 1, N, _p(rows, ctypes.c_double),
                     _p(r, ctypes.c_double), _p(x, ctypes.c_double))
        out[:, m] = x
    return out


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("kind,N", [("tri", 1), ("tri", 7), ("tri", 300), ("penta", 1), ("penta", 2),
                                    ("penta", 5), ("penta", 300)])
def test_df_sweep_matches_oracle(H, kind, N, adjoint):
    if kind == "tri":
        a, b, c = synth.random_tri_diagonals(seed=N, N=N)
        bh, ch = banded.tri_factor(a, b, c)
        fac = (a, bh, ch)
        ref_fn = (lambda r: banded.tri_solve_adjoint(a, bh, ch, r)) if adjoint else \
                 (lambda r: banded.tri_solve(a, bh, ch, r))
        P = 1
    else:
        diags = synth.random_penta_diagonals(seed=N, N=N)
        fac = banded.penta_factor(*diags)
        ref_fn = (lambda r: banded.penta_solve_adjoint(*fac, r)) if adjoint else \
                 (lambda r: banded.penta_solve(*fac, r))
        P = 2
    rows = prescaled_rows(P, fac, adjoint)
    rhs = synth.rhs_normal(seed=100 + N, N=N, M=6)
    x = df_sweep(H, P, rows, rhs, adjoint)
    ref = ref_fn(rhs)
    err = np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert np.max(err) <= 1e-13, np.max(err)


def test_df_sweep_hyperdiffusion_workload(H):
    N = 1024
    diags = matrices.hyperdiffusion_matrix(N, 0.25, "hinged")
    fac = banded.penta_factor(*diags)
    rows = prescaled_rows(2, fac, False)
    rhs = synth.rhs_normal(seed=2, N=N, M=4)
    x = df_sweep(H, 2, rows, rhs, False)
    ref = banded.penta_solve(*fac, rhs)
    err = np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert np.max(err) <= 1e-13, np.max(err)


def test_integer_fp64_multiply_is_bit_exact(H):
    """dmul_int (the FP64 product computed with integer instructions) must equal the
    FP64 multiply bit for bit: random bit patterns (zeros, subnormals, infinities,
    NaNs take the FP64 fallback), moderate values, and significands that sit on
    rounding ties."""
    rng = np.random.default_rng(123)
    n = 400000
    a = rng.integers(0, 2**63, n, dtype=np.uint64).view(np.float64) * np.where(rng.uniform(size=n) < 0.5, -1, 1)
    b = rng.integers(0, 2**63, n, dtype=np.uint64).view(np.float64)
    c = rng.uniform(-4, 4, n)
    d = rng.uniform(-4, 4, n)
    # significands ending in many ones / ties after the product
    e = (rng.integers(0, 2**52, n, dtype=np.uint64) | np.uint64(0xFFFFFF) | np.uint64(1023 << 52)).view(np.float64)
    f = np.ldexp(rng.uniform(1, 2, n), -20)
    special = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, 1e-308, 1e308, np.inf, -np.inf, np.nan, 2.0 ** -1022,
                        np.nextafter(2.0, 0.0)])
    xs = np.concatenate([a, c, e, np.repeat(special, len(special))])
    ys = np.concatenate([b, d, f, np.tile(special, len(special))])
    out = np.empty_like(xs)
    with np.errstate(all="ignore"):
        ref = xs * ys
    H.h_dmul_int(_p(xs, ctypes.c_double), _p(ys, ctypes.c_double), _p(out, ctypes.c_double), xs.size)
    same = (out.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(out) & np.isnan(ref))
    assert np.all(same), (xs[~same][:3], ys[~same][:3])
