"""CPU tests of the kernels' scalar arithmetic (csrc/peps_arith.cuh) compiled
for the host by tests/host/arith_host.cpp: the error-free transformations
are exact, the float-float operations and the compensated accumulator stay
within their error bounds against exact rational arithmetic, the two forms
of the QR's trailing update agree with the exact value, and the device
Philox4x32-10 reproduces the published known-answer vectors.

u = 2^-24 is the FP32 unit roundoff; float-float carries about u^2 = 2^-48."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1806_03761_gb300", "csrc")
U2 = Fr(1, 2 ** 48)
F = ctypes.POINTER(ctypes.c_float)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("arith") / "arith_host.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC,
                    os.path.join(HERE, "host", "arith_host.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    for name in ("h_add", "h_mul", "h_div"):
        getattr(L, name).argtypes = [F, F, F]
    L.h_two_sum.argtypes = [ctypes.c_float, ctypes.c_float, F]
    L.h_sqrt.argtypes = [F, F]
    L.h_from_double.argtypes = [ctypes.c_double, F]
    L.h_dot.argtypes = [F, F, ctypes.c_int, F]
    L.h_acc_merge.argtypes = [ctypes.c_float] * 4 + [F]
    L.h_update.argtypes = [F, F, F, ctypes.c_int, F, F]
    P32 = ctypes.POINTER(ctypes.c_uint32)
    L.h_philox.argtypes = [P32, ctypes.c_uint32, ctypes.c_uint32, P32]
    L.h_uniform53.argtypes = [ctypes.c_uint64]
    L.h_uniform53.restype = ctypes.c_double
    L.h_uniform_open52.argtypes = [ctypes.c_uint64]
    L.h_uniform_open52.restype = ctypes.c_double
    return L


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float32).ctypes.data_as(F)


def _out(n=2):
    o = np.zeros(n, np.float32)
    return o, o.ctypes.data_as(F)


def _ff(rng, n, lo_exp=-20, hi_exp=20):
    """n normalised float-float values (|lo| <= ulp(hi)/2) as an (n, 2) array."""
    hi = (rng.standard_normal(n) * 2.0 ** rng.integers(lo_exp, hi_exp, n)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    return np.stack([hi, lo], axis=1)


def _val(p):
    return Fr(float(p[0])) + Fr(float(p[1]))


def test_two_sum_is_exact(lib):
    rng = np.random.default_rng(1)
    a = (rng.standard_normal(4000) * 2.0 ** rng.integers(-30, 30, 4000)).astype(np.float32)
    b = (rng.standard_normal(4000) * 2.0 ** rng.integers(-30, 30, 4000)).astype(np.float32)
    b[:500] = -a[:500] * np.float32(1 + 2 ** -20)  # heavy cancellation
    o, po = _out()
    for x, y in zip(a, b):
        lib.h_two_sum(float(x), float(y), po)
        assert o[0] == np.float32(x) + np.float32(y)
        assert Fr(float(o[0])) + Fr(float(o[1])) == Fr(float(x)) + Fr(float(y))


@pytest.mark.parametrize("op,bound", [("add", 4), ("mul", 8), ("div", 16)])
def test_float_float_operations(lib, op, bound):
    """Relative error <= bound * u^2 of the exact result (sum, product,
    quotient of the float-float operands; measured worst over 3000 pairs:
    1.4, 2.8, 3.6 u^2)."""
    rng = np.random.default_rng({"add": 2, "mul": 3, "div": 4}[op])
    A, B = _ff(rng, 3000), _ff(rng, 3000)
    if op == "add":
        B[:300] = -A[:300]
        B[:300, 1] = (A[:300, 1] * np.float32(0.5)).astype(np.float32)  # partial cancellation
    fn = getattr(lib, "h_" + op)
    o, po = _out()
    worst = Fr(0)
    for a, b in zip(A, B):
        fn(_f(a), _f(b), po)
        va, vb = _val(a), _val(b)
        exact = va + vb if op == "add" else va * vb if op == "mul" else va / vb
        if exact == 0:
            assert _val(o) == 0
            continue
        err = abs(_val(o) - exact) / abs(exact)
        worst = max(worst, err)
    assert worst <= bound * U2, float(worst / U2)


def test_float_float_sqrt_and_conversion(lib):
    rng = np.random.default_rng(5)
    A = np.abs(_ff(rng, 2000))
    o, po = _out()
    for a in A:
        lib.h_sqrt(_f(a), po)
        r = _val(o)
        # r^2 = a (1 + d), |d| <= 2 * 16 u^2 for a relative error of 16 u^2 in r
        assert abs(r * r - _val(a)) <= 32 * U2 * _val(a)
    for x in rng.standard_normal(2000) * 2.0 ** rng.integers(-60, 60, 2000):
        lib.h_from_double(float(x), po)
        assert abs(_val(o) - Fr(float(x))) <= U2 * abs(Fr(float(x)))


@pytest.mark.parametrize("n", [1, 7, 28, 144])
def test_compensated_dot_product(lib, n):
    """sum x_i y_i with the compensated accumulator (every contraction and
    the QR's dot products): error <= (n^2 + 4n) u^2 sum |x_i y_i| (products
    rounded to within 2 u^2, the leading sum error-free, the FP32 correction
    term of size <= n u sum|x y| rounded n times), and on random data far
    below it: the median error stays within n u^2 of sum |x y| (measured:
    0.5, 0.8, 2.0 u^2 at n = 7, 28, 144; worst of 200, 3.4, 8.9, 22 u^2)."""
    rng = np.random.default_rng(10 + n)
    o, po = _out()
    rel = []
    for trial in range(200):
        X, Y = _ff(rng, n, -8, 8), _ff(rng, n, -8, 8)
        lib.h_dot(_f(X), _f(Y), n, po)
        exact = sum(_val(x) * _val(y) for x, y in zip(X, Y))
        scale = sum(abs(_val(x) * _val(y)) for x, y in zip(X, Y))
        err = abs(_val(o) - exact)
        assert err <= (n * n + 4 * n) * U2 * scale
        rel.append(float(err / scale))
    assert np.median(rel) <= n * 2.0 ** -48


def test_accumulator_merge(lib):
    """Two lanes' accumulators (s, c) merged by the warp reduction: the
    leading parts meet in an exact TwoSum, so s + c is the exact sum up to
    the two FP32 roundings of the correction terms, 2u (|c1| + |c2|) +
    2 u^2 (|s1| + |s2|), whichever lane merges."""
    rng = np.random.default_rng(20)
    o, po = _out()
    o2, po2 = _out()
    for _ in range(3000):
        s1, s2 = (rng.standard_normal(2) * 2.0 ** rng.integers(-10, 10, 2)).astype(np.float32)
        c1 = np.float32(rng.uniform(-4, 4) * np.spacing(abs(s1)))
        c2 = np.float32(rng.uniform(-4, 4) * np.spacing(abs(s2)))
        lib.h_acc_merge(float(s1), float(c1), float(s2), float(c2), po)
        lib.h_acc_merge(float(s2), float(c2), float(s1), float(c1), po2)
        assert o[0] == o2[0] and o[1] == o2[1]
        exact = Fr(float(s1)) + Fr(float(c1)) + Fr(float(s2)) + Fr(float(c2))
        got = Fr(float(o[0])) + Fr(float(o[1]))
        bound = Fr(2, 2 ** 24) * (abs(Fr(float(c1))) + abs(Fr(float(c2)))) + \
            2 * U2 * (abs(Fr(float(s1))) + abs(Fr(float(s2))))
        assert abs(got - exact) <= bound


@pytest.mark.parametrize("nb", [1, 4, 8])
def test_trailing_update_forms(lib, nb):
    """x - sum_s v_s w_s, as the compensated accumulation (the default QR
    trailing update) and as the chain of fused multiply-subtracts: both
    within (4 nb + 4) u^2 (|x| + sum |v_s w_s|) of the exact value, also
    when the result cancels."""
    rng = np.random.default_rng(30 + nb)
    a, pa = _out()
    c, pc = _out()
    for trial in range(1500):
        V, W = _ff(rng, nb, -4, 4), _ff(rng, nb, -4, 4)
        x = _ff(rng, 1, -4, 4)[0]
        if trial % 3 == 0:  # x close to sum v w: the update cancels
            s = float(sum(_val(v) * _val(w) for v, w in zip(V, W)))
            x = np.array([np.float32(s), np.float32(s - float(np.float32(s)))], np.float32)
        lib.h_update(_f(x), _f(V), _f(W), nb, pa, pc)
        exact = _val(x) - sum(_val(v) * _val(w) for v, w in zip(V, W))
        scale = abs(_val(x)) + sum(abs(_val(v) * _val(w)) for v, w in zip(V, W))
        assert abs(_val(a) - exact) <= (4 * nb + 4) * U2 * scale
        assert abs(_val(c) - exact) <= (4 * nb + 4) * U2 * scale


def test_device_philox_known_answers(lib):
    """The kernels' Philox4x32-10 against the published known-answer vectors
    (the same file pins the oracle's generator)."""
    n = 0
    ctr = (ctypes.c_uint32 * 4)()
    out = (ctypes.c_uint32 * 4)()
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        for i in range(4):
            ctr[i] = w[i]
        lib.h_philox(ctr, w[4], w[5], out)
        assert tuple(out) == tuple(w[6:10])
        n += 1
    assert n >= 3


def test_device_uniforms(lib):
    for x in (0, 1, 2 ** 11 - 1, 2 ** 11, 2 ** 63, 2 ** 64 - 1, 0x0123456789ABCDEF):
        assert lib.h_uniform53(x) == (x >> 11) * 2.0 ** -53
        p = lib.h_uniform_open52(x)
        assert p == ((x >> 12) + 0.5) * 2.0 ** -52 and 0.0 < p < 1.0
