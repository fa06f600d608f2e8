"""CPU checks of the double-float helpers (paper_1907_06487_gb300/csrc/df64.cuh)
behind the staged SymmSpMV executor's double-float row sums and the range
test of x_i in every executor that forms products off the FP64 pipe,
compiled for the host with contraction off and checked against exact
rational arithmetic: the split of a double into two floats (with and without
the range test), the error-free sums, the product, the branch-free integer
reassembly into a double, and a product of split doubles joined back into a
double.  The bounds are the ones the header states."""
import ctypes
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SHIM = os.path.join(HERE, "native", "df64_shim.cpp")


@pytest.fixture(scope="module")
def df(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("df64") / "libdf64.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", SHIM, "-o", out], check=True)
    lib = ctypes.CDLL(out)
    f, d, i = ctypes.c_float, ctypes.c_double, ctypes.c_int
    pf = ctypes.POINTER(f)
    lib.df_split.argtypes, lib.df_split.restype = [d, pf, pf], i
    lib.df_split_in_range.argtypes, lib.df_split_in_range.restype = [d, pf, pf], None
    lib.df_mul.argtypes, lib.df_mul.restype = [f, f, f, f, pf, pf], None
    lib.df_join.argtypes, lib.df_join.restype = [f, f], d
    lib.df_two_sum.argtypes, lib.df_two_sum.restype = [f, f, pf, pf], None
    lib.df_fast_two_sum.argtypes, lib.df_fast_two_sum.restype = [f, f, pf, pf], None
    lib.df_scatter.argtypes, lib.df_scatter.restype = [d, d], d
    lib.df_widen_mismatches.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.c_uint]
    lib.df_widen_mismatches.restype = ctypes.c_longlong
    return lib


def split(lib, v, checked=True):
    h, l = ctypes.c_float(), ctypes.c_float()
    if checked:
        st = lib.df_split(v, ctypes.byref(h), ctypes.byref(l))
    else:
        lib.df_split_in_range(v, ctypes.byref(h), ctypes.byref(l))
        st = 0
    return st, h.value, l.value


def f32(v):
    return float(np.float32(v))


def ulp32(v):
    return Fraction(float(np.spacing(np.float32(abs(v)))))


def rand_double(rng, emin=-50, emax=50):
    e = int(rng.integers(emin, emax + 1))
    m = int(rng.integers(0, 1 << 52))
    bits = (int(rng.integers(0, 2)) << 63) | ((e + 1023) << 52) | m
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


@pytest.mark.parametrize("checked", [True, False])
def test_split_bounds(df, checked):
    rng = np.random.default_rng(1)
    for _ in range(20000):
        v = rand_double(rng)
        st, h, l = split(df, v, checked)
        assert st == 0
        # hi is v truncated to 24 significant bits: same sign, |hi| <= |v| < |hi| (1 + 2^-23)
        assert math.copysign(1.0, h) == math.copysign(1.0, v)
        assert abs(h) <= abs(v) < abs(h) * (1 + 2.0 ** -23)
        assert f32(h) == h and f32(l) == l
        err = abs(Fraction(v) - Fraction(h) - Fraction(l))
        assert err < Fraction(2) ** -46 * abs(Fraction(v))


def test_split_edges(df):
    for v in (0.0, -0.0):
        st, h, l = split(df, v)
        assert (st, h, l) == (0, 0.0, 0.0)
    for v in (2.0 ** -50, -(2.0 ** 50) * (2 - 2.0 ** -52), 1.0, -1.5, 1.0 + 2.0 ** -52):
        st, h, l = split(df, v)
        assert st == 0 and Fraction(h) + Fraction(l) != 0
        assert split(df, v, checked=False)[1:] == (h, l)
    for v in (2.0 ** -51 * 1.9, 2.0 ** 51, -(2.0 ** 60), math.inf, -math.inf, math.nan, 5e-324, 1e300):
        st, h, l = split(df, v)
        assert st == 1 and h == 0.0 and l == 0.0


def test_two_sums_exact(df):
    rng = np.random.default_rng(2)
    s, e = ctypes.c_float(), ctypes.c_float()
    for _ in range(5000):
        a = f32(rng.normal() * 2.0 ** rng.integers(-30, 30))
        b = f32(rng.normal() * 2.0 ** rng.integers(-30, 30))
        df.df_two_sum(a, b, ctypes.byref(s), ctypes.byref(e))
        assert Fraction(s.value) + Fraction(e.value) == Fraction(a) + Fraction(b)
        assert s.value == f32(a + b)
        big, small = (a, b) if abs(a) >= abs(b) else (b, a)
        df.df_fast_two_sum(big, small, ctypes.byref(s), ctypes.byref(e))
        assert Fraction(s.value) + Fraction(e.value) == Fraction(a) + Fraction(b)


def test_mul_bound(df):
    rng = np.random.default_rng(3)
    ph, pl = ctypes.c_float(), ctypes.c_float()
    for _ in range(10000):
        a, b = rand_double(rng), rand_double(rng)
        _, ah, al = split(df, a)
        _, bh, bl = split(df, b)
        df.df_mul(ah, al, bh, bl, ctypes.byref(ph), ctypes.byref(pl))
        exact = (Fraction(ah) + Fraction(al)) * (Fraction(bh) + Fraction(bl))
        assert abs(Fraction(ph.value) + Fraction(pl.value) - exact) <= Fraction(2) ** -45 * abs(exact)
        assert abs(Fraction(pl.value)) <= ulp32(ph.value) / 2
        assert abs(ph.value) >= 2.0 ** -126  # normal


def check_join(df, h, l, ulps=2):
    r = df.df_join(h, l)
    exact = Fraction(h) + Fraction(l)
    assert math.copysign(1.0, r) == math.copysign(1.0, h)
    assert abs(Fraction(r) - exact) <= ulps * Fraction(math.ulp(abs(float(exact))))


def test_join(df):
    rng = np.random.default_rng(4)
    s, e = ctypes.c_float(), ctypes.c_float()
    n = 0
    while n < 20000:
        a = f32(rng.normal() * 2.0 ** rng.integers(-100, 100))
        b = f32(rng.normal() * 2.0 ** rng.integers(-100, 100))
        df.df_two_sum(a, b, ctypes.byref(s), ctypes.byref(e))
        if s.value == 0.0:
            continue
        check_join(df, s.value, e.value)
        n += 1
    # lo = 0 reproduces (double)hi exactly
    for h in (1.0, -3.5, f32(math.pi), f32(2.0 ** -100), f32(-(2.0 ** 120))):
        assert df.df_join(h, 0.0) == h and df.df_join(h, -0.0) == h


@pytest.mark.parametrize("k", [-100, -3, 0, 7, 90])
def test_join_power_of_two_borrow(df, k):
    """hi = +-2^k with lo of the opposite sign: the result falls into the
    binade below (the one case where the integer sum borrows)."""
    h = 2.0 ** k
    ulp = float(np.spacing(np.float32(h)))
    for hs in (1.0, -1.0):
        for sg in (1.0, -1.0):
            for frac in (0.5, 0.25, 0.3, 0.49999, 2.0 ** -20, 2.0 ** -28, 2.0 ** -40):
                lo = f32(sg * frac * ulp)
                check_join(df, hs * h, hs * lo)
    # also a mantissa of all ones (largest hi of its binade) with lo of either sign
    top = f32(h * (2 - 2.0 ** -23))
    for sg in (1.0, -1.0):
        check_join(df, top, f32(sg * 0.5 * float(np.spacing(np.float32(top)))))


def test_join_subnormal_lo(df):
    check_join(df, f32(2.0 ** -100), f32(2.0 ** -140))
    check_join(df, f32(-(2.0 ** -100)), f32(2.0 ** -149))
    check_join(df, f32(2.0 ** -102), f32(-(2.0 ** -127)))


def test_scatter_products(df):
    rng = np.random.default_rng(5)
    for _ in range(20000):
        a, x = rand_double(rng), rand_double(rng)
        q = df.df_scatter(a, x)
        exact = Fraction(a) * Fraction(x)
        assert abs(Fraction(q) - exact) <= Fraction(2) ** -44 * abs(exact)
    for a, x in ((1.0, 1.0), (0.5, 1.0), (-0.25, 3.0), (2.0 ** 50, 2.0 ** -50)):
        assert df.df_scatter(a, x) == a * x  # short mantissas are exact
    assert df.df_scatter(3.0, 0.0) == 0.0
    assert df.df_scatter(3.0, 2.0 ** 70) == 3.0 * 2.0 ** 70  # x outside the range: FP64
    assert math.isnan(df.df_scatter(3.0, math.nan))


def test_widen_is_the_exact_conversion(df):
    """Integer widening of FP32 values equals the (double) cast bit for bit:
    floats 65,537 and 65,521 bit patterns apart over the whole 32-bit range
    (all exponents, both signs, infinities, NaNs), every subnormal of both
    signs, and the special values."""
    assert df.df_widen_mismatches(0, 65537, 0xFFFFFFFF) == 0
    assert df.df_widen_mismatches(12345, 65521, 0xFFFFFFFF) == 0
    assert df.df_widen_mismatches(0, 1, 0x7FFFFF) == 0
    assert df.df_widen_mismatches(0x80000000, 1, 0x807FFFFF) == 0
