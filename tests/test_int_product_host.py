"""CPU checks of the product of two doubles on the integer pipes
(paper_1907_06487_gb300/csrc/int_product.cuh), compiled for the host and
checked against exact rational arithmetic: the result is the exact product
truncated toward zero, at most one unit in the last place further down (the
dropped low partial products), so within 2^-51 of it; signs, the ends of the
exponent range, significands of all ones, short significands (exact), FP32
values, and the whole transposed contribution a * x_r as the kernels form it."""
import ctypes
import math
import shutil
import struct
import subprocess
import os
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SHIM = os.path.join(HERE, "native", "int_product_shim.cpp")


@pytest.fixture(scope="module")
def ip(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("intprod") / "libintprod.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", SHIM, "-o", out], check=True)
    lib = ctypes.CDLL(out)
    d = ctypes.c_double
    lib.ip_mul.argtypes, lib.ip_mul.restype = [d, d], d
    lib.ip_mul_f32.argtypes, lib.ip_mul_f32.restype = [ctypes.c_float, d], d
    lib.ip_scatter.argtypes, lib.ip_scatter.restype = [d, d], d
    return lib


def rand_double(rng, emin=-50, emax=50):
    e = int(rng.integers(emin, emax + 1))
    m = int(rng.integers(0, 1 << 52))
    bits = (int(rng.integers(0, 2)) << 63) | ((e + 1023) << 52) | m
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def trunc53(q):
    """|q| truncated to 53 significant bits (q a nonzero Fraction)."""
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    ulp = Fraction(2) ** (e - 52)
    return (q // ulp) * ulp, ulp


def check(r, exact):
    assert r != 0.0 and math.isfinite(r)
    assert math.copysign(1.0, r) == (1.0 if exact > 0 else -1.0)
    t, ulp = trunc53(exact)
    short = t - abs(Fraction(r))
    # the truncation, or one unit in the last place below it
    assert short == 0 or short == ulp or (short < ulp and Fraction(abs(r)) < t), (r, float(exact))
    assert 0 <= abs(exact) - abs(Fraction(r)) < Fraction(2) ** -51 * abs(exact)
    return short == 0


def test_random_products(ip):
    rng = np.random.default_rng(11)
    exact_trunc = 0
    for _ in range(30000):
        a, x = rand_double(rng), rand_double(rng)
        exact_trunc += check(ip.ip_mul(a, x), Fraction(a) * Fraction(x))
    # the dropped partial products rarely move the result off the truncation
    assert exact_trunc > 29000


def test_edges(ip):
    top = 2.0 - 2.0 ** -52           # significand of all ones
    cases = [(1.0, 1.0), (top, top), (top, 1.0), (1.0 + 2.0 ** -52, 1.0 + 2.0 ** -52), (1.5, 1.5),
             (2.0 ** -50, 2.0 ** -50), (2.0 ** 50 * top, 2.0 ** 50 * top), (2.0 ** -50, 2.0 ** 50 * top),
             (math.sqrt(2.0), math.sqrt(2.0)), (3.0, 1.0 / 3.0), (0.1, 10.0)]
    for a, x in cases:
        for sa in (1.0, -1.0):
            for sx in (1.0, -1.0):
                check(ip.ip_mul(sa * a, sx * x), Fraction(sa * a) * Fraction(sx * x))
    # short significands multiply exactly
    for a, x in ((1.0, 1.0), (1.5, 3.0), (-0.25, 3.0), (2.0 ** 50, 2.0 ** -50), (0.5, -0.5), (6.5, 2.0 ** -20)):
        assert ip.ip_mul(a, x) == a * x
    # (1 + 2^-52)^2 = 1 + 2^-51 + 2^-104: truncated, not rounded
    assert ip.ip_mul(1.0 + 2.0 ** -52, 1.0 + 2.0 ** -52) == 1.0 + 2.0 ** -51
    # top * top = 4 - 2^-50 + 2^-104: all-ones significands make the dropped
    # partial products largest, so the result may sit one unit below the
    # truncation 4 - 2^-50; it never reaches 4
    assert ip.ip_mul(top, top) in (4.0 - 2.0 ** -50, 4.0 - 3 * 2.0 ** -51)


def test_float_values(ip):
    rng = np.random.default_rng(12)
    for _ in range(20000):
        a = float(np.float32(rand_double(rng, -40, 40)))
        x = rand_double(rng)
        check(ip.ip_mul_f32(a, x), Fraction(a) * Fraction(x))
    for a, x in ((1.0, 1.0), (-1.5, 2.0), (0.5, 0.75)):
        assert ip.ip_mul_f32(a, x) == a * x


def test_scatter_contributions(ip):
    rng = np.random.default_rng(13)
    for _ in range(10000):
        a, x = rand_double(rng), rand_double(rng)
        q = ip.ip_scatter(a, x)
        exact = Fraction(a) * Fraction(x)
        assert abs(Fraction(q) - exact) < Fraction(2) ** -51 * abs(exact)
    assert ip.ip_scatter(3.0, 0.0) == 0.0
    assert ip.ip_scatter(3.0, -0.0) == 0.0
    assert ip.ip_scatter(3.0, 2.0 ** 70) == 3.0 * 2.0 ** 70  # x outside the range: FP64
    assert ip.ip_scatter(3.0, 2.0 ** -60) == 3.0 * 2.0 ** -60
    assert math.isnan(ip.ip_scatter(3.0, math.nan))


def test_dropped_partial_products_at_their_largest(ip):
    """Significands whose low words are all ones make the dropped low by low
    product and the dropped carries of the cross products as large as they
    get: the result still sits at most one unit below the truncation."""
    rng = np.random.default_rng(14)
    low_ones = (1 << 21) - 1  # a significand's low 32 bits sit in bits 0..20 of the stored field, left-aligned by 11
    for _ in range(5000):
        bits = []
        for _ in range(2):
            hi = int(rng.integers(0, 1 << 31)) << 21
            e = int(rng.integers(-50, 51))
            bits.append((int(rng.integers(0, 2)) << 63) | ((e + 1023) << 52) | ((hi | low_ones) & ((1 << 52) - 1)))
        a, x = (struct.unpack("<d", struct.pack("<Q", b))[0] for b in bits)
        check(ip.ip_mul(a, x), Fraction(a) * Fraction(x))
