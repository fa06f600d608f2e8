// The product of two doubles on the integer pipes.
//
// The transposed update a_ij x_i of SymmSpMV (Alg. "SymmSpMV") is one
// multiply whose result goes straight to a reduction; on GB300 an FP64
// multiply issues to a pipe with about 1/70 of the FP32 rate.  Here the two
// 53-bit significands, left-aligned in 64 bits, are multiplied in 32-bit
// pieces by integer multiply-adds (the schoolbook product: the high by high
// partial product in full, the high halves of the two cross products, the
// low by low product and the carries out of the cross products' low halves
// dropped), the leading 53 bits of the 128-bit product are kept (truncated),
// and the sign and exponent are added as bit fields.  The x side is
// prepared once per row.
//
// Accuracy: the kept leading 64 bits fall short of the exact ones by less
// than 3 units, and the truncation to 53 bits drops less than 2^11 units of
// a value of at least 2^62, so the result is at most the exact product in
// magnitude and within 2^-51 of it, relative (|error| < 2^-52 (1 + 2^-8)).
//
// Domain: a and x nonzero, finite, with binary exponents in
// [df64::kEmin, df64::kEmax] (the same range the double-float helpers
// check), so that the product is a normal double.  Zero operands are the
// caller's to skip.
#pragma once
#include <cstdint>

#include "df64.cuh"

namespace intprod {

DF_HD uint32_t umulhi(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32);
#endif
}

// x prepared for int_product::mul: its significand with the leading bit set,
// left-aligned in m1:m0, and se = (x's sign in bit 31) + (E_x - 1024) in the
// exponent field, modulo 2^32 (E_x the biased exponent).
struct Factor {
    uint32_t m1, m0, se;
};

DF_HD Factor factor(double x) {
    const uint32_t H = df64::dhi(x), L = df64::dlo(x);
    Factor f;
    f.m1 = (H << 11) | (L >> 21) | 0x80000000u;
    f.m0 = L << 11;
    f.se = (H & 0x80000000u) + ((H & 0x7FF00000u) - (1024u << 20));
    return f;
}

// a * x from a's sign-and-exponent word sa (the high word of a double, the
// significand bits masked off) and its left-aligned significand a1:a0.
//   product of the significands, in units of 2^64:  t in [2^62, 2^64);
//   s = 1 when the significand product lies in [2, 4): 53 bits from 63 down,
//   else from 62 down; the biased exponent is E_a + E_x - 1023 + s.
// The high word is the sum of the fields: sa + se contributes both signs
// (their sum mod 2 lands in bit 31, nothing carries into it because the
// exponent stays in [1, 2046]) and E_a + E_x - 1024; s << 20 and the kept
// significand's leading bit (bit 20 of its high part) add the rest.
DF_HD double mul_fields(uint32_t sa, uint32_t a1, uint32_t a0, const Factor& f) {
    uint64_t t = static_cast<uint64_t>(a1) * f.m1 + umulhi(a1, f.m0);
    t += umulhi(a0, f.m1);
    const uint32_t th = static_cast<uint32_t>(t >> 32), tl = static_cast<uint32_t>(t);
    const uint32_t s = th >> 31;
    const uint32_t sh = 10u + s;
    const uint32_t mh = th >> sh;
    const uint32_t ml = (tl >> sh) | (th << (32u - sh));
    return df64::u2d(sa + f.se + (s << 20) + mh, ml);
}

DF_HD double mul(double a, const Factor& f) {
    const uint32_t H = df64::dhi(a), L = df64::dlo(a);
    return mul_fields(H & 0xFFF00000u, (H << 11) | (L >> 21) | 0x80000000u, L << 11, f);
}

// A float value: its 24-bit significand left-aligned in a1 (a0 = 0), its
// exponent re-biased to the double's.
DF_HD double mul(float a, const Factor& f) {
    const uint32_t u = df64::f2u(a);
    const uint32_t sa = (u & 0x80000000u) | ((((u >> 23) & 0xFFu) + 896u) << 20);
    return mul_fields(sa, (u << 8) | 0x80000000u, 0u, f);
}

}  // namespace intprod
