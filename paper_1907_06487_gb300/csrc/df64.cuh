// Double-float ("df64") arithmetic that keeps GB300's FP64 pipe free.
//
// On GB300 FP64 multiplies and adds issue to a pipe with about 1/70 of the
// FP32 rate (0.5 T DFMA/s against 35 T FFMA/s).  These helpers carry a double
// as an unevaluated sum hi + lo of two floats and do the per-entry work on
// the FP32 and integer pipes; the split itself avoids the FP64 subtraction
// lo = v - hi by reading the bits:
//   split:  double -> (hi, lo) with integer bit operations and one FP32
//           subtraction; hi = the leading 24 significant bits, lo = the next
//           23 bits, so |v - hi - lo| < 2^-46 |v|.  Defined for v = 0 and for
//           binary exponents in [kEmin, kEmax]; anything else is reported so
//           the caller can take that entry in FP64.
//   mul:    (ah, al) * (bh, bl) with Dekker's exact product (T. J. Dekker,
//           "A floating-point technique for extending the available
//           precision", 1971; the error term by one fused multiply-add) and
//           his fast TwoSum; Knuth's branch-free TwoSum (TAOCP vol. 2,
//           Sec. 4.2.2) is here for the tests.
//   join:   (hi, lo) -> double with integer operations: the bit pattern of
//           (double)hi plus lo in units of its last place.
// With |a|, |x| in [2^kEmin, 2^(kEmax+1)) no FP32 product over- or
// underflows: products stay within 2^(2 kEmin) .. 2^(2 kEmax + 2), far
// inside FP32's normal range.
//
// Every FP32 operation is an _rn intrinsic on the device (and plain IEEE
// arithmetic with contraction off on the host) so that the compiler can
// neither fuse a product into a following sum nor reassociate; the error-free
// transformations depend on each rounding happening exactly as written.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace df64 {

constexpr int kEmin = -50, kEmax = 50;

DF_HD uint32_t f2u(float v) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(v);
#else
    uint32_t u;
    std::memcpy(&u, &v, 4);
    return u;
#endif
}
DF_HD float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float v;
    std::memcpy(&v, &u, 4);
    return v;
#endif
}
DF_HD uint32_t dhi(double v) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__double2hiint(v));
#else
    uint64_t u;
    std::memcpy(&u, &v, 8);
    return static_cast<uint32_t>(u >> 32);
#endif
}
DF_HD uint32_t dlo(double v) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__double2loint(v));
#else
    uint64_t u;
    std::memcpy(&u, &v, 8);
    return static_cast<uint32_t>(u);
#endif
}
DF_HD double u2d(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
#else
    const uint64_t u = (static_cast<uint64_t>(hi) << 32) | lo;
    double v;
    std::memcpy(&v, &u, 8);
    return v;
#endif
}
DF_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz(static_cast<int>(x));
#else
    return x ? __builtin_clz(x) : 32;
#endif
}
DF_HD float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
DF_HD float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
DF_HD float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
DF_HD float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return __builtin_fmaf(a, b, c);
#endif
}

// (hi, lo) with hi + lo = v to 47 significant bits.  Returns 0 when v is zero
// (hi = lo = 0) or its binary exponent lies in [kEmin, kEmax]; returns 1
// otherwise (hi = lo = 0 as well): the caller then takes this entry in FP64.
DF_HD int split(double v, float& hi, float& lo) {
    const uint32_t H = dhi(v), L = dlo(v);
    const uint32_t e = (H >> 20) & 0x7FFu;
    const bool ok = e - static_cast<uint32_t>(1023 + kEmin) <= static_cast<uint32_t>(kEmax - kEmin);
    // (H:L) << 3 keeps the low 9 exponent bits and the top 23 mantissa bits in
    // one word; subtracting the bias difference (1023 - 127) << 23 leaves the
    // FP32 exponent there (in range it fits 8 bits, so the sign bit stays 0).
    const uint32_t t = ((H << 3) | (L >> 29)) - (896u << 23);
    const uint32_t hb = (t & 0x7FFFFFFFu) | (H & 0x80000000u);
    // lo: mantissa bits 28..6 of v, scaled by 2^(E-46).  With a float of
    // exponent E + 104 and that sign, base|m - base = m * 2^(E-46) exactly.
    const uint32_t base = (hb & 0xFF800000u) - (23u << 23);
    const float l = fsub(u2f(base | ((L >> 6) & 0x7FFFFFu)), u2f(base));
    hi = ok ? u2f(hb) : 0.0f;
    lo = ok ? l : 0.0f;
    return (!ok && ((H << 1) | L) != 0) ? 1 : 0;
}

// split for a value already known to be nonzero with its binary exponent in
// [kEmin, kEmax] (checked once for the stored values): no range test.
DF_HD void split_in_range(double v, float& hi, float& lo) {
    const uint32_t H = dhi(v), L = dlo(v);
    const uint32_t t = ((H << 3) | (L >> 29)) - (896u << 23);
    const uint32_t hb = (t & 0x7FFFFFFFu) | (H & 0x80000000u);
    const uint32_t base = (hb & 0xFF800000u) - (23u << 23);
    hi = u2f(hb);
    lo = fsub(u2f(base | ((L >> 6) & 0x7FFFFFu)), u2f(base));
}

// The double equal to a float, built from its bits with integer operations
// (the widening conversion issues to the FP64 pipe on GB300).  Exact for
// every float: normal (exponent + 896, mantissa << 29), zero, subnormal
// (normalised by its leading bit), infinity and NaN (payload kept, quiet bit
// set, as an IEEE conversion does).
DF_HD double widen(float v) {
    const uint32_t u = f2u(v);
    const uint32_t sign = u & 0x80000000u;
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t m = u & 0x7FFFFFu;
    uint32_t hi = sign | ((e + 896u) << 20) | (m >> 3);
    uint32_t lo = m << 29;
    if (e == 0xFFu) hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);  // NaN comes out quiet
    if (e == 0) {  // integer work only, so a predicated form costs no FP64 issue
        if (m == 0) {
            hi = sign;
            lo = 0;
        } else {
            const int p = 31 - clz32(m);  // leading bit of m * 2^-149
            const uint32_t f = (m << (23 - p)) & 0x7FFFFFu;
            hi = sign | (static_cast<uint32_t>(p + 874) << 20) | (f >> 3);
            lo = f << 29;
        }
    }
    return u2d(hi, lo);
}
DF_HD double widen(double v) { return v; }

// Zero test and split of a stored value (double: checked range, see above;
// float: its own hi part).
DF_HD bool is_zero(double v) { return ((dhi(v) << 1) | dlo(v)) == 0; }
DF_HD bool is_zero(float v) { return (f2u(v) << 1) == 0; }
DF_HD void split_value(double a, float& h, float& l) { split_in_range(a, h, l); }
DF_HD void split_value(float a, float& h, float& l) {
    h = a;
    l = 0.0f;
}

// Knuth's TwoSum: s + e = a + b exactly.
DF_HD void two_sum(float a, float b, float& s, float& e) {
    s = fadd(a, b);
    const float bb = fsub(s, a);
    e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
}

// Dekker's fast TwoSum, exact when |a| >= |b| (or a = 0).
DF_HD void fast_two_sum(float a, float b, float& s, float& e) {
    s = fadd(a, b);
    e = fsub(b, fsub(s, a));
}

// (ph, pl) ~ (ah + al)(bh + bl): Dekker's exact product of the hi parts (its
// error term by one fused multiply-add) plus the two cross terms; the al*bl
// term (below 2^-46 of the product) is dropped.  |pl| <= ulp(ph) / 2.  With
// both operands split from doubles in the range above, the error is below
// 2^-45 of the product and ph is a normal float.
DF_HD void mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    const float p = fmul(ah, bh);
    float e = ffma(ah, bh, -p);  // exact: ah * bh = p + e
    e = ffma(ah, bl, ffma(al, bh, e));
    fast_two_sum(p, e, ph, pl);
}

// The double hi + lo for hi a normal float of exponent >= -102 and
// |lo| <= ulp(hi) / 2 (lo may be zero or subnormal), within two units in the
// last place; integer operations only, no branches.  (double)|hi| is hi's bit
// pattern re-biased (exponent + 896, mantissa << 29); lo is added to it as an
// integer count of that double's last place, |lo| / 2^(E_hi - 52) truncated.
// The sum never carries out of the mantissa: the mantissa field of
// (double)hi is a multiple of 2^29 and |count| < 2^29.  A borrow happens only
// when hi is a power of two and lo has the opposite sign; the result then
// lies in the binade below, whose last place is half as large, so the count
// is doubled.
DF_HD double join(float hi, float lo) {
    const uint32_t hb = f2u(hi), lb = f2u(lo);
    const uint32_t eh = (hb >> 23) & 0xFFu;
    const uint32_t elr = (lb >> 23) & 0xFFu;
    const uint32_t el = elr ? elr : 1u;  // zero or subnormal lo: no implicit bit, exponent field 1
    const uint32_t m = (lb & 0x7FFFFFu) | (elr ? 0x800000u : 0u);
    const uint32_t rs = eh - el - 24u;   // >= 0 because |lo| <= ulp(hi) / 2
    uint32_t ml = rs < 32u ? ((m << 5) >> rs) : 0u;  // m * 2^(el - eh + 29)
    const uint32_t opposite = (hb ^ lb) >> 31;
    ml <<= opposite & ((hb & 0x7FFFFFu) == 0 ? 1u : 0u);
    const uint32_t mask = 0u - opposite;
    const int32_t sml = static_cast<int32_t>((ml ^ mask) - mask);
    const uint64_t d = ((static_cast<uint64_t>((hb >> 3) & 0x0FFFFFFFu) + (896u << 20)) << 32) |
                       static_cast<uint64_t>(hb << 29);
    const uint64_t r = d + static_cast<uint64_t>(static_cast<int64_t>(sml));
    return u2d(static_cast<uint32_t>(r >> 32) | (hb & 0x80000000u), static_cast<uint32_t>(r));
}

}  // namespace df64
