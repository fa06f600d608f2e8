// Host build of the double-float helpers (the staged executor's row sums, the
// range test of x_i), exported for the CPU tests (compiled with contraction
// off, so every FP32 operation rounds exactly as on the device).
#include <initializer_list>

#include "../../paper_1907_06487_gb300/csrc/df64.cuh"

extern "C" {

int df_split(double v, float* hi, float* lo) { return df64::split(v, *hi, *lo); }

void df_split_in_range(double v, float* hi, float* lo) { df64::split_in_range(v, *hi, *lo); }

void df_mul(float ah, float al, float bh, float bl, float* ph, float* pl) { df64::mul(ah, al, bh, bl, *ph, *pl); }

double df_join(float hi, float lo) { return df64::join(hi, lo); }

void df_two_sum(float a, float b, float* s, float* e) { df64::two_sum(a, b, *s, *e); }

void df_fast_two_sum(float a, float b, float* s, float* e) { df64::fast_two_sum(a, b, *s, *e); }

// A product a * xr of split doubles joined into a double: a (nonzero, in
// range) split without a test, xr split with the test; an xr outside the
// range is multiplied in FP64, a zero xr gives no contribution.
double df_scatter(double a, double xr) {
    float xh, xl;
    if (df64::split(xr, xh, xl)) return a * xr;
    if (xh == 0.0f) return 0.0;
    float ah, al, ph, pl;
    df64::split_in_range(a, ah, al);
    df64::mul(ah, al, xh, xl, ph, pl);
    return df64::join(ph, pl);
}

// Mismatches of df64::widen against the (double) cast over the floats whose
// bit patterns run from `start` to `end` in steps of `stride` (plus the
// special values), compared bit for bit.
long long df_widen_mismatches(unsigned start, unsigned stride, unsigned end) {
    long long bad = 0;
    auto check = [&](uint32_t u) {
        float f;
        std::memcpy(&f, &u, 4);
        const double a = df64::widen(f), b = static_cast<double>(f);
        uint64_t ua, ub;
        std::memcpy(&ua, &a, 8);
        std::memcpy(&ub, &b, 8);
        if (ua != ub) ++bad;
    };
    for (uint64_t u = start; u <= end; u += stride) check(static_cast<uint32_t>(u));
    for (uint32_t u : {0u, 0x80000000u, 1u, 0x80000001u, 0x7FFFFFu, 0x807FFFFFu, 0x800000u, 0x7F7FFFFFu,
                       0x7F800000u, 0xFF800000u, 0x7FC00000u, 0x7FA00001u, 0x3F800000u})
        check(u);
    return bad;
}

}  // extern "C"
