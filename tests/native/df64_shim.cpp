// Host build of the double-float helpers used by the SymmSpMV executor that
// forms the transposed products on the FP32 and integer pipes, exported for
// the CPU tests (compiled with contraction off, so every FP32 operation
// rounds exactly as on the device).
#include "../../paper_1907_06487_gb300/csrc/df64.cuh"

extern "C" {

int df_split(double v, float* hi, float* lo) { return df64::split(v, *hi, *lo); }

void df_split_in_range(double v, float* hi, float* lo) { df64::split_in_range(v, *hi, *lo); }

void df_mul(float ah, float al, float bh, float bl, float* ph, float* pl) { df64::mul(ah, al, bh, bl, *ph, *pl); }

double df_join(float hi, float lo) { return df64::join(hi, lo); }

void df_two_sum(float a, float b, float* s, float* e) { df64::two_sum(a, b, *s, *e); }

void df_fast_two_sum(float a, float b, float* s, float* e) { df64::fast_two_sum(a, b, *s, *e); }

// One transposed contribution a * xr as the kernel forms it: a (nonzero,
// in range) split without a test, xr split with the test; an xr outside the
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

}  // extern "C"
