// Host build of the integer-pipe product of two doubles
// (csrc/int_product.cuh), exported for the CPU tests.
#include "../../paper_1907_06487_gb300/csrc/int_product.cuh"

extern "C" {

double ip_mul(double a, double x) { return intprod::mul(a, intprod::factor(x)); }

double ip_mul_f32(float a, double x) { return intprod::mul(a, intprod::factor(x)); }

// One transposed contribution a * xr as a kernel forms it: xr checked by the
// double-float split's range test (outside: an FP64 multiply; zero: no
// contribution), a nonzero and in range (checked once per matrix).
double ip_scatter(double a, double xr) {
    float h, l;
    if (df64::split(xr, h, l)) return a * xr;
    if (h == 0.0f) return 0.0;
    return intprod::mul(a, intprod::factor(xr));
}

}  // extern "C"
