// *p += v as a reduction at L2 (red.global.add.f64): no value comes back.
// atomicAdd with its result unused usually compiles to the same, but not in
// kernels that also hold acquire/release operations (measured with ncu: every
// update of the one-launch executor came back as a returning atomic, a round
// trip each, until it was spelled out as below).  The kernels that wait on
// barriers or flags use this form.
#pragma once

__device__ __forceinline__ void red_add_f64(double* p, double v) {
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
