// Ceilings measured next to the kernels (race_probe_peaks).
//
// The paper bounds SymmSpMV by a roofline whose memory term it reports as a
// range, from the load-only to the copy bandwidth (Sec. 3, roofline model;
// Table "test bed").  On GB300 the copy figure comes from the driver's own
// measurement; the load-only figure and the FP64 fused multiply-add rate
// (the second roof of the FP64-heavy SymmSpMM) are measured here.
//   what = 0: load-only stream over in_d[0, n): 16-byte loads, grid-strided,
//             the words of each block folded by XOR into out_d[block] (so
//             nothing is elided, and no FP64 adds bound the loop);
//   what = 1: FP64 fused multiply-adds, eight independent chains of `iters`
//             per thread, each block's result stored to out_d[block].
// The grid is 4 blocks of 256 threads per SM; out_d holds one double per
// block (race_device_sms() * 4 <= 4096 on any current GPU).
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "race_internal.h"

namespace race_probe {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_load(const double2* __restrict__ in, int64_t n2, const double* tail,
                                                   int64_t ntail, double* out) {
    // the loaded words are folded with integer XORs: GB300's FP64 adder would
    // otherwise bound the loop (two additions per 16 bytes) below the HBM rate
    unsigned long long f0 = 0, f1 = 0, f2 = 0, f3 = 0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
    int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
    const longlong2* v = reinterpret_cast<const longlong2*>(in);
    for (; i + 3 * stride < n2; i += 4 * stride) {
        const longlong2 a = __ldcs(v + i), b = __ldcs(v + i + stride);
        const longlong2 c = __ldcs(v + i + 2 * stride), d = __ldcs(v + i + 3 * stride);
        f0 ^= static_cast<unsigned long long>(a.x ^ a.y);
        f1 ^= static_cast<unsigned long long>(b.x ^ b.y);
        f2 ^= static_cast<unsigned long long>(c.x ^ c.y);
        f3 ^= static_cast<unsigned long long>(d.x ^ d.y);
    }
    for (; i < n2; i += stride) {
        const longlong2 a = __ldcs(v + i);
        f0 ^= static_cast<unsigned long long>(a.x ^ a.y);
    }
    if (blockIdx.x == 0 && threadIdx.x < ntail) f1 ^= static_cast<unsigned long long>(__double_as_longlong(tail[threadIdx.x]));
    __shared__ unsigned long long red[kThreads];
    red[threadIdx.x] = (f0 ^ f1) ^ (f2 ^ f3);
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] ^= red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = __longlong_as_double(static_cast<long long>(red[0]));
}

__global__ void __launch_bounds__(kThreads) k_dfma(int32_t iters, double* out) {
    const double m = 1.0 + 1.0e-9 * (threadIdx.x + 1);
    double c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = 1.0e-3 * (q + 1) + blockIdx.x;
    for (int32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) c[q] = fma(c[q], m, 0.5);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += c[q];
    __shared__ double red[kThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads; ++k) t += red[k];
        out[blockIdx.x] = t;
    }
}

}  // namespace race_probe

extern "C" int race_probe_peaks(int32_t what, const double* in_d, int64_t n, double* out_d, int32_t iters,
                                void* stream) {
    if (!out_d || (what == 0 && (!in_d || n < 0 || (reinterpret_cast<uintptr_t>(in_d) & 15u))) ||
        (what == 1 && iters < 1) || (what != 0 && what != 1)) {
        race_set_detail("race_probe_peaks: bad argument (what 0 needs a 16-byte aligned input, what 1 iters >= 1)");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = race_device_sms() * 4;
    if (grid > 4096) {
        race_set_detail("race_probe_peaks: more than 4096 blocks");
        return RACE_ERR_UNSUPPORTED;
    }
    if (what == 0) {
        const int64_t n2 = n / 2;
        race_probe::k_load<<<grid, race_probe::kThreads, 0, st>>>(reinterpret_cast<const double2*>(in_d), n2,
                                                                   in_d + 2 * n2, n - 2 * n2, out_d);
    } else {
        race_probe::k_dfma<<<grid, race_probe::kThreads, 0, st>>>(iters, out_d);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_probe_peaks: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}
