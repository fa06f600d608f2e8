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

#include <algorithm>
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

// ---------------------------------------------------------------------------
// race_probe_reductions: the ways a GPU can combine the transposed update's
// contributions to one entry of b, timed on the same stream of target
// indices (the measurements behind the executors' use of reductions at L2):
//   mode 0: reduction at L2, red.global.add.f64 target[idx[i]] += 1;
//   mode 1: plain load, add and store of target[idx[i]] (what a
//           conflict-free schedule allows; indices that repeat race);
//   mode 2: FP64 atomic add in the block's shared memory, slot idx[i] % 4096;
//   mode 3: FP64 atomic add in the shared memory of the other block of a
//           two-block cluster (distributed shared memory), same slots;
//   mode 4: bulk reduction (cp.reduce.async.bulk .add.f64) of a 16-double
//           row from shared memory into target[16 idx[i] .. 16 idx[i] + 15].
// Modes 2 and 3 store each block's slot 0 into target[block] at the end.
// ---------------------------------------------------------------------------
namespace race_probe {

// indices are clamped to [0, hi] so that a wrong index array cannot leave the target
__device__ __forceinline__ int64_t clamp_index(int32_t v, int32_t hi) {
    return static_cast<int64_t>(min(static_cast<uint32_t>(v), static_cast<uint32_t>(hi)));
}

__global__ void __launch_bounds__(kThreads) k_red_global(const int32_t* __restrict__ idx, int64_t m, int32_t hi,
                                                         double* t) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * kThreads)
        atomicAdd(t + clamp_index(__ldg(idx + i), hi), 1.0);
}

__global__ void __launch_bounds__(kThreads) k_rmw_global(const int32_t* __restrict__ idx, int64_t m, int32_t hi,
                                                         double* t) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * kThreads) {
        const int64_t c = clamp_index(__ldg(idx + i), hi);
        t[c] = t[c] + 1.0;
    }
}

__global__ void __launch_bounds__(kThreads) k_red_shared(const int32_t* __restrict__ idx, int64_t m, double* t) {
    __shared__ double s[4096];
    for (int i = threadIdx.x; i < 4096; i += kThreads) s[i] = 0.0;
    __syncthreads();
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * kThreads)
        atomicAdd(s + (__ldg(idx + i) & 4095), 1.0);
    __syncthreads();
    if (threadIdx.x == 0) t[blockIdx.x] = s[0];
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads)
    k_red_cluster(const int32_t* __restrict__ idx, int64_t m, double* t) {
    __shared__ double s[4096];
    for (int i = threadIdx.x; i < 4096; i += kThreads) s[i] = 0.0;
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    uint32_t rank, remote;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(remote)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(s))), "r"(rank ^ 1u));
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * kThreads) {
        const uint32_t a = remote + static_cast<uint32_t>(__ldg(idx + i) & 4095) * 8u;
        asm volatile("red.shared::cluster.add.f64 [%0], %1;" ::"r"(a), "d"(1.0) : "memory");
    }
    // the peer's adds into this block's array finish before either block leaves
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (threadIdx.x == 0) t[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kThreads) k_bulk_rows(const int32_t* __restrict__ idx, int64_t m, int32_t hi,
                                                        double* t) {
    __shared__ __align__(128) double s[kThreads][16];
    for (int c = 0; c < 16; ++c) s[threadIdx.x][c] = 1.0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(&s[threadIdx.x][0]));
    int pend = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * kThreads) {
        double* dst = t + clamp_index(__ldg(idx + i), hi) * 16;
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], 128;" ::"l"(dst), "r"(sa)
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        if (++pend >= 8) {
            asm volatile("cp.async.bulk.wait_group.read 4;" ::: "memory");
            pend = 4;
        }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace race_probe

extern "C" int race_probe_reductions(int32_t mode, const int32_t* idx_d, int64_t m, int32_t max_index, double* target_d,
                                     int64_t n_target, void* stream) {
    const int grid = race_device_sms() * 8;  // even: whole clusters of two
    const int64_t need = mode == 4 ? 16 * (static_cast<int64_t>(max_index) + 1)
                                   : (mode == 2 || mode == 3 ? std::max<int64_t>(grid, max_index + 1)
                                                             : static_cast<int64_t>(max_index) + 1);
    if (mode < 0 || mode > 4 || !idx_d || !target_d || m < 0 || max_index < 0 || n_target < need ||
        (reinterpret_cast<uintptr_t>(target_d) & 15u)) {
        race_set_detail("race_probe_reductions: bad mode, NULL, or a target array too small for the indices "
                        "(16 (max_index + 1) doubles for mode 4; at least one per block for modes 2 and 3)");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (mode) {
        case 0: race_probe::k_red_global<<<grid, race_probe::kThreads, 0, st>>>(idx_d, m, max_index, target_d); break;
        case 1: race_probe::k_rmw_global<<<grid, race_probe::kThreads, 0, st>>>(idx_d, m, max_index, target_d); break;
        case 2: race_probe::k_red_shared<<<grid, race_probe::kThreads, 0, st>>>(idx_d, m, target_d); break;
        case 3: race_probe::k_red_cluster<<<grid, race_probe::kThreads, 0, st>>>(idx_d, m, target_d); break;
        default: race_probe::k_bulk_rows<<<grid, race_probe::kThreads, 0, st>>>(idx_d, m, max_index, target_d); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_probe_reductions: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}
