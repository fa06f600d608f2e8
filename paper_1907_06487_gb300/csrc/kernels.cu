// Device kernels and the compute entry points of the C ABI (sm_103a).
//
// SymmSpMV (Alg. "SymmSpMV"): each stored upper entry a_rc updates both
// b[r] (row sum, gathered) and b[c] (scattered).  The RACE phases make the
// scatter safe: leaves of one phase are distance-2 independent, so their
// write sets {rows} U {upper columns of the rows} are disjoint and no two
// concurrently running leaves touch the same entry of b.  One leaf runs on
// one group of G lanes: rows in order, the lanes sharing the row's
// nonzeros (the paper's SIMD-vectorised inner loop with VECWIDTH = G).
// Because a phase's write sets are disjoint, b is read and written with
// plain (non-atomic) loads and stores; the kernel boundary between phases
// orders the phases.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "df64.cuh"
#include "int_product.cuh"
#include "fp64_share.cuh"
#include "race_internal.h"

namespace {

constexpr int kBlock = 256;

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

template <int G>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// A stored value as a double; FP32 values are widened with integer
// operations (df64::widen), not on the FP64 pipe.
template <typename VT>
__device__ __forceinline__ double ldv(const VT* p) {
    return df64::widen(__ldg(p));
}

// One phase of SymmSpMV: leaves [0, nleaf) of this phase.
template <typename VT, int G>
__global__ void __launch_bounds__(kBlock) k_symm_phase(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                      const VT* __restrict__ val, const double* __restrict__ x,
                                                      double* b, const int32_t* __restrict__ llo,
                                                      const int32_t* __restrict__ lhi, int32_t nleaf) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * kBlock / G;
    for (int64_t q = gid; q < nleaf; q += ngroups) {
        const int32_t lo = __ldg(llo + q), hi = __ldg(lhi + q);
        int32_t rs = __ldg(rp + lo);
        for (int32_t r = lo; r < hi; ++r) {
            const int32_t re = __ldg(rp + r + 1);
            const double xr = __ldg(x + r);
            double tmp = 0.0;
            for (int32_t idx = rs + lane; idx < re; idx += G) {
                const double a = ldv(val + idx);
                if (idx == rs) {
                    tmp += a * xr;  // diagonal: first entry of the row
                } else {
                    const int32_t c = __ldg(col + idx);
                    tmp += a * __ldg(x + c);
                    b[c] += a * xr;
                }
            }
            tmp = group_sum<G>(tmp, mask);
            if (lane == 0) b[r] += tmp;
            __syncwarp(mask);
            rs = re;
        }
    }
}

// One phase of SymmSpMV with one CTA per leaf: the CTA's groups take the
// leaf's rows round-robin; updates inside the leaf use reductions at L2
// (red.global.add.f64).  Leaves of a phase are distance-2 independent, so no
// two CTAs ever update the same entry of b.
template <typename VT, int G>
__global__ void __launch_bounds__(kBlock) k_symm_phase_cta(const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col,
                                                          const VT* __restrict__ val, const double* __restrict__ x,
                                                          double* b, const int32_t* __restrict__ llo,
                                                          const int32_t* __restrict__ lhi, int32_t nleaf) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int grp = threadIdx.x / G;
    constexpr int kGroups = kBlock / G;
    for (int64_t q = blockIdx.x; q < nleaf; q += gridDim.x) {
        const int32_t lo = __ldg(llo + q), hi = __ldg(lhi + q);
        for (int32_t r = lo + grp; r < hi; r += kGroups) {
            const int32_t rs = __ldg(rp + r), re = __ldg(rp + r + 1);
            const double xr = __ldg(x + r);
            double tmp = 0.0;
            // four independent entries per lane and step (loads before uses)
            for (int32_t idx = rs + lane; idx < re; idx += 4 * G) {
                double a[4], xc[4];
                int32_t c[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int32_t j = idx + t * G;
                    const bool v = j < re;
                    a[t] = v ? ldv(val + j) : 0.0;
                    c[t] = v ? __ldg(col + j) : -1;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) xc[t] = c[t] >= 0 ? __ldg(x + c[t]) : 0.0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (c[t] < 0) continue;
                    tmp = fma(a[t], xc[t], tmp);
                    if (c[t] != r) atomicAdd(b + c[t], a[t] * xr);
                }
            }
            tmp = group_sum<G>(tmp, mask);
            if (lane == 0) atomicAdd(b + r, tmp);
        }
    }
}

// SymmSpMV without a schedule: all rows at once, every update a reduction
// at L2.  A comparison point only (correct for any row order).
template <typename VT, int G>
__global__ void __launch_bounds__(kBlock) k_symm_atomic(int32_t n, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                       const double* __restrict__ x, double* b) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * kBlock / G;
    for (int64_t r = gid; r < n; r += ngroups) {
        const int32_t rs = __ldg(rp + r), re = __ldg(rp + r + 1);
        const double xr = __ldg(x + r);
        double tmp = 0.0;
        for (int32_t idx = rs + lane; idx < re; idx += G) {
            const double a = ldv(val + idx);
            if (idx == rs) {
                tmp += a * xr;
            } else {
                const int32_t c = __ldg(col + idx);
                tmp += a * __ldg(x + c);
                atomicAdd(b + c, a * xr);
            }
        }
        tmp = group_sum<G>(tmp, mask);
        if (lane == 0) atomicAdd(b + r, tmp);
    }
}

// One phase of SymmSpMM with k right-hand sides (row-major n x k).  A warp
// runs one leaf; lane l serves column l % K of nonzero slot l / K.
template <typename VT, int K>
__global__ void __launch_bounds__(kBlock) k_symm_mm_phase(const int32_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                         const double* __restrict__ X, double* B,
                                                         const int32_t* __restrict__ llo,
                                                         const int32_t* __restrict__ lhi, int32_t nleaf) {
    constexpr int S = 32 / K;  // nonzero slots per warp
    const int lane = threadIdx.x & 31;
    const int c = lane % K, slot = lane / K;
    const int64_t wid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / 32;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * kBlock / 32;
    for (int64_t q = wid; q < nleaf; q += nwarps) {
        const int32_t lo = __ldg(llo + q), hi = __ldg(lhi + q);
        int32_t rs = __ldg(rp + lo);
        for (int32_t r = lo; r < hi; ++r) {
            const int32_t re = __ldg(rp + r + 1);
            const double xr = __ldg(X + static_cast<int64_t>(r) * K + c);
            double tmp = 0.0;
            for (int32_t idx = rs + slot; idx < re; idx += S) {
                const double a = ldv(val + idx);
                if (idx == rs) {
                    tmp += a * xr;
                } else {
                    const int64_t cc = __ldg(col + idx);
                    tmp += a * __ldg(X + cc * K + c);
                    B[cc * K + c] += a * xr;
                }
            }
#pragma unroll
            for (int o = 16; o >= K; o >>= 1) tmp += __shfl_xor_sync(0xffffffffu, tmp, o);
            if (slot == 0) B[static_cast<int64_t>(r) * K + c] += tmp;
            __syncwarp();
            rs = re;
        }
    }
}

// Alg. "SpMV using the CRS format" on the full matrix, G lanes per row.
template <typename VT, int G>
__global__ void __launch_bounds__(kBlock) k_spmv_full(int32_t n, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                     const double* __restrict__ x, double* __restrict__ b) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * kBlock / G;
    for (int64_t r = gid; r < n; r += ngroups) {
        const int32_t rs = __ldg(rp + r), re = __ldg(rp + r + 1);
        double tmp = 0.0;
        for (int32_t idx = rs + lane; idx < re; idx += G) tmp += ldv(val + idx) * __ldg(x + __ldg(col + idx));
        tmp = group_sum<G>(tmp, mask);
        if (lane == 0) b[r] = tmp;
    }
}

// Row-block streaming kernels.  A group of G lanes owns U consecutive rows;
// their nonzeros form one contiguous range that the lanes stream through
// (coalesced, two independent loads in flight per lane), each lane finding
// its row by comparing the index against the U+1 row starts.
template <int U>
__device__ __forceinline__ int row_of(int32_t idx, const int32_t (&rb)[U + 1]) {
    int u = 0;
#pragma unroll
    for (int j = 1; j < U; ++j) u += (idx >= rb[j]);
    return u;
}

// Alg. "SpMV using the CRS format", row-block streaming.
template <typename VT, int G, int U>
__global__ void __launch_bounds__(kBlock) k_spmv_rows(int32_t n, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                     const double* __restrict__ x, double* __restrict__ b) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * kBlock / G;
    const int64_t nblk = (static_cast<int64_t>(n) + U - 1) / U;
    for (int64_t blk = gid; blk < nblk; blk += ngroups) {
        const int32_t r0 = static_cast<int32_t>(blk * U);
        int32_t rb[U + 1];
#pragma unroll
        for (int j = 0; j <= U; ++j) rb[j] = __ldg(rp + min(r0 + j, n));
        double acc[U];
#pragma unroll
        for (int j = 0; j < U; ++j) acc[j] = 0.0;
        // four independent entries per lane and iteration
        for (int32_t idx = rb[0] + lane; idx < rb[U]; idx += 4 * G) {
            double a[4], p[4];
            int32_t c[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int32_t j = idx + t * G;
                const bool v = j < rb[U];
                a[t] = v ? ldv(val + j) : 0.0;
                c[t] = v ? __ldg(col + j) : -1;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) p[t] = c[t] >= 0 ? a[t] * __ldg(x + c[t]) : 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int u = row_of<U>(idx + t * G, rb);
#pragma unroll
                for (int j = 0; j < U; ++j) acc[j] += (u == j ? p[t] : 0.0);
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const double v = group_sum<G>(acc[j], mask);
            if (lane == j && r0 + j < n) b[r0 + j] = v;
        }
    }
}

// SymmSpMV over all rows at once, row-block streaming; the scatter of the
// transposed part and the row sums go to b as reductions at L2.
template <typename VT, int G, int U>
__global__ void __launch_bounds__(kBlock) k_symm_rows_red(int32_t n, const int32_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                         const double* __restrict__ x, double* b) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * kBlock / G;
    const int64_t nblk = (static_cast<int64_t>(n) + U - 1) / U;
    for (int64_t blk = gid; blk < nblk; blk += ngroups) {
        const int32_t r0 = static_cast<int32_t>(blk * U);
        int32_t rb[U + 1];
        double xr[U];
#pragma unroll
        for (int j = 0; j <= U; ++j) rb[j] = __ldg(rp + min(r0 + j, n));
#pragma unroll
        for (int j = 0; j < U; ++j) xr[j] = __ldg(x + min(r0 + j, n - 1));
        double acc[U];
#pragma unroll
        for (int j = 0; j < U; ++j) acc[j] = 0.0;
        // four independent entries per lane and iteration
        for (int32_t idx = rb[0] + lane; idx < rb[U]; idx += 4 * G) {
            double a[4], xc[4];
            int32_t c[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int32_t j = idx + t * G;
                const bool v = j < rb[U];
                a[t] = v ? ldv(val + j) : 0.0;
                c[t] = v ? __ldg(col + j) : -1;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) xc[t] = c[t] >= 0 ? __ldg(x + c[t]) : 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (c[t] < 0) continue;
                const int u = row_of<U>(idx + t * G, rb);
                double xrow = xr[0];
#pragma unroll
                for (int j = 1; j < U; ++j) xrow = (u == j) ? xr[j] : xrow;
                const double prod = a[t] * xc[t];
                if (c[t] != r0 + u) atomicAdd(b + c[t], a[t] * xrow);  // transposed part
#pragma unroll
                for (int j = 0; j < U; ++j) acc[j] += (u == j ? prod : 0.0);
            }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const double v = group_sum<G>(acc[j], mask);
            if (lane == j && r0 + j < n) atomicAdd(b + r0 + j, v);
        }
    }
}

// One row per thread, software-pipelined over the thread's rows (rows
// tid, tid + T, tid + 2T, ... with T threads in the grid, so a warp holds 32
// consecutive rows at each step).  Each iteration has three independent load
// groups in flight: the x gathers of row i, the val/col of row i+1 and the
// row pointers of row i+2.  The first P entries of a row live in registers;
// longer rows finish their tail with plain loads.
//   SYMM = false: b[r] = sum (full CRS, Alg. "SpMV using the CRS format").
//   SYMM = true : upper CRS; the transposed updates and the row sums are
//                 reductions at L2 into b (zeroed before).
template <typename VT, int P, bool SYMM>
__global__ void __launch_bounds__(kBlock) k_rows_pipe(int32_t n, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                     const double* __restrict__ x, double* b) {
    const int64_t T = static_cast<int64_t>(gridDim.x) * kBlock;
    int64_t r0 = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (r0 >= n) return;
    int64_t r1 = r0 + T;
    int32_t rs0 = __ldg(rp + r0), re0 = __ldg(rp + r0 + 1);
    int32_t rs1 = 0, re1 = 0;
    if (r1 < n) {
        rs1 = __ldg(rp + r1);
        re1 = __ldg(rp + r1 + 1);
    }
    double a0[P];
    int32_t c0[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const bool v = rs0 + p < re0;
        a0[p] = v ? ldv(val + rs0 + p) : 0.0;
        c0[p] = v ? __ldg(col + rs0 + p) : -1;
    }
    while (true) {
        // x gathers of the current row
        double x0[P];
#pragma unroll
        for (int p = 0; p < P; ++p) x0[p] = c0[p] >= 0 ? __ldg(x + c0[p]) : 0.0;
        const double xr = SYMM ? __ldg(x + r0) : 0.0;
        // val/col of the next row
        double a1[P];
        int32_t c1[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const bool v = rs1 + p < re1;
            a1[p] = v ? ldv(val + rs1 + p) : 0.0;
            c1[p] = v ? __ldg(col + rs1 + p) : -1;
        }
        // row pointers of the row after next
        const int64_t r2 = r1 + T;
        int32_t rs2 = 0, re2 = 0;
        if (r2 < n) {
            rs2 = __ldg(rp + r2);
            re2 = __ldg(rp + r2 + 1);
        }
        // current row
        double acc = 0.0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (c0[p] < 0) continue;
            acc += a0[p] * x0[p];
            if (SYMM && c0[p] != r0) atomicAdd(b + c0[p], a0[p] * xr);
        }
        for (int32_t j = rs0 + P; j < re0; ++j) {
            const double a = ldv(val + j);
            const int32_t c = __ldg(col + j);
            acc += a * __ldg(x + c);
            if (SYMM && c != r0) atomicAdd(b + c, a * xr);
        }
        if (SYMM) atomicAdd(b + r0, acc);
        else b[r0] = acc;
        // rotate the pipeline
        if (r1 >= n) break;
        r0 = r1;
        rs0 = rs1;
        re0 = re1;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            a0[p] = a1[p];
            c0[p] = c1[p];
        }
        r1 = r2;
        rs1 = rs2;
        re1 = re2;
    }
}

// SymmSpMM with K right-hand sides (row-major n x K), all rows at once: a
// group of K lanes owns a row, lane c serves column c, so the K values of
// a row of X or B are contiguous across the group.  Updates of B are
// reductions at L2 (B zeroed before).  R rows per group in flight.
// DF: the transposed updates a_ij X[i][c] by the integer product of the
// significands (int_product.cuh; off-diagonal values range-checked once),
// the row sums stay FP64; a row whose X[i][c] lies outside the range
// [2^-50, 2^51) scatters that column in FP64 after its main loop.
template <typename VT, int K, int R, bool DF>
__global__ void __launch_bounds__(kBlock) k_symm_mm_rows_red(int32_t n, const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const VT* __restrict__ val, const double* __restrict__ X,
                                                            double* B, int fp64_quarters) {
    const int c = threadIdx.x & (K - 1);
    // fp64_quarters of every four warp-wide row groups scatter in FP64
    // (warp-uniform, spread over the SM's FP64 units)
    const int64_t grp = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / K;
    const int64_t ngrp = static_cast<int64_t>(gridDim.x) * kBlock / K;
    for (int64_t r0 = grp; r0 < n; r0 += ngrp * R) {
        const bool warp64 = fp64_group(static_cast<uint32_t>(static_cast<uint64_t>(r0) / (32 / K)), fp64_quarters);
        int32_t js[R], je[R];
        double xr[R], acc[R];
        float xrh[R], xrl[R];
        intprod::Factor xf[R];
        bool xr64[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int64_t r = r0 + q * ngrp;
            const bool v = r < n;
            js[q] = v ? __ldg(rp + r) : 0;
            je[q] = v ? __ldg(rp + r + 1) : 0;
            xr[q] = v ? __ldg(X + r * K + c) : 0.0;
            acc[q] = 0.0;
            xr64[q] = DF && df64::split(xr[q], xrh[q], xrl[q]) != 0;  // the range test of x_r
            xf[q] = intprod::factor(xr[q]);
        }
        int32_t len = 0;
#pragma unroll
        for (int q = 0; q < R; ++q) len = max(len, je[q] - js[q]);
        // U entries of each of the R rows per step: all loads of a step are
        // issued before their uses (two dependent round trips per step, not
        // per entry)
        constexpr int U = 4;
        for (int32_t p = 0; p < len; p += U) {
            VT araw[R][U];
            double xc[R][U];
            int32_t cc[R][U];
#pragma unroll
            for (int q = 0; q < R; ++q)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool v = js[q] + p + u < je[q];
                    araw[q][u] = v ? __ldg(val + js[q] + p + u) : VT(0);
                    cc[q][u] = v ? __ldg(col + js[q] + p + u) : -1;
                }
#pragma unroll
            for (int q = 0; q < R; ++q)
#pragma unroll
                for (int u = 0; u < U; ++u)
                    xc[q][u] = cc[q][u] >= 0 ? __ldg(X + static_cast<int64_t>(cc[q][u]) * K + c) : 0.0;
#pragma unroll
            for (int q = 0; q < R; ++q)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (cc[q][u] < 0) continue;
                    const double a = df64::widen(araw[q][u]);
                    acc[q] = fma(a, xc[q][u], acc[q]);
                    if (p + u == 0) continue;  // the diagonal (first entry) has no transposed update
                    if constexpr (DF) {
                        if (warp64) {  // warp-uniform: this warp's share of FP64 products
                            if (!xr64[q]) atomicAdd(B + static_cast<int64_t>(cc[q][u]) * K + c, a * xr[q]);
                        } else if (xrh[q] != 0.0f && !df64::is_zero(araw[q][u])) {
                            atomicAdd(B + static_cast<int64_t>(cc[q][u]) * K + c, intprod::mul(araw[q][u], xf[q]));
                        }
                    } else {
                        atomicAdd(B + static_cast<int64_t>(cc[q][u]) * K + c, a * xr[q]);
                    }
                }
        }
        if constexpr (DF) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (!xr64[q]) continue;
                for (int32_t j = js[q] + 1; j < je[q]; ++j)
                    atomicAdd(B + static_cast<int64_t>(__ldg(col + j)) * K + c, ldv(val + j) * xr[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int64_t r = r0 + q * ngrp;
            if (r < n) atomicAdd(B + r * K + c, acc[q]);
        }
    }
}

// How a row of k_symm_mm_rows_df forms its transposed products: the integer
// product (int_product.cuh), FP64 multiplies, or none (x_r is zero).
enum MmScatter { kMmIntProd = 0, kMmFp64 = 1, kMmNone = 2 };

// One row of k_symm_mm_rows_df for the lane of right-hand side c: the FP64
// row sum is returned, the transposed updates go to B as reductions.  The
// mode is fixed for the whole row, so the entry loop carries no per-entry
// mode branches (3-9 % faster than choosing per entry).
template <typename VT, int K, int MODE>
__device__ __forceinline__ double mm_row_df(int32_t js, int32_t je, int c, const int32_t* __restrict__ col,
                                            const VT* __restrict__ val, const double* __restrict__ X, double* B,
                                            double xr, const intprod::Factor& xf) {
    double acc = 0.0;
    constexpr int U = 4;
    for (int32_t p = js; p < je; p += U) {
        VT araw[U];
        double xc[U];
        int32_t cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool v = p + u < je;
            araw[u] = v ? __ldg(val + p + u) : VT(0);
            cc[u] = v ? __ldg(col + p + u) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xc[u] = cc[u] >= 0 ? __ldg(X + static_cast<int64_t>(cc[u]) * K + c) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (cc[u] < 0) continue;
            const double a = df64::widen(araw[u]);
            acc = fma(a, xc[u], acc);
            if (p + u == js) continue;  // the diagonal (first entry) has no transposed update
            if constexpr (MODE == kMmIntProd) {
                if (!df64::is_zero(araw[u])) atomicAdd(B + static_cast<int64_t>(cc[u]) * K + c, intprod::mul(araw[u], xf));
            } else if constexpr (MODE == kMmFp64) {
                atomicAdd(B + static_cast<int64_t>(cc[u]) * K + c, a * xr);
            }
        }
    }
    return acc;
}

// SymmSpMM with the transposed products off the FP64 pipe, one row per group
// of K lanes (lane c owns right-hand side c) and rows strided over the grid.
// The lane's mode for the row: x_r outside the range [2^-50, 2^51) or a row
// group of the FP64 share (warp-uniform, fp64_quarters of every four, spread
// over the SM's FP64 units): FP64 multiplies; x_r zero: no transposed
// updates; else the integer product of the significands.
template <typename VT, int K>
__global__ void __launch_bounds__(kBlock, 6) k_symm_mm_rows_df(int32_t n, const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const VT* __restrict__ val, const double* __restrict__ X,
                                                           double* B, int fp64_quarters) {
    const int c = threadIdx.x & (K - 1);
    const int64_t grp = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / K;
    const int64_t ngrp = static_cast<int64_t>(gridDim.x) * kBlock / K;
    for (int64_t r = grp; r < n; r += ngrp) {
        const bool warp64 = fp64_group(static_cast<uint32_t>(static_cast<uint64_t>(r) / (32 / K)), fp64_quarters);
        const int32_t js = __ldg(rp + r), je = __ldg(rp + r + 1);
        const double xr = __ldg(X + r * K + c);
        float xrh, xrl;
        const int st = df64::split(xr, xrh, xrl);  // the range test of x_r
        const intprod::Factor xf = intprod::factor(xr);
        double acc;
        if (st != 0 || warp64) acc = mm_row_df<VT, K, kMmFp64>(js, je, c, col, val, X, B, xr, xf);
        else if (xrh == 0.0f) acc = mm_row_df<VT, K, kMmNone>(js, je, c, col, val, X, B, xr, xf);
        else acc = mm_row_df<VT, K, kMmIntProd>(js, je, c, col, val, X, B, xr, xf);
        atomicAdd(B + r * K + c, acc);
    }
}

// Diagnostics of race_probe_scatter, shaped like the row-parallel executors
// (one row per thread, four entries per step): mode 0 replays the transposed
// update's reductions with a constant value, mode 1 streams the column
// indices alone.
template <int MODE>
__global__ void __launch_bounds__(kBlock) k_probe_scatter(int32_t n, const int32_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col, double* b) {
    const int64_t T = static_cast<int64_t>(gridDim.x) * kBlock;
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x; r < n; r += T) {
        const int32_t row = static_cast<int32_t>(r);
        const int32_t lo = __ldg(rp + row), hi = __ldg(rp + row + 1);
        int32_t sum = 0;
        for (int32_t idx = lo; idx < hi; idx += 4) {
            int32_t c[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) c[t] = idx + t < hi ? __ldg(col + idx + t) : -1;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if constexpr (MODE == 0) {
                    if (c[t] >= 0 && c[t] != row) atomicAdd(b + c[t], 1.0);
                } else {
                    sum += c[t] >= 0 ? c[t] : 0;
                }
            }
        }
        if constexpr (MODE == 1) b[row] = static_cast<double>(sum);
    }
}

__global__ void k_permute(int32_t n, int32_t k, const int32_t* __restrict__ perm, const double* __restrict__ in,
                          double* __restrict__ out, int inverse) {
    const int64_t total = static_cast<int64_t>(n) * k;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t q = t / k, c = t % k;
        const int64_t o = __ldg(perm + q);
        if (inverse) out[o * k + c] = in[t];
        else out[t] = in[o * k + c];
    }
}

int sm_count() { return race_device_sms(); }

int grid_for(int64_t threads_needed, int blocks_per_sm = 0) {
    const int64_t per_sm = blocks_per_sm > 0 ? blocks_per_sm : (2048 / kBlock);
    const int64_t cap = static_cast<int64_t>(sm_count()) * per_sm;
    int64_t blocks = (threads_needed + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min(blocks, cap)));
}

int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string(what) + ": " + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

template <typename VT, int G>
void launch_phases(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const auto& sp = s->plan.stage_ptr;
    const VT* val = static_cast<const VT*>(s->d_val);
    for (size_t p = 0; p + 1 < sp.size(); ++p) {
        const int32_t nl = sp[p + 1] - sp[p];
        if (nl == 0) continue;
        k_symm_phase<VT, G><<<grid_for(static_cast<int64_t>(nl) * G), kBlock, 0, st>>>(
            s->d_rp, s->d_col, val, x, b, s->d_leaf_lo + sp[p], s->d_leaf_hi + sp[p], nl);
    }
}

template <typename VT, int G, int U>
void launch_rows_red_gu(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const int32_t n = s->plan.n;
    const int64_t groups = (static_cast<int64_t>(n) + U - 1) / U;
    k_symm_rows_red<VT, G, U><<<grid_for(groups * G, s->launch.blocks_per_sm), kBlock, 0, st>>>(
        n, s->d_rp, s->d_col, static_cast<const VT*>(s->d_val), x, b);
}

template <typename VT, int G, int U>
void launch_full_gu(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const int32_t n = s->plan.n;
    const int64_t groups = (static_cast<int64_t>(n) + U - 1) / U;
    k_spmv_rows<VT, G, U><<<grid_for(groups * G, s->full_launch.blocks_per_sm), kBlock, 0, st>>>(
        n, s->d_frp, s->d_fcol, static_cast<const VT*>(s->d_fval), x, b);
}

template <typename VT, bool SYMM>
void launch_pipe(int32_t n, const int32_t* rp, const int32_t* col, const void* val, const double* x, double* b,
                 const race_launch& l, cudaStream_t st) {
    const int g = grid_for(n, l.blocks_per_sm);
    const VT* v = static_cast<const VT*>(val);
    if (l.regs_per_row <= 4) k_rows_pipe<VT, 4, SYMM><<<g, kBlock, 0, st>>>(n, rp, col, v, x, b);
    else if (l.regs_per_row <= 8) k_rows_pipe<VT, 8, SYMM><<<g, kBlock, 0, st>>>(n, rp, col, v, x, b);
    else k_rows_pipe<VT, 16, SYMM><<<g, kBlock, 0, st>>>(n, rp, col, v, x, b);
}

#define RACE_U_SWITCH(FN, VT, GG, u_, ...)          \
    do {                                            \
        if ((u_) == 1) FN<VT, GG, 1>(__VA_ARGS__);   \
        else if ((u_) == 2) FN<VT, GG, 2>(__VA_ARGS__); \
        else if ((u_) == 4) FN<VT, GG, 4>(__VA_ARGS__); \
        else FN<VT, GG, 8>(__VA_ARGS__);             \
    } while (0)
#define RACE_GU_SWITCH(FN, VT, G, U, ...)                                  \
    do {                                                                   \
        const int g_ = (G), u_ = (U);                                      \
        if (g_ == 1) RACE_U_SWITCH(FN, VT, 1, u_, __VA_ARGS__);            \
        else if (g_ == 2) RACE_U_SWITCH(FN, VT, 2, u_, __VA_ARGS__);       \
        else if (g_ == 4) RACE_U_SWITCH(FN, VT, 4, u_, __VA_ARGS__);       \
        else if (g_ == 8) RACE_U_SWITCH(FN, VT, 8, u_, __VA_ARGS__);       \
        else if (g_ == 16) RACE_U_SWITCH(FN, VT, 16, u_, __VA_ARGS__);     \
        else RACE_U_SWITCH(FN, VT, 32, u_, __VA_ARGS__);                   \
    } while (0)

template <typename VT, int G>
void launch_phases_cta(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const auto& sp = s->plan.stage_ptr;
    const VT* val = static_cast<const VT*>(s->d_val);
    const int cap = sm_count() * (2048 / kBlock);
    for (size_t p = 0; p + 1 < sp.size(); ++p) {
        const int32_t nl = sp[p + 1] - sp[p];
        if (nl == 0) continue;
        k_symm_phase_cta<VT, G><<<std::min(nl, cap), kBlock, 0, st>>>(s->d_rp, s->d_col, val, x, b,
                                                                       s->d_leaf_lo + sp[p], s->d_leaf_hi + sp[p], nl);
    }
}

template <typename VT, int G>
void launch_atomic(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const int32_t n = s->plan.n;
    k_symm_atomic<VT, G><<<grid_for(static_cast<int64_t>(n) * G), kBlock, 0, st>>>(
        n, s->d_rp, s->d_col, static_cast<const VT*>(s->d_val), x, b);
}

template <typename VT>
int launch_symm_exec(const race_schedule* s, int exec, const double* x, double* b, cudaStream_t st) {
#define RACE_DISPATCH(FN)                          \
    switch (s->group_lanes) {                      \
        case 4: FN<VT, 4>(s, x, b, st); break;     \
        case 8: FN<VT, 8>(s, x, b, st); break;     \
        case 16: FN<VT, 16>(s, x, b, st); break;   \
        default: FN<VT, 32>(s, x, b, st); break;   \
    }
    if (exec == RACE_EXEC_LEAF_CTA) {
        if (s->group_lanes == 1) launch_phases_cta<VT, 1>(s, x, b, st);
        else if (s->group_lanes == 2) launch_phases_cta<VT, 2>(s, x, b, st);
        else RACE_DISPATCH(launch_phases_cta)
    } else if (exec == RACE_EXEC_ATOMIC) {
        RACE_DISPATCH(launch_atomic)
    } else if (exec == RACE_EXEC_ROWS_RED || (exec == RACE_EXEC_STREAM_RED && s->max_row_upper > 1024)) {
        RACE_GU_SWITCH(launch_rows_red_gu, VT, s->launch.group_lanes, s->launch.rows_per_group, s, x, b, st);
    } else if (exec == RACE_EXEC_STREAM_RED) {
        const int rc = race_stream_symm_red(s, x, b, st, sm_count());
        if (rc) return rc;
    } else if (exec == RACE_EXEC_PIPE_RED) {
        launch_pipe<VT, true>(s->plan.n, s->d_rp, s->d_col, s->d_val, x, b, s->launch, st);
    } else if (exec == RACE_EXEC_WINDOW_RED || exec == RACE_EXEC_WINDOW_RACE) {
        const bool race_mode = exec == RACE_EXEC_WINDOW_RACE;
        if ((race_mode ? s->win_race.ready : s->win_red.ready))
            race_window_launch(s, race_mode, x, b, st, sm_count());
        else  // a row longer than the window: the row-block kernel serves it
            RACE_GU_SWITCH(launch_rows_red_gu, VT, 1, 1, s, x, b, st);
    } else {
        RACE_DISPATCH(launch_phases)
    }
#undef RACE_DISPATCH
    return RACE_OK;
}

template <typename VT>
void launch_symm(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    switch (s->group_lanes) {
        case 4: launch_phases<VT, 4>(s, x, b, st); break;
        case 8: launch_phases<VT, 8>(s, x, b, st); break;
        case 16: launch_phases<VT, 16>(s, x, b, st); break;
        default: launch_phases<VT, 32>(s, x, b, st); break;
    }
}

template <typename VT, int K>
void launch_mm(const race_schedule* s, const double* X, double* B, cudaStream_t st) {
    const auto& sp = s->plan.stage_ptr;
    const VT* val = static_cast<const VT*>(s->d_val);
    for (size_t p = 0; p + 1 < sp.size(); ++p) {
        const int32_t nl = sp[p + 1] - sp[p];
        if (nl == 0) continue;
        k_symm_mm_phase<VT, K><<<grid_for(static_cast<int64_t>(nl) * 32), kBlock, 0, st>>>(
            s->d_rp, s->d_col, val, X, B, s->d_leaf_lo + sp[p], s->d_leaf_hi + sp[p], nl);
    }
}

template <typename VT>
int launch_mm_k(const race_schedule* s, int32_t k, const double* X, double* B, cudaStream_t st) {
    const bool phased = s->launch.executor < RACE_EXEC_ATOMIC || s->launch.executor == RACE_EXEC_PERSIST_GROUP ||
                        s->launch.executor == RACE_EXEC_PERSIST_CTA;
    if (!phased) {
        // row-parallel SpMM with reductions (R rows per group in flight)
        const int32_t n = s->plan.n;
        const int R = s->launch.rows_per_group >= 4 ? 4 : (s->launch.rows_per_group >= 2 ? 2 : 1);
        const VT* v = static_cast<const VT*>(s->d_val);
        const bool df = s->launch.executor == RACE_EXEC_DF64_RED || s->launch.executor == RACE_EXEC_SELL_DF64 ||
                        s->launch.executor == RACE_EXEC_PHASE_DF64;
        const int q64 = df ? s->launch.fp64_quarters : 0;
        if (df) {
            const int rc = race_df64_prepare(s);
            if (rc) return rc;
        }
#define RACE_MM_ROWS_DF(KK, DFV)                                                                                   \
    do {                                                                                                           \
        const int g = grid_for((static_cast<int64_t>(n) * KK + R - 1) / R, s->launch.blocks_per_sm);              \
        if (R == 4) k_symm_mm_rows_red<VT, KK, 4, DFV><<<g, kBlock, 0, st>>>(n, s->d_rp, s->d_col, v, X, B, q64);        \
        else if (R == 2) k_symm_mm_rows_red<VT, KK, 2, DFV><<<g, kBlock, 0, st>>>(n, s->d_rp, s->d_col, v, X, B, q64);   \
        else if (DFV) k_symm_mm_rows_df<VT, KK><<<g, kBlock, 0, st>>>(n, s->d_rp, s->d_col, v, X, B, q64);               \
        else k_symm_mm_rows_red<VT, KK, 1, DFV><<<g, kBlock, 0, st>>>(n, s->d_rp, s->d_col, v, X, B, q64);               \
    } while (0)
#define RACE_MM_ROWS(KK)                 \
    do {                                 \
        if (df) RACE_MM_ROWS_DF(KK, true);  \
        else RACE_MM_ROWS_DF(KK, false);    \
    } while (0)
        switch (k) {
            case 1: RACE_MM_ROWS(1); break;
            case 2: RACE_MM_ROWS(2); break;
            case 4: RACE_MM_ROWS(4); break;
            case 8: RACE_MM_ROWS(8); break;
            case 16: RACE_MM_ROWS(16); break;
            default: race_set_detail("k must be 1, 2, 4, 8 or 16"); return RACE_ERR_UNSUPPORTED;
        }
#undef RACE_MM_ROWS
#undef RACE_MM_ROWS_DF
        return RACE_OK;
    }
    switch (k) {
        case 1: launch_mm<VT, 1>(s, X, B, st); break;
        case 2: launch_mm<VT, 2>(s, X, B, st); break;
        case 4: launch_mm<VT, 4>(s, X, B, st); break;
        case 8: launch_mm<VT, 8>(s, X, B, st); break;
        case 16: launch_mm<VT, 16>(s, X, B, st); break;
        default: race_set_detail("k must be 1, 2, 4, 8 or 16"); return RACE_ERR_UNSUPPORTED;
    }
    return RACE_OK;
}

template <typename VT, int G>
void launch_full_g(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const int32_t n = s->plan.n;
    k_spmv_full<VT, G><<<grid_for(static_cast<int64_t>(n) * G), kBlock, 0, st>>>(
        n, s->d_frp, s->d_fcol, static_cast<const VT*>(s->d_fval), x, b);
}

template <typename VT>
void launch_full(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    switch (s->full_lanes) {
        case 4: launch_full_g<VT, 4>(s, x, b, st); break;
        case 8: launch_full_g<VT, 8>(s, x, b, st); break;
        case 16: launch_full_g<VT, 16>(s, x, b, st); break;
        default: launch_full_g<VT, 32>(s, x, b, st); break;
    }
}

int precheck(const race_schedule* s, const void* a, const void* b) {
    if (!s || !a || !b) {
        race_set_detail("NULL argument");
        return RACE_ERR_INVALID;
    }
    if (s->host_only) {
        race_set_detail("schedule was built with RACE_FLAG_HOST_ONLY");
        return RACE_ERR_UNSUPPORTED;
    }
    if (a == b) {
        race_set_detail("input and output alias");
        return RACE_ERR_INVALID;
    }
    return RACE_OK;
}

}  // namespace

extern "C" {

int symm_spmv(const race_schedule* s, const double* x_d, double* b_d, void* stream) {
    int rc = precheck(s, x_d, b_d);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b_d, 0, sizeof(double) * static_cast<size_t>(s->plan.n), st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("memset: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    if (s->launch.executor == RACE_EXEC_DF64_RED) return race_df64_launch(s, x_d, b_d, st);
    if (s->launch.executor == RACE_EXEC_SELL_DF64) return race_sell_launch(s, x_d, b_d, st);
    if (s->launch.executor == RACE_EXEC_STAGED) return race_staged_launch(s, s->launch, x_d, b_d, st, kStagedSpinLimit, 0);
    if (s->launch.executor == RACE_EXEC_PERSIST_GROUP || s->launch.executor == RACE_EXEC_PERSIST_CTA)
        return race_persist_launch(s, s->launch.executor, x_d, b_d, st);
    if (s->launch.executor == RACE_EXEC_PHASE_DF64) return race_df64_phase_launch(s, x_d, b_d, st);
    rc = s->val_type == RACE_F64 ? launch_symm_exec<double>(s, s->launch.executor, x_d, b_d, st)
                                 : launch_symm_exec<float>(s, s->launch.executor, x_d, b_d, st);
    if (rc) return rc;
    return check_launch("symm_spmv");
}

int symm_spmv_exec(const race_schedule* s, int32_t executor, const double* x_d, double* b_d, void* stream) {
    int rc = precheck(s, x_d, b_d);
    if (rc) return rc;
    if (executor < RACE_EXEC_LEAF_GROUP || executor > RACE_EXEC_PHASE_DF64) {
        race_set_detail("unknown executor");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b_d, 0, sizeof(double) * static_cast<size_t>(s->plan.n), st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("memset: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    if (executor == RACE_EXEC_DF64_RED) return race_df64_launch(s, x_d, b_d, st);
    if (executor == RACE_EXEC_SELL_DF64) return race_sell_launch(s, x_d, b_d, st);
    if (executor == RACE_EXEC_STAGED) return race_staged_launch(s, s->launch, x_d, b_d, st, kStagedSpinLimit, 0);
    if (executor == RACE_EXEC_PERSIST_GROUP || executor == RACE_EXEC_PERSIST_CTA)
        return race_persist_launch(s, executor, x_d, b_d, st);
    if (executor == RACE_EXEC_PHASE_DF64) return race_df64_phase_launch(s, x_d, b_d, st);
    rc = s->val_type == RACE_F64 ? launch_symm_exec<double>(s, executor, x_d, b_d, st)
                                 : launch_symm_exec<float>(s, executor, x_d, b_d, st);
    if (rc) return rc;
    return check_launch("symm_spmv_exec");
}

int symm_spmm(const race_schedule* s, int32_t k, const double* X_d, double* B_d, void* stream) {
    int rc = precheck(s, X_d, B_d);
    if (rc) return rc;
    if (k < 1 || k > 16) {
        race_set_detail("k must be in 1..16");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(B_d, 0, sizeof(double) * static_cast<size_t>(s->plan.n) * k, st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("memset: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    rc = s->val_type == RACE_F64 ? launch_mm_k<double>(s, k, X_d, B_d, st) : launch_mm_k<float>(s, k, X_d, B_d, st);
    if (rc) return rc;  // the detail is set where the error arose
    return check_launch("symm_spmm");
}

int spmv_full(const race_schedule* s, const double* x_d, double* b_d, void* stream) {
    int rc = precheck(s, x_d, b_d);
    if (rc) return rc;
    if (!s->d_frp) {
        rc = race_prepare_full(const_cast<race_schedule*>(s), stream);
        if (rc) return rc;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->full_launch.executor == 1 && s->max_row_full <= 1024) {
        rc = race_stream_full(s, x_d, b_d, st, sm_count());
        if (rc) return rc;
    } else if (s->full_launch.executor == 2 && s->val_type == RACE_F64)
        launch_pipe<double, false>(s->plan.n, s->d_frp, s->d_fcol, s->d_fval, x_d, b_d, s->full_launch, st);
    else if (s->full_launch.executor == 2)
        launch_pipe<float, false>(s->plan.n, s->d_frp, s->d_fcol, s->d_fval, x_d, b_d, s->full_launch, st);
    else if (s->val_type == RACE_F64)
        RACE_GU_SWITCH(launch_full_gu, double, s->full_launch.group_lanes, s->full_launch.rows_per_group, s, x_d, b_d, st);
    else
        RACE_GU_SWITCH(launch_full_gu, float, s->full_launch.group_lanes, s->full_launch.rows_per_group, s, x_d, b_d, st);
    return check_launch("spmv_full");
}

int race_set_launch(race_schedule* s, int32_t which, const race_launch* l) {
    if (!s || !l) {
        race_set_detail("NULL argument");
        return RACE_ERR_INVALID;
    }
    const bool g_ok = l->group_lanes == 1 || l->group_lanes == 2 || l->group_lanes == 4 || l->group_lanes == 8 || l->group_lanes == 16 || l->group_lanes == 32;
    const bool u_ok = l->rows_per_group == 1 || l->rows_per_group == 2 || l->rows_per_group == 4 || l->rows_per_group == 8;
    if (!g_ok || !u_ok || l->blocks_per_sm < 0 || l->blocks_per_sm > 2048 / kBlock ||
        l->executor < RACE_EXEC_LEAF_GROUP || l->executor > RACE_EXEC_PHASE_DF64 || l->regs_per_row < 0 ||
        l->regs_per_row > 16 || l->fp64_quarters < 0 || l->fp64_quarters > 4 || l->rowsum_fp64_quarters < 0 ||
        l->rowsum_fp64_quarters > 4 || (which != 0 && which != 1)) {
        race_set_detail("launch configuration out of range");
        return RACE_ERR_INVALID;
    }
    if (which == 0 && (l->executor == RACE_EXEC_DF64_RED || l->executor == RACE_EXEC_SELL_DF64 ||
                       l->executor == RACE_EXEC_PHASE_DF64)) {
        if (s->host_only) {
            race_set_detail("schedule was built with RACE_FLAG_HOST_ONLY");
            return RACE_ERR_UNSUPPORTED;
        }
        const int rc = l->executor == RACE_EXEC_SELL_DF64 ? race_sell_prepare(s) : race_df64_prepare(s);
        if (rc) return rc;
    }
    if (which == 0) {
        s->launch = *l;
        s->group_lanes = l->group_lanes;
    } else {
        s->full_launch = *l;
    }
    return RACE_OK;
}

int race_poll_status(race_schedule* s, void* stream) {
    if (!s) {
        race_set_detail("NULL schedule");
        return RACE_ERR_INVALID;
    }
    if (s->host_only || !s->d_status) return RACE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("status read: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    if (h != RACE_OK) {
        cudaMemsetAsync(s->d_status, 0, sizeof(int32_t), st);
        cudaStreamSynchronize(st);
        race_set_detail("a bounded device wait gave up");
        return h;
    }
    return RACE_OK;
}

int race_probe_scatter(const race_schedule* s, int32_t mode, double* b_d, void* stream) {
    int rc = precheck(s, s ? s->d_rp : nullptr, b_d);
    if (rc) return rc;
    if (mode != 0 && mode != 1) {
        race_set_detail("mode must be 0 (reductions) or 1 (column stream)");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int g = grid_for(s->plan.n, 4);
    if (mode == 0) k_probe_scatter<0><<<g, kBlock, 0, st>>>(s->plan.n, s->d_rp, s->d_col, b_d);
    else k_probe_scatter<1><<<g, kBlock, 0, st>>>(s->plan.n, s->d_rp, s->d_col, b_d);
    return check_launch("race_probe_scatter");
}

int race_get_launch(const race_schedule* s, int32_t which, race_launch* l) {
    if (!s || !l || (which != 0 && which != 1)) {
        race_set_detail("bad argument");
        return RACE_ERR_INVALID;
    }
    *l = which == 0 ? s->launch : s->full_launch;
    return RACE_OK;
}

static int permute_impl(const race_schedule* s, const double* in, double* out, int32_t k, void* stream, int inv) {
    int rc = precheck(s, in, out);
    if (rc) return rc;
    if (k < 1) {
        race_set_detail("k < 1");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_permute<<<grid_for(static_cast<int64_t>(s->plan.n) * k), kBlock, 0, st>>>(s->plan.n, k, s->d_perm, in, out, inv);
    return check_launch("race_permute");
}

int race_permute(const race_schedule* s, const double* in_d, double* out_d, int32_t k, void* stream) {
    return permute_impl(s, in_d, out_d, k, stream, 0);
}

int race_unpermute(const race_schedule* s, const double* in_d, double* out_d, int32_t k, void* stream) {
    return permute_impl(s, in_d, out_d, k, stream, 1);
}

}  // extern "C"
