// SymmSpMV with the transposed products off the FP64 pipe (executor
// RACE_EXEC_DF64_RED).
//
// GB300 runs FP64 at about 1/70 of its FP32 rate.  The FP64 SymmSpMV (Alg.
// "SymmSpMV") issues one FP64 multiply-add per stored upper entry for the row
// sums and one FP64 multiply per off-diagonal entry for the transposed part:
// on the 4-body XXZ Hamiltonian (26 sites) 151 M FP64 operations, 0.30 ms at
// the measured 0.5 T/s, against 0.17 ms of HBM traffic.  Here the row sums
// stay exact FP64 multiply-adds (80.7 M, 0.16 ms of FP64 pipe) and each
// transposed update a_ij x_i of a share of the row groups is formed on the
// integer pipes (int_product.cuh): x_i prepared once per row, the two
// significands multiplied in 32-bit pieces, sign and exponent added as bit
// fields, the result a double ready for its reduction at L2.  The other row
// groups multiply in FP64, so the two pipes share the work.  b, x and the
// stored values stay FP64.  (Dekker's double-float product on the FP32 pipe,
// df64.cuh, did this job before: about 30 integer and FP32 instructions per
// update against about 15, and an error of 2^-44 against 2^-51.)
//
// Accuracy: every transposed update is the exact product truncated, within
// 2^-51 of it (checked against rational arithmetic by the CPU tests), so
// |b_i - exact| stays below (2^-51 + n_i 2^-53) sum_j |a_ij x_j| for any row
// length: inside 1e-12 sum_j |a_ij x_j|.  Rows whose x_i is zero contribute
// no updates; rows whose x_i lies outside [2^-50, 2^51) scatter in FP64.
// Stored off-diagonal values must be zero or inside that range (checked once
// when the executor is prepared).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "df64.cuh"
#include "fp64_share.cuh"
#include "int_product.cuh"
#include "race_internal.h"

namespace {

constexpr int kBlock = 256;

template <int G>
__device__ __forceinline__ unsigned lane_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

__host__ __device__ __forceinline__ bool out_of_range(double v) {
    float h, l;
    return df64::split(v, h, l) != 0;
}
__host__ __device__ __forceinline__ bool out_of_range(float v) {
    const uint32_t u = df64::f2u(v);
    const int e = static_cast<int>((u >> 23) & 0xFFu) - 127;
    return (u << 1) != 0 && (e < df64::kEmin || e > df64::kEmax);
}

// How a row scatters its transposed part.
enum Scatter { kIntProd = 0, kFp64 = 1, kNone = 2 };

// One row's share of one lane: FP64 row sum returned, transposed updates
// sent to b.  B (4 or 8) independent entries per lane and iteration.
template <typename VT, int G, int MODE, int B>
__device__ __forceinline__ double lane_row(int32_t row, int32_t lo, int32_t hi, int lane,
                                           const int32_t* __restrict__ col, const VT* __restrict__ val,
                                           const double* __restrict__ x, double* b, double xr,
                                           const intprod::Factor& xf) {
    double acc = 0.0;
    for (int32_t idx = lo + lane; idx < hi; idx += B * G) {
        VT a[B];
        int32_t c[B];
        double xc[B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
            const int32_t j = idx + t * G;
            const bool v = j < hi;
            a[t] = v ? __ldg(val + j) : VT(0);
            c[t] = v ? __ldg(col + j) : -1;
        }
#pragma unroll
        for (int t = 0; t < B; ++t) xc[t] = c[t] >= 0 ? __ldg(x + c[t]) : 0.0;
#pragma unroll
        for (int t = 0; t < B; ++t) {
            if (c[t] < 0) continue;
            acc = fma(df64::widen(a[t]), xc[t], acc);
            if constexpr (MODE == kIntProd) {
                if (c[t] != row && !df64::is_zero(a[t])) atomicAdd(b + c[t], intprod::mul(a[t], xf));
            } else if constexpr (MODE == kFp64) {
                if (c[t] != row) atomicAdd(b + c[t], df64::widen(a[t]) * xr);
            }
        }
    }
    return acc;
}

// One row on its G lanes: the FP64 row sum (combined by shuffles) goes to
// b[row] as a reduction at L2, the transposed updates of the other rows land
// there too (b is zeroed first).  warp64: this row's transposed products in
// FP64 (warp-uniform).
template <typename VT, int G, int B>
__device__ __forceinline__ void row_df64(int32_t row, int lane, unsigned mask, bool warp64,
                                         const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, const double* __restrict__ x, double* b) {
    const int32_t lo = __ldg(rp + row), hi = __ldg(rp + row + 1);
    const double xr = __ldg(x + row);
    float xrh, xrl;
    const int st = df64::split(xr, xrh, xrl);  // the range test of x_i
    const intprod::Factor xf = intprod::factor(xr);
    double acc;
    if (st != 0) acc = lane_row<VT, G, kFp64, B>(row, lo, hi, lane, col, val, x, b, xr, xf);
    else if (xrh == 0.0f) acc = lane_row<VT, G, kNone, B>(row, lo, hi, lane, col, val, x, b, xr, xf);
    else if (warp64) acc = lane_row<VT, G, kFp64, B>(row, lo, hi, lane, col, val, x, b, xr, xf);
    else acc = lane_row<VT, G, kIntProd, B>(row, lo, hi, lane, col, val, x, b, xr, xf);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, G);
    if (lane == 0) atomicAdd(b + row, acc);
}

// G lanes per row, rows strided over the grid.
template <typename VT, int G, int B>
__global__ void __launch_bounds__(kBlock) k_symm_df64(int32_t n, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                     const double* __restrict__ x, double* b, int fp64_quarters) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = lane_mask<G>();
    // fp64_quarters of every four warp-wide row groups scatter with FP64
    // multiplies (warp-uniform, spread over the SM's FP64 units), the rest by
    // the integer product: the work is shared between the FP64 and integer
    // pipes
    const int64_t gid = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    const int64_t ngroups = static_cast<int64_t>(gridDim.x) * kBlock / G;
    for (int64_t r = gid; r < n; r += ngroups) {
        const bool warp64 = fp64_group(static_cast<uint32_t>(static_cast<uint64_t>(r) / (32 / G)), fp64_quarters);
        row_df64<VT, G, B>(static_cast<int32_t>(r), lane, mask, warp64, rp, col, val, x, b);
    }
}

// One phase of the schedule (executor RACE_EXEC_PHASE_DF64): the rows of the
// phase's leaves (rows[0, nrows), leaf after leaf), one per thread, a block
// per 256 of them and the blocks taking those in turn; first[q] is the first
// row of the q-th 256 when they are consecutive rows (no list to read), else
// -1.  The rows of one leaf may run in different blocks, so their updates of
// shared entries of b are L2 reductions; the leaves of a phase never share
// an entry of b (Sec. 4.2), and the phases run in order, one launch each.
template <typename VT, int B>
__global__ void __launch_bounds__(kBlock) k_symm_df64_phase(const int32_t* __restrict__ rows,
                                                           const int32_t* __restrict__ first, int32_t nrows,
                                                           const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const VT* __restrict__ val, const double* __restrict__ x,
                                                           double* b, int fp64_quarters, uint32_t group_base) {
    static_assert(kBlock == kPhaseBlockRows, "a block takes one entry of the first-row table");
    for (int32_t q = blockIdx.x; static_cast<int64_t>(q) * kBlock < nrows; q += gridDim.x) {
        const int32_t i = q * kBlock + static_cast<int32_t>(threadIdx.x);
        const bool warp64 = fp64_group(group_base + static_cast<uint32_t>(i >> 5), fp64_quarters);
        const int32_t f = __ldg(first + q);
        if (i < nrows) {
            const int32_t row = f >= 0 ? f + static_cast<int32_t>(threadIdx.x) : __ldg(rows + i);
            row_df64<VT, 1, B>(row, 0, 1u << (threadIdx.x & 31), warp64, rp, col, val, x, b);
        }
    }
}

int sm_count_of_device() { return race_device_sms(); }

template <typename VT, int G>
void launch_g(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const int64_t threads = static_cast<int64_t>(s->plan.n) * G;
    const int64_t per_sm = s->launch.blocks_per_sm > 0 ? s->launch.blocks_per_sm : (2048 / kBlock);
    const int64_t cap = static_cast<int64_t>(sm_count_of_device()) * per_sm;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min((threads + kBlock - 1) / kBlock, cap)));
    const bool mine = s->launch.executor == RACE_EXEC_DF64_RED;
    const int q64 = mine ? s->launch.fp64_quarters : 0;
    const VT* v = static_cast<const VT*>(s->d_val);
    if (mine && s->launch.regs_per_row >= 8)
        k_symm_df64<VT, G, 8><<<blocks, kBlock, 0, st>>>(s->plan.n, s->d_rp, s->d_col, v, x, b, q64);
    else
        k_symm_df64<VT, G, 4><<<blocks, kBlock, 0, st>>>(s->plan.n, s->d_rp, s->d_col, v, x, b, q64);
}

template <typename VT>
void launch_vt(const race_schedule* s, int G, const double* x, double* b, cudaStream_t st) {
    switch (G) {
        case 1: launch_g<VT, 1>(s, x, b, st); break;
        case 2: launch_g<VT, 2>(s, x, b, st); break;
        case 4: launch_g<VT, 4>(s, x, b, st); break;
        case 8: launch_g<VT, 8>(s, x, b, st); break;
        case 16: launch_g<VT, 16>(s, x, b, st); break;
        default: launch_g<VT, 32>(s, x, b, st); break;
    }
}

}  // namespace

int race_df64_prepare(const race_schedule* s) {
    int32_t st = s->df64_state.load(std::memory_order_acquire);
    if (st == 0) {
        // one pass over the host copy of the permuted matrix (threads that
        // race here compute the same answer)
        bool bad = false;
        const int32_t n = s->plan.n;
        for (int32_t r = 0; r < n && !bad; ++r)
            for (int32_t j = s->h_rp[r]; j < s->h_rp[r + 1]; ++j) {
                if (s->h_col[j] == r) continue;
                if (s->val_type == RACE_F64 ? out_of_range(s->h_val64[j]) : out_of_range(s->h_val32[j])) {
                    bad = true;
                    break;
                }
            }
        st = bad ? -1 : 1;
        s->df64_state.store(st, std::memory_order_release);
    }
    if (st == -1) {
        race_set_detail("an off-diagonal value outside the magnitude range [2^-50, 2^51) of the integer product");
        return RACE_ERR_UNSUPPORTED;
    }
    return RACE_OK;
}

int race_df64_phase_launch(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    int rc = race_df64_prepare(s);
    if (rc) return rc;
    const bool mine = s->launch.executor == RACE_EXEC_PHASE_DF64;
    const int64_t per_sm = mine && s->launch.blocks_per_sm > 0 ? s->launch.blocks_per_sm : (2048 / kBlock);
    const int64_t cap = static_cast<int64_t>(sm_count_of_device()) * per_sm;
    const int q64 = mine ? s->launch.fp64_quarters : 0;
    const bool b8 = mine && s->launch.regs_per_row >= 8;
    const auto& pp = s->phase_row_ptr;
    for (size_t p = 0; p + 1 < pp.size(); ++p) {
        const int64_t nr = pp[p + 1] - pp[p];
        if (nr == 0) continue;
        const int grid = static_cast<int>(std::min((nr + kBlock - 1) / kBlock, cap));
        const int32_t* rows = s->d_phase_rows + pp[p];
        const int32_t* first = s->d_phase_blk + s->phase_blk_ptr[p];
        const int32_t nr32 = static_cast<int32_t>(nr);
        const uint32_t base = static_cast<uint32_t>(pp[p] >> 5);
        if (s->val_type == RACE_F64) {
            const double* v = static_cast<const double*>(s->d_val);
            if (b8) k_symm_df64_phase<double, 8><<<grid, kBlock, 0, st>>>(rows, first, nr32, s->d_rp, s->d_col, v, x, b, q64, base);
            else k_symm_df64_phase<double, 4><<<grid, kBlock, 0, st>>>(rows, first, nr32, s->d_rp, s->d_col, v, x, b, q64, base);
        } else {
            const float* v = static_cast<const float*>(s->d_val);
            if (b8) k_symm_df64_phase<float, 8><<<grid, kBlock, 0, st>>>(rows, first, nr32, s->d_rp, s->d_col, v, x, b, q64, base);
            else k_symm_df64_phase<float, 4><<<grid, kBlock, 0, st>>>(rows, first, nr32, s->d_rp, s->d_col, v, x, b, q64, base);
        }
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_df64_phase: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

int race_df64_launch(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    int rc = race_df64_prepare(s);
    if (rc) return rc;
    const int G = s->launch.executor == RACE_EXEC_DF64_RED ? s->launch.group_lanes : 1;
    if (s->val_type == RACE_F64) launch_vt<double>(s, G, x, b, st);
    else launch_vt<float>(s, G, x, b, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_df64: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}
