// Streaming SpMV / SymmSpMV kernels: row blocks staged into shared memory by
// bulk copies (stream_engine.cuh), a persistent grid walking the blocks
// round-robin so that the blocks in flight form a contiguous window of rows
// (the level structure of the permuted matrix keeps x and b of that window
// in L2).
//
// Per block: (1) products of the block's nonzeros, all threads in parallel,
// each issuing independent x gathers; (2) row sums from the products.
//   kFull: Alg. "SpMV using the CRS format", b[row] = sum.
//   kSymmRed: Alg. "SymmSpMV" on the upper CRS; the transposed update
//             b[col] += a*x[row] and the row sum b[row] += sum are reductions
//             at L2 (red.global.add.f64), b zeroed beforehand.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "race_internal.h"
#include "stream_engine.cuh"

namespace race_dev {

constexpr int kThreads = 256;
enum Mode { kFull = 0, kSymmRed = 1 };

template <typename VT>
constexpr size_t stream_smem_bytes() {
    return sizeof(Stage<VT>) * kStages + sizeof(uint64_t) * kStages + sizeof(double) * (kChunk + 8) +
           sizeof(int32_t) * (kChunk + 8) + 128;
}

template <typename VT, int MODE>
__global__ void __launch_bounds__(kThreads) k_stream(int64_t nblk, const int32_t* __restrict__ blk_row,
                                                     const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                     const VT* __restrict__ val, const double* __restrict__ x,
                                                     double* b, int32_t* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    Stage<VT>* st = reinterpret_cast<Stage<VT>*>(base);
    uint64_t* bars = reinterpret_cast<uint64_t*>(st + kStages);
    double* prod = reinterpret_cast<double*>(bars + kStages);
    int32_t* rid = reinterpret_cast<int32_t*>(prod + kChunk + 8);
    const int tid = threadIdx.x;
    const int64_t first = blockIdx.x, stride = gridDim.x;

    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) mbar_init(&bars[q], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            const int64_t blk = first + q * stride;
            if (blk < nblk) issue_block(&st[q], &bars[q], block_geom(blk_row, rp, blk), val, col, rp);
        }
    }
    int64_t i = 0;
    bool failed = false;
    for (;; ++i) {
        const int64_t blk = first + i * stride;
        if (blk >= nblk) break;
        const int q = static_cast<int>(i % kStages);
        const BlockGeom g = block_geom(blk_row, rp, blk);
        const bool ok = mbar_wait(&bars[q], static_cast<uint32_t>((i / kStages) & 1));
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        Stage<VT>& S = st[q];
        const int nnz = g.e - g.s, off = g.s - g.s_al, nr = g.r1 - g.r0, roff = g.r0 - g.r0_al;
        if (MODE == kSymmRed) {
            for (int r = tid; r < nr; r += kThreads) {
                const int a = S.rp[roff + r] - g.s, z = S.rp[roff + r + 1] - g.s;
                for (int j = a; j < z; ++j) rid[j] = r;
            }
            __syncthreads();
        }
        // (1) products
        for (int j0 = tid; j0 < nnz; j0 += 4 * kThreads) {
            double xv[4];
            int32_t cj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u * kThreads;
                cj[u] = j < nnz ? S.col[off + j] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u * kThreads;
                xv[u] = j < nnz ? __ldg(x + cj[u]) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + u * kThreads;
                if (j >= nnz) continue;
                const double a = static_cast<double>(S.val[off + j]);
                if (MODE == kFull) {
                    prod[j] = a * xv[u];
                } else {
                    const int r = rid[j];
                    const int32_t row = g.r0 + r;
                    if (cj[u] == row) {
                        prod[j] = a * xv[u];  // diagonal: x[col] is x[row]
                    } else {
                        prod[j] = a * xv[u];
                        atomicAdd(b + cj[u], a * __ldg(x + row));
                    }
                }
            }
        }
        __syncthreads();
        // (2) row sums
        for (int r = tid; r < nr; r += kThreads) {
            const int a = S.rp[roff + r] - g.s, z = S.rp[roff + r + 1] - g.s;
            double sum = 0.0;
            for (int j = a; j < z; ++j) sum += prod[j];
            if (MODE == kFull) b[g.r0 + r] = sum;
            else atomicAdd(b + g.r0 + r, sum);
        }
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async();
            const int64_t nb = blk + kStages * stride;
            if (nb < nblk) issue_block(&S, &bars[q], block_geom(blk_row, rp, nb), val, col, rp);
        }
    }
    if (failed && tid == 0) {
        atomicExch(status, RACE_ERR_TIMEOUT);
        // drain the copies this block still has in flight (bounded)
        for (int64_t j = 1; j < kStages; ++j) {
            const int64_t blk = first + (i + j) * stride;
            if (blk < nblk) mbar_wait(&bars[(i + j) % kStages], static_cast<uint32_t>(((i + j) / kStages) & 1));
        }
    }
}

template <typename VT, int MODE>
int launch_stream(int64_t nblk, const int32_t* blk_row, const int32_t* rp, const int32_t* col, const VT* val,
                  const double* x, double* b, int32_t* status, int sm_count, int ctas_per_sm, cudaStream_t st) {
    static bool configured = false;
    const size_t smem = stream_smem_bytes<VT>();
    if (!configured) {
        cudaFuncSetAttribute(k_stream<VT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        configured = true;
    }
    if (nblk <= 0) return RACE_OK;
    const int per_sm = ctas_per_sm > 0 ? ctas_per_sm : 4;
    const int64_t grid = std::min<int64_t>(nblk, static_cast<int64_t>(sm_count) * per_sm);
    k_stream<VT, MODE><<<static_cast<int>(grid), kThreads, smem, st>>>(nblk, blk_row, rp, col, val, x, b, status);
    return RACE_OK;
}

}  // namespace race_dev

// Host-side entry points used by kernels.cu.
int race_stream_full(const race_schedule* s, const double* x, double* b, cudaStream_t st, int sm_count) {
    if (s->val_type == RACE_F64)
        return race_dev::launch_stream<double, race_dev::kFull>(
            s->n_fblk, s->d_fblk, s->d_frp, s->d_fcol, static_cast<const double*>(s->d_fval), x, b, s->d_status,
            sm_count, s->full_launch.blocks_per_sm, st);
    return race_dev::launch_stream<float, race_dev::kFull>(s->n_fblk, s->d_fblk, s->d_frp, s->d_fcol,
                                                           static_cast<const float*>(s->d_fval), x, b, s->d_status,
                                                           sm_count, s->full_launch.blocks_per_sm, st);
}

int race_stream_symm_red(const race_schedule* s, const double* x, double* b, cudaStream_t st, int sm_count) {
    if (s->val_type == RACE_F64)
        return race_dev::launch_stream<double, race_dev::kSymmRed>(
            s->n_blk, s->d_blk, s->d_rp, s->d_col, static_cast<const double*>(s->d_val), x, b, s->d_status,
            sm_count, s->launch.blocks_per_sm, st);
    return race_dev::launch_stream<float, race_dev::kSymmRed>(s->n_blk, s->d_blk, s->d_rp, s->d_col,
                                                              static_cast<const float*>(s->d_val), x, b, s->d_status,
                                                              sm_count, s->launch.blocks_per_sm, st);
}
