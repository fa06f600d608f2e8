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
#include <climits>
#include <cstdint>
#include <mutex>
#include <string>

#include "race_internal.h"
#include "stream_engine.cuh"
#include "red.cuh"

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
                        red_add_f64(b + cj[u], a * __ldg(x + row));
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
            else red_add_f64(b + g.r0 + r, sum);
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
    // set on every launch: the attribute is per device, and the call is cheap
    const size_t smem = stream_smem_bytes<VT>();
    const cudaError_t e =
        cudaFuncSetAttribute(k_stream<VT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_stream: shared-memory attribute: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
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

// ===========================================================================
// symm_spmv_noalloc: the streaming SymmSpMV for callers that may not
// allocate device memory.
//
// The streaming kernel above needs scratch memory besides its inputs and
// outputs: a table of row-block starts and a status word.  A schedule keeps
// them in memory that race_build allocates; this variant keeps them in one
// file-scope device array instead, fixed at load time, so the call itself
// allocates nothing.  The block table is rebuilt on the device at every call
// from the caller's row pointers (a block ends every 64 rows and whenever
// the next row starts in a new 512-entry chunk of the nonzeros, so a block
// holds at most 64 rows and 1023 nonzeros when no row is longer than 512).
// Blocks whose 16-byte-widened copies would read past the caller's arrays
// (the last one or two) are handled by a plain-load tail kernel instead.
// ===========================================================================
namespace race_noalloc {

constexpr int64_t kMaxRows = int64_t(1) << 24;    // 16,777,216 rows
constexpr int64_t kMaxNnz = int64_t(1) << 28;     // stored upper entries
constexpr int kGroupRows = 256;                   // rows per counting group
constexpr int64_t kMaxGroups = kMaxRows / kGroupRows;
constexpr int64_t kMaxBlocks = kMaxRows / 64 + kMaxNnz / 512 + 2;
constexpr int64_t kHeader = 64;  // [0] status [1] blocks [2] first unsafe [3] long row [4] bad row_ptr
constexpr int64_t kWords = kHeader + kMaxGroups + kMaxBlocks + 1;   // 3.4 MB in total

static __device__ __align__(256) int32_t g_scratch[kWords];

__device__ __forceinline__ bool starts_block(const int32_t* __restrict__ rp, int64_t r) {
    return (r % 64 == 0) || ((__ldg(rp + r) >> 9) != (__ldg(rp + r - 1) >> 9));
}

__global__ void k_reset(int32_t* sc) {
    if (threadIdx.x == 0) {
        sc[0] = RACE_OK;
        sc[1] = 0;
        sc[2] = INT32_MAX;
        sc[3] = 0;
        sc[4] = 0;
    }
}

// per 256-row group: number of block starts (one warp per group); flags any
// row longer than 512 entries (sc[3]) and row pointers that decrease, do not
// start at 0 or do not end at nnz (sc[4]); the block table is used only when
// neither flag is set
__global__ void k_count(int32_t n, int64_t nnz, const int32_t* __restrict__ rp, int32_t* sc) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t ngroups = (static_cast<int64_t>(n) + kGroupRows - 1) / kGroupRows;
    for (int64_t g = warp; g < ngroups; g += nwarps) {
        int32_t cnt = 0;
        bool longrow = false, bad = false;
        for (int k = 0; k < kGroupRows / 32; ++k) {
            const int64_t r = g * kGroupRows + k * 32 + lane;
            const bool f = r < n && starts_block(rp, r);
            if (r < n) {
                const int64_t len = static_cast<int64_t>(__ldg(rp + r + 1)) - __ldg(rp + r);
                longrow |= len > 512;
                bad |= len < 0;
                if (r == 0) bad |= __ldg(rp) != 0;
                if (r == n - 1) bad |= static_cast<int64_t>(__ldg(rp + n)) != nnz;
            }
            cnt += __popc(__ballot_sync(0xffffffffu, f));
        }
        if (__any_sync(0xffffffffu, longrow) && lane == 0) atomicExch(sc + 3, 1);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(sc + 4, 1);
        if (lane == 0) sc[kHeader + g] = cnt;
    }
}

// exclusive scan of the group counts in place (one block of 1024 threads)
__global__ void __launch_bounds__(1024) k_scan(int32_t ngroups, int32_t* sc) {
    __shared__ int32_t part[1024];
    int32_t* c = sc + kHeader;
    const int t = threadIdx.x;
    const int32_t per = (ngroups + 1023) / 1024;
    const int32_t beg = min(t * per, ngroups), end = min(beg + per, ngroups);
    int32_t sum = 0;
    for (int32_t i = beg; i < end; ++i) sum += c[i];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = part[t] - sum;
    for (int32_t i = beg; i < end; ++i) {
        const int32_t v = c[i];
        c[i] = run;
        run += v;
    }
    if (t == 1023) sc[1] = part[1023];
}

// block starts in row order, then the sentinel n
__global__ void k_write(int32_t n, const int32_t* __restrict__ rp, int32_t* sc) {
    // malformed row pointers (flagged by k_count, which ran before on the same
    // stream) could give more block starts than the table holds: write none
    if (sc[4] != 0 || sc[1] > kMaxBlocks) return;
    int32_t* tbl = sc + kHeader + kMaxGroups;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t ngroups = (static_cast<int64_t>(n) + kGroupRows - 1) / kGroupRows;
    for (int64_t g = warp; g < ngroups; g += nwarps) {
        int32_t pos = sc[kHeader + g];
        for (int k = 0; k < kGroupRows / 32; ++k) {
            const int64_t r = g * kGroupRows + k * 32 + lane;
            const bool f = r < n && starts_block(rp, r);
            const unsigned m = __ballot_sync(0xffffffffu, f);
            if (f) tbl[pos + __popc(m & lt)] = static_cast<int32_t>(r);
            pos += __popc(m);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tbl[sc[1]] = n;
}

// first block whose widened copies would leave [0, nnz) or [0, n]
__global__ void k_safe(int32_t n, int64_t nnz, const int32_t* __restrict__ rp, int32_t* sc) {
    if (sc[4] != 0 || sc[1] > kMaxBlocks) return;
    const int32_t* tbl = sc + kHeader + kMaxGroups;
    const int32_t nb = sc[1];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nb;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t r0 = tbl[i], r1 = tbl[i + 1];
        const int64_t s = __ldg(rp + r0), e = __ldg(rp + r1);
        const int64_t s_al = s & ~int64_t(3), n_el = ((e - s_al) + 3) & ~int64_t(3);
        const int64_t r0_al = r0 & ~3, n_rp = ((r1 + 1 - r0_al) + 3) & ~int64_t(3);
        if (s_al + n_el > nnz || r0_al + n_rp > int64_t(n) + 1) atomicMin(sc + 2, static_cast<int32_t>(i));
    }
}

// rows from the first unsafe block to n: one thread per row, plain loads
__global__ void k_tail(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* b, const int32_t* sc) {
    const int32_t* tbl = sc + kHeader + kMaxGroups;
    const int32_t first = min(sc[2], sc[1]);
    const int32_t r_begin = tbl[first];
    for (int64_t r = r_begin + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double xr = __ldg(x + r);
        double acc = 0.0;
        for (int32_t j = __ldg(rp + r); j < __ldg(rp + r + 1); ++j) {
            const int32_t c = __ldg(col + j);
            const double a = __ldg(val + j);
            acc += a * __ldg(x + c);
            if (c != r) red_add_f64(b + c, a * xr);
        }
        red_add_f64(b + r, acc);
    }
}

std::mutex g_setup_mutex;
int32_t* g_scratch_ptr[64] = {nullptr};
int g_sm[64] = {0};

}  // namespace race_noalloc

extern "C" int symm_spmv_noalloc(int32_t n, int64_t nnz, const int32_t* row_ptr_d, const int32_t* col_d,
                                 const double* val_d, const double* x_d, double* b_d, void* stream) {
    using namespace race_noalloc;
    if (n < 1 || nnz < n || !row_ptr_d || !col_d || !val_d || !x_d || !b_d) {
        race_set_detail("symm_spmv_noalloc: n < 1, nnz < n or a NULL pointer");
        return RACE_ERR_INVALID;
    }
    if (static_cast<const void*>(x_d) == static_cast<const void*>(b_d)) {
        race_set_detail("symm_spmv_noalloc: x and b alias");
        return RACE_ERR_INVALID;
    }
    if ((reinterpret_cast<uintptr_t>(row_ptr_d) | reinterpret_cast<uintptr_t>(col_d) |
         reinterpret_cast<uintptr_t>(val_d)) & 15u) {
        // the row blocks are staged by bulk copies, which start at 16-byte boundaries
        race_set_detail("symm_spmv_noalloc: row_ptr, col and val must be 16-byte aligned");
        return RACE_ERR_INVALID;
    }
    if (n > kMaxRows || nnz > kMaxNnz) {
        race_set_detail("symm_spmv_noalloc: at most 16,777,216 rows and 268,435,456 stored entries "
                        "(fixed scratch of the non-allocating path)");
        return RACE_ERR_OVERFLOW;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        race_set_detail("symm_spmv_noalloc: no usable current device");
        return RACE_ERR_CUDA;
    }
    int32_t* sc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            // first call on this device: the host-side symbol is only a stand-in,
            // the kernels need the array's device address
            e = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_scratch_ptr[dev]), g_scratch);
            if (e != cudaSuccess) {
                g_scratch_ptr[dev] = nullptr;
                race_set_detail(std::string("symm_spmv_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return RACE_ERR_CUDA;
            }
            cudaDeviceGetAttribute(&g_sm[dev], cudaDevAttrMultiProcessorCount, dev);
            if (g_sm[dev] <= 0) g_sm[dev] = 1;
        }
        sc = g_scratch_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t ngroups = static_cast<int32_t>((static_cast<int64_t>(n) + kGroupRows - 1) / kGroupRows);
    const int gw = static_cast<int>(std::min<int64_t>((static_cast<int64_t>(ngroups) * 32 + 255) / 256, g_sm[dev] * 8));
    k_reset<<<1, 32, 0, st>>>(sc);
    k_count<<<gw, 256, 0, st>>>(n, nnz, row_ptr_d, sc);
    k_scan<<<1, 1024, 0, st>>>(ngroups, sc);
    k_write<<<gw, 256, 0, st>>>(n, row_ptr_d, sc);
    k_safe<<<g_sm[dev] * 4, 256, 0, st>>>(n, nnz, row_ptr_d, sc);
    int32_t head[5] = {0, 0, 0, 0, 0};
    e = cudaMemcpyAsync(head, sc, sizeof(head), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("symm_spmv_noalloc: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    if (head[4]) {
        race_set_detail("symm_spmv_noalloc: row_ptr decreases, row_ptr[0] != 0 or row_ptr[n] != nnz");
        return RACE_ERR_INVALID;
    }
    if (head[3]) {
        race_set_detail("symm_spmv_noalloc: a row has more than 512 stored entries");
        return RACE_ERR_UNSUPPORTED;
    }
    // b is written only once the request has been accepted
    e = cudaMemsetAsync(b_d, 0, sizeof(double) * static_cast<size_t>(n), st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("symm_spmv_noalloc: memset: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    const int64_t n_safe = std::min(head[2], head[1]);
    const int32_t* tbl = sc + kHeader + kMaxGroups;
    race_dev::launch_stream<double, race_dev::kSymmRed>(n_safe, tbl, row_ptr_d, col_d, val_d, x_d, b_d, sc, g_sm[dev],
                                                          4, st);
    k_tail<<<g_sm[dev] * 2, 256, 0, st>>>(n, row_ptr_d, col_d, val_d, x_d, b_d, sc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(head, sc, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("symm_spmv_noalloc: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    if (head[0] != RACE_OK) {
        race_set_detail("symm_spmv_noalloc: a bounded device wait gave up");
        return head[0];
    }
    return RACE_OK;
}
