// Matrix powers Y[:, q] = A^(q+1) x, q = 0..p-1 (race_matrix_powers).
//
// The paper's conclusion names in-place matrix powers among the kernels a
// level-based formulation serves.  "In place" here: the p powers are the p
// columns of the caller's n x p array Y, each computed from the previous
// column; no other vector storage is used.  Two modes:
//
//   RACE_MPK_SWEEPS     p SymmSpMV sweeps with the schedule's executor, one
//                       column after the other (Alg. "SymmSpMV" each).
//   RACE_MPK_WAVEFRONT  one cooperative launch over (power, row block)
//                       items.  In the level order of the permuted matrix
//                       (Sec. 4.1) the rows of a level couple only to the
//                       neighbouring levels, so power q of a stretch of rows
//                       needs power q-1 only on that stretch and just beyond
//                       it.  The matrix is cut into blocks of `rows`
//                       consecutive rows; reach[t] is the last block that
//                       the columns of block t's rows fall in.  Item (q, t)
//                       adds the contributions of block t's rows to column q
//                       (row sums and transposed updates, reductions at L2
//                       into the zeroed column) from column q-1 (or x); it
//                       may start once items (q-1, 0..reach[t]) are done,
//                       because every contribution to a row comes from rows
//                       at or before it.  Items are handed out through one
//                       ticket counter in the order of key = t + q * step
//                       (step = lag + 1 + blocks / p, lag = max_t (reach[t] -
//                       t)): every item an item waits for carries a smaller
//                       ticket, and with the grid resident (cooperative
//                       launch) the waits end.  The powers of a stretch of
//                       rows are computed while its rows of the matrix are
//                       recent in L2 when the wavefront (about p * step
//                       blocks) fits there.
//
// Arithmetic as RACE_EXEC_DF64_RED: FP64 row sums; the transposed products
// in FP64 in fp64_quarters / 4 of each warp's row groups and by the integer
// product of the significands (int_product.cuh) in the rest (relative error
// below 2^-51 each).  The columns of Y are read through L2
// only (ld.global.cg): they are written by reductions during the launch.
// Every wait on a done flag is bounded; one that gives up records
// RACE_ERR_TIMEOUT in the schedule's status word and its block leaves the
// loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "df64.cuh"
#include "int_product.cuh"
#include "fp64_share.cuh"
#include "race_internal.h"
#include "red.cuh"

namespace race_mpk {

constexpr int kThreads = 256;
constexpr int kMaxPowers = 64;
constexpr int32_t kRows = 2048;           // rows per wavefront block
constexpr uint32_t kSpinLimit = 1u << 24;  // polls (with a 100 ns pause) of one done flag
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The rows of one warp (row per lane) applied to src, accumulated into dst;
// tp64: this warp forms its transposed products in FP64 (also taken when a
// lane's x_i lies outside the split's range; the caller passes tp64 when a
// stored off-diagonal value does).
template <int B>
__device__ __forceinline__ void warp_rows(int32_t row, bool live, const int32_t* __restrict__ rp,
                                          const int32_t* __restrict__ col, const double* __restrict__ val,
                                          const double* src, double* dst, bool tp64) {
    const int32_t lo = live ? __ldg(rp + row) : 0;
    const int32_t len = live ? __ldg(rp + row + 1) - lo : 0;
    const int32_t maxlen = __reduce_max_sync(kFull, len);
    const double xr = live ? __ldcg(src + row) : 0.0;
    float xrh = 0.0f, xrl = 0.0f;
    const int xbad = df64::split(xr, xrh, xrl);  // the range test of x_i
    const intprod::Factor xf = intprod::factor(xr);
    const bool use64 = tp64 || __any_sync(kFull, live && xbad != 0);  // warp-uniform choice
    const bool scatter = !df64::is_zero(xr);
    double acc = 0.0;
    for (int32_t j = 0; j < maxlen; j += B) {
        double a[B], xc[B];
        int32_t c[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const bool v = j + u < len;
            a[u] = v ? __ldg(val + lo + j + u) : 0.0;
            c[u] = v ? __ldg(col + lo + j + u) : -1;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) xc[u] = c[u] >= 0 ? __ldcg(src + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (c[u] < 0) continue;
            acc = fma(a[u], xc[u], acc);
            if (c[u] == row || !scatter) continue;
            if (use64) {
                red_add_f64(dst + c[u], a[u] * xr);
            } else if (!df64::is_zero(a[u])) {
                red_add_f64(dst + c[u], intprod::mul(a[u], xf));
            }
        }
    }
    if (live) red_add_f64(dst + row, acc);
}

template <int B>
__global__ void __launch_bounds__(kThreads) k_mpk_wave(int32_t n, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ col, const double* __restrict__ val,
                                                       const double* x, double* Y, int32_t p, int32_t rows,
                                                       int32_t nblk, int32_t step, const int32_t* __restrict__ reach,
                                                       int32_t* flags, int32_t* status, int fp64_quarters) {
    __shared__ long long s_ticket;
    __shared__ int32_t s_known[kMaxPowers];
    __shared__ int32_t s_abort;
    for (int i = threadIdx.x; i < p; i += kThreads) s_known[i] = 0;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    // flags: the ticket counter (64 bits), then per power a hint (every block
    // below it is known done), then the done flags of every power and block
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(flags);
    int32_t* hint = flags + 2;
    int32_t* done = flags + 2 + p;
    const long long total = (static_cast<long long>(nblk) + static_cast<long long>(p - 1) * step) * p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = static_cast<long long>(atomicAdd(ctr, 1ull));
        __syncthreads();
        const long long tk = s_ticket;
        __syncthreads();  // every thread holds the ticket before thread 0 draws the next
        if (tk >= total) break;
        const int32_t q = static_cast<int32_t>(tk % p);
        const long long t64 = tk / p - static_cast<long long>(q) * step;
        if (t64 < 0 || t64 >= nblk) continue;
        const int32_t t = static_cast<int32_t>(t64);
        if (q > 0) {
            if (threadIdx.x == 0) {
                // power q - 1 complete on blocks 0 .. reach[t]
                const int32_t need = __ldg(reach + t);
                // start past what this block or any other has verified already
                int32_t k = max(s_known[q - 1], ld_acquire(hint + q - 1));
                bool ok = true;
                for (; k <= need && ok; ++k) {
                    const int32_t* f = done + static_cast<long long>(q - 1) * nblk + k;
                    uint32_t it = 0;
                    while (ld_acquire(f) == 0) {
                        if (++it >= kSpinLimit) {
                            ok = false;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                if (ok) {
                    s_known[q - 1] = k;
                    __threadfence();
                    atomicMax(hint + q - 1, k);
                } else {
                    s_abort = 1;
                    atomicExch(status, RACE_ERR_TIMEOUT);
                }
            }
            __syncthreads();
            if (s_abort) break;
        }
        const double* src = q == 0 ? x : Y + static_cast<long long>(q - 1) * n;
        double* dst = Y + static_cast<long long>(q) * n;
        const int32_t r0 = t * rows, r1 = min(n, r0 + rows);
        for (int32_t base = r0 + warp * 32; base < r1; base += kThreads)
            warp_rows<B>(base + lane, base + lane < r1, rp, col, val, src, dst,
                         fp64_group(static_cast<uint32_t>(base >> 5) + static_cast<uint32_t>(q), fp64_quarters));
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) st_release(done + static_cast<long long>(q) * nblk + t, 1);
    }
}

// Block structure of the wavefront (host, once per schedule).
int prepare(race_schedule* s, cudaStream_t st) {
    MpkState& m = s->mpk;
    if (m.d_reach) return RACE_OK;
    const int32_t n = s->plan.n;
    const int32_t rows = kRows;
    const int32_t nblk = static_cast<int32_t>((static_cast<int64_t>(n) + rows - 1) / rows);
    std::vector<int32_t> reach(static_cast<size_t>(nblk));
    int32_t lag = 0;
    for (int32_t t = 0; t < nblk; ++t) {
        int32_t hi = t;
        const int32_t r1 = std::min(n, (t + 1) * rows);
        for (int32_t r = t * rows; r < r1; ++r)
            if (s->h_rp[r + 1] > s->h_rp[r]) hi = std::max(hi, s->h_col[s->h_rp[r + 1] - 1] / rows);
        // columns come sorted, so the last one of a row is its largest
        reach[static_cast<size_t>(t)] = hi;
        lag = std::max(lag, hi - t);
    }
    cudaError_t e = cudaMalloc(&m.d_reach, sizeof(int32_t) * static_cast<size_t>(nblk));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m.d_reach, reach.data(), sizeof(int32_t) * static_cast<size_t>(nblk),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vector goes out of scope
    if (e != cudaSuccess) {
        if (m.d_reach) cudaFree(m.d_reach);
        m.d_reach = nullptr;
        race_set_detail(std::string("race_matrix_powers: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RACE_ERR_NOMEM : RACE_ERR_CUDA;
    }
    m.rows = rows;
    m.nblk = nblk;
    m.lag = lag;
    return RACE_OK;
}

int wavefront(race_schedule* s, int32_t p, const double* x, double* Y, cudaStream_t st) {
    int rc = prepare(s, st);
    if (rc) return rc;
    MpkState& m = s->mpk;
    if (m.flag_powers < p) {
        if (m.d_flags) cudaFree(m.d_flags);
        m.d_flags = nullptr;
        m.flag_powers = 0;
        const cudaError_t e =
            cudaMalloc(&m.d_flags, sizeof(int32_t) * (2 + static_cast<size_t>(p) * (1 + static_cast<size_t>(m.nblk))));
        if (e != cudaSuccess) {
            m.d_flags = nullptr;
            race_set_detail(std::string("race_matrix_powers: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? RACE_ERR_NOMEM : RACE_ERR_CUDA;
        }
        m.flag_powers = p;
    }
    const bool df = race_df64_prepare(s) == RACE_OK;  // off-diagonal values in the split's range
    const int q64 = df ? s->launch.fp64_quarters : 4;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mpk_wave<4>, kThreads, 0);
    if (e != cudaSuccess || per_sm < 1) {
        race_set_detail("race_matrix_powers: no resident block");
        return RACE_ERR_CUDA;
    }
    const int grid = race_device_sms() * per_sm;
    const int32_t step = m.lag + 1 + (grid + p - 1) / p;
    e = cudaMemsetAsync(m.d_flags, 0, sizeof(int32_t) * (2 + static_cast<size_t>(p) * (1 + static_cast<size_t>(m.nblk))),
                        st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(Y, 0, sizeof(double) * static_cast<size_t>(s->plan.n) * static_cast<size_t>(p), st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_matrix_powers: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    int32_t n = s->plan.n, rows = m.rows, nblk = m.nblk;
    const int32_t* rp = s->d_rp;
    const int32_t* col = s->d_col;
    const double* val = static_cast<const double*>(s->d_val);
    const int32_t* reach = m.d_reach;
    int32_t* flags = m.d_flags;
    int32_t* status = s->d_status;
    int pp = p;
    int32_t stp = step;
    void* args[] = {&n, &rp, &col, &val, &x, &Y, &pp, &rows, &nblk, &stp, &reach, &flags, &status,
                    const_cast<int*>(&q64)};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_mpk_wave<4>), dim3(grid), dim3(kThreads), args, 0,
                                    st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("race_matrix_powers: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

}  // namespace race_mpk

extern "C" int race_matrix_powers(race_schedule* s, int32_t p, const double* x_d, double* Y_d, int32_t mode,
                                  void* stream) {
    if (!s || !x_d || !Y_d || p < 1 || p > race_mpk::kMaxPowers ||
        (mode != RACE_MPK_SWEEPS && mode != RACE_MPK_WAVEFRONT)) {
        race_set_detail("race_matrix_powers: NULL argument, p outside 1..64 or unknown mode");
        return RACE_ERR_INVALID;
    }
    if (s->host_only) {
        race_set_detail("schedule was built with RACE_FLAG_HOST_ONLY");
        return RACE_ERR_UNSUPPORTED;
    }
    const size_t n = static_cast<size_t>(s->plan.n);
    const char* xb = reinterpret_cast<const char*>(x_d);
    const char* yb = reinterpret_cast<const char*>(Y_d);
    if (xb + n * sizeof(double) > yb && yb + n * static_cast<size_t>(p) * sizeof(double) > xb) {
        race_set_detail("race_matrix_powers: x overlaps Y");
        return RACE_ERR_INVALID;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mode == RACE_MPK_SWEEPS) {
        for (int32_t q = 0; q < p; ++q) {
            const int rc = symm_spmv(s, q == 0 ? x_d : Y_d + (q - 1) * n, Y_d + q * n, stream);
            if (rc) return rc;
        }
        return RACE_OK;
    }
    if (s->val_type != RACE_F64) {
        race_set_detail("race_matrix_powers: the wavefront mode serves FP64-stored values");
        return RACE_ERR_UNSUPPORTED;
    }
    return race_mpk::wavefront(s, p, x_d, Y_d, st);
}
