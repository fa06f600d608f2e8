// SymmSpMV on a SELL-32-sigma copy of the permuted upper matrix (executor
// RACE_EXEC_SELL_DF64).
//
// The row-per-lane CRS kernels gather each lane's own row, so one warp load
// touches up to 32 different sectors and the L1 pipe, not HBM, saturates.
// SELL-C-sigma (Kreutzer, Hager, Wellein, Fehske, Bishop, "A unified sparse
// matrix data format for efficient general sparse matrix-vector
// multiplication on modern processors with wide SIMD units", 2014) stores
// chunks of C = 32 rows column by column: entry j of the chunk's lane l sits
// at off[k] + 32 j + l, so every warp load of values and columns is one
// contiguous 256- (or 128-) byte line, and all lanes of a chunk loop the same
// number of times.  Within windows of sigma = 1024 consecutive rows the rows
// are sorted by length (descending, stable), which keeps the padding small
// (1.5 % on the XXZ Hamiltonian, 0.8 % on the 27-point stencil) and the
// RACE/BFS locality of x and b intact.  Padding entries have column -1 and
// value 0.
//
// Arithmetic as RACE_EXEC_DF64_RED: FP64 row sums (one multiply-add per
// entry), transposed updates a_ij x_i by the integer product of the
// significands (int_product.cuh), both sent to b as reductions at L2 on a
// zeroed b.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "df64.cuh"
#include "int_product.cuh"
#include "race_internal.h"

namespace {

constexpr int kBlock = 256;
constexpr int kChunk = 32;
constexpr int64_t kWinChunks = kSellSigma / kChunk;  // chunks per sorting window


// One warp per chunk (grid-strided).  U entries of the lane's row per step,
// all loads of a step issued before their uses.
template <typename VT, int U>
__global__ void __launch_bounds__(kBlock) k_symm_sell(int64_t n_chunks, const int64_t* __restrict__ off,
                                                     const int32_t* __restrict__ srow, const int32_t* __restrict__ col,
                                                     const VT* __restrict__ val, const double* __restrict__ x,
                                                     double* b) {
    const int lane = threadIdx.x & (kChunk - 1);
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (kBlock / kChunk);
    const int64_t full_windows = n_chunks / kWinChunks;
    for (int64_t i = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / kChunk; i < n_chunks; i += nwarps) {
        // Chunks are sorted by width within each window, so a plain grid
        // stride would hand every warp the same position (and width) in every
        // window; rotating the position by the window index spreads them.
        const int64_t win = i / kWinChunks;
        const int64_t k = win < full_windows ? win * kWinChunks + (i + win) % kWinChunks : i;
        const int64_t o = __ldg(off + k);
        const int32_t w = static_cast<int32_t>((__ldg(off + k + 1) - o) / kChunk);
        const int32_t row = __ldg(srow + k * kChunk + lane);
        const double xr = row >= 0 ? __ldg(x + row) : 0.0;
        float xrh, xrl;
        const int st = df64::split(xr, xrh, xrl);  // the range test of x_r
        const bool scatter = st == 0 && xrh != 0.0f;
        const intprod::Factor xf = intprod::factor(xr);
        const VT* vp = val + o + lane;
        const int32_t* cp = col + o + lane;
        double acc = 0.0;
        for (int32_t j = 0; j < w; j += U) {  // the last step is predicated, not a serial tail
            VT a[U];
            int32_t c[U];
            double xc[U];
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const bool v = j + t < w;
                a[t] = v ? __ldg(vp + static_cast<int64_t>(j + t) * kChunk) : VT(0);
                c[t] = v ? __ldg(cp + static_cast<int64_t>(j + t) * kChunk) : -1;
            }
#pragma unroll
            for (int t = 0; t < U; ++t) xc[t] = c[t] >= 0 ? __ldg(x + c[t]) : 0.0;
#pragma unroll
            for (int t = 0; t < U; ++t) {
                acc = fma(df64::widen(a[t]), xc[t], acc);
                if (scatter && c[t] >= 0 && c[t] != row && !df64::is_zero(a[t]))
                    atomicAdd(b + c[t], intprod::mul(a[t], xf));
            }
        }
        if (st != 0) {  // x_row outside the split's range: this row scatters in FP64
            for (int32_t jj = 0; jj < w; ++jj) {
                const int32_t c = __ldg(cp + static_cast<int64_t>(jj) * kChunk);
                if (c >= 0 && c != row) atomicAdd(b + c, df64::widen(__ldg(vp + static_cast<int64_t>(jj) * kChunk)) * xr);
            }
        }
        if (row >= 0) atomicAdd(b + row, acc);
    }
}

int sm_count_here() {
    static int count = 0;
    if (count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (count <= 0) count = 1;
    }
    return count;
}

template <typename VT>
void launch_vt(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    const SellSet& q = s->sell;
    const int64_t per_sm = s->launch.blocks_per_sm > 0 ? s->launch.blocks_per_sm : (2048 / kBlock);
    const int64_t cap = static_cast<int64_t>(sm_count_here()) * per_sm;
    const int64_t need = (q.n_chunks * kChunk + kBlock - 1) / kBlock;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min(need, cap)));
    const VT* v = static_cast<const VT*>(q.d_val);
    const int u = s->launch.executor == RACE_EXEC_SELL_DF64 ? s->launch.regs_per_row : 8;
    if (u >= 16)
        k_symm_sell<VT, 16><<<blocks, kBlock, 0, st>>>(q.n_chunks, q.d_off, q.d_row, q.d_col, v, x, b);
    else if (u >= 8)
        k_symm_sell<VT, 8><<<blocks, kBlock, 0, st>>>(q.n_chunks, q.d_off, q.d_row, q.d_col, v, x, b);
    else
        k_symm_sell<VT, 4><<<blocks, kBlock, 0, st>>>(q.n_chunks, q.d_off, q.d_row, q.d_col, v, x, b);
}
}  // namespace

void race_make_sell(int32_t n, const int32_t* rp, const int32_t* col, const double* v64, const float* v32,
                    int32_t sigma, SellHost& out) {
    std::vector<int32_t> order(static_cast<size_t>(n));
    std::iota(order.begin(), order.end(), 0);
    for (int32_t w0 = 0; w0 < n; w0 += sigma) {
        const int32_t w1 = std::min(n, w0 + sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [rp](int32_t a, int32_t b) {
            return rp[a + 1] - rp[a] > rp[b + 1] - rp[b];
        });
    }
    const int64_t n_chunks = (static_cast<int64_t>(n) + kChunk - 1) / kChunk;
    out.row.assign(static_cast<size_t>(n_chunks * kChunk), -1);
    out.off.assign(static_cast<size_t>(n_chunks + 1), 0);
    for (int64_t k = 0; k < n_chunks; ++k) {
        int32_t w = 0;
        for (int l = 0; l < kChunk; ++l) {
            const int64_t i = k * kChunk + l;
            if (i >= n) break;
            const int32_t r = order[static_cast<size_t>(i)];
            out.row[static_cast<size_t>(i)] = r;
            w = std::max(w, rp[r + 1] - rp[r]);
        }
        out.off[static_cast<size_t>(k + 1)] = out.off[static_cast<size_t>(k)] + static_cast<int64_t>(w) * kChunk;
    }
    const size_t total = static_cast<size_t>(out.off.back());
    out.col.assign(total, -1);
    if (v64) out.val64.assign(total, 0.0);
    else out.val32.assign(total, 0.0f);
    for (int64_t k = 0; k < n_chunks; ++k) {
        for (int l = 0; l < kChunk; ++l) {
            const int32_t r = out.row[static_cast<size_t>(k * kChunk + l)];
            if (r < 0) continue;
            for (int32_t j = 0; j < rp[r + 1] - rp[r]; ++j) {
                const size_t d = static_cast<size_t>(out.off[static_cast<size_t>(k)] + static_cast<int64_t>(j) * kChunk + l);
                const int32_t src = rp[r] + j;
                out.col[d] = col[src];
                if (v64) out.val64[d] = v64[src];
                else out.val32[d] = v32[src];
            }
        }
    }
}

int race_sell_prepare(const race_schedule* s) {
    SellSet& q = s->sell;
    if (q.ready) return RACE_OK;
    int rc = race_df64_prepare(s);
    if (rc) return rc;
    const int32_t n = s->plan.n;
    SellHost h;
    const bool f64 = s->val_type == RACE_F64;
    race_make_sell(n, s->h_rp.data(), s->h_col.data(), f64 ? s->h_val64.data() : nullptr,
                   f64 ? nullptr : s->h_val32.data(), kSellSigma, h);
    const size_t total = h.col.size();
    const size_t vbytes = (f64 ? sizeof(double) : sizeof(float)) * std::max<size_t>(total, 1);
    cudaError_t e = cudaMalloc(&q.d_off, sizeof(int64_t) * h.off.size());
    if (e == cudaSuccess) e = cudaMalloc(&q.d_row, sizeof(int32_t) * std::max<size_t>(h.row.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&q.d_col, sizeof(int32_t) * std::max<size_t>(total, 1));
    if (e == cudaSuccess) e = cudaMalloc(&q.d_val, vbytes);
    if (e == cudaSuccess) e = cudaMemcpy(q.d_off, h.off.data(), sizeof(int64_t) * h.off.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !h.row.empty())
        e = cudaMemcpy(q.d_row, h.row.data(), sizeof(int32_t) * h.row.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && total)
        e = cudaMemcpy(q.d_col, h.col.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && total)
        e = cudaMemcpy(q.d_val, f64 ? static_cast<const void*>(h.val64.data()) : static_cast<const void*>(h.val32.data()),
                       vbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        race_free_sell(q);
        race_set_detail(std::string("SELL upload: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    q.n_chunks = static_cast<int64_t>(h.off.size()) - 1;
    q.n_stored = static_cast<int64_t>(total);
    q.ready = true;
    return RACE_OK;
}

void race_free_sell(SellSet& q) {
    void* p[] = {q.d_off, q.d_row, q.d_col, q.d_val};
    for (void* v : p)
        if (v) cudaFree(v);
    q = SellSet();
}

int race_sell_launch(const race_schedule* s, const double* x, double* b, cudaStream_t st) {
    int rc = race_sell_prepare(s);
    if (rc) return rc;
    if (s->sell.n_chunks == 0) return RACE_OK;
    if (s->val_type == RACE_F64) launch_vt<double>(s, x, b, st);
    else launch_vt<float>(s, x, b, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_sell: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}
