// Symmetric Gauss-Seidel and symmetric Kaczmarz sweeps under a RACE
// schedule: the paper names both solvers among the kernels with distance-k
// dependencies that the same schedules serve.
//
// One sweep is a forward pass over the phases in order and a backward pass
// over them in reverse order.  Inside a phase every leaf runs on one group of
// G lanes, its rows one after the other (ascending forward, descending
// backward), each updated in place from the current x:
//     x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii
// on the full CRS of the permuted matrix (built once, as for spmv_full).
// Leaves of a phase share no edge (the schedules are distance-2 colourings,
// stronger than the distance 1 this kernel needs), so no lane reads an entry
// of x that another leaf of the phase writes; inside a leaf the group
// synchronises after every row, so the next row reads the new value.  One
// launch per phase and pass.  A zero diagonal gives inf or nan, as the serial
// method would; nothing traps.
//
// Kaczmarz projects x onto row i's hyperplane instead,
//     f = (b_i - sum_j a_ij x_j) / sum_j a_ij^2,   x_j <- x_j + f a_ij  (all j),
// writing x at every column of the row: rows of concurrent leaves share no
// column (distance-2 independence), and the lanes of a group update distinct
// columns of their row.  The butterfly reductions leave every lane of the
// group with the same f.  A zero row gives inf or nan.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

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

// One phase of one pass: leaf q of the phase on lanes [q*G, q*G + G).
template <typename VT, int G, bool BACKWARD, bool KACZ>
__global__ void __launch_bounds__(kBlock) k_gs_phase(const int32_t* __restrict__ frp, const int32_t* __restrict__ fcol,
                                                    const VT* __restrict__ fval, const double* __restrict__ b,
                                                    double* x, const int32_t* __restrict__ leaf_lo,
                                                    const int32_t* __restrict__ leaf_hi, int32_t nleaves) {
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t leaf = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) / G;
    if (leaf >= nleaves) return;  // all G lanes of a group share the leaf index
    const int32_t lo = __ldg(leaf_lo + leaf), hi = __ldg(leaf_hi + leaf);
    for (int32_t k = 0; k < hi - lo; ++k) {
        const int32_t r = BACKWARD ? hi - 1 - k : lo + k;
        double s = 0.0, d = 0.0;  // Gauss-Seidel: off-diagonal sum, diagonal; Kaczmarz: a.x, |a|^2
        const int32_t beg = __ldg(frp + r), end = __ldg(frp + r + 1);
        // U entries per lane and step, all loads of a step issued before their uses
        constexpr int U = 4;
        for (int32_t t0 = beg + lane; t0 < end; t0 += U * G) {
            int32_t c[U];
            double a[U], xc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t t = t0 + u * G;
                c[u] = t < end ? __ldg(fcol + t) : -1;
                a[u] = t < end ? static_cast<double>(__ldg(fval + t)) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) xc[u] = c[u] >= 0 ? x[c[u]] : 0.0;  // plain loads: x changes during the launch
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (c[u] < 0) continue;
                if constexpr (KACZ) {
                    s += a[u] * xc[u];
                    d += a[u] * a[u];
                } else {
                    if (c[u] == r) d += a[u];
                    else s += a[u] * xc[u];
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            s += __shfl_xor_sync(mask, s, o, G);
            d += __shfl_xor_sync(mask, d, o, G);
        }
        if constexpr (KACZ) {
            const double f = (__ldg(b + r) - s) / d;
            for (int32_t t = beg + lane; t < end; t += G) x[__ldg(fcol + t)] += f * static_cast<double>(__ldg(fval + t));
        } else {
            if (lane == 0) x[r] = (__ldg(b + r) - s) / d;
        }
        __syncwarp(mask);  // the group's next row reads the updated x
    }
}

template <typename VT, int G, bool KACZ>
void sweep(const race_schedule* s, const double* b, double* x, int32_t sweeps, cudaStream_t st) {
    const auto& sp = s->plan.stage_ptr;
    const int32_t nph = static_cast<int32_t>(sp.size()) - 1;
    const VT* fval = static_cast<const VT*>(s->d_fval);
    for (int32_t w = 0; w < sweeps; ++w)
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t i = 0; i < nph; ++i) {
                const int32_t p = pass == 0 ? i : nph - 1 - i;
                const int32_t nl = sp[p + 1] - sp[p];
                if (nl == 0) continue;
                const int grid = static_cast<int>((static_cast<int64_t>(nl) * G + kBlock - 1) / kBlock);
                if (pass == 0)
                    k_gs_phase<VT, G, false, KACZ><<<grid, kBlock, 0, st>>>(s->d_frp, s->d_fcol, fval, b, x,
                                                                     s->d_leaf_lo + sp[p], s->d_leaf_hi + sp[p], nl);
                else
                    k_gs_phase<VT, G, true, KACZ><<<grid, kBlock, 0, st>>>(s->d_frp, s->d_fcol, fval, b, x,
                                                                    s->d_leaf_lo + sp[p], s->d_leaf_hi + sp[p], nl);
            }
}

template <typename VT, bool KACZ>
void sweep_vt(const race_schedule* s, const double* b, double* x, int32_t sweeps, cudaStream_t st) {
    switch (s->group_lanes) {
        case 1: sweep<VT, 1, KACZ>(s, b, x, sweeps, st); break;
        case 2: sweep<VT, 2, KACZ>(s, b, x, sweeps, st); break;
        case 4: sweep<VT, 4, KACZ>(s, b, x, sweeps, st); break;
        case 16: sweep<VT, 16, KACZ>(s, b, x, sweeps, st); break;
        case 32: sweep<VT, 32, KACZ>(s, b, x, sweeps, st); break;
        default: sweep<VT, 8, KACZ>(s, b, x, sweeps, st); break;
    }
}

// True when no two leaves of one phase hold rows at distance <= 2, i.e. the
// closed neighbourhoods of their rows (the entries of x a Kaczmarz update
// writes) are disjoint.  Schedules with one-level stage-0 groups are
// write-disjoint for half storage only and fail this.
bool kacz_independent(const race_schedule* s) {
    const int32_t n = s->plan.n;
    const auto& rp = s->h_rp;
    const auto& col = s->h_col;
    std::vector<int64_t> off(static_cast<size_t>(n) + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t)
            if (col[t] != r) {
                ++off[r + 1];
                ++off[col[t] + 1];
            }
    for (int32_t r = 0; r < n; ++r) off[r + 1] += off[r];
    std::vector<int32_t> nbr(static_cast<size_t>(off[n]));
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t)
            if (col[t] != r) {
                nbr[fill[r]++] = col[t];
                nbr[fill[col[t]]++] = r;
            }
    std::vector<int32_t> owner(static_cast<size_t>(n), -1), phase(static_cast<size_t>(n), -1);
    const auto& sp = s->plan.stage_ptr;
    auto claim = [&](int32_t c, int32_t ph, int32_t q) {
        if (phase[c] == ph && owner[c] != q) return false;
        phase[c] = ph;
        owner[c] = q;
        return true;
    };
    for (size_t ph = 0; ph + 1 < sp.size(); ++ph)
        for (int32_t q = sp[ph]; q < sp[ph + 1]; ++q)
            for (int32_t r = s->plan.leaf_lo[q]; r < s->plan.leaf_hi[q]; ++r) {
                if (!claim(r, static_cast<int32_t>(ph), q)) return false;
                for (int64_t e = off[r]; e < off[r + 1]; ++e)
                    if (!claim(nbr[e], static_cast<int32_t>(ph), q)) return false;
            }
    return true;
}

template <bool KACZ>
int run(const race_schedule* s, const double* b_d, double* x_d, int32_t sweeps, void* stream, const char* name) {
    if (!s || !b_d || !x_d) {
        race_set_detail("NULL argument");
        return RACE_ERR_INVALID;
    }
    if (s->host_only) {
        race_set_detail("schedule was built with RACE_FLAG_HOST_ONLY");
        return RACE_ERR_UNSUPPORTED;
    }
    if (static_cast<const void*>(b_d) == static_cast<const void*>(x_d)) {
        race_set_detail("b and x alias");
        return RACE_ERR_INVALID;
    }
    if (sweeps < 0) {
        race_set_detail("sweeps < 0");
        return RACE_ERR_INVALID;
    }
    if (KACZ) {
        int32_t ks = s->kacz_state.load(std::memory_order_acquire);
        if (ks == 0) {
            ks = kacz_independent(s) ? 1 : -1;  // threads that race here compute the same answer
            s->kacz_state.store(ks, std::memory_order_release);
        }
        if (ks < 0) {
            race_set_detail("the schedule's phases are not distance-2 independent on the full rows "
                            "(RACE_FLAG_ONE_LEVEL_STAGE0): a Kaczmarz update writes every column of its row");
            return RACE_ERR_UNSUPPORTED;
        }
    }
    if (!s->d_frp) {
        const int rc = race_prepare_full(const_cast<race_schedule*>(s), stream);
        if (rc) return rc;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->val_type == RACE_F64) sweep_vt<double, KACZ>(s, b_d, x_d, sweeps, st);
    else sweep_vt<float, KACZ>(s, b_d, x_d, sweeps, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string(name) + ": " + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

}  // namespace

extern "C" int symm_gs(const race_schedule* s, const double* b_d, double* x_d, int32_t sweeps, void* stream) {
    return run<false>(s, b_d, x_d, sweeps, stream, "symm_gs");
}

extern "C" int symm_kacz(const race_schedule* s, const double* b_d, double* x_d, int32_t sweeps, void* stream) {
    return run<true>(s, b_d, x_d, sweeps, stream, "symm_kacz");
}
