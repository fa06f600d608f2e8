// RACE execution in one launch (executors RACE_EXEC_PERSIST_GROUP and
// RACE_EXEC_PERSIST_CTA): the leaves of every phase in one cooperative
// launch, consecutive phases separated by a grid barrier.  This is the
// execution of Sec. 4.4.3 (the leaves of one colour run concurrently, a
// synchronisation separates the colours) on the schedule's tree flattened
// into global phases, with the kernel boundaries of RACE_EXEC_LEAF_GROUP /
// _LEAF_CTA replaced by barriers inside one kernel.
//
//   PERSIST_GROUP  one leaf per group of G lanes, the leaf's rows in order,
//                  b updated by plain loads and stores (the paper's model: a
//                  leaf runs on one worker and writes b without atomics).
//                  b is read and written through L2 (ld/st .cg): another
//                  SM's L1 may still hold a line of b from an earlier phase.
//   PERSIST_CTA    one leaf per block, the leaf's rows in parallel (four
//                  entries per lane and step), updates inside a leaf as L2
//                  reductions, as RACE_EXEC_LEAF_CTA.
// The leaves of a phase are distance-2 independent (Sec. 4.2), so no two
// workers of one phase touch the same entry of b.
//
// The grid barrier is an arrival counter and a generation word.  Thread 0 of a block makes the block's
// writes visible (a device-wide fence), arrives, and polls the generation a
// bounded number of times; the last arrival resets the counter and releases
// the next generation.  The pause between polls backs off, since the blocks
// without a leaf wait through the whole phase.  A wait that gives up records
// RACE_ERR_TIMEOUT in the schedule's status word and its block leaves the
// kernel, so every later barrier gives up too: the launch always ends, and
// race_poll_status reports the timeout.  race_probe_barrier_timeout launches
// the kernel expecting one block more than it has, a wrong worker count made
// on the host, so the first barrier gives up in every block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "df64.cuh"
#include "red.cuh"
#include "race_internal.h"

namespace race_persist {

constexpr int kBlock = 256;
// polls of one barrier wait; the pause between polls doubles from 64 ns up to
// 4 us, so a wait gives up after about 4 s (the probe's after about 16 ms)
constexpr uint32_t kSpinLimit = 1u << 20;
constexpr uint32_t kProbeSpinLimit = 1u << 12;
constexpr uint32_t kPauseMinNs = 64, kPauseMaxNs = 4096;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~static_cast<unsigned>(G - 1));
    }
}

template <int G>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// Arrive at the grid barrier and wait for the release of generation gen + 1
// (thread 0 of the block only).  Returns 0 when the wait gave up.
__device__ int arrive_and_wait(uint32_t* bar, uint32_t& gen, uint32_t expected, uint32_t spin_limit,
                               int32_t* status) {
    __threadfence();  // the block's writes to b before its arrival
    const uint32_t arrived = atomicAdd(bar, 1u) + 1u;
    int ok = 1;
    if (arrived == expected) {
        atomicExch(bar, 0u);  // ready for the next barrier before anyone passes this one
        __threadfence();
        st_release(bar + 1, gen + 1u);
    } else {
        // the blocks without work wait here for the whole phase: the pause
        // backs off so that their polls of one L2 line stay rare
        uint32_t it = 0, pause = kPauseMinNs;
        while (ld_acquire(bar + 1) == gen) {
            if (++it >= spin_limit) {
                ok = 0;
                atomicExch(status, RACE_ERR_TIMEOUT);
                break;
            }
            __nanosleep(pause);
            pause = min(pause * 2u, kPauseMaxNs);
        }
    }
    ++gen;
    return ok;
}

// Leaf [lo, hi) on the G lanes of one group, rows in order (Alg.
// "SymmSpMV" on the leaf's rows): the diagonal is each row's first entry.
template <typename VT, int G>
__device__ __forceinline__ void leaf_group(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                           const VT* __restrict__ val, const double* __restrict__ x, double* b,
                                           int32_t lo, int32_t hi, int lane, unsigned mask) {
    int32_t rs = __ldg(rp + lo);
    for (int32_t r = lo; r < hi; ++r) {
        const int32_t re = __ldg(rp + r + 1);
        const double xr = __ldg(x + r);
        double tmp = 0.0;
        for (int32_t idx = rs + lane; idx < re; idx += G) {
            const double a = df64::widen(__ldg(val + idx));
            if (idx == rs) {
                tmp = fma(a, xr, tmp);
            } else {
                const int32_t c = __ldg(col + idx);
                tmp = fma(a, __ldg(x + c), tmp);
                __stcg(b + c, __ldcg(b + c) + a * xr);
            }
        }
        tmp = group_sum<G>(tmp, mask);
        if (lane == 0) __stcg(b + r, __ldcg(b + r) + tmp);
        __syncwarp(mask);  // the next row may update what this one wrote
        rs = re;
    }
}

// Leaf [lo, hi) on one block: rows in parallel, four entries per lane and
// step, updates as reductions at L2.
template <typename VT>
__device__ __forceinline__ void leaf_cta(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, const double* __restrict__ x, double* b,
                                         int32_t lo, int32_t hi) {
    for (int32_t r = lo + static_cast<int32_t>(threadIdx.x); r < hi; r += kBlock) {
        const int32_t rs = __ldg(rp + r), re = __ldg(rp + r + 1);
        const double xr = __ldg(x + r);
        double tmp = 0.0;
        for (int32_t idx = rs; idx < re; idx += 4) {
            double a[4], xc[4];
            int32_t c[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool v = idx + t < re;
                a[t] = v ? df64::widen(__ldg(val + idx + t)) : 0.0;
                c[t] = v ? __ldg(col + idx + t) : -1;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) xc[t] = c[t] >= 0 ? __ldg(x + c[t]) : 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (c[t] < 0) continue;
                tmp = fma(a[t], xc[t], tmp);
                if (c[t] != r) red_add_f64(b + c[t], a[t] * xr);
            }
        }
        red_add_f64(b + r, tmp);
    }
}

// The words after the barrier's two: a leaf ticket per phase, then the
// counters that rank the blocks (kTiers, then kSmSlots).
constexpr int kTiers = 32;
constexpr int kSmSlots = 1024;
inline size_t bar_words(size_t nphase) { return 2 + nphase + kTiers + kSmSlots; }

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t v;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
    return v;
}

// All phases of the schedule; leaves of phase p are [stage[p], stage[p+1]).
//
// Which workers take the leaves: at the start each block gets a rank, its
// slot on its SM (0 for the first block there, 1 for the next, ...) times
// the SM count plus its place among the blocks of that slot, so that the
// ranks below the SM count lie on distinct SMs.  In a phase of nl leaves
// the workers of rank below nl (blocks, or lane groups ranked group-major
// over the blocks) draw the leaves from the phase's ticket counter until
// none is left: the leaves of a small phase spread over the SMs instead of
// piling onto a few, and every leaf is drawn exactly once whatever the ranks
// turn out to be (rank 0 always exists and always draws).
template <typename VT, int G, bool CTA>
__global__ void __launch_bounds__(kBlock) k_symm_persist(const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                        const double* __restrict__ x, double* b,
                                                        const int32_t* __restrict__ llo,
                                                        const int32_t* __restrict__ lhi,
                                                        const int32_t* __restrict__ stage, int32_t nphase,
                                                        uint32_t* bar, int32_t* status, uint32_t expected,
                                                        uint32_t spin_limit, uint32_t n_sm) {
    __shared__ int s_go;
    __shared__ int32_t s_q;
    __shared__ uint32_t s_rank;
    uint32_t gen = 0;
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    if (threadIdx.x == 0) {
        uint32_t* tier_ctr = bar + 2 + nphase;
        uint32_t* sm_slot = tier_ctr + kTiers;
        const uint32_t slot = min(atomicAdd(sm_slot + (sm_id() % kSmSlots), 1u), static_cast<uint32_t>(kTiers - 1));
        s_rank = slot * n_sm + atomicAdd(tier_ctr + slot, 1u);
    }
    __syncthreads();
    const uint32_t rank = s_rank;
    const uint32_t grank = (threadIdx.x / G) * gridDim.x + rank;  // lane groups, group-major
    for (int32_t p = 0; p < nphase; ++p) {
        const int32_t l0 = __ldg(stage + p), l1 = __ldg(stage + p + 1);
        const uint32_t nl = static_cast<uint32_t>(l1 - l0);
        uint32_t* ticket = bar + 2 + p;
        if constexpr (CTA) {
            for (; rank < nl;) {
                if (threadIdx.x == 0) s_q = l0 + static_cast<int32_t>(atomicAdd(ticket, 1u));
                __syncthreads();
                const int32_t q = s_q;
                __syncthreads();  // every thread holds q before thread 0 draws again
                if (q >= l1) break;
                leaf_cta<VT>(rp, col, val, x, b, __ldg(llo + q), __ldg(lhi + q));
            }
        } else {
            for (; grank < nl;) {
                int32_t q = 0;
                if (lane == 0) q = l0 + static_cast<int32_t>(atomicAdd(ticket, 1u));
                q = __shfl_sync(mask, q, 0, G);
                if (q >= l1) break;
                leaf_group<VT, G>(rp, col, val, x, b, __ldg(llo + q), __ldg(lhi + q), lane, mask);
            }
        }
        if (p + 1 == nphase) break;
        __syncthreads();  // the whole block is done with phase p
        if (threadIdx.x == 0) s_go = arrive_and_wait(bar, gen, expected, spin_limit, status);
        __syncthreads();
        if (!s_go) return;
    }
}

template <typename VT, int G, bool CTA>
int launch(const race_schedule* s, const double* x, double* b, cudaStream_t st, uint32_t extra_arrivals,
           uint32_t spin_limit) {
    const void* fn = reinterpret_cast<const void*>(k_symm_persist<VT, G, CTA>);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_symm_persist<VT, G, CTA>, kBlock, 0);
    if (e != cudaSuccess || per_sm < 1) {
        race_set_detail("k_symm_persist: no resident block");
        return RACE_ERR_CUDA;
    }
    // the same number of blocks on every SM: race_launch.blocks_per_sm when the
    // schedule's launch names this executor and asks for fewer than fit
    if (s->launch.executor == (CTA ? RACE_EXEC_PERSIST_CTA : RACE_EXEC_PERSIST_GROUP) && s->launch.blocks_per_sm > 0)
        per_sm = std::min(per_sm, s->launch.blocks_per_sm);
    const auto& sp = s->plan.stage_ptr;
    const int grid = per_sm * race_device_sms();
    e = cudaMemsetAsync(s->d_bar, 0, sizeof(uint32_t) * bar_words(sp.size() - 1), st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_persist: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    const int32_t* rp = s->d_rp;
    const int32_t* col = s->d_col;
    const VT* val = static_cast<const VT*>(s->d_val);
    const int32_t* llo = s->d_leaf_lo;
    const int32_t* lhi = s->d_leaf_hi;
    const int32_t* stage = s->d_stage;
    int32_t nphase = static_cast<int32_t>(sp.size()) - 1;
    uint32_t* bar = s->d_bar;
    int32_t* status = s->d_status;
    uint32_t expected = static_cast<uint32_t>(grid) + extra_arrivals;
    uint32_t n_sm = static_cast<uint32_t>(race_device_sms());
    void* args[] = {&rp, &col, &val, &x, &b, &llo, &lhi, &stage, &nphase, &bar, &status, &expected, &spin_limit, &n_sm};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, st);
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_persist: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

template <typename VT>
int launch_vt(const race_schedule* s, bool cta, const double* x, double* b, cudaStream_t st, uint32_t extra,
              uint32_t spin) {
    if (cta) return launch<VT, 1, true>(s, x, b, st, extra, spin);
    switch (s->group_lanes) {
        case 1: return launch<VT, 1, false>(s, x, b, st, extra, spin);
        case 2: return launch<VT, 2, false>(s, x, b, st, extra, spin);
        case 4: return launch<VT, 4, false>(s, x, b, st, extra, spin);
        case 8: return launch<VT, 8, false>(s, x, b, st, extra, spin);
        case 16: return launch<VT, 16, false>(s, x, b, st, extra, spin);
        default: return launch<VT, 32, false>(s, x, b, st, extra, spin);
    }
}

int run(const race_schedule* s, int32_t executor, const double* x, double* b, cudaStream_t st, uint32_t extra,
        uint32_t spin) {
    if (s->plan.stage_ptr.size() < 2 || s->plan.n == 0) return RACE_OK;
    const bool cta = executor == RACE_EXEC_PERSIST_CTA;
    return s->val_type == RACE_F64 ? launch_vt<double>(s, cta, x, b, st, extra, spin)
                                   : launch_vt<float>(s, cta, x, b, st, extra, spin);
}

}  // namespace race_persist

size_t race_persist_bar_words(size_t stage_ptr_size) {
    return race_persist::bar_words(stage_ptr_size > 0 ? stage_ptr_size - 1 : 0);
}

int race_persist_launch(const race_schedule* s, int32_t executor, const double* x, double* b, cudaStream_t st) {
    return race_persist::run(s, executor, x, b, st, 0u, race_persist::kSpinLimit);
}

extern "C" int race_probe_barrier_timeout(const race_schedule* s, const double* x_d, double* b_d, void* stream) {
    if (!s || !x_d || !b_d || x_d == b_d) {
        race_set_detail("race_probe_barrier_timeout: NULL or aliasing argument");
        return RACE_ERR_INVALID;
    }
    if (s->host_only) {
        race_set_detail("schedule was built with RACE_FLAG_HOST_ONLY");
        return RACE_ERR_UNSUPPORTED;
    }
    if (s->plan.stage_ptr.size() < 3) {
        race_set_detail("race_probe_barrier_timeout: the schedule has a single phase (no barrier)");
        return RACE_ERR_UNSUPPORTED;
    }
    return race_persist::run(s, RACE_EXEC_PERSIST_CTA, x_d, b_d, static_cast<cudaStream_t>(stream), 1u,
                             race_persist::kProbeSpinLimit);
}
