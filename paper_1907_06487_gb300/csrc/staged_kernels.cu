// Warp-tile staged SymmSpMV (executor RACE_EXEC_STAGED).
//
// Alg. "SymmSpMV" on the permuted upper CRS, all rows at once: the row sum
// b_i += sum_j a_ij x_j and the transposed update b_j += a_ij x_i (j != i)
// both go to L2 as reductions (red.global.add.f64), b zeroed first.
//
// Work unit: a warp tile, the 32 consecutive rows [32 t, 32 t + 32); lane l
// owns row 32 t + l.  One elected lane copies the tile's stored values and
// column indices into a per-warp shared-memory stage with the bulk-copy
// engine (cp.async.bulk, the TMA's one-dimensional form; completion counted
// in bytes on an mbarrier), widened to 16-byte boundaries (the device arrays
// carry 8 zeroed padding elements).  With two stages per warp the copy of
// its next tile is in flight while its lanes walk the current one out of
// shared memory; with one stage the block is half the size, so twice as many
// warps stay resident and hide the copy instead.  The matrix stream thus reaches the SM as whole lines
// without passing the L1 load path, which is left to the x gathers and the
// reductions.  A tile with more than kCap stored entries is read from global
// memory directly.  The grid is persistent: warp g takes tiles g, g + W,
// g + 2W, ..., so the tiles in flight form one moving window of rows whose x
// and b stay in L2.
//
// Arithmetic.  GB300 runs FP64 at about 1/70 of its FP32 rate.  Per warp
// (by quarters of the warp index) the row sums run either as FP64 fused
// multiply-adds or in double-float arithmetic (df64.cuh: Dekker products of
// the split operands, summed as a float pair with Knuth's TwoSum), and the
// transposed products either as FP64 multiplies or by the integer product of
// the significands (int_product.cuh).  The FP64 row sums go to the first quarters and the FP64
// transposed products to the last ones, so a warp does at most one FP64
// operation per stored entry unless both shares exceed half.  x, b and the
// stored values stay FP64 (or FP32-stored values, widened exactly).
//
// Accuracy of a double-float row sum over n <= kDfRowMax entries: every
// product carries a relative error below 2^-44 (split of both operands,
// Dekker's product with the low cross term dropped) and every float-pair
// addition an absolute error below 3 * 2^-48 (|partial sum| + |product|),
// so the row sum lies within (2^-44 + 3 (n + 1) 2^-48) sum_j |a_ij x_j|,
// below 1e-12 sum_j |a_ij x_j| for n <= 64.  Longer rows, and entries whose
// stored value or gathered x lies outside the split's exponent range
// [2^-50, 2^51) (zero excepted), are taken in FP64 by a second pass over the
// row, entered only by warps that need it.
//
// Every mbarrier wait is bounded (spin_limit polls); a wait that gives up
// records RACE_ERR_TIMEOUT in the schedule's status word, and the warp waits
// (bounded) for the copy it still has in flight before it leaves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "df64.cuh"
#include "int_product.cuh"
#include "race_internal.h"
#include "stream_engine.cuh"
#include "red.cuh"

namespace race_stg {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kCap = 512;      // stored entries of a staged tile
constexpr int kDfRowMax = 64;  // longest row summed in double-float
constexpr unsigned kFull = 0xffffffffu;

template <typename VT>
struct alignas(16) TileStage {
    VT val[kCap + 8];
    int32_t col[kCap + 8];
};

template <typename VT, int NS>
constexpr size_t staged_smem_bytes() {
    return sizeof(TileStage<VT>) * NS * kWarps + sizeof(uint64_t) * NS * kWarps + 128;
}

struct Tile {
    int32_t r0, r1;  // rows [r0, r1)
    int32_t s, e;    // stored entries [s, e)
    int32_t s_al;    // s rounded down to a multiple of 4 (16 bytes of col)
    uint32_t n_el;   // widened entry count, a multiple of 4
    bool staged;
};

__device__ __forceinline__ Tile tile_of(int64_t t, int32_t n, const int32_t* __restrict__ rp) {
    Tile g;
    g.r0 = static_cast<int32_t>(t * 32);
    g.r1 = min(n, g.r0 + 32);
    g.s = __ldg(rp + g.r0);
    g.e = __ldg(rp + g.r1);
    g.s_al = g.s & ~3;
    g.n_el = static_cast<uint32_t>((g.e - g.s_al + 3) & ~3);
    g.staged = g.e - g.s <= kCap;
    return g;
}

// One lane: arm the stage's mbarrier with the byte count, then issue the
// two bulk copies (values, columns) that complete it.
template <typename VT>
__device__ __forceinline__ void issue(TileStage<VT>* st, uint64_t* bar, const Tile& g, const VT* val,
                                      const int32_t* col, uint32_t extra_tx) {
    race_dev::mbar_expect_tx(bar, g.n_el * static_cast<uint32_t>(sizeof(VT) + sizeof(int32_t)) + extra_tx);
    race_dev::bulk_g2s(st->val, val + g.s_al, g.n_el * static_cast<uint32_t>(sizeof(VT)), bar);
    race_dev::bulk_g2s(st->col, col + g.s_al, g.n_el * static_cast<uint32_t>(sizeof(int32_t)), bar);
}

template <bool SMEM, typename T>
__device__ __forceinline__ T ldx(const T* p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

// Split of a stored value; nonzero return: outside the split's range.
__device__ __forceinline__ int split_stored(double a, float& h, float& l) { return df64::split(a, h, l); }
__device__ __forceinline__ int split_stored(float a, float& h, float& l) {
    h = a;
    l = 0.0f;
    const uint32_t u = __float_as_uint(a);
    const int e = static_cast<int>((u >> 23) & 0xFFu) - 127;
    return ((u << 1) != 0 && (e < df64::kEmin || e > df64::kEmax)) ? 1 : 0;
}

// (sh, sl) += (ph, pl): TwoSum of the high parts, the low parts added, renormalised.
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float ph, float pl) {
    float s, e;
    df64::two_sum(sh, ph, s, e);
    e = df64::fadd(e, df64::fadd(sl, pl));
    df64::fast_two_sum(s, e, sh, sl);
}

// df64::join needs a normal high part of binary exponent >= -102.
__device__ __forceinline__ bool joinable(float h) { return ((__float_as_uint(h) >> 23) & 0xFFu) >= 25u; }

// The rows of one tile, one per lane; the lane's entries are sv[lo .. lo+len)
// and sc[lo .. lo+len) (shared memory when SMEM, else global memory).
template <typename VT, int B, bool SMEM, bool RS64, bool TP64>
__device__ __forceinline__ void tile_rows(int32_t row, bool live, int32_t lo, int32_t len, int32_t maxlen,
                                          const VT* __restrict__ sv, const int32_t* __restrict__ sc,
                                          const double* __restrict__ x, double* b) {
    const double xr = live ? __ldg(x + row) : 0.0;
    float xrh = 0.0f, xrl = 0.0f;
    const int xr_bad = TP64 ? 0 : df64::split(xr, xrh, xrl);  // the range test of x_i
    const intprod::Factor xf = intprod::factor(xr);
    const bool scatter = !df64::is_zero(xr);  // x_i = 0: the row makes no transposed update
    const bool rs_df = !RS64 && len <= kDfRowMax;
    double acc = 0.0;
    float sh = 0.0f, sl = 0.0f;
    bool defer = live && !RS64 && !rs_df;
    for (int32_t j = 0; j < maxlen; j += B) {
        VT a[B];
        int32_t c[B];
        double xc[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const bool v = j + u < len;
            a[u] = v ? ldx<SMEM>(sv + lo + j + u) : VT(0);
            c[u] = v ? ldx<SMEM>(sc + lo + j + u) : -1;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) xc[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            if (c[u] < 0) continue;
            float ah = 0.0f, al = 0.0f;
            int abad = 0;
            if constexpr (!RS64 || !TP64) abad = split_stored(a[u], ah, al);
            if constexpr (RS64) {
                acc = fma(df64::widen(a[u]), xc[u], acc);
            } else {
                if (rs_df) {
                    float xh, xl;
                    const int xb = df64::split(xc[u], xh, xl);
                    if (abad | xb) {
                        defer = true;
                    } else {
                        float ph, pl;
                        df64::mul(ah, al, xh, xl, ph, pl);
                        ff_acc(sh, sl, ph, pl);
                    }
                }
            }
            if (c[u] != row && scatter) {
                if constexpr (TP64) {
                    red_add_f64(b + c[u], df64::widen(a[u]) * xr);
                } else {
                    if (abad | xr_bad) {
                        defer = true;
                    } else if (!df64::is_zero(a[u])) {
                        red_add_f64(b + c[u], intprod::mul(a[u], xf));
                    }
                }
            }
        }
    }
    // FP64 pass over the rows that deferred entries (rare; whole warp enters or none)
    const bool any_defer = __any_sync(kFull, defer);
    if (any_defer && defer) {
        for (int32_t j = 0; j < len; ++j) {
            const VT av = ldx<SMEM>(sv + lo + j);
            const int32_t cj = ldx<SMEM>(sc + lo + j);
            float ah, al;
            const int abad = split_stored(av, ah, al);
            if constexpr (!RS64) {
                const double xv = __ldg(x + cj);
                float xh, xl;
                if (!rs_df || abad || df64::split(xv, xh, xl)) acc = fma(df64::widen(av), xv, acc);
            }
            if constexpr (!TP64) {
                if (cj != row && scatter && (abad || xr_bad)) red_add_f64(b + cj, df64::widen(av) * xr);
            }
        }
    }
    double total = acc;
    if constexpr (!RS64) {
        const bool zero = (__float_as_uint(sh) << 1) == 0;
        const bool easy = zero || joinable(sh);
        double v = zero ? 0.0 : df64::join(sh, sl);
        if (__any_sync(kFull, !easy)) {  // the sum cancelled below 2^-102 in some lane (rare)
            if (!easy) v = df64::widen(sh) + df64::widen(sl);
        }
        total = any_defer ? acc + v : v;
    }
    if (live) red_add_f64(b + row, total);
}

template <typename VT, int B, int NS, bool RS64, bool TP64>
__device__ __forceinline__ void warp_loop(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                          const VT* __restrict__ val, const double* __restrict__ x, double* b,
                                          TileStage<VT>* my, uint64_t* bar, int64_t t, int64_t tw, int64_t ntiles,
                                          uint32_t spin_limit, uint32_t extra_tx, int32_t* status) {
    const int lane = threadIdx.x & 31;
    Tile g = tile_of(t, n, rp);
    if (lane == 0 && g.staged) issue(&my[0], &bar[0], g, val, col, extra_tx);
    uint32_t phase = 0;  // bit q: parity of stage q's next completion
    int q = 0;
    bool failed = false, next_issued = false;
    for (; t < ntiles; t += tw) {
        const int64_t tn = t + tw;
        Tile gn{};
        next_issued = false;
        if (NS == 2 && tn < ntiles) {
            gn = tile_of(tn, n, rp);
            if (gn.staged) {
                // stage q ^ 1 was last read by the previous tile (finished before its __syncwarp)
                if (lane == 0) {
                    race_dev::fence_proxy_async();
                    issue(&my[q ^ 1], &bar[q ^ 1], gn, val, col, extra_tx);
                }
                next_issued = true;
            }
        }
        const int32_t row = g.r0 + lane;
        const bool live = row < g.r1;
        const int32_t lo = live ? __ldg(rp + row) : 0;
        const int32_t len = live ? __ldg(rp + row + 1) - lo : 0;
        const int32_t maxlen = __reduce_max_sync(kFull, len);
        if (g.staged) {
            const bool ok = race_dev::mbar_wait_n(&bar[q], (phase >> q) & 1u, spin_limit);
            phase ^= 1u << q;
            if (!__all_sync(kFull, ok)) {
                failed = true;
                break;
            }
            tile_rows<VT, B, true, RS64, TP64>(row, live, lo - g.s_al, len, maxlen, my[q].val, my[q].col, x, b);
        } else {
            tile_rows<VT, B, false, RS64, TP64>(row, live, lo, len, maxlen, val, col, x, b);
        }
        __syncwarp();
        if constexpr (NS == 2) {
            g = gn;
            q ^= 1;
        } else if (tn < ntiles) {
            // one stage: the next tile's copy goes into the stage just read
            g = tile_of(tn, n, rp);
            if (lane == 0 && g.staged) {
                race_dev::fence_proxy_async();
                issue(&my[0], &bar[0], g, val, col, extra_tx);
            }
        }
    }
    if (failed) {
        if (lane == 0) atomicExch(status, RACE_ERR_TIMEOUT);
        // the next tile's copy may still be in flight: let it land before the block leaves
        if (next_issued) race_dev::mbar_wait_n(&bar[q ^ 1], (phase >> (q ^ 1)) & 1u, spin_limit);
    }
}

template <typename VT, int B, int NS>
__global__ void __launch_bounds__(kThreads) k_symm_staged(int32_t n, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                          const double* __restrict__ x, double* b, int rs64_quarters,
                                                          int tp64_quarters, uint32_t spin_limit, uint32_t extra_tx,
                                                          int32_t* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    TileStage<VT>* stages = reinterpret_cast<TileStage<VT>*>(base);
    uint64_t* bars = reinterpret_cast<uint64_t*>(stages + NS * kWarps);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TileStage<VT>* my = stages + NS * w;
    uint64_t* bar = bars + NS * w;
    if (lane == 0) {
        for (int q = 0; q < NS; ++q) race_dev::mbar_init(&bar[q], 1);
        race_dev::mbar_fence_init();
    }
    __syncwarp();
    const int64_t ntiles = (static_cast<int64_t>(n) + 31) / 32;
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kWarps + w;
    const int64_t tw = static_cast<int64_t>(gridDim.x) * kWarps;
    if (gw >= ntiles) return;
    // the warp's quarter (fixed for its whole loop): every four consecutive
    // warps take all four, and the warps an SM deals to one sub-partition
    // (same gw mod 4) cycle through them, so each sub-partition's FP64 unit
    // gets its share
    const int quarter = static_cast<int>((gw + (gw >> 2)) & 3);
    const bool rs64 = quarter < rs64_quarters;
    const bool tp64 = 3 - quarter < tp64_quarters;
#define RACE_STG_LOOP(R, T) \
    warp_loop<VT, B, NS, R, T>(n, rp, col, val, x, b, my, bar, gw, tw, ntiles, spin_limit, extra_tx, status)
    if (rs64) {
        if (tp64) RACE_STG_LOOP(true, true);
        else RACE_STG_LOOP(true, false);
    } else {
        if (tp64) RACE_STG_LOOP(false, true);
        else RACE_STG_LOOP(false, false);
    }
#undef RACE_STG_LOOP
}

template <typename VT, int B, int NS>
int launch(const race_schedule* s, const race_launch& l, const double* x, double* b, cudaStream_t st,
           uint32_t spin_limit, uint32_t extra_tx) {
    const size_t smem = staged_smem_bytes<VT, NS>();
    cudaError_t e = cudaFuncSetAttribute(k_symm_staged<VT, B, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_staged: shared-memory attribute: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    const int32_t n = s->plan.n;
    const int64_t ntiles = (static_cast<int64_t>(n) + 31) / 32;
    // blocks of this size that fit one SM's 228 KB of shared memory (1 KB reserved per block)
    const int resident = static_cast<int>(std::min<size_t>(8, (228u * 1024u) / (smem + 1024u)));
    const int per_sm = l.blocks_per_sm > 0 ? std::min(l.blocks_per_sm, resident) : resident;
    const int64_t blocks =
        std::max<int64_t>(1, std::min<int64_t>((ntiles + kWarps - 1) / kWarps,
                                               static_cast<int64_t>(race_device_sms()) * per_sm));
    k_symm_staged<VT, B, NS><<<static_cast<int>(blocks), kThreads, smem, st>>>(
        n, s->d_rp, s->d_col, static_cast<const VT*>(s->d_val), x, b, l.rowsum_fp64_quarters, l.fp64_quarters,
        spin_limit, extra_tx, s->d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        race_set_detail(std::string("k_symm_staged: ") + cudaGetErrorString(e));
        return RACE_ERR_CUDA;
    }
    return RACE_OK;
}

template <typename VT>
int launch_vt(const race_schedule* s, const race_launch& l, const double* x, double* b, cudaStream_t st,
              uint32_t spin, uint32_t extra) {
    const bool two = l.rows_per_group >= 2;  // pipeline stages per warp
    if (l.regs_per_row >= 8)
        return two ? launch<VT, 8, 2>(s, l, x, b, st, spin, extra) : launch<VT, 8, 1>(s, l, x, b, st, spin, extra);
    return two ? launch<VT, 4, 2>(s, l, x, b, st, spin, extra) : launch<VT, 4, 1>(s, l, x, b, st, spin, extra);
}

}  // namespace race_stg

int race_staged_launch(const race_schedule* s, const race_launch& l, const double* x, double* b, cudaStream_t st,
                       uint32_t spin_limit, uint32_t extra_tx) {
    if (s->val_type == RACE_F64) return race_stg::launch_vt<double>(s, l, x, b, st, spin_limit, extra_tx);
    return race_stg::launch_vt<float>(s, l, x, b, st, spin_limit, extra_tx);
}

// Diagnostic for the bounded waits: every stage's mbarrier expects 16 bytes
// more than its two copies deliver, so each wait gives up after a short
// spin while no copy is left in flight (the copies complete; only the
// count stays short).  The kernel records RACE_ERR_TIMEOUT in the schedule's
// status word, which race_poll_status reports and clears.
extern "C" int race_probe_wait_timeout(const race_schedule* s, const double* x_d, double* b_d, void* stream) {
    if (!s || !x_d || !b_d || static_cast<const void*>(x_d) == static_cast<const void*>(b_d)) {
        race_set_detail("race_probe_wait_timeout: NULL or aliasing arguments");
        return RACE_ERR_INVALID;
    }
    if (s->host_only) {
        race_set_detail("schedule was built with RACE_FLAG_HOST_ONLY");
        return RACE_ERR_UNSUPPORTED;
    }
    race_launch l = s->launch;
    l.executor = RACE_EXEC_STAGED;
    l.rows_per_group = 2;
    l.regs_per_row = 4;
    l.blocks_per_sm = 1;
    l.fp64_quarters = 4;
    l.rowsum_fp64_quarters = 4;
    const int rc = race_staged_launch(s, l, x_d, b_d, static_cast<cudaStream_t>(stream), 1u << 12, 16u);
    return rc;
}
