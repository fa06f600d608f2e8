// Shared-memory window executors of SymmSpMV (Alg. "SymmSpMV").
//
// A tile is a run of consecutive rows [lo, hi) of the permuted upper CRS.
// Its write set W = {lo..hi-1} U {upper columns >= hi of its rows} (the
// "external" targets, sorted) has at most kWindow entries.  Each stored
// entry carries a 16-bit local index into W instead of its global column.
// A thread block processes a tile in three steps:
//   1. stage x[W] into shared memory and zero the window of b;
//   2. one thread per row: row sum from the staged x; the transposed update
//      a*x[row] and the row sum go to the shared window (shared-memory
//      atomics, no global traffic);
//   3. flush the window to b, coalesced (W is sorted):
//        RED mode:  reductions at L2 (tiles run in any order, one launch);
//        RACE mode: plain load/add/store.  The tiles of one RACE leaf run in
//                   order on one block, one launch per phase; leaves of a
//                   phase are distance-2 independent (Eq. "corollary_dk"), so
//                   their write sets are disjoint and no other block touches
//                   the same entries of b during the phase.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "race_internal.h"

namespace race_win {

constexpr int kThreads = 256;

template <typename VT>
__device__ __forceinline__ double ldv(const VT* p) {
    return static_cast<double>(__ldg(p));
}

// units: for RED, one unit per tile; for RACE, one unit per leaf of the
// phase, its tiles [unit_tile[u], unit_tile[u+1]).
template <typename VT, bool RACE>
__global__ void __launch_bounds__(kThreads) k_window(int32_t n_units, const int32_t* __restrict__ unit_tile,
                                                     const int32_t* __restrict__ tiles,  // lo, hi, ext_off, ext_len
                                                     const int32_t* __restrict__ rp, const VT* __restrict__ val,
                                                     const uint16_t* __restrict__ lidx, const int32_t* __restrict__ ext,
                                                     const double* __restrict__ x, double* b) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* sx = reinterpret_cast<double*>(smem);
    double* sb = sx + kWindowCap;
    int32_t* sw = reinterpret_cast<int32_t*>(sb + kWindowCap);
    const int tid = threadIdx.x;
    for (int32_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int32_t t0 = RACE ? __ldg(unit_tile + u) : u;
        const int32_t t1 = RACE ? __ldg(unit_tile + u + 1) : u + 1;
        for (int32_t t = t0; t < t1; ++t) {
            const int32_t lo = __ldg(tiles + 4 * t), hi = __ldg(tiles + 4 * t + 1);
            const int32_t eoff = __ldg(tiles + 4 * t + 2), elen = __ldg(tiles + 4 * t + 3);
            const int32_t nr = hi - lo, w = nr + elen;
            __syncthreads();  // previous tile's flush has read the window
            for (int32_t i = tid; i < w; i += kThreads) {
                const int32_t g = i < nr ? lo + i : __ldg(ext + eoff + (i - nr));
                sw[i] = g;
                sx[i] = __ldg(x + g);
                sb[i] = 0.0;
            }
            __syncthreads();
            for (int32_t i = tid; i < nr; i += kThreads) {
                const int32_t r = lo + i;
                const int32_t js = __ldg(rp + r), je = __ldg(rp + r + 1);
                const double xr = sx[i];
                double acc = 0.0;
                for (int32_t j = js; j < je; ++j) {
                    const double a = ldv(val + j);
                    const int32_t l = __ldg(lidx + j);
                    acc += a * sx[l];
                    if (j != js) atomicAdd(sb + l, a * xr);  // transposed part
                }
                atomicAdd(sb + i, acc);
            }
            __syncthreads();
            for (int32_t i = tid; i < w; i += kThreads) {
                const double v = sb[i];
                if (RACE) {
                    b[sw[i]] += v;
                } else {
                    atomicAdd(b + sw[i], v);
                }
            }
        }
    }
}

size_t smem_bytes() { return kWindowCap * (2 * sizeof(double) + sizeof(int32_t)); }

template <typename VT, bool RACE>
void configure() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_window<VT, RACE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_bytes()));
        done = true;
    }
}

}  // namespace race_win

// Host-side construction of the tiles of one row range [lo, hi) of the
// permuted upper CRS, appended to the output arrays.  A tile grows row by
// row while (rows + external targets) <= cap.
void race_make_tiles(const int32_t* rp, const int32_t* col, int32_t lo, int32_t hi, int32_t cap,
                     std::vector<int32_t>& tiles, std::vector<int32_t>& ext, std::vector<uint16_t>& lidx,
                     std::vector<int32_t>& mark, int32_t& stamp) {
    int32_t r = lo;
    std::vector<int32_t> cur;
    while (r < hi) {
        ++stamp;
        const int32_t tlo = r;
        int32_t n_ext = 0;
        cur.clear();
        while (r < hi) {
            // count new externals of row r (columns > r not yet marked)
            int32_t add = 0;
            for (int32_t j = rp[r] + 1; j < rp[r + 1]; ++j)
                if (mark[col[j]] != stamp) ++add;
            const int32_t leaving = (mark[r] == stamp) ? 1 : 0;  // r turns from external into a row
            const int32_t w_after = (r + 1 - tlo) + n_ext - leaving + add;
            if (w_after > cap && r > tlo) break;
            n_ext -= leaving;
            for (int32_t j = rp[r] + 1; j < rp[r + 1]; ++j)
                if (mark[col[j]] != stamp) {
                    mark[col[j]] = stamp;
                    cur.push_back(col[j]);
                    ++n_ext;
                }
            mark[r] = stamp;
            ++r;
        }
        const int32_t thi = r;
        // externals: marked columns >= thi, sorted
        std::vector<int32_t> e;
        e.reserve(cur.size());
        for (int32_t c : cur)
            if (c >= thi) e.push_back(c);
        std::sort(e.begin(), e.end());
        e.erase(std::unique(e.begin(), e.end()), e.end());
        tiles.push_back(tlo);
        tiles.push_back(thi);
        tiles.push_back(static_cast<int32_t>(ext.size()));
        tiles.push_back(static_cast<int32_t>(e.size()));
        const int32_t nr = thi - tlo;
        for (int32_t q = tlo; q < thi; ++q)
            for (int32_t j = rp[q]; j < rp[q + 1]; ++j) {
                const int32_t c = col[j];
                int32_t l;
                if (c < thi) {
                    l = c - tlo;
                } else {
                    l = nr + static_cast<int32_t>(std::lower_bound(e.begin(), e.end(), c) - e.begin());
                }
                lidx[j] = static_cast<uint16_t>(l);
            }
        ext.insert(ext.end(), e.begin(), e.end());
    }
}

int race_window_launch(const race_schedule* s, bool race_mode, const double* x, double* b, cudaStream_t st,
                       int sm_count) {
    using namespace race_win;
    const size_t smem = smem_bytes();
    const int per_sm = s->launch.blocks_per_sm > 0 ? s->launch.blocks_per_sm : 5;
    if (!race_mode) {
        const int32_t nt = s->win_red.n_tiles;
        if (nt == 0) return RACE_OK;
        const int grid = std::min<int64_t>(nt, static_cast<int64_t>(sm_count) * per_sm);
        if (s->val_type == RACE_F64) {
            configure<double, false>();
            k_window<double, false><<<grid, kThreads, smem, st>>>(nt, nullptr, s->win_red.d_tiles, s->d_rp,
                                                                  static_cast<const double*>(s->d_val),
                                                                  s->win_red.d_lidx, s->win_red.d_ext, x, b);
        } else {
            configure<float, false>();
            k_window<float, false><<<grid, kThreads, smem, st>>>(nt, nullptr, s->win_red.d_tiles, s->d_rp,
                                                                 static_cast<const float*>(s->d_val),
                                                                 s->win_red.d_lidx, s->win_red.d_ext, x, b);
        }
        return RACE_OK;
    }
    const auto& sp = s->plan.stage_ptr;
    for (size_t p = 0; p + 1 < sp.size(); ++p) {
        const int32_t nl = sp[p + 1] - sp[p];
        if (nl == 0) continue;
        const int grid = std::min<int64_t>(nl, static_cast<int64_t>(sm_count) * per_sm);
        const int32_t* ut = s->win_race.d_unit_tile + sp[p];
        if (s->val_type == RACE_F64) {
            configure<double, true>();
            k_window<double, true><<<grid, kThreads, smem, st>>>(nl, ut, s->win_race.d_tiles, s->d_rp,
                                                                 static_cast<const double*>(s->d_val),
                                                                 s->win_race.d_lidx, s->win_race.d_ext, x, b);
        } else {
            configure<float, true>();
            k_window<float, true><<<grid, kThreads, smem, st>>>(nl, ut, s->win_race.d_tiles, s->d_rp,
                                                                static_cast<const float*>(s->d_val),
                                                                s->win_race.d_lidx, s->win_race.d_ext, x, b);
        }
    }
    return RACE_OK;
}
