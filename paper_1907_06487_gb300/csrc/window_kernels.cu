// Shared-memory window executors of SymmSpMV (Alg. "SymmSpMV").
//
// A tile is a run of consecutive rows [lo, hi) of the permuted upper CRS.
// Its write set W = {lo..hi-1} U {upper columns >= hi of its rows} (the
// "external" targets, sorted) has at most kWindowCap entries, and the tile
// makes at most kContribCap contributions (one row sum per row and one
// transposed update per stored off-diagonal entry).
//
// Layout (built on the host, per tile):
//   - the tile's rows are ordered by length (longest first) into slots of
//     32; a chunk of 32 slots stores its entries column-major (entry p of
//     slot s at p*32 + s), padded to the chunk's longest row, so a warp's
//     loads of val / local index / position are contiguous (SELL-32-sigma
//     with sigma = the tile);
//   - every entry carries its column as a 16-bit index into W and the
//     16-bit position of its transposed contribution in a per-tile buffer
//     where contributions are grouped by target (a transpose computed once
//     at build time); seg[i]..seg[i+1] is the group of target i.
// A thread block processes a tile in three steps:
//   1. stage x[W] into shared memory;
//   2. one lane per row slot: row sum from the staged x; each transposed
//      contribution a*x[row] and the row sum are stored (plain stores, each
//      position written once) into the contribution buffer;
//   3. one thread per target sums its group and flushes it to b:
//        RED mode:  reduction at L2 (tiles in any order, one launch);
//        RACE mode: plain load/add/store.  The tiles of one RACE leaf run in
//                   order on one block, one launch per phase.  Leaves of a
//                   phase are distance-2 independent (Eq. "corollary_dk"),
//                   so their write sets are disjoint: no two blocks touch
//                   the same entry of b during a phase.
// No atomics in shared memory; in RACE mode none in global memory either.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "race_internal.h"

namespace race_win {

constexpr int kThreads = 256;
constexpr uint16_t kPadIdx = 0xFFFF;

// Tile header: 8 int32 per tile.
enum : int { kLo = 0, kHi, kExtOff, kExtLen, kEntOff, kSlotOff, kSegOff, kNChunk };

template <typename VT>
__device__ __forceinline__ double ldv(const VT* p) {
    return static_cast<double>(__ldg(p));
}

template <typename VT, bool RACE>
__global__ void __launch_bounds__(kThreads) k_window(
    int32_t n_units, const int32_t* __restrict__ unit_tile, const int32_t* __restrict__ hdr,
    const int32_t* __restrict__ ext, const VT* __restrict__ val, const uint16_t* __restrict__ lidx,
    const uint16_t* __restrict__ pos, const uint16_t* __restrict__ slot_row, const uint16_t* __restrict__ rs_pos,
    const uint16_t* __restrict__ chunk_len, const uint16_t* __restrict__ seg, const double* __restrict__ x,
    double* b) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* sx = reinterpret_cast<double*>(smem);
    double* sc = sx + kWindowCap;  // contribution buffer
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int32_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int32_t t0 = RACE ? __ldg(unit_tile + u) : u;
        const int32_t t1 = RACE ? __ldg(unit_tile + u + 1) : u + 1;
        for (int32_t t = t0; t < t1; ++t) {
            const int32_t* h = hdr + 8 * static_cast<int64_t>(t);
            const int32_t lo = __ldg(h + kLo), hi = __ldg(h + kHi), eoff = __ldg(h + kExtOff);
            const int32_t elen = __ldg(h + kExtLen), ent = __ldg(h + kEntOff), soff = __ldg(h + kSlotOff);
            const int32_t goff = __ldg(h + kSegOff), nch = __ldg(h + kNChunk);
            const int32_t nr = hi - lo, w = nr + elen;
            __syncthreads();  // the previous tile is flushed
            for (int32_t i = tid; i < w; i += kThreads) sx[i] = __ldg(x + (i < nr ? lo + i : __ldg(ext + eoff + i - nr)));
            __syncthreads();
            // chunks of 32 slots; entry offsets accumulate over the chunks
            int32_t cbase = ent;
            int32_t q = 0;
            for (int32_t k = warp; k < nch; k += kThreads / 32) {
                // entry base of chunk k: sum of 32*len over chunks before it
                for (; q < k; ++q) cbase += 32 * __ldg(chunk_len + soff / 32 + q);
                const int32_t len = __ldg(chunk_len + soff / 32 + k);
                const int32_t slot = soff + k * 32 + lane;
                const uint16_t lr = __ldg(slot_row + slot);
                const double xr = lr != kPadIdx ? sx[lr] : 0.0;
                double acc = 0.0;
                int32_t p = 0;
                for (; p + 2 <= len; p += 2) {
                    const int64_t e0 = cbase + static_cast<int64_t>(p) * 32 + lane, e1 = e0 + 32;
                    const double a0 = ldv(val + e0), a1 = ldv(val + e1);
                    const uint16_t l0 = __ldg(lidx + e0), l1 = __ldg(lidx + e1);
                    const uint16_t p0 = __ldg(pos + e0), p1 = __ldg(pos + e1);
                    if (l0 != kPadIdx) {
                        acc += a0 * sx[l0];
                        if (p > 0) sc[p0] = a0 * xr;
                    }
                    if (l1 != kPadIdx) {
                        acc += a1 * sx[l1];
                        sc[p1] = a1 * xr;
                    }
                }
                if (p < len) {
                    const int64_t e0 = cbase + static_cast<int64_t>(p) * 32 + lane;
                    const double a0 = ldv(val + e0);
                    const uint16_t l0 = __ldg(lidx + e0), p0 = __ldg(pos + e0);
                    if (l0 != kPadIdx) {
                        acc += a0 * sx[l0];
                        if (p > 0) sc[p0] = a0 * xr;
                    }
                }
                if (lr != kPadIdx) sc[__ldg(rs_pos + slot)] = acc;
            }
            __syncthreads();
            for (int32_t i = tid; i < w; i += kThreads) {
                const int32_t a = __ldg(seg + goff + i), z = __ldg(seg + goff + i + 1);
                double v = 0.0;
                for (int32_t j = a; j < z; ++j) v += sc[j];
                const int32_t g = i < nr ? lo + i : __ldg(ext + eoff + i - nr);
                if (RACE) {
                    b[g] += v;
                } else {
                    atomicAdd(b + g, v);
                }
            }
        }
    }
}

size_t smem_bytes() { return sizeof(double) * (kWindowCap + kContribCap); }

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

// ---------------------------------------------------------------------------
// Host construction of the tiles of rows [lo, hi), appended to `out`.
// A tile grows row by row while |W| <= kWindowCap, its contributions
// <= kContribCap and its rows <= 1024.
void race_make_tiles(const int32_t* rp, const int32_t* col, const double* val, int32_t lo, int32_t hi,
                     WindowHost& out, std::vector<int32_t>& mark, int32_t& stamp) {
    using race_win::kPadIdx;
    int32_t r = lo;
    std::vector<int32_t> cand, ext, slots, cnt;
    while (r < hi) {
        ++stamp;
        const int32_t tlo = r;
        int32_t n_ext = 0, n_contrib = 0;
        cand.clear();
        while (r < hi) {
            int32_t add = 0;
            for (int32_t j = rp[r] + 1; j < rp[r + 1]; ++j)
                if (mark[col[j]] != stamp) ++add;
            const int32_t leaving = (mark[r] == stamp) ? 1 : 0;  // r turns from target into row
            const int32_t rows = r + 1 - tlo;
            const int32_t w_after = rows + n_ext - leaving + add;
            const int32_t k_after = n_contrib + (rp[r + 1] - rp[r]);
            if (r > tlo && (w_after > kWindowCap || k_after > kContribCap || rows > 1024)) break;
            n_ext -= leaving;
            n_contrib = k_after;
            for (int32_t j = rp[r] + 1; j < rp[r + 1]; ++j)
                if (mark[col[j]] != stamp) {
                    mark[col[j]] = stamp;
                    cand.push_back(col[j]);
                    ++n_ext;
                }
            mark[r] = stamp;
            ++r;
        }
        const int32_t thi = r, nr = thi - tlo;
        ext.clear();
        for (int32_t c : cand)
            if (c >= thi) ext.push_back(c);
        std::sort(ext.begin(), ext.end());
        const int32_t w = nr + static_cast<int32_t>(ext.size());
        auto local = [&](int32_t c) -> int32_t {
            return c < thi ? c - tlo
                           : nr + static_cast<int32_t>(std::lower_bound(ext.begin(), ext.end(), c) - ext.begin());
        };
        // slots: rows by length, longest first (stable), padded to 32
        slots.resize(nr);
        std::iota(slots.begin(), slots.end(), 0);
        std::stable_sort(slots.begin(), slots.end(), [&](int32_t a, int32_t b2) {
            return (rp[tlo + a + 1] - rp[tlo + a]) > (rp[tlo + b2 + 1] - rp[tlo + b2]);
        });
        const int32_t nslot = (nr + 31) / 32 * 32, nch = nslot / 32;
        // contributions per target: row sums + transposed updates
        cnt.assign(w + 1, 0);
        for (int32_t i = 0; i < nr; ++i) {
            cnt[i + 1] += 1;
            for (int32_t j = rp[tlo + i] + 1; j < rp[tlo + i + 1]; ++j) cnt[local(col[j]) + 1] += 1;
        }
        for (int32_t i = 0; i < w; ++i) cnt[i + 1] += cnt[i];
        const size_t seg_off = out.seg.size();
        for (int32_t i = 0; i <= w; ++i) out.seg.push_back(static_cast<uint16_t>(cnt[i]));
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        // header
        out.hdr.push_back(tlo);
        out.hdr.push_back(thi);
        out.hdr.push_back(static_cast<int32_t>(out.ext.size()));
        out.hdr.push_back(static_cast<int32_t>(ext.size()));
        out.hdr.push_back(static_cast<int32_t>(out.val.size()));
        out.hdr.push_back(static_cast<int32_t>(out.slot_row.size()));
        out.hdr.push_back(static_cast<int32_t>(seg_off));
        out.hdr.push_back(nch);
        out.ext.insert(out.ext.end(), ext.begin(), ext.end());
        // chunks
        for (int32_t k = 0; k < nch; ++k) {
            int32_t len = 0;
            for (int32_t s = 0; s < 32; ++s) {
                const int32_t q = k * 32 + s;
                if (q < nr) len = std::max(len, rp[tlo + slots[q] + 1] - rp[tlo + slots[q]]);
            }
            out.chunk_len.push_back(static_cast<uint16_t>(len));
            const size_t base = out.val.size();
            out.val.resize(base + static_cast<size_t>(len) * 32, 0.0);
            out.lidx.resize(base + static_cast<size_t>(len) * 32, kPadIdx);
            out.pos.resize(base + static_cast<size_t>(len) * 32, 0);
            for (int32_t s = 0; s < 32; ++s) {
                const int32_t q = k * 32 + s;
                if (q >= nr) {
                    out.slot_row.push_back(kPadIdx);
                    out.rs_pos.push_back(0);
                    continue;
                }
                const int32_t i = slots[q], row = tlo + i;
                out.slot_row.push_back(static_cast<uint16_t>(i));
                out.rs_pos.push_back(static_cast<uint16_t>(fill[i]++));
                for (int32_t j = rp[row]; j < rp[row + 1]; ++j) {
                    const int32_t p = j - rp[row];
                    const size_t e = base + static_cast<size_t>(p) * 32 + s;
                    const int32_t l = local(col[j]);
                    out.val[e] = val[j];
                    out.lidx[e] = static_cast<uint16_t>(l);
                    if (p > 0) out.pos[e] = static_cast<uint16_t>(fill[l]++);
                }
            }
        }
        // the slot table is padded to whole chunks already; keep chunk_len
        // indexable as slot_off / 32 + k
    }
}

int race_window_launch(const race_schedule* s, bool race_mode, const double* x, double* b, cudaStream_t st,
                       int sm_count) {
    using namespace race_win;
    const WindowSet& w = race_mode ? s->win_race : s->win_red;
    const size_t smem = smem_bytes();
    const int per_sm = s->launch.blocks_per_sm > 0 ? s->launch.blocks_per_sm : 4;
    auto go = [&](int32_t n_units, const int32_t* unit_tile, int grid) {
        if (s->val_type == RACE_F64) {
            if (race_mode) configure<double, true>(); else configure<double, false>();
            auto k = race_mode ? k_window<double, true> : k_window<double, false>;
            k<<<grid, kThreads, smem, st>>>(n_units, unit_tile, w.d_hdr, w.d_ext, static_cast<const double*>(w.d_val),
                                           w.d_lidx, w.d_pos, w.d_slot_row, w.d_rs_pos, w.d_chunk_len, w.d_seg, x, b);
        } else {
            if (race_mode) configure<float, true>(); else configure<float, false>();
            auto k = race_mode ? k_window<float, true> : k_window<float, false>;
            k<<<grid, kThreads, smem, st>>>(n_units, unit_tile, w.d_hdr, w.d_ext, static_cast<const float*>(w.d_val),
                                           w.d_lidx, w.d_pos, w.d_slot_row, w.d_rs_pos, w.d_chunk_len, w.d_seg, x, b);
        }
    };
    if (!race_mode) {
        if (w.n_tiles == 0) return RACE_OK;
        go(w.n_tiles, nullptr, static_cast<int>(std::min<int64_t>(w.n_tiles, static_cast<int64_t>(sm_count) * per_sm)));
        return RACE_OK;
    }
    const auto& sp = s->plan.stage_ptr;
    for (size_t p = 0; p + 1 < sp.size(); ++p) {
        const int32_t nl = sp[p + 1] - sp[p];
        if (nl == 0) continue;
        go(nl, w.d_unit_tile + sp[p], static_cast<int>(std::min<int64_t>(nl, static_cast<int64_t>(sm_count) * per_sm)));
    }
    return RACE_OK;
}
