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
//                   order on one block, one launch per phase.  The write
//                   sets of the leaves of a phase are disjoint (distance-2
//                   independent leaves, Eq. "corollary_dk", or stage-0
//                   groups of one level, whose rows write b only in their
//                   own and the next level), and the flush touches W only:
//                   no two blocks touch the same entry of b during a phase.
// No atomics in shared memory; in RACE mode none in global memory either.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "race_internal.h"

namespace race_win {

constexpr int kThreads = 128;
constexpr uint16_t kPadIdx = 0xFFFF;

// Tile header: 8 int32 per tile.  kChunkOff indexes chunk_off, whose entry
// c is the first stored entry of chunk c (the next entry closes it).
enum : int { kLo = 0, kHi, kExtOff, kExtLen, kChunkOff, kSlotOff, kSegOff, kNChunk };

template <typename VT>
__device__ __forceinline__ double ldv(const VT* p) {
    return static_cast<double>(__ldg(p));
}

template <typename VT, bool RACE>
__global__ void __launch_bounds__(kThreads) k_window(
    int32_t n_units, const int32_t* __restrict__ unit_tile, const int32_t* __restrict__ hdr,
    const int32_t* __restrict__ ext, const VT* __restrict__ val, const uint16_t* __restrict__ lidx,
    const uint16_t* __restrict__ pos, const uint16_t* __restrict__ slot_row, const uint16_t* __restrict__ rs_pos,
    const int32_t* __restrict__ chunk_off, const uint16_t* __restrict__ seg, const double* __restrict__ x,
    double* b) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* sx = reinterpret_cast<double*>(smem);
    double* sc = sx + kWindowCap;  // contribution buffer
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kPer = kWindowCap / kThreads;  // window entries per thread
    for (int32_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int32_t t0 = RACE ? __ldg(unit_tile + u) : u;
        const int32_t t1 = RACE ? __ldg(unit_tile + u + 1) : u + 1;
        for (int32_t t = t0; t < t1; ++t) {
            const int32_t* h = hdr + 8 * static_cast<int64_t>(t);
            const int32_t lo = __ldg(h + kLo), hi = __ldg(h + kHi), eoff = __ldg(h + kExtOff);
            const int32_t elen = __ldg(h + kExtLen), coff = __ldg(h + kChunkOff), soff = __ldg(h + kSlotOff);
            const int32_t goff = __ldg(h + kSegOff), nch = __ldg(h + kNChunk);
            const int32_t nr = hi - lo, w = nr + elen;
            // 1. stage x[W]: every index load first, then every x load
            int32_t gi[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int32_t i = tid + q * kThreads;
                gi[q] = i < nr ? lo + i : (i < w ? __ldg(ext + eoff + i - nr) : -1);
            }
            double xv[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) xv[q] = gi[q] >= 0 ? __ldg(x + gi[q]) : 0.0;
            __syncthreads();  // the previous tile's window is flushed
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (gi[q] >= 0) sx[tid + q * kThreads] = xv[q];
            __syncthreads();
            // 2. one warp per chunk of 32 row slots, four entries per lane in flight
            for (int32_t k = warp; k < nch; k += kThreads / 32) {
                const int32_t c0 = __ldg(chunk_off + coff + k), c1 = __ldg(chunk_off + coff + k + 1);
                const int32_t len = (c1 - c0) >> 5;
                const int32_t slot = soff + k * 32 + lane;
                const uint16_t lr = __ldg(slot_row + slot);
                const uint16_t rsp = __ldg(rs_pos + slot);
                const double xr = lr != kPadIdx ? sx[lr] : 0.0;
                double acc = 0.0;
                for (int32_t p = 0; p < len; p += 4) {
                    double a[4];
                    uint16_t l[4], ps[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool v = p + q < len;
                        const int64_t e = c0 + static_cast<int64_t>(p + q) * 32 + lane;
                        a[q] = v ? ldv(val + e) : 0.0;
                        l[q] = v ? __ldg(lidx + e) : kPadIdx;
                        ps[q] = v ? __ldg(pos + e) : 0;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (l[q] == kPadIdx) continue;
                        acc += a[q] * sx[l[q]];
                        if (p + q > 0) sc[ps[q]] = a[q] * xr;  // entry 0 is the diagonal
                    }
                }
                if (lr != kPadIdx) sc[rsp] = acc;
            }
            __syncthreads();
            // 3. flush: one thread per window entry, all segment bounds loaded first
            int32_t sa[kPer], sz[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int32_t i = tid + q * kThreads;
                sa[q] = i < w ? __ldg(seg + goff + i) : 0;
                sz[q] = i < w ? __ldg(seg + goff + i + 1) : 0;
            }
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                if (gi[q] < 0) continue;
                double v = 0.0;
                for (int32_t j = sa[q]; j < sz[q]; ++j) v += sc[j];
                if (RACE) {
                    b[gi[q]] += v;
                } else {
                    atomicAdd(b + gi[q], v);
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
        if (out.chunk_off.empty()) out.chunk_off.push_back(0);
        out.hdr.push_back(static_cast<int32_t>(out.chunk_off.size()) - 1);
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
            const size_t base = out.val.size();
            out.chunk_off.push_back(static_cast<int32_t>(base + static_cast<size_t>(len) * 32));
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
    }
}

int race_window_launch(const race_schedule* s, bool race_mode, const double* x, double* b, cudaStream_t st,
                       int sm_count) {
    using namespace race_win;
    const WindowSet& w = race_mode ? s->win_race : s->win_red;
    const size_t smem = smem_bytes();
    const int per_sm = s->launch.blocks_per_sm > 0 ? s->launch.blocks_per_sm : 9;
    auto go = [&](int32_t n_units, const int32_t* unit_tile, int grid) {
        if (s->val_type == RACE_F64) {
            if (race_mode) configure<double, true>(); else configure<double, false>();
            auto k = race_mode ? k_window<double, true> : k_window<double, false>;
            k<<<grid, kThreads, smem, st>>>(n_units, unit_tile, w.d_hdr, w.d_ext, static_cast<const double*>(w.d_val),
                                           w.d_lidx, w.d_pos, w.d_slot_row, w.d_rs_pos, w.d_chunk_off, w.d_seg, x, b);
        } else {
            if (race_mode) configure<float, true>(); else configure<float, false>();
            auto k = race_mode ? k_window<float, true> : k_window<float, false>;
            k<<<grid, kThreads, smem, st>>>(n_units, unit_tile, w.d_hdr, w.d_ext, static_cast<const float*>(w.d_val),
                                           w.d_lidx, w.d_pos, w.d_slot_row, w.d_rs_pos, w.d_chunk_off, w.d_seg, x, b);
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
