// Host side of the C ABI: input validation and canonicalisation, the
// symmetric permutation of the upper CRS, device upload, export, getters.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "race_internal.h"
#include "race_plan_ops.h"

namespace {
thread_local std::string g_detail;

int fail(int code, const std::string& why) {
    g_detail = why;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_detail = std::string(what) + ": " + cudaGetErrorString(e);
    return RACE_ERR_CUDA;
}

void release_device(race_schedule* s) {
    void* ptrs[] = {s->d_rp, s->d_col, s->d_val, s->d_leaf_lo, s->d_leaf_hi, s->d_perm,
                    s->d_frp, s->d_fcol, s->d_fval, s->d_blk, s->d_fblk, s->d_status,
                    s->mpk.d_reach, s->mpk.d_flags, s->d_stage, s->d_bar, s->d_phase_rows, s->d_phase_blk};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    s->mpk = MpkState();
    s->d_stage = nullptr;
    s->d_bar = nullptr;
    s->d_phase_rows = nullptr;
    s->d_phase_blk = nullptr;
    s->d_rp = s->d_col = s->d_leaf_lo = s->d_leaf_hi = s->d_perm = s->d_frp = s->d_fcol = nullptr;
    s->d_blk = s->d_fblk = s->d_status = nullptr;
    s->d_val = s->d_fval = nullptr;
    s->df64_state.store(0);
    race_free_sell(s->sell);
    for (WindowSet* w : {&s->win_red, &s->win_race}) {
        void* wp[] = {w->d_hdr, w->d_ext, w->d_val, w->d_lidx, w->d_pos, w->d_slot_row, w->d_rs_pos,
                      w->d_chunk_off, w->d_seg, w->d_unit_tile};
        for (void* p : wp)
            if (p) cudaFree(p);
        *w = WindowSet();
    }
}

// Streamed arrays get kStreamPad zeroed elements after their end so that
// copies widened to 16-byte multiples stay inside the allocation.
constexpr size_t kStreamPad = 8;

template <typename T>
int upload(const std::vector<T>& h, T** d, cudaStream_t st, size_t pad = kStreamPad) {
    const size_t bytes = (h.size() + pad) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(RACE_ERR_NOMEM, "cudaMalloc") : cuda_fail(e, "cudaMalloc");
    e = cudaMemsetAsync(*d, 0, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (!h.empty()) {
        e = cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    }
    return RACE_OK;
}

// Canonical rows: diagonal first, strictly increasing columns, explicit 0.0
// diagonal when the input has none (the diagonal is the first entry of each
// row in Alg. "SymmSpMV").  Values kept in double here.
int canonicalize(const race_csr_upper* a, std::vector<int32_t>& rp, std::vector<int32_t>& col,
                 std::vector<double>& val) {
    const int32_t n = a->n;
    if (a->row_ptr[0] != 0) return fail(RACE_ERR_INVALID, "row_ptr[0] != 0");
    if (static_cast<int64_t>(a->row_ptr[n]) != a->nnz) return fail(RACE_ERR_INVALID, "row_ptr[n] != nnz");
    for (int32_t i = 0; i < n; ++i)
        if (a->row_ptr[i + 1] < a->row_ptr[i]) return fail(RACE_ERR_INVALID, "row_ptr not monotone");
    rp.assign(static_cast<size_t>(n) + 1, 0);
    col.clear();
    val.clear();
    col.reserve(static_cast<size_t>(a->nnz) + n);
    val.reserve(static_cast<size_t>(a->nnz) + n);
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int32_t i = 0; i < n; ++i) {
        row.clear();
        bool diag = false;
        for (int64_t t = a->row_ptr[i]; t < a->row_ptr[i + 1]; ++t) {
            const int32_t c = a->col[t];
            if (c < i || c >= n) return fail(RACE_ERR_INVALID, "column below the diagonal or out of range in row " + std::to_string(i));
            const double v = a->val_type == RACE_F32 ? static_cast<double>(static_cast<const float*>(a->val)[t])
                                                     : static_cast<const double*>(a->val)[t];
            if (!std::isfinite(v)) return fail(RACE_ERR_INVALID, "non-finite value in row " + std::to_string(i));
            diag |= (c == i);
            row.push_back({c, t});
        }
        std::sort(row.begin(), row.end());
        for (size_t q = 1; q < row.size(); ++q)
            if (row[q].first == row[q - 1].first) return fail(RACE_ERR_INVALID, "duplicate column in row " + std::to_string(i));
        if (!diag) {
            col.push_back(i);
            val.push_back(0.0);
        }
        for (auto& e : row) {
            col.push_back(e.first);
            val.push_back(a->val_type == RACE_F32 ? static_cast<double>(static_cast<const float*>(a->val)[e.second])
                                                  : static_cast<const double*>(a->val)[e.second]);
        }
        if (col.size() >= static_cast<size_t>(INT32_MAX)) return fail(RACE_ERR_OVERFLOW, "nnz >= 2^31");
        rp[i + 1] = static_cast<int32_t>(col.size());
    }
    return RACE_OK;
}

// Upper CRS of P A P^T: the entry (i, j) moves to row min(P i, P j),
// column max(P i, P j); each row sorted by column (diagonal first).
void permute_upper(int32_t n, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                   const std::vector<double>& val, const std::vector<int32_t>& perm, std::vector<int32_t>& prp,
                   std::vector<int32_t>& pcol, std::vector<double>& pval) {
    std::vector<int32_t> where(n);
    for (int32_t q = 0; q < n; ++q) where[perm[q]] = q;
    prp.assign(static_cast<size_t>(n) + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) ++prp[std::min(where[i], where[col[t]]) + 1];
    for (int32_t i = 0; i < n; ++i) prp[i + 1] += prp[i];
    std::vector<std::pair<int32_t, double>> tmp(col.size());
    std::vector<int32_t> fill(prp.begin(), prp.end() - 1);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            const int32_t u = where[i], w = where[col[t]];
            tmp[fill[std::min(u, w)]++] = {std::max(u, w), val[t]};
        }
    for (int32_t r = 0; r < n; ++r)
        std::sort(tmp.begin() + prp[r], tmp.begin() + prp[r + 1],
                  [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) { return x.first < y.first; });
    pcol.resize(col.size());
    pval.resize(col.size());
    for (size_t q = 0; q < tmp.size(); ++q) {
        pcol[q] = tmp[q].first;
        pval[q] = tmp[q].second;
    }
}

int pick_lanes(int64_t nnz, int32_t n) {
    const double per_row = n > 0 ? static_cast<double>(nnz) / n : 1.0;
    if (per_row <= 4.5) return 4;
    if (per_row <= 9.0) return 8;
    if (per_row <= 18.0) return 16;
    return 32;
}
}  // namespace

void race_set_detail(const std::string& s) { g_detail = s; }

int race_device_sms() {
    // one slot per device ordinal; 0 = not looked up yet (a race between two
    // threads stores the same value twice)
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev >= 64) {
        int c = 0;
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return c > 0 ? c : 1;
    }
    int c = cache[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        if (c <= 0) c = 1;
        cache[dev].store(c, std::memory_order_relaxed);
    }
    return c;
}

std::vector<int32_t> race_row_blocks(const int32_t* rp, int32_t n, int32_t max_nnz, int32_t max_rows) {
    std::vector<int32_t> out(1, 0);
    int32_t r0 = 0;
    while (r0 < n) {
        int32_t r = r0 + 1;
        while (r < n && r - r0 < max_rows && rp[r + 1] - rp[r0] <= max_nnz) ++r;
        out.push_back(r);
        r0 = r;
    }
    return out;
}

int32_t race_max_row(const int32_t* rp, int32_t n) {
    int32_t m = 0;
    for (int32_t r = 0; r < n; ++r) m = std::max(m, rp[r + 1] - rp[r]);
    return m;
}

// Device half of race_build (and of race_upload): uploads the permuted
// matrix and schedule, builds the row blocks and the window tiles.
static int upload_schedule(race_schedule* s, cudaStream_t st) {
    int rc = RACE_OK;
    const int32_t n_rows = s->plan.n;
    
    cudaGetDevice(&s->device);
    if ((rc = upload(s->h_rp, &s->d_rp, st)) || (rc = upload(s->h_col, &s->d_col, st)) ||
        (rc = upload(s->plan.leaf_lo, &s->d_leaf_lo, st)) || (rc = upload(s->plan.leaf_hi, &s->d_leaf_hi, st)) ||
        (rc = upload(s->plan.perm, &s->d_perm, st))) {
        return rc;
    }
    if (s->val_type == RACE_F64) {
        double* d = nullptr;
        rc = upload(s->h_val64, &d, st);
        s->d_val = d;
    } else {
        float* d = nullptr;
        rc = upload(s->h_val32, &d, st);
        s->d_val = d;
    }
    if (rc == RACE_OK) {
        std::vector<int32_t> blk = race_row_blocks(s->h_rp.data(), n_rows, 1024, 256);
        s->n_blk = static_cast<int64_t>(blk.size()) - 1;
        s->max_row_upper = race_max_row(s->h_rp.data(), n_rows);
        rc = upload(blk, &s->d_blk, st);
    }
    if (rc == RACE_OK) {
        std::vector<int32_t> z(1, 0);
        rc = upload(z, &s->d_status, st);
    }
    if (rc == RACE_OK) rc = upload(s->plan.stage_ptr, &s->d_stage, st);
    if (rc == RACE_OK) {
        // the rows of every phase's leaves, phase after phase
        const auto& sp = s->plan.stage_ptr;
        std::vector<int32_t> rows;
        rows.reserve(static_cast<size_t>(n_rows));
        s->phase_row_ptr.assign(1, 0);
        for (size_t p = 0; p + 1 < sp.size(); ++p) {
            for (int32_t q = sp[p]; q < sp[p + 1]; ++q)
                for (int32_t r = s->plan.leaf_lo[static_cast<size_t>(q)]; r < s->plan.leaf_hi[static_cast<size_t>(q)]; ++r)
                    rows.push_back(r);
            s->phase_row_ptr.push_back(static_cast<int64_t>(rows.size()));
        }
        // per block of 256 rows of a phase: its first row if the rows are consecutive
        std::vector<int32_t> blk;
        s->phase_blk_ptr.assign(1, 0);
        for (size_t p = 0; p + 1 < s->phase_row_ptr.size(); ++p) {
            for (int64_t i0 = s->phase_row_ptr[p]; i0 < s->phase_row_ptr[p + 1]; i0 += kPhaseBlockRows) {
                const int64_t i1 = std::min<int64_t>(i0 + kPhaseBlockRows, s->phase_row_ptr[p + 1]);
                bool run = true;
                for (int64_t i = i0 + 1; i < i1 && run; ++i) run = rows[static_cast<size_t>(i)] == rows[static_cast<size_t>(i - 1)] + 1;
                blk.push_back(run ? rows[static_cast<size_t>(i0)] : -1);
            }
            s->phase_blk_ptr.push_back(static_cast<int64_t>(blk.size()));
        }
        rc = upload(rows, &s->d_phase_rows, st);
        if (rc == RACE_OK) rc = upload(blk, &s->d_phase_blk, st);
    }
    if (rc == RACE_OK) {
        // barrier words, a leaf ticket per phase, block-ranking counters
        std::vector<uint32_t> z(race_persist_bar_words(s->plan.stage_ptr.size()), 0u);
        rc = upload(z, &s->d_bar, st);
    }
    if (rc == RACE_OK && s->max_row_upper + 1 <= kWindowCap && s->want_windows) {
        // window executors: flat tiles over all rows, and tiles of every
        // RACE leaf in phase order
        const int32_t n = n_rows;
        std::vector<int32_t> mark(n, 0);
        int32_t stamp = 0;
        std::vector<double> v64;
        const double* vals = s->h_val64.data();
        if (s->val_type == RACE_F32) {
            v64.assign(s->h_val32.begin(), s->h_val32.end());
            vals = v64.data();
        }
        for (int mode = 0; mode < 2 && rc == RACE_OK; ++mode) {
            WindowSet& w = mode == 0 ? s->win_red : s->win_race;
            WindowHost wh;
            std::vector<int32_t> unit_tile;
            if (mode == 0) {
                race_make_tiles(s->h_rp.data(), s->h_col.data(), vals, 0, n, wh, mark, stamp);
            } else {
                const auto& lo = s->plan.leaf_lo;
                const auto& hi = s->plan.leaf_hi;
                for (size_t q = 0; q < lo.size(); ++q) {
                    unit_tile.push_back(static_cast<int32_t>(wh.hdr.size() / 8));
                    race_make_tiles(s->h_rp.data(), s->h_col.data(), vals, lo[q], hi[q], wh, mark, stamp);
                }
                unit_tile.push_back(static_cast<int32_t>(wh.hdr.size() / 8));
            }
            w.n_tiles = static_cast<int32_t>(wh.hdr.size() / 8);
            rc = upload(wh.hdr, &w.d_hdr, st);
            if (rc == RACE_OK) rc = upload(wh.ext, &w.d_ext, st);
            if (rc == RACE_OK) {
                if (s->val_type == RACE_F64) {
                    double* d = nullptr;
                    rc = upload(wh.val, &d, st);
                    w.d_val = d;
                } else {
                    std::vector<float> f(wh.val.begin(), wh.val.end());
                    float* d = nullptr;
                    rc = upload(f, &d, st);
                    w.d_val = d;
                }
            }
            if (rc == RACE_OK) rc = upload(wh.lidx, &w.d_lidx, st);
            if (rc == RACE_OK) rc = upload(wh.pos, &w.d_pos, st);
            if (rc == RACE_OK) rc = upload(wh.slot_row, &w.d_slot_row, st);
            if (rc == RACE_OK) rc = upload(wh.rs_pos, &w.d_rs_pos, st);
            if (rc == RACE_OK) rc = upload(wh.chunk_off, &w.d_chunk_off, st);
            if (rc == RACE_OK) rc = upload(wh.seg, &w.d_seg, st);
            if (rc == RACE_OK && mode == 1) rc = upload(unit_tile, &w.d_unit_tile, st);
            if (rc == RACE_OK) {
                // host vectors go out of scope: finish the copies first
                cudaError_t e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) rc = cuda_fail(e, "window upload");
            }
            w.ready = (rc == RACE_OK);
        }
    }
    if (rc == RACE_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "upload");
    }
    if (rc != RACE_OK) {
        return rc;
    }
    return rc;
}

// Matrix checks shared by race_build and race_import (the rest is checked
// entry by entry by canonicalize).
static int check_matrix(const race_csr_upper* a) {
    if (a->n <= 0) return fail(RACE_ERR_INVALID, "n <= 0");
    if (a->nnz < 0 || (a->nnz > 0 && (!a->col || !a->val)) || !a->row_ptr) return fail(RACE_ERR_INVALID, "NULL matrix array");
    if (a->nnz + a->n >= static_cast<int64_t>(INT32_MAX)) return fail(RACE_ERR_OVERFLOW, "nnz + n >= 2^31");
    if (a->val_type != RACE_F64 && a->val_type != RACE_F32) return fail(RACE_ERR_INVALID, "val_type");
    return RACE_OK;
}

// True when no two leaves of one phase update the same entry of b: a leaf's
// rows write b at their own index and at every stored column (Alg.
// "SymmSpMV"), so the write sets of concurrent leaves must be disjoint
// (the distance-2 condition of Sec. 4.2).
static bool phases_conflict_free(const race::Plan& plan, const std::vector<int32_t>& rp, const std::vector<int32_t>& col) {
    std::vector<int32_t> phase_of(static_cast<size_t>(plan.n), -1), leaf_of(static_cast<size_t>(plan.n), -1);
    for (size_t ph = 0; ph + 1 < plan.stage_ptr.size(); ++ph)
        for (int32_t q = plan.stage_ptr[ph]; q < plan.stage_ptr[ph + 1]; ++q)
            for (int32_t r = plan.leaf_lo[static_cast<size_t>(q)]; r < plan.leaf_hi[static_cast<size_t>(q)]; ++r)
                for (int32_t t = rp[static_cast<size_t>(r)]; t < rp[static_cast<size_t>(r) + 1]; ++t) {
                    const size_t c = static_cast<size_t>(col[static_cast<size_t>(t)]);
                    if (phase_of[c] == static_cast<int32_t>(ph) && leaf_of[c] != q) return false;
                    phase_of[c] = static_cast<int32_t>(ph);
                    leaf_of[c] = q;
                }
    return true;
}

// Common tail of race_build and race_import: value storage, launch
// defaults and (unless host-only) the device upload.
static int finish_schedule(race_schedule* s, int32_t val_type, int32_t group_lanes, uint32_t flags, void* stream,
                           race_schedule** out) {
    try {
        s->val_type = val_type;
        if (val_type == RACE_F32) {
            s->h_val32.assign(s->h_val64.begin(), s->h_val64.end());
            std::vector<double>().swap(s->h_val64);
        }
    } catch (const std::bad_alloc&) {
        delete s;
        return fail(RACE_ERR_NOMEM, "host allocation during build");
    }
    s->group_lanes = group_lanes ? group_lanes : pick_lanes(static_cast<int64_t>(s->h_col.size()), s->plan.n);
    s->launch.executor = RACE_EXEC_LEAF_GROUP;
    s->launch.group_lanes = s->group_lanes;
    s->launch.rows_per_group = 4;
    s->launch.blocks_per_sm = 0;
    s->launch.regs_per_row = 8;
    s->host_only = (flags & RACE_FLAG_HOST_ONLY) ? 1 : 0;
    s->want_windows = (flags & RACE_FLAG_NO_WINDOWS) ? 0 : 1;
    if (!s->host_only) {
        const int rc = upload_schedule(s, static_cast<cudaStream_t>(stream));
        if (rc != RACE_OK) {
            release_device(s);
            delete s;
            return rc;
        }
    }
    *out = s;
    return RACE_OK;
}

extern "C" {

void race_default_params(race_params* p, int32_t n_workers) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dist_k = 2;
    p->n_workers = n_workers;
    p->eps[0] = 0.8;
    p->eps[1] = 0.8;
    for (int i = 2; i < 8; ++i) p->eps[i] = 0.5;
    p->max_depth = -1;
    p->balance = RACE_BAL_ROWS;
    p->group_lanes = 0;
    p->flags = 0;
}

int race_build(const race_csr_upper* a, const race_params* p, void* stream, race_schedule** out) {
    if (!out) return fail(RACE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!a || !p) return fail(RACE_ERR_INVALID, "NULL argument");
    int rc = check_matrix(a);
    if (rc != RACE_OK) return rc;
    if (p->dist_k != 2) return fail(RACE_ERR_UNSUPPORTED, "only distance-2 colouring (SymmSpMV) is built");
    if (p->n_workers < 1) return fail(RACE_ERR_INVALID, "n_workers < 1");
    for (int i = 0; i < 8; ++i)
        if (!(p->eps[i] >= 0.5 && p->eps[i] < 1.0)) return fail(RACE_ERR_INVALID, "eps_s outside [0.5, 1)");
    if (p->balance != RACE_BAL_ROWS && p->balance != RACE_BAL_NNZ) return fail(RACE_ERR_INVALID, "balance");
    if (p->group_lanes != 0 && p->group_lanes != 4 && p->group_lanes != 8 && p->group_lanes != 16 && p->group_lanes != 32)
        return fail(RACE_ERR_INVALID, "group_lanes must be 0, 4, 8, 16 or 32");
    if ((p->flags & RACE_FLAG_PSEUDO_PERIPHERAL) && (p->flags & RACE_FLAG_NATURAL_ORDER))
        return fail(RACE_ERR_INVALID, "RACE_FLAG_PSEUDO_PERIPHERAL has no effect with RACE_FLAG_NATURAL_ORDER");
    if (p->flags & ~(RACE_FLAG_HOST_ONLY | RACE_FLAG_NO_WINDOWS | RACE_FLAG_NATURAL_ORDER | RACE_FLAG_PSEUDO_PERIPHERAL |
                     RACE_FLAG_RCM | RACE_FLAG_ONE_LEVEL_STAGE0))
        return fail(RACE_ERR_INVALID, "unknown flag bits");

    race_schedule* s = new (std::nothrow) race_schedule();
    if (!s) return fail(RACE_ERR_NOMEM, "host allocation");
    try {
        std::vector<int32_t> rp, col;
        std::vector<double> val;
        rc = canonicalize(a, rp, col, val);
        if (rc != RACE_OK) {
            delete s;
            return rc;
        }
        if (p->flags & RACE_FLAG_RCM) {
            // the construction runs on the RCM-ordered matrix; its permutation
            // is then composed with the RCM order (new -> RCM label -> input)
            const std::vector<int32_t> order = race::rcm_order(a->n, rp.data(), col.data());
            std::vector<int32_t> rp1, col1;
            std::vector<double> val1;
            permute_upper(a->n, rp, col, val, order, rp1, col1, val1);
            if (p->flags & RACE_FLAG_NATURAL_ORDER) race::natural_plan(a->n, *p, s->plan);
            else race::build_plan(a->n, rp1.data(), col1.data(), *p, s->plan);
            for (int32_t& v : s->plan.perm) v = order[static_cast<size_t>(v)];
        } else if (p->flags & RACE_FLAG_NATURAL_ORDER) {
            race::natural_plan(a->n, *p, s->plan);
        } else {
            race::build_plan(a->n, rp.data(), col.data(), *p, s->plan);
        }
        permute_upper(a->n, rp, col, val, s->plan.perm, s->h_rp, s->h_col, s->h_val64);
    } catch (const std::bad_alloc&) {
        delete s;
        return fail(RACE_ERR_NOMEM, "host allocation during build");
    }
    return finish_schedule(s, a->val_type, p->group_lanes, p->flags, stream, out);
}

int race_build_coloring(const race_csr_upper* a, int32_t method, int32_t block_rows, int32_t n_workers, uint32_t flags,
                        void* stream, race_schedule** out) {
    if (!out) return fail(RACE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!a) return fail(RACE_ERR_INVALID, "NULL argument");
    int rc = check_matrix(a);
    if (rc != RACE_OK) return rc;
    if (method != RACE_COLOR_MC && method != RACE_COLOR_ABMC) return fail(RACE_ERR_INVALID, "unknown colouring method");
    if (method == RACE_COLOR_ABMC && (block_rows < 1 || block_rows > 4096))
        return fail(RACE_ERR_INVALID, "block_rows must be in 1..4096");
    if (n_workers < 1) return fail(RACE_ERR_INVALID, "n_workers < 1");
    if (flags & ~(RACE_FLAG_HOST_ONLY | RACE_FLAG_NO_WINDOWS | RACE_FLAG_RCM))
        return fail(RACE_ERR_INVALID, "race_build_coloring takes RACE_FLAG_HOST_ONLY, _NO_WINDOWS and _RCM");
    race_params p;
    race_default_params(&p, n_workers);
    race_schedule* s = new (std::nothrow) race_schedule();
    if (!s) return fail(RACE_ERR_NOMEM, "host allocation");
    try {
        std::vector<int32_t> rp, col;
        std::vector<double> val;
        rc = canonicalize(a, rp, col, val);
        if (rc != RACE_OK) {
            delete s;
            return rc;
        }
        if (flags & RACE_FLAG_RCM) {
            const std::vector<int32_t> order = race::rcm_order(a->n, rp.data(), col.data());
            std::vector<int32_t> rp1, col1;
            std::vector<double> val1;
            permute_upper(a->n, rp, col, val, order, rp1, col1, val1);
            race::coloring_plan(a->n, rp1.data(), col1.data(), method, block_rows, p, s->plan);
            for (int32_t& v : s->plan.perm) v = order[static_cast<size_t>(v)];
        } else {
            race::coloring_plan(a->n, rp.data(), col.data(), method, block_rows, p, s->plan);
        }
        permute_upper(a->n, rp, col, val, s->plan.perm, s->h_rp, s->h_col, s->h_val64);
    } catch (const std::bad_alloc&) {
        delete s;
        return fail(RACE_ERR_NOMEM, "host allocation during build");
    }
    return finish_schedule(s, a->val_type, 0, flags, stream, out);
}

int race_import(const race_csr_upper* a, const void* image, size_t size, uint32_t flags, void* stream,
                race_schedule** out) {
    if (!out) return fail(RACE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!a || !image) return fail(RACE_ERR_INVALID, "NULL argument");
    if (flags & ~(RACE_FLAG_HOST_ONLY | RACE_FLAG_NO_WINDOWS))
        return fail(RACE_ERR_INVALID, "race_import takes only RACE_FLAG_HOST_ONLY and RACE_FLAG_NO_WINDOWS");
    int rc = check_matrix(a);
    if (rc != RACE_OK) return rc;
    race_schedule* s = new (std::nothrow) race_schedule();
    if (!s) return fail(RACE_ERR_NOMEM, "host allocation");
    try {
        std::vector<int32_t> rp, col;
        std::vector<double> val;
        rc = canonicalize(a, rp, col, val);
        if (rc != RACE_OK) {
            delete s;
            return rc;
        }
        std::string why;
        if (!race::import_plan(image, size, a->n, s->plan, why)) {
            delete s;
            return fail(RACE_ERR_INVALID, "schedule image: " + why);
        }
        permute_upper(a->n, rp, col, val, s->plan.perm, s->h_rp, s->h_col, s->h_val64);
        if (!phases_conflict_free(s->plan, s->h_rp, s->h_col)) {
            delete s;
            return fail(RACE_ERR_INVALID, "schedule image: two leaves of one phase update the same entry of b "
                                          "(not a distance-2 colouring of this matrix)");
        }
    } catch (const std::bad_alloc&) {
        delete s;
        return fail(RACE_ERR_NOMEM, "host allocation during import");
    }
    return finish_schedule(s, a->val_type, 0, flags, stream, out);
}

int race_upload(race_schedule* s, void* stream) {
    if (!s) return fail(RACE_ERR_INVALID, "NULL schedule");
    if (!s->host_only) return RACE_OK;
    cudaGetDevice(&s->device);
    int rc = upload_schedule(s, static_cast<cudaStream_t>(stream));
    if (rc != RACE_OK) {
        release_device(s);
        return rc;
    }
    s->host_only = 0;
    return RACE_OK;
}

int race_prepare_full(race_schedule* s, void* stream) {
    if (!s) return fail(RACE_ERR_INVALID, "NULL schedule");
    if (s->host_only) return fail(RACE_ERR_UNSUPPORTED, "host-only schedule");
    if (s->d_frp) return RACE_OK;
    const int32_t n = s->plan.n;
    const int64_t nnz_full = 2 * static_cast<int64_t>(s->h_col.size()) - n;
    if (nnz_full >= INT32_MAX) return fail(RACE_ERR_OVERFLOW, "full nnz >= 2^31");
    std::vector<int32_t> frp(static_cast<size_t>(n) + 1, 0), fcol(static_cast<size_t>(nnz_full));
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = s->h_rp[r]; t < s->h_rp[r + 1]; ++t) {
            ++frp[r + 1];
            if (s->h_col[t] != r) ++frp[s->h_col[t] + 1];
        }
    for (int32_t r = 0; r < n; ++r) frp[r + 1] += frp[r];
    std::vector<int32_t> fill(frp.begin(), frp.end() - 1);
    std::vector<double> fval64;
    std::vector<float> fval32;
    if (s->val_type == RACE_F64) fval64.resize(static_cast<size_t>(nnz_full));
    else fval32.resize(static_cast<size_t>(nnz_full));
    auto put = [&](int32_t row, int32_t c, int32_t t) {
        const int32_t q = fill[row]++;
        fcol[q] = c;
        if (s->val_type == RACE_F64) fval64[q] = s->h_val64[t];
        else fval32[q] = s->h_val32[t];
    };
    // lower part first (rows r < c in increasing order), then the upper part,
    // so every full row is sorted by column
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = s->h_rp[r] + 1; t < s->h_rp[r + 1]; ++t) put(s->h_col[t], r, t);
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = s->h_rp[r]; t < s->h_rp[r + 1]; ++t) put(r, s->h_col[t], t);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload(frp, &s->d_frp, st);
    if (rc == RACE_OK) rc = upload(fcol, &s->d_fcol, st);
    if (rc == RACE_OK) {
        if (s->val_type == RACE_F64) {
            double* d = nullptr;
            rc = upload(fval64, &d, st);
            s->d_fval = d;
        } else {
            float* d = nullptr;
            rc = upload(fval32, &d, st);
            s->d_fval = d;
        }
    }
    if (rc == RACE_OK) {
        std::vector<int32_t> blk = race_row_blocks(frp.data(), n, 1024, 256);
        s->n_fblk = static_cast<int64_t>(blk.size()) - 1;
        s->max_row_full = race_max_row(frp.data(), n);
        rc = upload(blk, &s->d_fblk, st);
    }
    if (rc == RACE_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "full upload");
    }
    s->nnz_full = nnz_full;
    const double per_row = static_cast<double>(nnz_full) / n;
    s->full_lanes = per_row <= 4.5 ? 4 : per_row <= 9.0 ? 8 : per_row <= 18.0 ? 16 : 32;
    if (s->full_launch.group_lanes == 0) {
        s->full_launch.executor = 1;
        s->full_launch.group_lanes = s->full_lanes;
        s->full_launch.rows_per_group = 4;
        s->full_launch.blocks_per_sm = 0;
        s->full_launch.regs_per_row = 16;
    }
    return rc;
}

int race_get_perm(const race_schedule* s, int32_t* perm_host) {
    if (!s || !perm_host) return fail(RACE_ERR_INVALID, "NULL argument");
    std::memcpy(perm_host, s->plan.perm.data(), sizeof(int32_t) * s->plan.perm.size());
    return RACE_OK;
}

int race_get_matrix(const race_schedule* s, int32_t* row_ptr, int32_t* col, void* val) {
    if (!s) return fail(RACE_ERR_INVALID, "NULL schedule");
    if (row_ptr) std::memcpy(row_ptr, s->h_rp.data(), sizeof(int32_t) * s->h_rp.size());
    if (col) std::memcpy(col, s->h_col.data(), sizeof(int32_t) * s->h_col.size());
    if (val) {
        if (s->val_type == RACE_F64) std::memcpy(val, s->h_val64.data(), sizeof(double) * s->h_val64.size());
        else std::memcpy(val, s->h_val32.data(), sizeof(float) * s->h_val32.size());
    }
    return RACE_OK;
}

int race_get_phases(const race_schedule* s, int32_t* stage_ptr, int32_t* leaf_lo, int32_t* leaf_hi) {
    if (!s) return fail(RACE_ERR_INVALID, "NULL schedule");
    if (stage_ptr) std::memcpy(stage_ptr, s->plan.stage_ptr.data(), sizeof(int32_t) * s->plan.stage_ptr.size());
    if (leaf_lo) std::memcpy(leaf_lo, s->plan.leaf_lo.data(), sizeof(int32_t) * s->plan.leaf_lo.size());
    if (leaf_hi) std::memcpy(leaf_hi, s->plan.leaf_hi.data(), sizeof(int32_t) * s->plan.leaf_hi.size());
    return RACE_OK;
}

int race_get_info(const race_schedule* s, race_info* info) {
    if (!s || !info) return fail(RACE_ERR_INVALID, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n = s->plan.n;
    info->nnz_upper = static_cast<int64_t>(s->h_col.size());
    info->n_levels = s->plan.n_levels;
    info->n_phases = static_cast<int32_t>(s->plan.stage_ptr.size()) - 1;
    info->n_leaves = static_cast<int32_t>(s->plan.leaf_lo.size());
    info->n_nodes = static_cast<int32_t>(s->plan.nodes.size());
    int32_t depth = 0;
    for (const auto& t : s->plan.nodes) depth = std::max(depth, t.stage + 1);
    info->depth = depth;
    info->n_workers = s->plan.n_workers;
    info->val_type = s->val_type;
    info->group_lanes = s->group_lanes;
    info->eta = s->plan.eta;
    info->neff_root = s->plan.nodes[0].neff;
    return RACE_OK;
}

int race_export(const race_schedule* s, void* buf, size_t* size) {
    if (!s || !size) return fail(RACE_ERR_INVALID, "NULL argument");
    std::vector<uint8_t> img = race::export_plan(s->plan);
    if (!buf) {
        *size = img.size();
        return RACE_OK;
    }
    if (*size < img.size()) {
        *size = img.size();
        return fail(RACE_ERR_INVALID, "export buffer too small");
    }
    std::memcpy(buf, img.data(), img.size());
    *size = img.size();
    return RACE_OK;
}

void race_free(race_schedule* s) {
    if (!s) return;
    release_device(s);
    delete s;
}

const char* race_strerror(int code) {
    switch (code) {
        case RACE_OK: return "ok";
        case RACE_ERR_INVALID: return "invalid argument or malformed matrix";
        case RACE_ERR_OVERFLOW: return "size exceeds the int32 layout";
        case RACE_ERR_NOMEM: return "out of memory";
        case RACE_ERR_CUDA: return "CUDA runtime error";
        case RACE_ERR_TIMEOUT: return "bounded device wait gave up";
        case RACE_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown error code";
    }
}

const char* race_last_error_detail(void) { return g_detail.c_str(); }

}  // extern "C"
