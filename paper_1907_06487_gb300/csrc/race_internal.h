// Internal declarations shared by the library's translation units.
#pragma once
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/race.h"

namespace race {

// One node of the RACE tree (Sec. 4.4.3, tree of Fig. "internal tree").
struct TreeNode {
    int32_t stage = -1;       // s of T_s(i); the root T_{-1}(0) has -1
    int32_t color = 0;        // 0 red, 1 blue
    int32_t lo = 0, hi = 0;   // rows [lo, hi) in the final permuted order
    int32_t n_threads = 1;    // n_t(T_s(i))
    int32_t thread_lo = 0;    // first thread id (ids are consecutive)
    int32_t n_levels = 0;     // parent levels spanned by this group
    int32_t n_sub = 0;        // own levels when it was split (0 = not split)
    int32_t phase_count = 1;
    int32_t phase_off = 0;
    int64_t size = 0;         // rows (or nnz weight) of the group
    int64_t neff = 0;         // effective row count (Sec. 5)
    std::vector<int32_t> kids;
};

// Host-side result of the schedule construction.
struct Plan {
    int32_t n = 0, n_workers = 1, dist_k = 2, balance = 0, max_depth = -1;
    double eps[8] = {0};
    int32_t n_levels = 0;                  // BFS levels of the whole graph
    std::vector<int32_t> perm;             // perm[new] = old
    std::vector<TreeNode> nodes;           // nodes[0] = root
    std::vector<int32_t> stage_ptr;        // n_phases + 1
    std::vector<int32_t> leaf_lo, leaf_hi; // flattened non-empty leaves
    double eta = 0.0;
};

// Builds the RACE plan for the symmetric graph given by an upper CRS whose
// rows are canonical (diagonal first, strictly increasing columns).
void build_plan(int32_t n, const int32_t* row_ptr, const int32_t* col, const race_params& p, Plan& out);

// The plan of RACE_FLAG_NATURAL_ORDER: identity permutation, one phase
// holding one leaf with every row.
void natural_plan(int32_t n, const race_params& p, Plan& out);

// The MC / ABMC schedules of race_build_coloring (coloring.cpp): one phase
// per colour, one leaf per unit (a row, or a block of block_rows rows).
void coloring_plan(int32_t n, const int32_t* rp, const int32_t* col, int32_t method, int32_t block_rows,
                   const race_params& p, Plan& out);

// Canonical export image (layout documented in race.h).
std::vector<uint8_t> export_plan(const Plan& plan);

}  // namespace race

// Capacities of the shared-memory windows of the window executors: write
// set entries per tile, and contributions (row sums + transposed updates).
constexpr int32_t kWindowCap = 1024;
constexpr int32_t kContribCap = 2048;

// Host image of the tiles of one window executor (see window_kernels.cu).
struct WindowHost {
    std::vector<int32_t> hdr;        // 8 int32 per tile
    std::vector<int32_t> ext;        // external targets, sorted per tile
    std::vector<double> val;         // entries, chunk-major (32 slots, column-major)
    std::vector<uint16_t> lidx;      // window index of every entry (0xFFFF = padding)
    std::vector<uint16_t> pos;       // contribution position of every off-diagonal entry
    std::vector<uint16_t> slot_row;  // local row of every slot (0xFFFF = padding)
    std::vector<uint16_t> rs_pos;    // contribution position of every slot's row sum
    std::vector<int32_t> chunk_off;  // first entry of every chunk (+ final end)
    std::vector<uint16_t> seg;       // per tile: contribution groups of the w targets (w+1)
};

// Device tiles of one window executor.
struct WindowSet {
    int32_t n_tiles = 0;
    int32_t* d_hdr = nullptr;
    int32_t* d_ext = nullptr;
    void* d_val = nullptr;           // double or float, as the schedule's values
    uint16_t* d_lidx = nullptr;
    uint16_t* d_pos = nullptr;
    uint16_t* d_slot_row = nullptr;
    uint16_t* d_rs_pos = nullptr;
    int32_t* d_chunk_off = nullptr;
    uint16_t* d_seg = nullptr;
    int32_t* d_unit_tile = nullptr;  // RACE mode: first tile of every leaf (+1)
    bool ready = false;
};

// SELL-32-sigma copy of the permuted upper matrix (sell_kernels.cu): chunks
// of 32 rows stored column by column; entry j of lane l of chunk k at
// off[k] + 32 j + l; row[32 k + l] is the row of that lane (-1: none);
// padding entries have column -1 and value 0.
constexpr int32_t kSellSigma = 1024;  // rows sorted by length within windows of this size

struct SellHost {
    std::vector<int64_t> off;
    std::vector<int32_t> row, col;
    std::vector<double> val64;
    std::vector<float> val32;
};

struct SellSet {
    int64_t n_chunks = 0, n_stored = 0;
    int64_t* d_off = nullptr;
    int32_t* d_row = nullptr;
    int32_t* d_col = nullptr;
    void* d_val = nullptr;
    bool ready = false;
};

// Level-wavefront matrix powers (mpk_kernels.cu): row blocks of `rows`
// rows; reach[t] = the last block that rows of block t touch; `lag` = max_t
// (reach[t] - t); the flags (a ticket counter, then one done flag per power
// and block) are allocated on first use for up to `flag_powers` powers.
struct MpkState {
    int32_t rows = 0, nblk = 0, lag = 0, flag_powers = 0;
    int32_t* d_reach = nullptr;
    int32_t* d_flags = nullptr;
};

// The opaque handle of the C ABI.
struct race_schedule {
    race::Plan plan;
    int32_t val_type = RACE_F64;
    int32_t group_lanes = 8;
    int32_t host_only = 0;
    int32_t want_windows = 1;
    // permuted upper CRS, host copies
    std::vector<int32_t> h_rp, h_col;
    std::vector<double> h_val64;
    std::vector<float> h_val32;
    // device copies
    int32_t* d_rp = nullptr;
    int32_t* d_col = nullptr;
    void* d_val = nullptr;
    int32_t* d_leaf_lo = nullptr;
    int32_t* d_leaf_hi = nullptr;
    int32_t* d_perm = nullptr;
    // full CRS for the spmv_full baseline (lazy)
    int32_t* d_frp = nullptr;
    int32_t* d_fcol = nullptr;
    void* d_fval = nullptr;
    int64_t nnz_full = 0;
    int32_t full_lanes = 8;
    int32_t device = 0;
    int32_t* d_blk = nullptr;   // row-block starts of the upper CRS (streaming)
    int64_t n_blk = 0;
    int32_t* d_fblk = nullptr;  // row-block starts of the full CRS
    int64_t n_fblk = 0;
    int32_t* d_status = nullptr;  // device status word (RACE_ERR_TIMEOUT)
    int32_t* d_stage = nullptr;   // plan.stage_ptr on the device (one-launch executors)
    // the rows of every phase's leaves, phase after phase (RACE_EXEC_PHASE_DF64);
    // phase_row_ptr[p] = the first of phase p.  Per 256 of a phase's rows (one
    // block's share, phase_blk_ptr[p] = the first of phase p), d_phase_blk
    // holds their first row when they are consecutive rows, else -1.
    std::vector<int64_t> phase_row_ptr, phase_blk_ptr;
    int32_t* d_phase_rows = nullptr;
    int32_t* d_phase_blk = nullptr;
    uint32_t* d_bar = nullptr;    // one-launch executors: barrier words, leaf tickets, block ranking
    int32_t max_row_upper = 0, max_row_full = 0;
    WindowSet win_red, win_race;  // window executors (flat tiles / RACE leaves)
    // executor with the transposed products off the FP64 pipe: off-diagonal
    // values range-checked on first use
    // (0 = not checked, 1 = ready, -1 = a value out of range)
    mutable std::atomic<int32_t> df64_state{0};
    mutable SellSet sell;  // built on first use of RACE_EXEC_SELL_DF64
    race_launch launch{};       // symm_spmv executor and shape
    race_launch full_launch{};  // spmv_full shape
    // symm_kacz: phases checked on first use for distance-2 independence on
    // the full rows (0 = not checked, 1 = independent, -1 = not)
    mutable std::atomic<int32_t> kacz_state{0};
    MpkState mpk;  // matrix powers, level wavefront (built on first use)
};

// Row blocks for the streaming kernels: consecutive rows with at most
// max_nnz nonzeros and max_rows rows each (a longer row gets a block alone).
std::vector<int32_t> race_row_blocks(const int32_t* rp, int32_t n, int32_t max_nnz, int32_t max_rows);
int32_t race_max_row(const int32_t* rp, int32_t n);

// Streaming launchers (stream_kernels.cu).
int race_stream_full(const race_schedule* s, const double* x, double* b, cudaStream_t st, int sm_count);
int race_stream_symm_red(const race_schedule* s, const double* x, double* b, cudaStream_t st, int sm_count);

// Window executors (window_kernels.cu).
void race_make_tiles(const int32_t* rp, const int32_t* col, const double* val, int32_t lo, int32_t hi,
                     WindowHost& out, std::vector<int32_t>& mark, int32_t& stamp);
int race_window_launch(const race_schedule* s, bool race_mode, const double* x, double* b, cudaStream_t st,
                       int sm_count);

// Double-float executor (df64_kernels.cu): preparation (range check of the
// off-diagonal values on the host copy of the matrix, once per schedule; no
// device work) and the launch, which prepares on first use.
int race_df64_prepare(const race_schedule* s);
int race_df64_launch(const race_schedule* s, const double* x, double* b, cudaStream_t st);
// The arithmetic of RACE_EXEC_DF64_RED phase by phase (RACE_EXEC_PHASE_DF64).
int race_df64_phase_launch(const race_schedule* s, const double* x, double* b, cudaStream_t st);
// Rows of a phase one block of RACE_EXEC_PHASE_DF64 takes at a time.
constexpr int32_t kPhaseBlockRows = 256;

// SELL executor (sell_kernels.cu): layout construction, upload on first use,
// release, launch.
void race_make_sell(int32_t n, const int32_t* rp, const int32_t* col, const double* v64, const float* v32,
                    int32_t sigma, SellHost& out);
int race_sell_prepare(const race_schedule* s);
void race_free_sell(SellSet& q);
int race_sell_launch(const race_schedule* s, const double* x, double* b, cudaStream_t st);

// Warp-tile staged executor (staged_kernels.cu).  spin_limit bounds every
// mbarrier wait (polls); extra_tx is added to every stage's expected byte
// count (0 in production; the timeout probe overstates it so that every wait
// gives up while no copy stays in flight).
constexpr uint32_t kStagedSpinLimit = 1u << 26;
int race_staged_launch(const race_schedule* s, const race_launch& l, const double* x, double* b, cudaStream_t st,
                       uint32_t spin_limit, uint32_t extra_tx);

// One-launch executors (persist_kernels.cu): every phase in one cooperative
// launch with bounded grid barriers between phases.
int race_persist_launch(const race_schedule* s, int32_t executor, const double* x, double* b, cudaStream_t st);
// Words of s->d_bar for a schedule of stage_ptr_size - 1 phases.
size_t race_persist_bar_words(size_t stage_ptr_size);

// Multiprocessor count of the current device (cached per device).
int race_device_sms();

// Error detail for race_last_error_detail (thread-local).
void race_set_detail(const std::string& s);
