// Many matrices in one CUDA graph, and a launch-shape autotuner.
//
// A batch holds one SymmSpMV / SymmSpMM per schedule, captured once from
// the caller's stream into a CUDA graph and replayed with one graph launch:
// the small matrices of a batch are launch-latency bound, and a graph
// removes the per-launch host cost.  The autotuner times the candidate
// launch shapes of one schedule on the caller's buffers (CUDA events on the
// caller's stream) and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "race_internal.h"

struct race_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t count = 0;
    int32_t k = 1;
};

namespace {
int run_one(race_schedule* s, int32_t k, const double* X, double* B, cudaStream_t st) {
    return k == 1 ? symm_spmv(s, X, B, st) : symm_spmm(s, k, X, B, st);
}

int cuda_err(cudaError_t e, const char* what) {
    race_set_detail(std::string(what) + ": " + cudaGetErrorString(e));
    return RACE_ERR_CUDA;
}
}  // namespace

constexpr int kBranches = 8;

extern "C" {

int race_batch_create(race_schedule* const* s, int32_t count, int32_t k, const double* const* X_d,
                      double* const* B_d, void* stream, race_batch** out) {
    if (!out) {
        race_set_detail("out is NULL");
        return RACE_ERR_INVALID;
    }
    *out = nullptr;
    if (!s || !X_d || !B_d || count < 1 || k < 1 || k > 16) {
        race_set_detail("race_batch_create: bad argument");
        return RACE_ERR_INVALID;
    }
    for (int32_t i = 0; i < count; ++i)
        if (!s[i] || s[i]->host_only || !X_d[i] || !B_d[i]) {
            race_set_detail("race_batch_create: NULL or host-only entry " + std::to_string(i));
            return RACE_ERR_INVALID;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!st) {
        race_set_detail("race_batch_create: capture needs a non-default stream");
        return RACE_ERR_INVALID;
    }
    race_batch* b = new (std::nothrow) race_batch();
    if (!b) return RACE_ERR_NOMEM;
    b->count = count;
    b->k = k;
    // The matrices are independent: the graph runs them as kBranches parallel
    // branches (forked from and joined into `stream` by events), each matrix
    // on the branch with the least stored work so far, largest first.
    const int nb = std::min<int32_t>(kBranches, count);
    std::vector<cudaStream_t> br(static_cast<size_t>(nb), nullptr);
    std::vector<cudaEvent_t> ev(static_cast<size_t>(nb) + 1, nullptr);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < nb && e == cudaSuccess; ++j) e = cudaStreamCreateWithFlags(&br[j], cudaStreamNonBlocking);
    for (int j = 0; j <= nb && e == cudaSuccess; ++j) e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
    auto release = [&]() {
        for (cudaStream_t x : br)
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
    };
    if (e != cudaSuccess) {
        release();
        delete b;
        return cuda_err(e, "race_batch_create: streams");
    }
    std::vector<int32_t> order(static_cast<size_t>(count));
    for (int32_t i = 0; i < count; ++i) order[static_cast<size_t>(i)] = i;
    std::stable_sort(order.begin(), order.end(), [s](int32_t a, int32_t c) {
        return s[a]->h_col.size() > s[c]->h_col.size();
    });
    std::vector<int64_t> load(static_cast<size_t>(nb), 0);
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        release();
        delete b;
        return cuda_err(e, "cudaStreamBeginCapture");
    }
    int rc = RACE_OK;
    e = cudaEventRecord(ev[nb], st);
    for (int j = 0; j < nb && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(br[j], ev[nb], 0);
    if (e != cudaSuccess) rc = cuda_err(e, "race_batch_create: fork");
    for (int32_t i : order) {
        if (rc != RACE_OK) break;
        const int j = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        load[static_cast<size_t>(j)] += static_cast<int64_t>(s[i]->h_col.size());
        rc = run_one(s[i], k, X_d[i], B_d[i], br[j]);
    }
    for (int j = 0; j < nb && rc == RACE_OK; ++j) {
        e = cudaEventRecord(ev[j], br[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[j], 0);
        if (e != cudaSuccess) rc = cuda_err(e, "race_batch_create: join");
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    release();
    if (rc != RACE_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        delete b;
        return rc != RACE_OK ? rc : cuda_err(e, "cudaStreamEndCapture");
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        delete b;
        return cuda_err(e, "cudaGraphInstantiate");
    }
    *out = b;
    return RACE_OK;
}

int race_batch_launch(race_batch* b, void* stream) {
    if (!b || !b->exec) {
        race_set_detail("race_batch_launch: NULL batch");
        return RACE_ERR_INVALID;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RACE_OK : cuda_err(e, "cudaGraphLaunch");
}

void race_batch_free(race_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

int race_autotune(race_schedule* s, int32_t k, const double* X_d, double* B_d, int32_t reps, void* stream,
                  race_launch* best, float* best_us) {
    if (!s || !X_d || !B_d || k < 1 || k > 16 || reps < 1) {
        race_set_detail("race_autotune: bad argument");
        return RACE_ERR_INVALID;
    }
    if (s->host_only) {
        race_set_detail("race_autotune: host-only schedule");
        return RACE_ERR_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the executor with the transposed products off the FP64 pipe competes
    // when the matrix's values allow it
    const bool df = race_df64_prepare(s) == RACE_OK;
    std::vector<race_launch> cand;
    for (int bps : {0, 4, 6}) {
        if (k == 1) {
            if (bps != 6) {
                for (int g : {1, 2, 4}) cand.push_back({RACE_EXEC_ROWS_RED, g, 1, bps, 8, 0});
                for (int p : {4, 8}) cand.push_back({RACE_EXEC_PIPE_RED, 1, 1, bps, p, 0});
            }
            if (df)
                for (int g : {1, 2})
                    for (int q : {0, 1, 2})
                        for (int u : {4, 8}) cand.push_back({RACE_EXEC_DF64_RED, g, 1, bps, u, q});
        } else {
            if (bps != 6)
                for (int r : {1, 2, 4}) cand.push_back({RACE_EXEC_ROWS_RED, 1, r, bps, 8, 0});
            if (df)
                for (int r : {1, 2})
                    for (int q : {0, 1, 2}) cand.push_back({RACE_EXEC_DF64_RED, 1, r, bps, 4, q});
        }
    }
    const race_launch keep = s->launch;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RACE_ERR_CUDA;
    float best_t = 1e30f;
    race_launch best_l = keep;
    int rc = RACE_OK;
    for (const race_launch& l : cand) {
        s->launch = l;
        rc = run_one(s, k, X_d, B_d, st);  // warm-up
        if (rc != RACE_OK) break;
        cudaEventRecord(e0, st);
        for (int32_t r = 0; r < reps && rc == RACE_OK; ++r) rc = run_one(s, k, X_d, B_d, st);
        cudaEventRecord(e1, st);
        if (rc != RACE_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_err(e, "race_autotune");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = ms * 1000.f / reps;
        if (us < best_t) {
            best_t = us;
            best_l = l;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->launch = rc == RACE_OK ? best_l : keep;
    s->group_lanes = s->launch.group_lanes;
    if (best) *best = s->launch;
    if (best_us) *best_us = best_t;
    return rc;
}

}  // extern "C"
