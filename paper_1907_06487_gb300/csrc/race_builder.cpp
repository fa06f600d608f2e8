// RACE schedule construction on the host (paper Sec. 4 and 5).
//
// Steps, in the paper's order:
//   1. level construction by breadth-first search from a root (Alg.
//      "Construction of levels", Eq. "level"), levels stored consecutively;
//   2. distance-2 colouring by aggregating >= k adjacent levels into level
//      groups coloured red/blue alternately (Sec. 4.2, Eq. "corollary_dk");
//   3. epsilon-driven pairing of level groups with thread counts (Sec.
//      4.4.3 steps 1-3) and load balancing with worker weights (Alg. "Load
//      Balancing", Sec. 4.3 / 4.4.3 step 4);
//   4. recursion into groups that own more than one thread, on the group
//      plus its distance-1 halo (Sec. 4.4.2);
//   5. the tree's effective row counts and efficiency eta (Sec. 5), and a
//      flattening of the tree into globally synchronised phases for the GPU.
//
// Interpretation choices where the paper is silent or garbled:
//   - root = last vertex of the (sub)graph in its current order (with
//     RACE_FLAG_PSEUDO_PERIPHERAL, stage-0 roots move to a pseudo-peripheral
//     vertex of their component);
//   - islands restart from the last unvisited group vertex at level
//     (highest level reached so far) + 2;
//   - vertices of one level keep their current relative order;
//   - weight a = sum(size) * n_t(parent) / size(parent) as a single FP64
//     division of exact integers; b = max(1, round half away from zero);
//     eps = 1 - |a - b| must exceed eps_s strictly;
//   - after b is fixed a pair grows only while a' <= b, keeping the first
//     strictly best eps; when no further pair can be formed, fewer than 2k
//     levels would remain, or the threads are used up, the remaining levels
//     join the last pair, which receives every thread not yet assigned;
//   - a pair of n levels starts as floor(n/2) red levels and the rest blue;
//   - load balancing uses u_i = size_i / worker_i and the colour mean
//     sum(size) / sum(worker); the group visited at rank r is the r-th
//     entry of the |deviation| ranking;
//   - phases: red children first, blue children after the longest red
//     child; a node needs (max red phases) + (max blue phases).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "race_internal.h"
#include "race_plan_ops.h"

namespace race {
namespace {

struct Graph {
    std::vector<int64_t> off;
    std::vector<int32_t> nbr;
};

// Undirected adjacency without self loops.
Graph make_graph(int32_t n, const int32_t* rp, const int32_t* col) {
    Graph g;
    g.off.assign(static_cast<size_t>(n) + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t) {
            const int32_t c = col[t];
            if (c == r) continue;
            ++g.off[r + 1];
            ++g.off[c + 1];
        }
    std::partial_sum(g.off.begin(), g.off.end(), g.off.begin());
    g.nbr.resize(static_cast<size_t>(g.off[n]));
    std::vector<int64_t> cur(g.off.begin(), g.off.end() - 1);
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t) {
            const int32_t c = col[t];
            if (c == r) continue;
            g.nbr[cur[r]++] = c;
            g.nbr[cur[c]++] = r;
        }
    return g;
}

// George and Liu's pseudo-peripheral vertex of v's connected component
// (ACM TOMS 5, 1979): from the current start, take a vertex of minimum
// degree (lowest index on ties) among those farthest away; move there while
// its eccentricity is larger, stop at the first start that is not beaten.
class PeripheralFinder {
public:
    explicit PeripheralFinder(const Graph& g) : g_(g) {}

    int32_t find(int32_t v) {
        std::vector<int32_t> far, far_u;
        int32_t ecc = eccentricity(v, far);
        for (;;) {
            int32_t u = far[0];
            for (int32_t w : far) {
                const int64_t dw = degree(w), du = degree(u);
                if (dw < du || (dw == du && w < u)) u = w;
            }
            const int32_t ecc_u = eccentricity(u, far_u);
            if (ecc_u <= ecc) return v;
            v = u;
            ecc = ecc_u;
            far.swap(far_u);
        }
    }

    int64_t degree(int32_t v) const { return g_.off[v + 1] - g_.off[v]; }

private:
    // Eccentricity of v; `far` receives the vertices at that distance.
    int32_t eccentricity(int32_t v, std::vector<int32_t>& far) {
        if (mark_.empty()) mark_.assign(g_.off.size() - 1, 0);
        const uint32_t s = ++stamp_;
        std::vector<int32_t> front(1, v), next;
        mark_[static_cast<size_t>(v)] = s;
        int32_t ecc = 0;
        for (;;) {
            next.clear();
            for (int32_t u : front)
                for (int64_t e = g_.off[u]; e < g_.off[u + 1]; ++e) {
                    const int32_t w = g_.nbr[e];
                    if (mark_[static_cast<size_t>(w)] == s) continue;
                    mark_[static_cast<size_t>(w)] = s;
                    next.push_back(w);
                }
            if (next.empty()) break;
            front.swap(next);
            ++ecc;
        }
        far.swap(front);
        return ecc;
    }

    const Graph& g_;
    std::vector<uint32_t> mark_;
    uint32_t stamp_ = 0;
};

struct LevelSet {
    int32_t count = 0;
    std::vector<int64_t> weight;  // balancing unit per level
    std::vector<int32_t> rows;    // vertices per level
};

class Builder {
public:
    Builder(int32_t n, const int32_t* rp, const int32_t* col, const race_params& p, Plan& plan)
        : n_(n), p_(p), plan_(plan), g_(make_graph(n, rp, col)) {
        weight_.resize(n);
        for (int32_t v = 0; v < n; ++v)
            weight_[v] = (p.balance == RACE_BAL_NNZ) ? 1 + (g_.off[v + 1] - g_.off[v]) : 1;
        seq_.resize(n);
        std::iota(seq_.begin(), seq_.end(), 0);
        in_group_.assign(n, 0);
        in_halo_.assign(n, 0);
        seen_.assign(n, 0);
        depth_of_.assign(n, 0);
    }

    void run() {
        TreeNode root;
        root.stage = -1;
        root.lo = 0;
        root.hi = n_;
        root.n_threads = p_.n_workers;
        root.size = std::accumulate(weight_.begin(), weight_.end(), int64_t{0});
        plan_.nodes.clear();
        plan_.nodes.push_back(root);
        // depth-first over an explicit stack; children are processed in
        // level order (the result does not depend on the order)
        std::vector<int32_t> todo;
        if (p_.max_depth != 0) todo.push_back(0);
        bool first = true;
        while (!todo.empty()) {
            const int32_t id = todo.back();
            todo.pop_back();
            std::vector<int32_t> kids = split(id, first);
            first = false;
            for (auto it = kids.rbegin(); it != kids.rend(); ++it) {
                const TreeNode& k = plan_.nodes[*it];
                const bool may = p_.max_depth < 0 || k.stage + 1 < p_.max_depth;
                if (k.n_threads > 1 && may && k.hi > k.lo) todo.push_back(*it);
            }
        }
        plan_.perm = seq_;
        finish_tree();
    }

private:
    // Level construction for the group seq_[lo, hi) (Alg. "Construction of
    // levels"); the whole graph for the root, else group + distance-1 halo.
    LevelSet levels(int32_t lo, int32_t hi, bool whole) {
        ++stamp_;
        const uint32_t s = stamp_;
        for (int32_t q = lo; q < hi; ++q) in_group_[seq_[q]] = s;
        if (!whole) {
            for (int32_t q = lo; q < hi; ++q) {
                const int32_t v = seq_[q];
                in_halo_[v] = s;
                for (int64_t e = g_.off[v]; e < g_.off[v + 1]; ++e) in_halo_[g_.nbr[e]] = s;
            }
        }
        auto usable = [&](int32_t v) { return whole || in_halo_[v] == s; };
        int32_t left = hi - lo;   // group vertices not reached yet
        int32_t cursor = hi;      // scan position for the next root
        int32_t top = -1;         // highest level reached
        std::vector<int32_t> front, next;
        while (left > 0) {
            do { --cursor; } while (seen_[seq_[cursor]] == s);
            const int32_t root = (whole && (p_.flags & RACE_FLAG_PSEUDO_PERIPHERAL)) ? pp_.find(seq_[cursor])
                                                                                     : seq_[cursor];
            int32_t lev = top < 0 ? 0 : top + 2;
            seen_[root] = s;
            depth_of_[root] = lev;
            left -= (in_group_[root] == s);
            top = std::max(top, lev);
            front.assign(1, root);
            while (!front.empty()) {
                next.clear();
                for (int32_t u : front)
                    for (int64_t e = g_.off[u]; e < g_.off[u + 1]; ++e) {
                        const int32_t w = g_.nbr[e];
                        if (seen_[w] == s || !usable(w)) continue;
                        seen_[w] = s;
                        depth_of_[w] = lev + 1;
                        left -= (in_group_[w] == s);
                        next.push_back(w);
                    }
                if (!next.empty()) top = std::max(top, lev + 1);
                front.swap(next);
                ++lev;
            }
        }
        LevelSet ls;
        int32_t deepest = -1;
        for (int32_t q = lo; q < hi; ++q) deepest = std::max(deepest, depth_of_[seq_[q]]);
        ls.count = deepest + 1;
        ls.weight.assign(ls.count, 0);
        ls.rows.assign(ls.count, 0);
        for (int32_t q = lo; q < hi; ++q) {
            const int32_t v = seq_[q];
            ls.rows[depth_of_[v]] += 1;
            ls.weight[depth_of_[v]] += weight_[v];
        }
        // stable regrouping of seq_[lo, hi) by level
        std::vector<int32_t> slot(ls.count, 0);
        for (int32_t l = 1; l < ls.count; ++l) slot[l] = slot[l - 1] + ls.rows[l - 1];
        scratch_.resize(static_cast<size_t>(hi - lo));
        for (int32_t q = lo; q < hi; ++q) {
            const int32_t v = seq_[q];
            scratch_[slot[depth_of_[v]]++] = v;
        }
        std::copy(scratch_.begin(), scratch_.end(), seq_.begin() + lo);
        return ls;
    }

    struct Pair {
        int32_t first_level, end_level, threads;
    };

    // Sec. 4.4.3 steps 1-3: aggregate levels into pairs of level groups.
    std::vector<Pair> pair_levels(const LevelSet& ls, int32_t threads, double eps, int32_t k) const {
        const int64_t total = std::accumulate(ls.weight.begin(), ls.weight.end(), int64_t{0});
        auto share = [&](int64_t w) {
            return total > 0 ? static_cast<double>(w * static_cast<int64_t>(threads)) / static_cast<double>(total)
                             : 0.0;
        };
        std::vector<Pair> out;
        int32_t used = 0, at = 0;
        while (at < ls.count) {
            int64_t w = 0;
            int32_t stop = at;
            double target = 0.0, best = -1.0;
            bool ok = false;
            while (stop < ls.count && !ok) {
                w += ls.weight[stop++];
                const double a = share(w);
                target = std::max(1.0, std::round(a));
                best = 1.0 - std::fabs(a - target);
                ok = (stop - at >= 2 * k) && best > eps;
            }
            if (!ok) {
                if (out.empty()) {
                    out.push_back({at, ls.count, threads});
                } else {
                    used -= out.back().threads;
                    out.back().end_level = ls.count;
                    out.back().threads = threads - used;
                }
                return out;
            }
            int32_t pick = stop;
            for (int32_t e = stop; e < ls.count;) {
                w += ls.weight[e++];
                const double a = share(w);
                if (a > target) break;
                const double cand = 1.0 - std::fabs(a - target);
                if (cand > best) {
                    best = cand;
                    pick = e;
                }
            }
            const int32_t b = static_cast<int32_t>(target);
            if (ls.count - pick < 2 * k || used + b >= threads) {
                out.push_back({at, ls.count, threads - used});
                return out;
            }
            out.push_back({at, pick, b});
            used += b;
            at = pick;
        }
        return out;
    }

    // Alg. "Load Balancing" with worker weights over level groups ptr[].
    void balance(const LevelSet& ls, std::vector<int32_t>& ptr, const std::vector<int32_t>& worker, int32_t k) const {
        const int32_t len = static_cast<int32_t>(worker.size());
        std::vector<int64_t> prefix(ls.count + 1, 0);
        for (int32_t l = 0; l < ls.count; ++l) prefix[l + 1] = prefix[l] + ls.weight[l];
        int64_t wsum[2] = {0, 0};
        for (int32_t i = 0; i < len; ++i) wsum[i % 2] += worker[i];
        auto deviation = [&](const std::vector<int32_t>& tp, std::vector<double>& dev) {
            int64_t csum[2] = {0, 0};
            for (int32_t i = 0; i < len; ++i) csum[i % 2] += prefix[tp[i + 1]] - prefix[tp[i]];
            const double mean[2] = {wsum[0] ? static_cast<double>(csum[0]) / static_cast<double>(wsum[0]) : 0.0,
                                    wsum[1] ? static_cast<double>(csum[1]) / static_cast<double>(wsum[1]) : 0.0};
            double acc = 0.0;
            for (int32_t i = 0; i < len; ++i) {
                const double per = static_cast<double>(prefix[tp[i + 1]] - prefix[tp[i]]) /
                                   static_cast<double>(worker[i]);
                dev[i] = per - mean[i % 2];
                acc += dev[i] * dev[i];
            }
            return acc / static_cast<double>(len);
        };
        auto move_level = [](std::vector<int32_t>& tp, int32_t from, int32_t to) {
            if (from > to)
                for (int32_t j = to + 1; j <= from; ++j) ++tp[j];
            else
                for (int32_t j = from + 1; j <= to; ++j) --tp[j];
        };
        std::vector<double> dev(len), scratch(len);
        std::vector<int32_t> by_abs(len), by_signed(len), trial;
        for (;;) {
            const double var = deviation(ptr, dev);
            std::iota(by_abs.begin(), by_abs.end(), 0);
            std::stable_sort(by_abs.begin(), by_abs.end(),
                             [&](int32_t a, int32_t b) { return std::fabs(dev[a]) > std::fabs(dev[b]); });
            std::iota(by_signed.begin(), by_signed.end(), 0);
            std::stable_sort(by_signed.begin(), by_signed.end(), [&](int32_t a, int32_t b) { return dev[a] < dev[b]; });
            bool moved = false;
            for (int32_t r = 0; r < len && !moved; ++r) {
                const int32_t t = by_abs[r];
                trial = ptr;
                bool changed = false;
                if (dev[t] < 0.0) {
                    for (int32_t q = len - 1; q >= 0; --q) {
                        const int32_t donor = by_signed[q];
                        if (donor != t && trial[donor + 1] - trial[donor] > k) {
                            move_level(trial, donor, t);
                            changed = true;
                            break;
                        }
                    }
                } else if (trial[t + 1] - trial[t] > k && by_signed[0] != t) {
                    move_level(trial, t, by_signed[0]);
                    changed = true;
                }
                if (changed && deviation(trial, scratch) < var) {
                    ptr.swap(trial);
                    moved = true;
                }
            }
            if (!moved) return;
        }
    }

    // Split one node into its stage-(s+1) level groups; returns child ids.
    std::vector<int32_t> split(int32_t id, bool whole) {
        const int32_t lo = plan_.nodes[id].lo, hi = plan_.nodes[id].hi;
        const int32_t threads = plan_.nodes[id].n_threads;
        const int32_t stage = plan_.nodes[id].stage + 1;
        LevelSet ls = levels(lo, hi, whole);
        plan_.nodes[id].n_sub = ls.count;
        if (whole) plan_.n_levels = ls.count;
        // levels per group: k = 2 (Sec. 4.2); with RACE_FLAG_ONE_LEVEL_STAGE0
        // one level per stage-0 group (upper storage in level order: a row of
        // level j writes b only in levels j and j + 1, so same-colour groups
        // one level apart stay write-disjoint)
        const int32_t k = (whole && (p_.flags & RACE_FLAG_ONE_LEVEL_STAGE0)) ? 1 : p_.dist_k;
        if (ls.count < 2 * k) return {};
        const double eps = p_.eps[std::min(stage, 7)];
        const std::vector<Pair> pairs = pair_levels(ls, threads, eps, k);
        std::vector<int32_t> ptr;
        std::vector<int32_t> worker;
        for (const Pair& pr : pairs) {
            ptr.push_back(pr.first_level);
            ptr.push_back(pr.first_level + (pr.end_level - pr.first_level) / 2);
            worker.push_back(pr.threads);
            worker.push_back(pr.threads);
        }
        ptr.push_back(ls.count);
        balance(ls, ptr, worker, k);
        std::vector<int32_t> kids;
        int32_t row = lo, tid = plan_.nodes[id].thread_lo;
        for (size_t gi = 0; gi + 1 < ptr.size(); ++gi) {
            TreeNode c;
            c.stage = stage;
            c.color = static_cast<int32_t>(gi % 2);
            c.n_threads = worker[gi];
            c.thread_lo = tid;
            c.n_levels = ptr[gi + 1] - ptr[gi];
            int32_t rows = 0;
            for (int32_t l = ptr[gi]; l < ptr[gi + 1]; ++l) {
                rows += ls.rows[l];
                c.size += ls.weight[l];
            }
            c.lo = row;
            c.hi = row + rows;
            row += rows;
            if (c.color == 1) tid += c.n_threads;
            kids.push_back(static_cast<int32_t>(plan_.nodes.size()));
            plan_.nodes.push_back(std::move(c));
        }
        plan_.nodes[id].kids = kids;
        return kids;
    }

    // Effective row counts, phase counts and offsets; leaves per phase.
    void finish_tree() {
        std::vector<TreeNode>& nd = plan_.nodes;
        // children are always created after their parent: a reverse sweep
        // visits every child before its parent
        for (int32_t i = static_cast<int32_t>(nd.size()) - 1; i >= 0; --i) {
            if (nd[i].kids.empty()) {
                nd[i].neff = nd[i].size;
                nd[i].phase_count = 1;
                continue;
            }
            int64_t nr = 0, nb = 0;
            int32_t pr = 0, pb = 0;
            for (int32_t c : nd[i].kids) {
                if (nd[c].color == 0) {
                    nr = std::max(nr, nd[c].neff);
                    pr = std::max(pr, nd[c].phase_count);
                } else {
                    nb = std::max(nb, nd[c].neff);
                    pb = std::max(pb, nd[c].phase_count);
                }
            }
            nd[i].neff = nr + nb;
            nd[i].phase_count = pr + pb;
        }
        for (size_t i = 0; i < nd.size(); ++i) {
            if (nd[i].kids.empty()) continue;
            int32_t pr = 0;
            for (int32_t c : nd[i].kids)
                if (nd[c].color == 0) pr = std::max(pr, nd[c].phase_count);
            for (int32_t c : nd[i].kids) nd[c].phase_off = nd[i].phase_off + (nd[c].color == 0 ? 0 : pr);
        }
        const int32_t phases = nd[0].phase_count;
        std::vector<std::vector<std::pair<int32_t, int32_t>>> per(phases);
        for (const TreeNode& t : nd)
            if (t.kids.empty() && t.hi > t.lo) per[t.phase_off].push_back({t.lo, t.hi});
        plan_.stage_ptr.assign(1, 0);
        plan_.leaf_lo.clear();
        plan_.leaf_hi.clear();
        for (auto& v : per) {
            std::sort(v.begin(), v.end());
            for (auto& r : v) {
                plan_.leaf_lo.push_back(r.first);
                plan_.leaf_hi.push_back(r.second);
            }
            plan_.stage_ptr.push_back(static_cast<int32_t>(plan_.leaf_lo.size()));
        }
        plan_.eta = static_cast<double>(nd[0].size) /
                    (static_cast<double>(nd[0].neff) * static_cast<double>(plan_.n_workers));
    }

    int32_t n_;
    race_params p_;
    Plan& plan_;
    Graph g_;
    std::vector<int64_t> weight_;
    std::vector<int32_t> seq_;                       // position -> vertex
    std::vector<uint32_t> in_group_, in_halo_, seen_;
    std::vector<int32_t> depth_of_;
    std::vector<int32_t> scratch_;
    uint32_t stamp_ = 0;
    PeripheralFinder pp_{g_};
};

template <typename T>
void emit(std::vector<uint8_t>& o, T v) {
    uint8_t b[sizeof(T)];
    std::memcpy(b, &v, sizeof(T));
    o.insert(o.end(), b, b + sizeof(T));
}

void emit_node(const std::vector<TreeNode>& nd, int32_t i, std::vector<uint8_t>& o) {
    const TreeNode& t = nd[i];
    for (int32_t v : {t.stage, t.color, t.lo, t.hi, t.n_threads, t.thread_lo, t.n_levels, t.n_sub,
                      static_cast<int32_t>(t.kids.size()), t.phase_count, t.phase_off})
        emit<int32_t>(o, v);
    emit<int64_t>(o, t.size);
    emit<int64_t>(o, t.neff);
    for (int32_t c : t.kids) emit_node(nd, c, o);
}

}  // namespace

void build_plan(int32_t n, const int32_t* row_ptr, const int32_t* col, const race_params& p, Plan& out) {
    out = Plan();
    out.n = n;
    out.n_workers = p.n_workers;
    out.dist_k = p.dist_k;
    out.balance = p.balance;
    out.max_depth = p.max_depth;
    for (int i = 0; i < 8; ++i) out.eps[i] = p.eps[i];
    Builder b(n, row_ptr, col, p, out);
    b.run();
}

std::vector<int32_t> rcm_order(int32_t n, const int32_t* row_ptr, const int32_t* col) {
    const Graph g = make_graph(n, row_ptr, col);
    PeripheralFinder pf(g);
    std::vector<int32_t> cm;
    cm.reserve(static_cast<size_t>(n));
    std::vector<uint8_t> seen(static_cast<size_t>(n), 0);
    std::vector<int32_t> kids;
    for (int32_t v = 0; v < n; ++v) {
        if (seen[static_cast<size_t>(v)]) continue;
        // Cuthill-McKee from a pseudo-peripheral vertex of v's component:
        // breadth first, each vertex's newly reached neighbours appended by
        // increasing degree (lowest index on ties)
        const int32_t start = pf.find(v);
        size_t head = cm.size();
        cm.push_back(start);
        seen[static_cast<size_t>(start)] = 1;
        while (head < cm.size()) {
            const int32_t u = cm[head++];
            kids.clear();
            for (int64_t e = g.off[u]; e < g.off[u + 1]; ++e) {
                const int32_t w = g.nbr[e];
                if (seen[static_cast<size_t>(w)]) continue;
                seen[static_cast<size_t>(w)] = 1;
                kids.push_back(w);
            }
            std::sort(kids.begin(), kids.end(), [&](int32_t a, int32_t b) {
                const int64_t da = pf.degree(a), db = pf.degree(b);
                return da < db || (da == db && a < b);
            });
            cm.insert(cm.end(), kids.begin(), kids.end());
        }
    }
    std::reverse(cm.begin(), cm.end());
    return cm;
}

void natural_plan(int32_t n, const race_params& p, Plan& out) {
    out = Plan();
    out.n = n;
    out.n_workers = p.n_workers;
    out.dist_k = p.dist_k;
    out.balance = p.balance;
    out.max_depth = 0;
    for (int i = 0; i < 8; ++i) out.eps[i] = p.eps[i];
    out.perm.resize(static_cast<size_t>(n));
    for (int32_t i = 0; i < n; ++i) out.perm[static_cast<size_t>(i)] = i;
    TreeNode root;
    root.lo = 0;
    root.hi = n;
    root.n_threads = 1;
    root.size = n;
    root.neff = n;
    out.nodes.push_back(root);
    out.stage_ptr = {0};
    if (n > 0) {
        out.stage_ptr.push_back(1);
        out.leaf_lo = {0};
        out.leaf_hi = {n};
    }
    // one leaf holds every row: N_eff = n, eta = n / (N_eff * N_t)
    out.eta = p.n_workers > 0 ? 1.0 / p.n_workers : 1.0;
}

std::vector<uint8_t> export_plan(const Plan& plan) {
    std::vector<uint8_t> o;
    const int32_t phases = static_cast<int32_t>(plan.stage_ptr.size()) - 1;
    for (int32_t v : {0x45434152, 1, plan.n, plan.n_workers, plan.dist_k, plan.balance, plan.max_depth,
                      static_cast<int32_t>(plan.nodes.size()), phases,
                      static_cast<int32_t>(plan.leaf_lo.size()), 0, 0})
        emit<int32_t>(o, v);
    for (int i = 0; i < 8; ++i) emit<double>(o, plan.eps[i]);
    emit<double>(o, plan.eta);
    for (int32_t v : plan.perm) emit<int32_t>(o, v);
    for (int32_t v : plan.stage_ptr) emit<int32_t>(o, v);
    for (size_t i = 0; i < plan.leaf_lo.size(); ++i) {
        emit<int32_t>(o, plan.leaf_lo[i]);
        emit<int32_t>(o, plan.leaf_hi[i]);
    }
    emit_node(plan.nodes, 0, o);
    return o;
}

namespace {

// Bounds-checked little-endian reader over an export image.
struct Reader {
    const uint8_t* p;
    size_t left;
    template <typename T>
    bool get(T& v) {
        if (left < sizeof(T)) return false;
        std::memcpy(&v, p, sizeof(T));
        p += sizeof(T);
        left -= sizeof(T);
        return true;
    }
};

}  // namespace

bool import_plan(const void* buf, size_t size, int32_t n, Plan& out, std::string& why) {
    out = Plan();
    Reader rd{static_cast<const uint8_t*>(buf), size};
    int32_t h[12];
    for (int32_t& v : h)
        if (!rd.get(v)) return why = "image shorter than its header", false;
    if (h[0] != 0x45434152 || h[1] != 1) return why = "not a schedule image (magic or version)", false;
    if (h[2] != n) return why = "image was built for another number of rows", false;
    const int32_t n_nodes = h[7], n_phases = h[8], n_leaves = h[9];
    if (h[3] < 1 || h[4] != 2 || (h[5] != RACE_BAL_ROWS && h[5] != RACE_BAL_NNZ) || h[6] < -1 || n_nodes < 1 ||
        n_phases < 0 || n_leaves < 0 || h[10] != 0 || h[11] != 0)
        return why = "header field out of range", false;
    // the remaining size is fixed by the header's counts
    const uint64_t want = 8ull * 9 + 4ull * static_cast<uint64_t>(n) + 4ull * (static_cast<uint64_t>(n_phases) + 1) +
                          8ull * static_cast<uint64_t>(n_leaves) + static_cast<uint64_t>(n_nodes) * (11 * 4 + 2 * 8);
    if (rd.left != want) return why = "image size does not match its header", false;
    out.n = n;
    out.n_workers = h[3];
    out.dist_k = h[4];
    out.balance = h[5];
    out.max_depth = h[6];
    for (double& e : out.eps) rd.get(e);
    rd.get(out.eta);
    for (double e : out.eps)
        if (!(e >= 0.5 && e < 1.0)) return why = "eps_s outside [0.5, 1)", false;
    out.perm.resize(static_cast<size_t>(n));
    std::vector<uint8_t> hit(static_cast<size_t>(n), 0);
    for (int32_t& v : out.perm) {
        rd.get(v);
        if (v < 0 || v >= n || hit[static_cast<size_t>(v)]) return why = "perm is not a permutation", false;
        hit[static_cast<size_t>(v)] = 1;
    }
    out.stage_ptr.resize(static_cast<size_t>(n_phases) + 1);
    for (int32_t& v : out.stage_ptr) rd.get(v);
    if (out.stage_ptr.front() != 0 || out.stage_ptr.back() != n_leaves)
        return why = "phase offsets do not span the leaves", false;
    for (size_t q = 1; q < out.stage_ptr.size(); ++q)
        if (out.stage_ptr[q] < out.stage_ptr[q - 1]) return why = "phase offsets decrease", false;
    out.leaf_lo.resize(static_cast<size_t>(n_leaves));
    out.leaf_hi.resize(static_cast<size_t>(n_leaves));
    std::fill(hit.begin(), hit.end(), 0);
    for (int32_t q = 0; q < n_leaves; ++q) {
        int32_t lo, hi;
        rd.get(lo);
        rd.get(hi);
        if (lo < 0 || lo >= hi || hi > n) return why = "leaf row range out of bounds or empty", false;
        for (int32_t r = lo; r < hi; ++r) {
            if (hit[static_cast<size_t>(r)]) return why = "a row belongs to two leaves", false;
            hit[static_cast<size_t>(r)] = 1;
        }
        out.leaf_lo[static_cast<size_t>(q)] = lo;
        out.leaf_hi[static_cast<size_t>(q)] = hi;
    }
    for (uint8_t v : hit)
        if (!v) return why = "a row belongs to no leaf", false;
    // the tree in preorder; an explicit stack of (node, children still to read)
    out.nodes.resize(static_cast<size_t>(n_nodes));
    std::vector<std::pair<int32_t, int32_t>> open;
    for (int32_t id = 0; id < n_nodes; ++id) {
        if (id > 0 && open.empty()) return why = "tree has more than one root", false;
        TreeNode& t = out.nodes[static_cast<size_t>(id)];
        int32_t kids = 0;
        for (int32_t* f : {&t.stage, &t.color, &t.lo, &t.hi, &t.n_threads, &t.thread_lo, &t.n_levels, &t.n_sub, &kids,
                           &t.phase_count, &t.phase_off})
            rd.get(*f);
        rd.get(t.size);
        rd.get(t.neff);
        if (t.lo < 0 || t.lo > t.hi || t.hi > n || kids < 0 || kids > n_nodes - 1 - id || t.stage < -1 ||
            (t.color != 0 && t.color != 1) || t.n_threads < 1)
            return why = "tree node field out of range", false;
        if (!open.empty()) {
            out.nodes[static_cast<size_t>(open.back().first)].kids.push_back(id);
            if (--open.back().second == 0) open.pop_back();
        }
        if (kids > 0) open.emplace_back(id, kids);
    }
    if (!open.empty()) return why = "tree ends before its last child", false;
    out.n_levels = out.nodes[0].n_sub;
    return true;
}

}  // namespace race
