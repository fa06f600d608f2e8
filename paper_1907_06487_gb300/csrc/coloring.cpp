// Multicolouring schedules, the comparison methods of the paper (Sec. 3.3 and
// Sec. 6.3): plain multicolouring (MC) and algebraic block multicolouring
// (ABMC).  Written from the paper's description, not from COLPACK or METIS:
//   MC    every row is a unit; units are coloured so that no two rows of one
//         colour lie within distance 2 of each other in the symmetric graph
//         (the distance-2 condition SymmSpMV's writes need, Sec. 4.2);
//   ABMC  the matrix is first cut into blocks of block_rows consecutive rows
//         (the partitioning step; the paper uses METIS, here the blocks
//         follow the given, typically RCM, order), then the blocks are
//         coloured so that no two rows of different blocks of one colour lie
//         within distance 2.
// The colouring is first fit in unit order: unit u takes the smallest colour
// that no earlier unit within distance 2 of it holds.  The permutation lists
// the units colour by colour (units in index order, rows in order inside a
// unit); each colour is one phase and each unit one leaf, so every executor
// runs these schedules unchanged (the leaf executors phase by phase, the
// row-parallel ones on the permuted matrix).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "race_internal.h"

namespace race {

void coloring_plan(int32_t n, const int32_t* rp, const int32_t* col, int32_t method, int32_t block_rows,
                   const race_params& p, Plan& out) {
    out = Plan();
    out.n = n;
    out.n_workers = p.n_workers;
    out.dist_k = 2;
    out.balance = p.balance;
    out.max_depth = 0;
    for (int i = 0; i < 8; ++i) out.eps[i] = p.eps[i];
    const int32_t bs = method == RACE_COLOR_MC ? 1 : block_rows;
    const int32_t units = n > 0 ? (n + bs - 1) / bs : 0;
    // symmetric adjacency without self-loops
    std::vector<int64_t> aptr(static_cast<size_t>(n) + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t)
            if (col[t] != r) {
                ++aptr[static_cast<size_t>(r) + 1];
                ++aptr[static_cast<size_t>(col[t]) + 1];
            }
    for (int32_t r = 0; r < n; ++r) aptr[static_cast<size_t>(r) + 1] += aptr[static_cast<size_t>(r)];
    std::vector<int32_t> adj(static_cast<size_t>(aptr[static_cast<size_t>(n)]));
    {
        std::vector<int64_t> fill(aptr.begin(), aptr.end() - 1);
        for (int32_t r = 0; r < n; ++r)
            for (int32_t t = rp[r]; t < rp[r + 1]; ++t)
                if (col[t] != r) {
                    adj[static_cast<size_t>(fill[static_cast<size_t>(r)]++)] = col[t];
                    adj[static_cast<size_t>(fill[static_cast<size_t>(col[t])]++)] = r;
                }
    }
    // first-fit colouring of the units; mark[c] == u: colour c is taken near unit u
    std::vector<int32_t> color(static_cast<size_t>(units), -1), mark;
    int32_t ncol = 0;
    auto note = [&](int32_t v, int32_t u) {
        const int32_t c = color[static_cast<size_t>(v / bs)];
        if (c >= 0) mark[static_cast<size_t>(c)] = u;
    };
    for (int32_t u = 0; u < units; ++u) {
        const int32_t r0 = u * bs, r1 = std::min(n, r0 + bs);
        for (int32_t r = r0; r < r1; ++r) {
            note(r, u);
            for (int64_t a = aptr[static_cast<size_t>(r)]; a < aptr[static_cast<size_t>(r) + 1]; ++a) {
                const int32_t w = adj[static_cast<size_t>(a)];
                note(w, u);
                for (int64_t b = aptr[static_cast<size_t>(w)]; b < aptr[static_cast<size_t>(w) + 1]; ++b)
                    note(adj[static_cast<size_t>(b)], u);
            }
        }
        int32_t c = 0;
        while (c < ncol && mark[static_cast<size_t>(c)] == u) ++c;
        if (c == ncol) {
            ++ncol;
            mark.push_back(-1);
        }
        color[static_cast<size_t>(u)] = c;
    }
    // units colour by colour; one phase per colour, one leaf per unit
    std::vector<int32_t> count(static_cast<size_t>(ncol) + 1, 0);
    for (int32_t u = 0; u < units; ++u) ++count[static_cast<size_t>(color[static_cast<size_t>(u)]) + 1];
    for (int32_t c = 0; c < ncol; ++c) count[static_cast<size_t>(c) + 1] += count[static_cast<size_t>(c)];
    std::vector<int32_t> order(static_cast<size_t>(units));
    {
        std::vector<int32_t> fill(count.begin(), count.end() - 1);
        for (int32_t u = 0; u < units; ++u) order[static_cast<size_t>(fill[static_cast<size_t>(color[static_cast<size_t>(u)])]++)] = u;
    }
    out.perm.reserve(static_cast<size_t>(n));
    out.stage_ptr.assign(count.begin(), count.end());
    int64_t neff = 0;
    for (int32_t c = 0; c < ncol; ++c) {
        int32_t longest = 0;
        for (int32_t q = count[static_cast<size_t>(c)]; q < count[static_cast<size_t>(c) + 1]; ++q) {
            const int32_t u = order[static_cast<size_t>(q)];
            const int32_t r0 = u * bs, r1 = std::min(n, r0 + bs);
            out.leaf_lo.push_back(static_cast<int32_t>(out.perm.size()));
            for (int32_t r = r0; r < r1; ++r) out.perm.push_back(r);
            out.leaf_hi.push_back(static_cast<int32_t>(out.perm.size()));
            longest = std::max(longest, r1 - r0);
        }
        neff += longest;  // the longest leaf of each phase lies on the critical path
    }
    TreeNode root;
    root.lo = 0;
    root.hi = n;
    root.n_threads = std::max(1, p.n_workers);
    root.size = n;
    root.neff = neff;
    out.nodes.push_back(root);
    out.eta = neff > 0 ? std::min(1.0, static_cast<double>(n) / (static_cast<double>(neff) * root.n_threads)) : 1.0;
}

}  // namespace race
