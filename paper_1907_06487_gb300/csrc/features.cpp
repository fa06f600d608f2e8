// Matrix features for the RACE-parameter predictor (host, O(nnz)).
//
// The epsilon parameters act on the level structure of the graph (Sec.
// 4.4.3, Sec. 5.1), so most features describe the BFS levels from the root
// the schedule uses (the last vertex; islands restart from the last
// unvisited vertex two levels further on):
//   0 log10 n                       8  coefficient of variation of level sizes
//   1 log10 nnz (full)              9  index of the largest level / N_l
//   2 mean row length (full)       10  log10(1 + number of islands)
//   3 CV of row length             11  fraction of edges inside one level
//   4 max / mean row length        12  bandwidth of the level order / n
//   5 log10 N_l                    13  sum |s_{i+1} - s_i| / n over levels
//   6 log10 (n / N_l)              14  share of rows in the 10 % largest levels
//   7 largest level / n            15  log10 (nnz / N_l)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "race_internal.h"

extern "C" int race_features(const race_csr_upper* a, float* feat) {
    if (!a || !feat || a->n <= 0 || !a->row_ptr || (a->nnz > 0 && !a->col)) {
        race_set_detail("race_features: bad argument");
        return RACE_ERR_INVALID;
    }
    const int32_t n = a->n;
    std::vector<int64_t> off(static_cast<size_t>(n) + 1, 0);
    for (int32_t r = 0; r < n; ++r)
        for (int64_t t = a->row_ptr[r]; t < a->row_ptr[r + 1]; ++t) {
            const int32_t c = a->col[t];
            if (c < r || c >= n) {
                race_set_detail("race_features: not an upper-triangle CRS");
                return RACE_ERR_INVALID;
            }
            if (c == r) continue;
            ++off[r + 1];
            ++off[c + 1];
        }
    std::partial_sum(off.begin(), off.end(), off.begin());
    std::vector<int32_t> nbr(static_cast<size_t>(off[n]));
    {
        std::vector<int64_t> cur(off.begin(), off.end() - 1);
        for (int32_t r = 0; r < n; ++r)
            for (int64_t t = a->row_ptr[r]; t < a->row_ptr[r + 1]; ++t) {
                const int32_t c = a->col[t];
                if (c == r) continue;
                nbr[cur[r]++] = c;
                nbr[cur[c]++] = r;
            }
    }
    // row lengths of the full matrix (degree + diagonal)
    double sum = 0, sum2 = 0, mx = 0;
    for (int32_t r = 0; r < n; ++r) {
        const double len = static_cast<double>(off[r + 1] - off[r] + 1);
        sum += len;
        sum2 += len * len;
        mx = std::max(mx, len);
    }
    const double mean = sum / n;
    const double cv = std::sqrt(std::max(0.0, sum2 / n - mean * mean)) / mean;
    // levels
    std::vector<int32_t> lev(n, -1), front, next;
    int32_t top = -1, islands = 0, scan = n - 1;
    int64_t visited = 0;
    while (visited < n) {
        while (lev[scan] >= 0) --scan;
        const int32_t l0 = top < 0 ? 0 : top + 2;
        ++islands;
        lev[scan] = l0;
        ++visited;
        top = std::max(top, l0);
        front.assign(1, scan);
        int32_t l = l0;
        while (!front.empty()) {
            next.clear();
            for (int32_t u : front)
                for (int64_t e = off[u]; e < off[u + 1]; ++e)
                    if (lev[nbr[e]] < 0) {
                        lev[nbr[e]] = l + 1;
                        next.push_back(nbr[e]);
                    }
            visited += static_cast<int64_t>(next.size());
            if (!next.empty()) top = std::max(top, l + 1);
            front.swap(next);
            ++l;
        }
    }
    const int32_t nl = top + 1;
    std::vector<double> sz(nl, 0.0);
    for (int32_t v = 0; v < n; ++v) sz[lev[v]] += 1.0;
    std::vector<double> nonempty;
    for (double s : sz)
        if (s > 0) nonempty.push_back(s);
    const double lmean = static_cast<double>(n) / nonempty.size();
    double lvar = 0, lmax = 0, growth = 0;
    int32_t argmax = 0;
    for (int32_t i = 0; i < nl; ++i) {
        if (sz[i] > lmax) {
            lmax = sz[i];
            argmax = i;
        }
        if (i + 1 < nl) growth += std::fabs(sz[i + 1] - sz[i]);
    }
    for (double s : nonempty) lvar += (s - lmean) * (s - lmean);
    lvar /= nonempty.size();
    std::vector<double> sorted = nonempty;
    std::sort(sorted.rbegin(), sorted.rend());
    const size_t top10 = std::max<size_t>(1, sorted.size() / 10);
    double share = 0;
    for (size_t i = 0; i < top10; ++i) share += sorted[i];
    // positions in level order (stable by index) for the bandwidth
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return lev[x] < lev[y]; });
    std::vector<int32_t> posn(n);
    for (int32_t q = 0; q < n; ++q) posn[order[q]] = q;
    int64_t same = 0, edges = 0, bw = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
            const int32_t v = nbr[e];
            if (v < u) continue;
            ++edges;
            if (lev[u] == lev[v]) ++same;
            bw = std::max<int64_t>(bw, std::abs(static_cast<int64_t>(posn[u]) - posn[v]));
        }
    const double nnz_full = static_cast<double>(off[n] + n);
    float f[16];
    f[0] = static_cast<float>(std::log10(static_cast<double>(n)));
    f[1] = static_cast<float>(std::log10(nnz_full));
    f[2] = static_cast<float>(mean);
    f[3] = static_cast<float>(cv);
    f[4] = static_cast<float>(mx / mean);
    f[5] = static_cast<float>(std::log10(static_cast<double>(nl)));
    f[6] = static_cast<float>(std::log10(static_cast<double>(n) / nl));
    f[7] = static_cast<float>(lmax / n);
    f[8] = static_cast<float>(std::sqrt(lvar) / lmean);
    f[9] = static_cast<float>(static_cast<double>(argmax) / nl);
    f[10] = static_cast<float>(std::log10(1.0 + islands));
    f[11] = static_cast<float>(edges ? static_cast<double>(same) / edges : 0.0);
    f[12] = static_cast<float>(static_cast<double>(bw) / n);
    f[13] = static_cast<float>(growth / n);
    f[14] = static_cast<float>(share / n);
    f[15] = static_cast<float>(std::log10(nnz_full / nl));
    std::memcpy(feat, f, sizeof(f));
    return RACE_OK;
}
