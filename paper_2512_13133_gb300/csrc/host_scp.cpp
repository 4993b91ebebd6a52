// a11 (host): surprisal-based lazy-greedy set cover (Sec. 3.3, Eqs. 7-9) and
// the coarse-to-fine closed loop (Sec. 3.1, stages 2-4).  Plain host C++ that
// consumes the pass lists produced on the GPU.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <vector>

#include "pcl.h"

namespace {

struct Graph {
    std::vector<uint64_t> off;
    std::vector<uint32_t> adj;
};

// undirected CSR with duplicate edges and self loops removed
bool build_graph(const pcl_pair *e, uint64_t m, uint32_t n, Graph &g) {
    std::vector<uint64_t> deg(n + 1, 0);
    for (uint64_t i = 0; i < m; ++i) {
        if (e[i].a >= n || e[i].b >= n) return false;
        if (e[i].a == e[i].b) continue;
        ++deg[e[i].a];
        ++deg[e[i].b];
    }
    g.off.assign(n + 1, 0);
    for (uint32_t i = 0; i < n; ++i) g.off[i + 1] = g.off[i] + deg[i];
    g.adj.assign(g.off[n], 0);
    std::vector<uint64_t> pos(g.off.begin(), g.off.end() - 1);
    for (uint64_t i = 0; i < m; ++i) {
        if (e[i].a == e[i].b) continue;
        g.adj[pos[e[i].a]++] = e[i].b;
        g.adj[pos[e[i].b]++] = e[i].a;
    }
    // sort + unique each list, compact
    std::vector<uint64_t> noff(n + 1, 0);
    uint64_t w = 0;
    for (uint32_t i = 0; i < n; ++i) {
        auto b = g.adj.begin() + (int64_t)g.off[i], en = g.adj.begin() + (int64_t)g.off[i + 1];
        std::sort(b, en);
        auto u = std::unique(b, en);
        noff[i] = w;
        for (auto it = b; it != u; ++it) g.adj[w++] = *it;
    }
    noff[n] = w;
    g.adj.resize(w);
    g.off.swap(noff);
    return true;
}

// lazy greedy over graph g; fills rep_of (UINT32_MAX if never covered, which
// cannot happen) and the selection order
void lazy_greedy(const Graph &g, uint32_t n, std::vector<uint32_t> &rep_of, std::vector<uint32_t> &order) {
    // S_i = floor(2^32 / f_i), f_i = 1 + |neighbours(i)| (Eqs. 7-8, fixed point)
    std::vector<uint64_t> w(n);
    for (uint32_t i = 0; i < n; ++i) w[i] = (1ull << 32) / (1ull + (g.off[i + 1] - g.off[i]));
    std::vector<uint8_t> unc(n, 1);
    rep_of.assign(n, UINT32_MAX);
    order.clear();
    // key: (score, -index) -- larger first
    using Key = std::pair<uint64_t, int64_t>;
    std::priority_queue<Key> heap;
    auto gain = [&](uint32_t j) {
        uint64_t s = w[j];  // j is uncovered whenever it is evaluated
        for (uint64_t t = g.off[j]; t < g.off[j + 1]; ++t)
            if (unc[g.adj[t]]) s += w[g.adj[t]];
        return s;
    };
    for (uint32_t j = 0; j < n; ++j) heap.push(Key(gain(j), -(int64_t)j));
    uint32_t left = n;
    while (left && !heap.empty()) {
        const Key top = heap.top();
        heap.pop();
        const uint32_t j = (uint32_t)(-top.second);
        if (!unc[j]) continue;  // covered meanwhile: no longer a candidate
        const uint64_t gj = gain(j);
        bool take = (gj == top.first);
        if (!take) {
            while (!heap.empty() && !unc[(uint32_t)(-heap.top().second)]) heap.pop();
            // stored scores bound the true gains from above (submodularity),
            // so beating the best stored key beats every true key
            take = heap.empty() || Key(gj, -(int64_t)j) >= heap.top();
            if (!take) heap.push(Key(gj, -(int64_t)j));
        }
        if (!take) continue;
        order.push_back(j);
        if (unc[j]) { unc[j] = 0; rep_of[j] = j; --left; }
        for (uint64_t t = g.off[j]; t < g.off[j + 1]; ++t) {
            const uint32_t k = g.adj[t];
            if (unc[k]) { unc[k] = 0; rep_of[k] = j; --left; }
        }
    }
}

}  // namespace

extern "C" {

pcl_status pcl_setcover(const pcl_pair *h_edges, uint64_t n_edges, uint32_t n_nodes, uint32_t *h_rep_of,
                        uint32_t *h_order, uint32_t *n_selected) {
    if ((n_edges && !h_edges) || (n_nodes && (!h_rep_of || !h_order)) || !n_selected) return PCL_ERR_INVALID;
    Graph g;
    if (!build_graph(h_edges, n_edges, n_nodes, g)) return PCL_ERR_INVALID;
    std::vector<uint32_t> rep, order;
    lazy_greedy(g, n_nodes, rep, order);
    std::copy(rep.begin(), rep.end(), h_rep_of);
    std::copy(order.begin(), order.end(), h_order);
    *n_selected = (uint32_t)order.size();
    return PCL_OK;
}

pcl_status pcl_cluster_loop(const pcl_pair *h_pairs, const uint8_t *h_strict, const uint8_t *h_relaxed, uint64_t m,
                            uint32_t n, uint32_t *h_rep_of, uint32_t *n_clusters, uint32_t *n_rounds) {
    if ((m && (!h_pairs || !h_strict || !h_relaxed)) || (n && !h_rep_of) || !n_clusters || !n_rounds)
        return PCL_ERR_INVALID;
    for (uint64_t i = 0; i < m; ++i)
        if (h_pairs[i].a >= n || h_pairs[i].b >= n) return PCL_ERR_INVALID;
    // strict-pass adjacency (for orphans)
    std::vector<pcl_pair> strict_edges;
    for (uint64_t i = 0; i < m; ++i)
        if (h_strict[i]) strict_edges.push_back(h_pairs[i]);
    Graph sg;
    build_graph(strict_edges.data(), strict_edges.size(), n, sg);
    auto strict_ok = [&](uint32_t a, uint32_t b) {
        return std::binary_search(sg.adj.begin() + (int64_t)sg.off[a], sg.adj.begin() + (int64_t)sg.off[a + 1], b);
    };
    std::vector<uint32_t> rep_of(n, UINT32_MAX);
    std::vector<uint8_t> is_rep(n, 0);
    std::vector<uint32_t> remaining(n);
    for (uint32_t i = 0; i < n; ++i) remaining[i] = i;
    std::vector<uint32_t> loc(n, UINT32_MAX);
    uint32_t rounds = 0, clusters = 0;
    while (!remaining.empty()) {
        ++rounds;
        for (uint32_t t = 0; t < remaining.size(); ++t) loc[remaining[t]] = t;
        std::vector<pcl_pair> sub;
        for (uint64_t i = 0; i < m; ++i) {
            if (!h_relaxed[i]) continue;
            const uint32_t a = loc[h_pairs[i].a], b = loc[h_pairs[i].b];
            if (a != UINT32_MAX && b != UINT32_MAX) sub.push_back(pcl_pair{a, b});
        }
        const uint32_t nr = (uint32_t)remaining.size();
        Graph g;
        build_graph(sub.data(), sub.size(), nr, g);
        std::vector<uint32_t> rep_local, order;
        lazy_greedy(g, nr, rep_local, order);
        if (order.empty()) break;  // cannot happen for a non-empty set
        for (uint32_t j : order) {
            const uint32_t gj = remaining[j];
            rep_of[gj] = gj;
            is_rep[gj] = 1;
            ++clusters;
        }
        std::vector<uint32_t> orphans;
        for (uint32_t k = 0; k < nr; ++k) {
            const uint32_t r = rep_local[k];
            if (r == k) continue;
            const uint32_t gk = remaining[k], gr = remaining[r];
            if (strict_ok(gr, gk)) rep_of[gk] = gr;
            else orphans.push_back(gk);
        }
        for (uint32_t t = 0; t < nr; ++t) loc[remaining[t]] = UINT32_MAX;
        // orphans: the lowest-index representative so far that passes strictly
        std::sort(orphans.begin(), orphans.end());
        std::vector<uint32_t> next;
        for (uint32_t k : orphans) {
            uint32_t best = UINT32_MAX;
            for (uint64_t t = sg.off[k]; t < sg.off[k + 1]; ++t) {
                const uint32_t r = sg.adj[t];
                if (is_rep[r] && r < best) best = r;
            }
            if (best != UINT32_MAX) rep_of[k] = best;
            else next.push_back(k);
        }
        remaining.swap(next);
    }
    std::copy(rep_of.begin(), rep_of.end(), h_rep_of);
    *n_clusters = clusters;
    *n_rounds = rounds;
    return remaining.empty() ? PCL_OK : PCL_ERR_INVALID;
}

}  // extern "C"
