// schedule.cpp -- edge schedules (Sec. 6, Alg. 1): partitions of E into
// matchings, visited in order every iteration.
//
//  round robin   complete graphs: the circle method.  With m = n (n even) or
//                n + 1 (n odd, one dummy vertex), vertex m-1 stays fixed and
//                round r = 0..m-2 pairs (r, m-1) and ((r+k) mod (m-1),
//                (r-k) mod (m-1)) for k = 1..m/2-1; pairs with the dummy are
//                dropped.  n-1 perfect matchings for even n.
//  greedy colour edges in (u,v)-lexicographic order take the smallest colour
//                used at neither end; the colour classes, in colour order, are
//                the matchings (at most 2*maxdeg - 1 of them).
//  Alg. 1        repeat: scan the remaining edges in (u,v) order, keep every
//                edge whose ends are both still free (a maximal matching),
//                push it, remove it.
// Within a matching edges are listed in (u,v) order.
#include <algorithm>
#include <cstdint>
#include <unordered_set>
#include <vector>

#include "mplpp.h"
#include "host.h"

namespace mplpp {

namespace {

uint64_t key(int u, int v) { return (static_cast<uint64_t>(static_cast<uint32_t>(u)) << 32) | static_cast<uint32_t>(v); }

void emit(std::vector<std::vector<int>> &classes, const std::vector<int> &eu, const std::vector<int> &ev,
          std::vector<int> &off, std::vector<int> &order)
{
    off.assign(1, 0);
    order.clear();
    for (auto &c : classes) {
        std::sort(c.begin(), c.end(), [&](int a, int b) {
            return eu[a] != eu[b] ? eu[a] < eu[b] : ev[a] < ev[b];
        });
        for (int e : c) order.push_back(e);
        off.push_back(static_cast<int>(order.size()));
    }
}

std::vector<int> lex_order(const std::vector<int> &eu, const std::vector<int> &ev)
{
    std::vector<int> idx(eu.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = static_cast<int>(i);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return eu[a] != eu[b] ? eu[a] < eu[b] : ev[a] < ev[b]; });
    return idx;
}

}  // namespace

std::string check_graph(int n, const std::vector<int> &eu, const std::vector<int> &ev)
{
    if (n < 1) return "n_nodes must be >= 1";
    std::unordered_set<uint64_t> seen;
    seen.reserve(eu.size() * 2);
    for (size_t e = 0; e < eu.size(); ++e) {
        if (eu[e] < 0 || ev[e] >= n || eu[e] >= ev[e]) return "edge " + std::to_string(e) + " must satisfy 0 <= u < v < n";
        if (!seen.insert(key(eu[e], ev[e])).second) return "duplicate edge " + std::to_string(e);
    }
    return "";
}

std::string build_schedule(int kind, int n, const std::vector<int> &eu, const std::vector<int> &ev,
                           std::vector<int> &off, std::vector<int> &order)
{
    std::string err = check_graph(n, eu, ev);
    if (!err.empty()) return err;
    const int E = static_cast<int>(eu.size());
    std::vector<std::vector<int>> classes;
    if (kind == MPLPP_SCHED_ROUND_ROBIN) {
        if (static_cast<long long>(E) != static_cast<long long>(n) * (n - 1) / 2)
            return "round-robin schedule needs the complete graph";
        // every pair is present (no duplicates, E = n(n-1)/2): index them
        std::vector<int> id(static_cast<size_t>(n) * n, -1);
        for (int e = 0; e < E; ++e) id[static_cast<size_t>(eu[e]) * n + ev[e]] = e;
        const int m = (n % 2 == 0) ? n : n + 1;
        for (int r = 0; r < m - 1; ++r) {
            std::vector<int> c;
            auto add = [&](int a, int b) {
                if (a >= n || b >= n) return;
                const int u = std::min(a, b), v = std::max(a, b);
                c.push_back(id[static_cast<size_t>(u) * n + v]);
            };
            add(r, m - 1);
            for (int k = 1; k < m / 2; ++k) add((r + k) % (m - 1), ((r - k) % (m - 1) + (m - 1)) % (m - 1));
            if (!c.empty()) classes.push_back(std::move(c));
        }
    } else if (kind == MPLPP_SCHED_GREEDY_COLOR) {
        std::vector<std::vector<char>> used(n);
        for (int e : lex_order(eu, ev)) {
            auto &a = used[eu[e]];
            auto &b = used[ev[e]];
            size_t c = 0;
            while ((c < a.size() && a[c]) || (c < b.size() && b[c])) ++c;
            if (a.size() <= c) a.resize(c + 1, 0);
            if (b.size() <= c) b.resize(c + 1, 0);
            a[c] = b[c] = 1;
            if (classes.size() <= c) classes.resize(c + 1);
            classes[c].push_back(e);
        }
    } else if (kind == MPLPP_SCHED_ALG1) {
        std::vector<int> remaining = lex_order(eu, ev);
        std::vector<int> busy(n, -1);
        int round = 0;
        while (!remaining.empty()) {
            std::vector<int> c, rest;
            for (int e : remaining) {
                if (busy[eu[e]] == round || busy[ev[e]] == round) {
                    rest.push_back(e);
                } else {
                    busy[eu[e]] = busy[ev[e]] = round;
                    c.push_back(e);
                }
            }
            classes.push_back(std::move(c));
            remaining.swap(rest);
            ++round;
        }
    } else {
        return "unknown schedule kind";
    }
    emit(classes, eu, ev, off, order);
    return "";
}

std::string check_schedule(int n, const std::vector<int> &eu, const std::vector<int> &ev, const std::vector<int> &off,
                           const std::vector<int> &order)
{
    const int E = static_cast<int>(eu.size());
    if (off.empty() || off.front() != 0 || off.back() != E || static_cast<int>(order.size()) != E)
        return "schedule offsets must start at 0 and end at n_edges";
    std::vector<int> seen(E, 0), mark(n, -1);
    for (size_t k = 0; k + 1 < off.size(); ++k) {
        if (off[k + 1] < off[k]) return "schedule offsets must be non-decreasing";
        for (int i = off[k]; i < off[k + 1]; ++i) {
            const int e = order[i];
            if (e < 0 || e >= E) return "schedule edge id out of range";
            if (seen[e]++) return "edge " + std::to_string(e) + " appears twice in the schedule";
            if (mark[eu[e]] == static_cast<int>(k) || mark[ev[e]] == static_cast<int>(k))
                return "matching " + std::to_string(k) + " has two edges sharing a node";
            mark[eu[e]] = mark[ev[e]] = static_cast<int>(k);
        }
    }
    return "";
}

}  // namespace mplpp

extern "C" mplpp_status mplpp_schedule(int32_t kind, int32_t n_nodes, int32_t n_edges, const int32_t *edge_u,
                                       const int32_t *edge_v, int32_t *matching_off, int32_t *edge_order,
                                       int32_t *n_matchings)
{
    if (n_edges < 0 || (n_edges > 0 && (!edge_u || !edge_v || !edge_order)) || !matching_off || !n_matchings)
        return MPLPP_E_INVALID;
    std::vector<int> eu(edge_u, edge_u + n_edges), ev(edge_v, edge_v + n_edges), off, order;
    if (!mplpp::build_schedule(kind, n_nodes, eu, ev, off, order).empty()) return MPLPP_E_INVALID;
    for (size_t i = 0; i < off.size(); ++i) matching_off[i] = off[i];
    for (size_t i = 0; i < order.size(); ++i) edge_order[i] = order[i];
    *n_matchings = static_cast<int32_t>(off.size()) - 1;
    return MPLPP_OK;
}
