// Band-k ordering for k = 3 (rows, super-rows, super-super-rows): Sec. 2.2, Listing 2.
//
// The paper coarsens the matrix graph level by level, puts each coarse level in a
// weighted bandwidth-limiting order, expands the coarse nodes again reordering the
// vertices inside each one, and takes the coarse nodes as the super-rows (and
// super-super-rows).  It names neither the coarsening, nor the weights, nor the orders;
// the reading implemented here:
//   G0  graph of A + A^T without self-loops, edge weights 1.
//   CM  Cuthill-McKee sequence with the reverse-Cuthill-McKee start rules (least-degree
//       component start, George-Liu pseudo-peripheral search, at most 8 moves).
//   1   G0 -> G1: walk CM(G0); each unassigned vertex seeds an aggregate that grows one
//       vertex at a time by the adjacent unassigned vertex with the fewest unassigned
//       neighbours, then the largest edge weight into it, then the smallest index, up to
//       sr vertices.  G1 edge weight = number of G0 edges between two aggregates.
//   2   G1 -> G2 the same with CM(G1) and cap ssr (in G1 vertices).
//   3   order G2 by weighted reverse Cuthill-McKee (neighbours by weight descending,
//       degree, index; sequence reversed).
//   4/5 expand G2 -> G1 -> G0: the members of each coarse node, in coarse order, by a
//       breadth-first walk inside the node (neighbours by weight descending, degree,
//       index) from the member most connected to what is already placed; when nothing
//       placed touches the node, from the member farthest (inside the node) from the
//       members with edges leaving it (ties: smaller outside weight, then index), or,
//       with no edge leaving it, from its pseudo-peripheral vertex.
// The result: perm (perm[new] = old) and variable sr_ptr / ssr_ptr (sizes <= sr, ssr).
// Deterministic: every choice is keyed on integers.
#include <algorithm>
#include <cstdint>
#include <tuple>
#include <vector>

#include "csrk_internal.h"

namespace csrk {
namespace {

struct WGraph {
    std::vector<int64_t> start;   // n + 1
    std::vector<int32_t> nbr;     // ascending
    std::vector<int64_t> w;       // edge weights, parallel to nbr
    int32_t n() const { return (int32_t)start.size() - 1; }
    int32_t deg(int32_t v) const { return (int32_t)(start[v + 1] - start[v]); }
};

void graph_of(const CsrHost& a, WGraph& g) {
    const int32_t n = a.n;
    // A + A^T without the diagonal: rows merged with the transpose's rows
    std::vector<int64_t> tstart((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) tstart[a.colidx[p] + 1]++;
    for (int32_t i = 0; i < n; ++i) tstart[i + 1] += tstart[i];
    std::vector<int32_t> trow(tstart[n]);
    std::vector<int64_t> fill(tstart.begin(), tstart.end() - 1);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) trow[fill[a.colidx[p]]++] = i;
    g.start.assign((size_t)n + 1, 0);
    g.nbr.clear();
    std::vector<int32_t> merged;
    for (int32_t i = 0; i < n; ++i) {
        merged.clear();
        std::set_union(a.colidx.begin() + a.rowptr[i], a.colidx.begin() + a.rowptr[i + 1],
                       trow.begin() + tstart[i], trow.begin() + tstart[i + 1], std::back_inserter(merged));
        for (int32_t v : merged)
            if (v != i) g.nbr.push_back(v);
        g.start[i + 1] = (int64_t)g.nbr.size();
    }
    g.w.assign(g.nbr.size(), 1);
}

// Breadth-first level structure from root over vertices with !blocked[v]; returns the depth
// and leaves the reached vertices in `order` with the last level from last_at on.
template <typename Blocked>
int32_t levels(const WGraph& g, int32_t root, Blocked blocked, std::vector<int32_t>& tag, int32_t t,
               std::vector<int32_t>& order, size_t& last_at) {
    order.clear();
    order.push_back(root);
    tag[root] = t;
    size_t begin = 0;
    int32_t depth = 0;
    while (begin < order.size()) {
        const size_t end = order.size();
        last_at = begin;
        ++depth;
        for (size_t q = begin; q < end; ++q) {
            const int32_t v = order[q];
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                const int32_t u = g.nbr[e];
                if (!blocked(u) && tag[u] != t) {
                    tag[u] = t;
                    order.push_back(u);
                }
            }
        }
        begin = end;
    }
    return depth;
}

// George-Liu search from `root` with the least-(key, index) vertex of the last level.
template <typename Blocked, typename Key>
int32_t pseudo_peripheral(const WGraph& g, int32_t root, Blocked blocked, Key key, std::vector<int32_t>& tag,
                          int32_t& t, std::vector<int32_t>& l1, std::vector<int32_t>& l2) {
    size_t last = 0;
    int32_t depth = levels(g, root, blocked, tag, t++, l1, last);
    for (int moves = 0; moves < 8; ++moves) {
        int32_t c = -1;
        for (size_t q = last; q < l1.size(); ++q) {
            const int32_t v = l1[q];
            if (c < 0 || key(v) < key(c) || (key(v) == key(c) && v < c)) c = v;
        }
        size_t last2 = 0;
        const int32_t d2 = levels(g, c, blocked, tag, t++, l2, last2);
        if (d2 <= depth) break;
        root = c;
        depth = d2;
        l1.swap(l2);
        last = last2;
    }
    return root;
}

// Cuthill-McKee sequence over all components; weighted = neighbours by (weight desc,
// degree, index), else by (degree, index).
void cm_sequence(const WGraph& g, bool weighted, std::vector<int32_t>& seq) {
    const int32_t n = g.n();
    seq.clear();
    seq.reserve(n);
    if (n == 0) return;
    std::vector<int32_t> by_deg(n);
    for (int32_t v = 0; v < n; ++v) by_deg[v] = v;
    std::stable_sort(by_deg.begin(), by_deg.end(), [&](int32_t a, int32_t b) { return g.deg(a) < g.deg(b); });
    std::vector<uint8_t> visited(n, 0);
    std::vector<int32_t> tag(n, -1), l1, l2;
    int32_t t = 0;
    size_t cursor = 0;
    std::vector<std::tuple<int64_t, int32_t, int32_t>> kids;
    auto blocked = [&](int32_t u) { return visited[u] != 0; };
    auto degkey = [&](int32_t v) { return g.deg(v); };
    while ((int32_t)seq.size() < n) {
        while (visited[by_deg[cursor]]) ++cursor;
        const int32_t root = pseudo_peripheral(g, by_deg[cursor], blocked, degkey, tag, t, l1, l2);
        size_t head = seq.size();
        seq.push_back(root);
        visited[root] = 1;
        while (head < seq.size()) {
            const int32_t v = seq[head++];
            kids.clear();
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                const int32_t u = g.nbr[e];
                if (!visited[u]) kids.emplace_back(weighted ? -g.w[e] : 0, g.deg(u), u);
            }
            std::sort(kids.begin(), kids.end());
            for (auto& kd : kids) {
                visited[std::get<2>(kd)] = 1;
                seq.push_back(std::get<2>(kd));
            }
        }
    }
}

// Aggregates of at most cap vertices seeded in `seeds` order; each grows by the adjacent
// unassigned vertex with the fewest unassigned neighbours, then the largest edge weight
// into the aggregate, then the smallest index.
void aggregate(const WGraph& g, const std::vector<int32_t>& seeds, int32_t cap, std::vector<int32_t>& agg,
               std::vector<int64_t>& gstart, std::vector<int32_t>& gmem) {
    const int32_t n = g.n();
    agg.assign(n, -1);
    gstart.assign(1, 0);
    gmem.clear();
    gmem.reserve(n);
    std::vector<int32_t> free_nb(n);
    for (int32_t v = 0; v < n; ++v) free_nb[v] = g.deg(v);
    std::vector<int64_t> conn(n, 0);     // edge weight into the growing aggregate
    std::vector<int32_t> cand;           // unassigned vertices touching it (conn > 0)
    auto take = [&](int32_t v, int32_t id) {
        agg[v] = id;
        gmem.push_back(v);
        for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
            const int32_t u = g.nbr[e];
            free_nb[u]--;
            if (agg[u] < 0) {
                if (conn[u] == 0) cand.push_back(u);
                conn[u] += g.w[e];
            }
        }
    };
    for (int32_t s : seeds) {
        if (agg[s] >= 0) continue;
        const int32_t id = (int32_t)gstart.size() - 1;
        const size_t first = gmem.size();
        cand.clear();
        take(s, id);
        while ((int32_t)(gmem.size() - first) < cap) {
            int32_t best = -1;
            size_t bi = 0;
            for (size_t i = 0; i < cand.size(); ++i) {
                const int32_t u = cand[i];
                if (agg[u] >= 0) continue;   // taken since it entered the list
                if (best < 0 || free_nb[u] < free_nb[best] ||
                    (free_nb[u] == free_nb[best] && (conn[u] > conn[best] || (conn[u] == conn[best] && u < best)))) {
                    best = u;
                    bi = i;
                }
            }
            if (best < 0) break;
            cand[bi] = cand.back();
            cand.pop_back();
            take(best, id);
        }
        for (int32_t u : cand) conn[u] = 0;   // reset the scratch for the next aggregate
        gstart.push_back((int64_t)gmem.size());
    }
}

// The graph of the aggregates: edge weight = summed weights of the edges between them.
void coarse_graph(const WGraph& g, const std::vector<int32_t>& agg, const std::vector<int64_t>& gstart,
                  const std::vector<int32_t>& gmem, WGraph& c) {
    const int32_t ng = (int32_t)gstart.size() - 1;
    c.start.assign((size_t)ng + 1, 0);
    c.nbr.clear();
    c.w.clear();
    std::vector<int64_t> acc(ng, 0);
    std::vector<int32_t> touched;
    for (int32_t a = 0; a < ng; ++a) {
        touched.clear();
        for (int64_t q = gstart[a]; q < gstart[a + 1]; ++q) {
            const int32_t v = gmem[q];
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                const int32_t b = agg[g.nbr[e]];
                if (b == a) continue;
                if (acc[b] == 0) touched.push_back(b);
                acc[b] += g.w[e];
            }
        }
        std::sort(touched.begin(), touched.end());
        for (int32_t b : touched) {
            c.nbr.push_back(b);
            c.w.push_back(acc[b]);
            acc[b] = 0;
        }
        c.start[a + 1] = (int64_t)c.nbr.size();
    }
}

// Steps 4 / 5 for one coarse node: appends its members, in order, to `out`.
struct Expander {
    const WGraph& g;
    std::vector<uint8_t> placed;
    std::vector<int32_t> in_set;     // == id while v belongs to the current node
    std::vector<int32_t> remaining;  // == id while v is in the node and not yet placed
    std::vector<int32_t> tag, l1, l2, dist, cand, queue;
    int32_t t = 0;
    std::vector<std::tuple<int64_t, int32_t, int32_t>> kids;

    explicit Expander(const WGraph& gr)
        : g(gr), placed(gr.n(), 0), in_set(gr.n(), -1), remaining(gr.n(), -1), tag(gr.n(), -1),
          dist(gr.n(), -1) {}

    int32_t start_vertex(int32_t id) {
        // (a) most connected to placed vertices
        int32_t best = -1;
        int64_t best_w = 0;
        for (int32_t v : cand) {
            int64_t wp = 0;
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e)
                if (placed[g.nbr[e]]) wp += g.w[e];
            if (wp > best_w) {   // cand ascending: ties keep the smaller index
                best_w = wp;
                best = v;
            }
        }
        if (best >= 0) return best;
        // (b) farthest from the members with edges leaving the node
        queue.clear();
        std::vector<int64_t> outside(cand.size(), 0);
        for (size_t i = 0; i < cand.size(); ++i) {
            const int32_t v = cand[i];
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e)
                if (in_set[g.nbr[e]] != id) outside[i] += g.w[e];
            dist[v] = -1;
        }
        for (size_t i = 0; i < cand.size(); ++i)
            if (outside[i] > 0) {
                dist[cand[i]] = 0;
                queue.push_back(cand[i]);
            }
        if (!queue.empty()) {
            for (size_t head = 0; head < queue.size(); ++head) {
                const int32_t v = queue[head];
                for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                    const int32_t u = g.nbr[e];
                    if (remaining[u] == id && dist[u] < 0) {
                        dist[u] = dist[v] + 1;
                        queue.push_back(u);
                    }
                }
            }
            const int32_t far = (int32_t)cand.size() + 1;
            int32_t s = -1, sd = 0;
            int64_t so = 0;
            for (size_t i = 0; i < cand.size(); ++i) {
                const int32_t v = cand[i];
                const int32_t d = dist[v] < 0 ? far : dist[v];
                if (s < 0 || d > sd || (d == sd && outside[i] < so)) {
                    s = v;
                    sd = d;
                    so = outside[i];
                }
            }
            return s;
        }
        // (c) pseudo-peripheral vertex of the node's own edges
        auto blocked = [&](int32_t u) { return remaining[u] != id; };
        auto ideg = [&](int32_t v) {
            int32_t d = 0;
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) d += (remaining[g.nbr[e]] == id);
            return d;
        };
        int32_t root = cand[0];
        for (int32_t v : cand)
            if (ideg(v) < ideg(root)) root = v;
        return pseudo_peripheral(g, root, blocked, ideg, tag, t, l1, l2);
    }

    void expand(int32_t id, const int32_t* members, int64_t count, std::vector<int32_t>& out) {
        for (int64_t q = 0; q < count; ++q) {
            in_set[members[q]] = id;
            remaining[members[q]] = id;
        }
        int64_t left = count;
        while (left > 0) {
            cand.clear();
            for (int64_t q = 0; q < count; ++q)
                if (remaining[members[q]] == id) cand.push_back(members[q]);
            std::sort(cand.begin(), cand.end());
            const int32_t s = start_vertex(id);
            remaining[s] = -1;
            placed[s] = 1;
            out.push_back(s);
            --left;
            queue.clear();
            queue.push_back(s);
            for (size_t head = 0; head < queue.size(); ++head) {
                const int32_t v = queue[head];
                kids.clear();
                for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                    const int32_t u = g.nbr[e];
                    if (remaining[u] == id) kids.emplace_back(-g.w[e], g.deg(u), u);
                }
                std::sort(kids.begin(), kids.end());
                for (auto& kd : kids) {
                    const int32_t u = std::get<2>(kd);
                    remaining[u] = -1;
                    placed[u] = 1;
                    out.push_back(u);
                    queue.push_back(u);
                    --left;
                }
            }
        }
    }
};

}  // namespace

void bandk_permutation(const CsrHost& a, int32_t sr, int32_t ssr, std::vector<int32_t>& perm,
                       std::vector<int32_t>& sr_ptr, std::vector<int32_t>& ssr_ptr) {
    const int32_t n = a.n;
    perm.clear();
    sr_ptr.assign(1, 0);
    ssr_ptr.assign(1, 0);
    if (n == 0) return;
    WGraph g0, g1, g2;
    graph_of(a, g0);
    std::vector<int32_t> seq, agg1, agg2, gmem1, gmem2;
    std::vector<int64_t> gs1, gs2;
    cm_sequence(g0, false, seq);
    aggregate(g0, seq, sr, agg1, gs1, gmem1);
    coarse_graph(g0, agg1, gs1, gmem1, g1);
    cm_sequence(g1, false, seq);
    aggregate(g1, seq, ssr, agg2, gs2, gmem2);
    coarse_graph(g1, agg2, gs2, gmem2, g2);
    std::vector<int32_t> order2;
    cm_sequence(g2, true, order2);
    std::reverse(order2.begin(), order2.end());
    // expand G2 -> G1: each aggregate's members sorted ascending first (the walk is keyed
    // on indices, so the stored member order does not matter)
    std::vector<int32_t> order1;
    order1.reserve(g1.n());
    {
        Expander ex(g1);
        std::vector<int32_t> mem;
        for (int32_t b : order2) {
            mem.assign(gmem2.begin() + gs2[b], gmem2.begin() + gs2[b + 1]);
            const size_t before = order1.size();
            ex.expand(b, mem.data(), (int64_t)mem.size(), order1);
            ssr_ptr.push_back(ssr_ptr.back() + (int32_t)(order1.size() - before));
        }
    }
    perm.reserve(n);
    {
        Expander ex(g0);
        for (int32_t c : order1) {
            const size_t before = perm.size();
            ex.expand(c, gmem1.data() + gs1[c], gs1[c + 1] - gs1[c], perm);
            sr_ptr.push_back(sr_ptr.back() + (int32_t)(perm.size() - before));
        }
    }
}

}  // namespace csrk
