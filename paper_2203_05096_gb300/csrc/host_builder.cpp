// Host-side CSR-k builder: validation, reverse Cuthill-McKee, symmetric permutation,
// super-row / super-super-row pointers (Sec. 2.2), per-SSR descriptors, and FP64 ->
// FP32 / BF16 narrowing.  Everything here is integer or bit-exact work: the same inputs
// give the same arrays on every host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "csrk_internal.h"

namespace csrk {

// ---------------------------------------------------------------- threading helper
void parallel_for(int64_t n, int64_t grain, void (*fn)(int64_t, int64_t, void*), void* ctx) {
    unsigned hw = std::thread::hardware_concurrency();
    int64_t nthreads = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 1, 32));
    nthreads = std::min<int64_t>(nthreads, (n + grain - 1) / std::max<int64_t>(grain, 1));
    if (nthreads <= 1) {
        if (n > 0) fn(0, n, ctx);
        return;
    }
    std::vector<std::thread> pool;
    int64_t chunk = (n + nthreads - 1) / nthreads;
    for (int64_t t = 0; t < nthreads; ++t) {
        int64_t b = t * chunk, e = std::min(n, b + chunk);
        if (b >= e) break;
        pool.emplace_back([=] { fn(b, e, ctx); });
    }
    for (auto& th : pool) th.join();
}

// As parallel_for, but every range except the last is a whole number of `grain` items and
// starts at a multiple of it (callers index per-range results by start / grain).
static void parallel_for_ranges(int64_t n, int64_t grain, void (*fn)(int64_t, int64_t, void*), void* ctx) {
    if (n <= 0) return;
    const int64_t blocks = (n + grain - 1) / grain;
    unsigned hw = std::thread::hardware_concurrency();
    const int64_t nthreads = std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 32, blocks}));
    if (nthreads <= 1) {
        for (int64_t b = 0; b < n; b += grain) fn(b, std::min(n, b + grain), ctx);
        return;
    }
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < nthreads; ++t)
        pool.emplace_back([=] {
            for (int64_t k = t; k < blocks; k += nthreads) fn(k * grain, std::min(n, (k + 1) * grain), ctx);
        });
    for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------- ingest
int ingest_csr(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
               CsrHost& out, std::string& err) {
    if (n < 0) { err = "n must be >= 0"; return CSRK_ERR_ARG; }
    if (!rowptr) { err = "rowptr is NULL"; return CSRK_ERR_ARG; }
    if (rowptr[0] != 0) { err = "rowptr[0] must be 0"; return CSRK_ERR_MATRIX; }
    for (int32_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) {
            err = "rowptr decreases at row " + std::to_string(i);
            return CSRK_ERR_MATRIX;
        }
    }
    int64_t nnz = rowptr[n];
    if (nnz > 0 && (!colidx || !vals)) { err = "colidx/vals is NULL"; return CSRK_ERR_ARG; }
    out.n = n;
    out.rowptr.assign(rowptr, rowptr + n + 1);
    out.colidx.resize(nnz);
    out.vals.resize(nnz);
    std::vector<std::pair<int32_t, double>> row;
    for (int32_t i = 0; i < n; ++i) {
        int64_t b = rowptr[i], e = rowptr[i + 1];
        bool sorted = true;
        for (int64_t p = b; p < e; ++p) {
            int32_t c = colidx[p];
            if (c < 0 || c >= n) {
                err = "column " + std::to_string(c) + " out of range in row " + std::to_string(i);
                return CSRK_ERR_MATRIX;
            }
            if (p > b && c <= colidx[p - 1]) sorted = false;
        }
        if (sorted) {
            std::memcpy(&out.colidx[b], colidx + b, sizeof(int32_t) * (e - b));
            std::memcpy(&out.vals[b], vals + b, sizeof(double) * (e - b));
            continue;
        }
        row.clear();
        for (int64_t p = b; p < e; ++p) row.emplace_back(colidx[p], vals[p]);
        std::stable_sort(row.begin(), row.end(),
                         [](const auto& u, const auto& v) { return u.first < v.first; });
        for (size_t q = 0; q < row.size(); ++q) {
            if (q > 0 && row[q].first == row[q - 1].first) {
                err = "repeated column " + std::to_string(row[q].first) + " in row " +
                      std::to_string(i);
                return CSRK_ERR_MATRIX;
            }
            out.colidx[b + q] = row[q].first;
            out.vals[b + q] = row[q].second;
        }
    }
    return CSRK_OK;
}

// ---------------------------------------------------------------- RCM
namespace {

struct Graph {
    std::vector<int64_t> start;   // n + 1
    std::vector<int32_t> nbr;     // sorted distinct neighbours, no self-loops
    int32_t deg(int32_t v) const { return (int32_t)(start[v + 1] - start[v]); }
};

// Rows [b, e) of the symmetry check: every off-diagonal (i, j) has its (j, i).  Threads
// take disjoint row ranges; the answer does not depend on their number or order.
struct SymCtx {
    const CsrHost* a;
    std::vector<uint8_t>* ok;   // one flag per range start
    int64_t grain;
};
void sym_rows(int64_t b, int64_t e, void* vctx) {
    const SymCtx& c = *static_cast<const SymCtx*>(vctx);
    const CsrHost& a = *c.a;
    bool ok = true;
    for (int64_t i = b; i < e && ok; ++i) {
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) {
            const int32_t j = a.colidx[p];
            if (j == i) continue;
            const int32_t* lo = a.colidx.data() + a.rowptr[j];
            const int32_t* hi = a.colidx.data() + a.rowptr[j + 1];
            if (!std::binary_search(lo, hi, (int32_t)i)) {
                ok = false;
                break;
            }
        }
    }
    if (!ok) (*c.ok)[(size_t)(b / c.grain)] = 0;
}

bool pattern_is_symmetric(const CsrHost& a) {
    const int64_t grain = 16384;
    std::vector<uint8_t> ok((size_t)((a.n + grain - 1) / grain) + 1, 1);
    SymCtx ctx{&a, &ok, grain};
    parallel_for_ranges(a.n, grain, sym_rows, &ctx);
    for (uint8_t f : ok)
        if (!f) return false;
    return true;
}

// Copy rows [b, e) of A's pattern without the diagonal into the neighbour lists.
struct NbrCtx {
    const CsrHost* a;
    Graph* g;
};
void copy_nbr_rows(int64_t b, int64_t e, void* vctx) {
    const NbrCtx& c = *static_cast<const NbrCtx*>(vctx);
    for (int64_t i = b; i < e; ++i) {
        int64_t w = c.g->start[i];
        for (int64_t p = c.a->rowptr[i]; p < c.a->rowptr[i + 1]; ++p)
            if (c.a->colidx[p] != i) c.g->nbr[w++] = c.a->colidx[p];
    }
}

// Neighbour lists of A + A^T.  For a symmetric pattern this is A's pattern minus the
// diagonal (rows are already sorted and distinct).
void symmetrised_graph(const CsrHost& a, Graph& g) {
    const int32_t n = a.n;
    g.start.assign((size_t)n + 1, 0);
    if (pattern_is_symmetric(a)) {
        for (int32_t i = 0; i < n; ++i) {
            int64_t d = 0;
            for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) d += (a.colidx[p] != i);
            g.start[i + 1] = g.start[i] + d;
        }
        g.nbr.resize(g.start[n]);
        NbrCtx ctx{&a, &g};
        parallel_for_ranges(n, 16384, copy_nbr_rows, &ctx);
        return;
    }
    // General case: merge each row with the matching column of A (via the transpose).
    std::vector<int64_t> tstart((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) tstart[a.colidx[p] + 1]++;
    for (int32_t i = 0; i < n; ++i) tstart[i + 1] += tstart[i];
    std::vector<int32_t> trow(tstart[n]);
    std::vector<int64_t> fill(tstart.begin(), tstart.end() - 1);
    for (int32_t i = 0; i < n; ++i)   // rows ascending -> each transposed list ascending
        for (int64_t p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) trow[fill[a.colidx[p]]++] = i;
    std::vector<int32_t> merged;
    g.nbr.clear();
    for (int32_t i = 0; i < n; ++i) {
        merged.clear();
        std::set_union(a.colidx.begin() + a.rowptr[i], a.colidx.begin() + a.rowptr[i + 1],
                       trow.begin() + tstart[i], trow.begin() + tstart[i + 1],
                       std::back_inserter(merged));
        for (int32_t v : merged)
            if (v != i) g.nbr.push_back(v);
        g.start[i + 1] = (int64_t)g.nbr.size();
    }
}

// Breadth-first level structure from root over vertices with placed[v] == 0.  Fills
// `order` with the reached vertices level by level; returns the level count and the
// offset where the last level begins.
// Large levels are expanded by several threads: each claims a vertex by swapping the tag
// into seen_tag (exactly one thread sees the old value) and collects its finds, which are
// appended in thread order.  The order inside a level then varies from run to run, but the
// SET of vertices of every level does not, and the callers use only the depth and the last
// level's set (the start search picks its least-degree, smallest-index vertex).
struct LevelCtx {
    const Graph* g;
    const uint8_t* placed;
    int32_t* seen_tag;
    int32_t tag;
    const int32_t* frontier;
    std::vector<std::vector<int32_t>>* found;   // one list per range of the frontier
    int64_t grain;
};
void expand_level(int64_t b, int64_t e, void* vctx) {
    const LevelCtx& c = *static_cast<const LevelCtx*>(vctx);
    std::vector<int32_t>& out = (*c.found)[(size_t)(b / c.grain)];
    out.clear();
    for (int64_t q = b; q < e; ++q) {
        const int32_t v = c.frontier[q];
        for (int64_t k = c.g->start[v]; k < c.g->start[v + 1]; ++k) {
            const int32_t u = c.g->nbr[k];
            if (c.placed[u] || __atomic_load_n(&c.seen_tag[u], __ATOMIC_RELAXED) == c.tag) continue;
            if (__atomic_exchange_n(&c.seen_tag[u], c.tag, __ATOMIC_RELAXED) != c.tag) out.push_back(u);
        }
    }
}

int32_t level_structure(const Graph& g, int32_t root, const std::vector<uint8_t>& placed,
                        std::vector<int32_t>& seen_tag, int32_t tag,
                        std::vector<int32_t>& order, size_t& last_level_at) {
    constexpr int64_t PAR_LEVEL = 8192, GRAIN = 2048;
    std::vector<std::vector<int32_t>> found;
    order.clear();
    order.push_back(root);
    seen_tag[root] = tag;
    size_t level_begin = 0;
    int32_t depth = 0;
    while (level_begin < order.size()) {
        size_t level_end = order.size();
        last_level_at = level_begin;
        ++depth;
        const int64_t width = (int64_t)(level_end - level_begin);
        if (width >= PAR_LEVEL) {
            found.resize((size_t)((width + GRAIN - 1) / GRAIN));
            LevelCtx ctx{&g, placed.data(), seen_tag.data(), tag, order.data() + level_begin, &found, GRAIN};
            parallel_for_ranges(width, GRAIN, expand_level, &ctx);
            for (size_t f = 0; f < (size_t)((width + GRAIN - 1) / GRAIN); ++f)
                order.insert(order.end(), found[f].begin(), found[f].end());
            level_begin = level_end;
            continue;
        }
        for (size_t q = level_begin; q < level_end; ++q) {
            int32_t v = order[q];
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                int32_t u = g.nbr[e];
                if (!placed[u] && seen_tag[u] != tag) {
                    seen_tag[u] = tag;
                    order.push_back(u);
                }
            }
        }
        level_begin = level_end;
    }
    return depth;
}

}  // namespace

void rcm_permutation(const CsrHost& a, std::vector<int32_t>& perm) {
    const int32_t n = a.n;
    perm.assign(n, 0);
    if (n == 0) return;
    Graph g;
    symmetrised_graph(a, g);

    // Candidate start vertices in (degree, index) order: a counting sort by degree keeps
    // indices ascending within a degree.
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v) maxdeg = std::max(maxdeg, g.deg(v));
    std::vector<int32_t> bucket((size_t)maxdeg + 2, 0);
    for (int32_t v = 0; v < n; ++v) bucket[g.deg(v) + 1]++;
    for (int32_t d = 0; d <= maxdeg; ++d) bucket[d + 1] += bucket[d];
    std::vector<int32_t> by_degree(n);
    for (int32_t v = 0; v < n; ++v) by_degree[bucket[g.deg(v)]++] = v;

    std::vector<uint8_t> placed(n, 0);
    std::vector<int32_t> seen_tag(n, -1);
    std::vector<int32_t> levels, levels2;
    std::vector<int32_t> cm;
    cm.reserve(n);
    std::vector<std::pair<int32_t, int32_t>> kids;
    int32_t tag = 0;
    size_t cursor = 0;
    while ((int32_t)cm.size() < n) {
        while (placed[by_degree[cursor]]) ++cursor;
        int32_t root = by_degree[cursor];
        size_t last_at = 0;
        int32_t depth = level_structure(g, root, placed, seen_tag, tag++, levels, last_at);
        for (int moves = 0; moves < 8; ++moves) {
            int32_t cand = -1;
            for (size_t q = last_at; q < levels.size(); ++q) {
                int32_t v = levels[q];
                if (cand < 0 || g.deg(v) < g.deg(cand) || (g.deg(v) == g.deg(cand) && v < cand))
                    cand = v;
            }
            size_t last2 = 0;
            int32_t depth2 = level_structure(g, cand, placed, seen_tag, tag++, levels2, last2);
            if (depth2 <= depth) break;
            root = cand;
            depth = depth2;
            levels.swap(levels2);
            last_at = last2;
        }
        // Cuthill-McKee from root.
        size_t head = cm.size();
        cm.push_back(root);
        placed[root] = 1;
        while (head < cm.size()) {
            int32_t v = cm[head++];
            kids.clear();
            for (int64_t e = g.start[v]; e < g.start[v + 1]; ++e) {
                int32_t u = g.nbr[e];
                if (!placed[u]) kids.emplace_back(g.deg(u), u);
            }
            std::sort(kids.begin(), kids.end());
            for (auto& kd : kids) {
                placed[kd.second] = 1;
                cm.push_back(kd.second);
            }
        }
    }
    for (int32_t i = 0; i < n; ++i) perm[i] = cm[n - 1 - i];
}

// ---------------------------------------------------------------- B = P A P^T
namespace {
struct PermCtx {
    const CsrHost* a;
    const int32_t* perm;
    const int32_t* iperm;
    CsrHost* b;
};
void permute_rows(int64_t lo, int64_t hi, void* vctx) {
    auto* c = (PermCtx*)vctx;
    const CsrHost& a = *c->a;
    CsrHost& b = *c->b;
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = lo; i < hi; ++i) {
        int32_t old = c->perm[i];
        int64_t src = a.rowptr[old], len = a.rowptr[old + 1] - src;
        int64_t dst = b.rowptr[i];
        row.resize(len);
        for (int64_t q = 0; q < len; ++q)
            row[q] = {c->iperm[a.colidx[src + q]], a.vals[src + q]};
        // columns are distinct, so a plain sort on the new index is deterministic
        std::sort(row.begin(), row.end(),
                  [](const auto& u, const auto& v) { return u.first < v.first; });
        for (int64_t q = 0; q < len; ++q) {
            b.colidx[dst + q] = row[q].first;
            b.vals[dst + q] = row[q].second;
        }
    }
}
}  // namespace

void permute_symmetric(const CsrHost& a, const std::vector<int32_t>& perm, CsrHost& b) {
    const int32_t n = a.n;
    std::vector<int32_t> iperm(n);
    for (int32_t i = 0; i < n; ++i) iperm[perm[i]] = i;
    b.n = n;
    b.rowptr.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i)
        b.rowptr[i + 1] = b.rowptr[i] + (a.rowptr[perm[i] + 1] - a.rowptr[perm[i]]);
    b.colidx.resize(a.colidx.size());
    b.vals.resize(a.vals.size());
    PermCtx ctx{&a, perm.data(), iperm.data(), &b};
    parallel_for(n, 4096, permute_rows, &ctx);
}

// ---------------------------------------------------------------- pointers
void fixed_pointers(int32_t n, int32_t sr, int32_t ssr, std::vector<int32_t>& sr_ptr,
                    std::vector<int32_t>& ssr_ptr) {
    int64_t nsr = ((int64_t)n + sr - 1) / sr;
    sr_ptr.resize(nsr + 1);
    for (int64_t s = 0; s <= nsr; ++s) sr_ptr[s] = (int32_t)std::min<int64_t>(s * sr, n);
    int64_t nssr = (nsr + ssr - 1) / ssr;
    ssr_ptr.resize(nssr + 1);
    for (int64_t t = 0; t <= nssr; ++t) ssr_ptr[t] = (int32_t)std::min<int64_t>(t * ssr, nsr);
}

bool check_pointers(int32_t n, const std::vector<int32_t>& sr_ptr,
                    const std::vector<int32_t>& ssr_ptr, std::string& err) {
    if (sr_ptr.empty() || sr_ptr.front() != 0 || sr_ptr.back() != n) {
        err = "sr_ptr must start at 0 and end at n";
        return false;
    }
    for (size_t s = 1; s < sr_ptr.size(); ++s)
        if (sr_ptr[s] < sr_ptr[s - 1]) { err = "sr_ptr decreases"; return false; }
    int32_t nsr = (int32_t)sr_ptr.size() - 1;
    if (ssr_ptr.empty() || ssr_ptr.front() != 0 || ssr_ptr.back() != nsr) {
        err = "ssr_ptr must start at 0 and end at the number of super-rows";
        return false;
    }
    for (size_t t = 1; t < ssr_ptr.size(); ++t)
        if (ssr_ptr[t] < ssr_ptr[t - 1]) { err = "ssr_ptr decreases"; return false; }
    return true;
}

void build_descs(const CsrHost& b, const std::vector<int32_t>& sr_ptr,
                 const std::vector<int32_t>& ssr_ptr, std::vector<SsrDesc>& desc,
                 TileStats& st) {
    size_t nssr = ssr_ptr.size() - 1;
    desc.resize(nssr);
    st = TileStats{};
    for (size_t t = 0; t < nssr; ++t) {
        SsrDesc d{};
        d.s0 = ssr_ptr[t];
        d.s1 = ssr_ptr[t + 1];
        d.r0 = sr_ptr[d.s0];
        d.r1 = sr_ptr[d.s1];
        d.p0 = b.rowptr[d.r0];
        d.p1 = b.rowptr[d.r1];
        int32_t lo = 0;
        for (int64_t p = d.p0; p < d.p1; ++p)
            if (p == d.p0 || b.colidx[p] < lo) lo = b.colidx[p];
        d.cbase = lo;
        desc[t] = d;
        st.max_srs = std::max(st.max_srs, d.s1 - d.s0);
        st.max_rows = std::max(st.max_rows, d.r1 - d.r0);
        st.max_nnz = std::max<int64_t>(st.max_nnz, (int64_t)d.p1 - d.p0);
    }
    for (size_t s = 0; s + 1 < sr_ptr.size(); ++s)
        st.max_sr_rows = std::max(st.max_sr_rows, sr_ptr[s + 1] - sr_ptr[s]);
    const int32_t covered = sr_ptr.empty() ? 0 : sr_ptr.back();   // long rows lie beyond
    for (int32_t i = 0; i < covered; ++i)
        st.max_row_len = std::max(st.max_row_len, b.rowptr[i + 1] - b.rowptr[i]);
}

// Delta-coded 16-bit columns: a row's first entry holds its column minus the SSR's
// cbase, every further entry the step from the previous column (columns ascend within a
// row).  Exact when every code is at most 65,535; returns false and leaves col16 empty
// otherwise.
bool compress_columns(const CsrHost& b, const std::vector<SsrDesc>& desc, std::vector<uint16_t>& col16) {
    col16.assign(b.colidx.size(), 0);
    for (const SsrDesc& d : desc)
        for (int32_t r = d.r0; r < d.r1; ++r)
            for (int64_t p = b.rowptr[r]; p < b.rowptr[r + 1]; ++p) {
                const int64_t code = p == b.rowptr[r] ? (int64_t)b.colidx[p] - d.cbase
                                                      : (int64_t)b.colidx[p] - b.colidx[p - 1];
                if (code < 0 || code > 65535) {
                    col16.clear();
                    return false;
                }
                col16[p] = (uint16_t)code;
            }
    return true;
}

// x windows of kernel 5.  Columns are grouped in aligned blocks of XWIN_ALIGN elements;
// an SSR's window is the list of runs of blocks holding its columns (runs whose gap is at
// most XWIN_GAP blocks merged), each run copied to shared memory at a running offset.
struct XwinCtx {
    const CsrHost* b;
    const std::vector<SsrDesc>* desc;
    std::vector<std::vector<int32_t>>* runs;   // per SSR: (start, base) pairs, then the sentinel pair
    std::vector<uint16_t>* colx;
    std::vector<uint8_t>* ok;
};

static void xwin_ssrs(int64_t t0, int64_t t1, void* vctx) {
    auto* c = static_cast<XwinCtx*>(vctx);
    const CsrHost& b = *c->b;
    std::vector<int32_t> blocks;
    for (int64_t t = t0; t < t1; ++t) {
        const SsrDesc& d = (*c->desc)[t];
        std::vector<int32_t>& run = (*c->runs)[t];
        run.clear();
        blocks.clear();
        for (int64_t p = d.p0; p < d.p1; ++p) blocks.push_back(b.colidx[p] / XWIN_ALIGN);
        std::sort(blocks.begin(), blocks.end());
        blocks.erase(std::unique(blocks.begin(), blocks.end()), blocks.end());
        // runs of blocks: [first, last] inclusive
        int64_t base = 0;
        size_t i = 0;
        int32_t exact_end = 0;
        while (i < blocks.size()) {
            const int32_t first = blocks[i];
            int32_t last = first;
            while (i + 1 < blocks.size() && blocks[i + 1] - last <= XWIN_GAP + 1) last = blocks[++i];
            ++i;
            const int64_t start = (int64_t)first * XWIN_ALIGN;
            const int64_t end = std::min<int64_t>((int64_t)(last + 1) * XWIN_ALIGN, b.n);
            run.push_back((int32_t)start);
            run.push_back((int32_t)base);
            exact_end = (int32_t)(base + (end - start));
            base += (int64_t)(last - first + 1) * XWIN_ALIGN;
        }
        run.push_back(exact_end);      // sentinel: elements the copies cover (the last run may end at n)
        run.push_back((int32_t)std::min<int64_t>(base, INT32_MAX));   // and the aligned window length
        if (base > 65536) {
            (*c->ok)[t] = 0;
            continue;
        }
        // window-local code of every nonzero: its run's base + offset into the run
        const size_t nrun = run.size() / 2 - 1;
        for (int64_t p = d.p0; p < d.p1; ++p) {
            const int32_t col = b.colidx[p];
            size_t lo = 0, hi = nrun;   // last run whose start <= col
            while (hi - lo > 1) {
                const size_t mid = (lo + hi) / 2;
                if (run[2 * mid] <= col) lo = mid;
                else hi = mid;
            }
            (*c->colx)[p] = (uint16_t)(run[2 * lo + 1] + (col - run[2 * lo]));
        }
    }
}

bool build_xwin(const CsrHost& b, const std::vector<SsrDesc>& desc, std::vector<SsrDesc>& xdesc,
                std::vector<int32_t>& win, std::vector<int32_t>& wptr, std::vector<uint16_t>& colx,
                int32_t& max_win, int64_t& total_runs) {
    const size_t nssr = desc.size();
    std::vector<std::vector<int32_t>> runs(nssr);
    std::vector<uint8_t> ok(nssr, 1);
    colx.assign(b.colidx.size(), 0);
    XwinCtx ctx{&b, &desc, &runs, &colx, &ok};
    parallel_for(nssr, 64, xwin_ssrs, &ctx);
    for (uint8_t f : ok)
        if (!f) {
            colx.clear();
            return false;
        }
    xdesc = desc;
    win.clear();
    wptr.assign(nssr + 1, 0);
    max_win = 0;
    total_runs = 0;
    for (size_t t = 0; t < nssr; ++t) {
        const std::vector<int32_t>& run = runs[t];
        const int32_t nrun = (int32_t)run.size() / 2 - 1;
        win.insert(win.end(), run.begin(), run.end() - 2);
        wptr[t + 1] = wptr[t] + nrun;
        xdesc[t].cbase = run[2 * nrun];   // elements the copies cover
        xdesc[t].aux = nrun;
        max_win = std::max(max_win, run.back());
        total_runs += nrun;
    }
    win.push_back(0);   // one pair of padding after the last run
    win.push_back(0);
    return true;
}

void build_row_order(const CsrHost& b, const std::vector<int32_t>& sr_ptr, const std::vector<SsrDesc>& desc,
                     std::vector<uint16_t>& ord, int64_t& slots_natural, int64_t& slots_ordered) {
    const int32_t covered = sr_ptr.empty() ? 0 : sr_ptr.back();
    ord.assign((size_t)covered, 0);
    slots_natural = slots_ordered = 0;
    std::vector<int32_t> rows;
    auto len = [&](int32_t r) { return b.rowptr[r + 1] - b.rowptr[r]; };
    for (const SsrDesc& d : desc) {
        rows.resize((size_t)(d.r1 - d.r0));
        for (int32_t j = 0; j < d.r1 - d.r0; ++j) rows[j] = d.r0 + j;
        std::stable_sort(rows.begin(), rows.end(), [&](int32_t a, int32_t c) { return len(a) > len(c); });
        for (int32_t j = 0; j < d.r1 - d.r0; ++j) ord[d.r0 + j] = (uint16_t)(rows[j] - d.r0);
        // warp passes: 32 positions at a time inside each super-row
        for (int32_t sr = d.s0; sr < d.s1; ++sr)
            for (int32_t q = sr_ptr[sr]; q < sr_ptr[sr + 1]; q += 32) {
                int32_t mn = 0, mo = 0;
                for (int32_t k = q; k < std::min(q + 32, sr_ptr[sr + 1]); ++k) {
                    mn = std::max(mn, len(k));
                    mo = std::max(mo, len(rows[k - d.r0]));
                }
                slots_natural += mn;
                slots_ordered += mo;
            }
    }
}

// ---------------------------------------------------------------- narrowing
void narrow_f32(const double* in, float* out, int64_t n) {
    // The C conversion is IEEE round-to-nearest-even in the default rounding mode.
    for (int64_t i = 0; i < n; ++i) out[i] = (float)in[i];
}

// Round an FP64 value to the nearest BF16 (8 significant bits, FP32's exponent range,
// subnormals kept), ties to even, working on the FP64 bit pattern so that no
// intermediate rounding happens.
uint16_t f64_to_bf16(double d) {
    uint64_t u;
    std::memcpy(&u, &d, sizeof u);
    const uint16_t sign = (uint16_t)((u >> 48) & 0x8000u);
    const uint64_t mag = u & 0x7FFFFFFFFFFFFFFFull;
    if (mag > 0x7FF0000000000000ull) return sign | 0x7FC0u;       // NaN -> quiet NaN
    if (mag == 0x7FF0000000000000ull) return sign | 0x7F80u;      // +-Inf
    const int biased = (int)(mag >> 52);
    if (biased == 0) return sign;   // zero or FP64 subnormal: far below half a BF16 quantum
    const int e = biased - 1023;                                  // value = sig * 2^(e-52)
    const uint64_t sig = (mag & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    // Keep `keep` = sig >> shift significant bits: 8 for normal targets, fewer when the
    // result lands in BF16's subnormal range (quantum 2^-133).
    int shift = (e >= -126) ? 45 : 45 + (-126 - e);
    if (shift >= 64) return sign;                                 // < 2^-134 rounds to 0
    uint64_t keep = sig >> shift;
    const uint64_t rem = sig & ((1ull << shift) - 1);
    const uint64_t half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (keep & 1))) ++keep;
    if (e >= -126) {
        int ex = e;
        if (keep == 0x100) {   // mantissa carry into the next binade
            keep >>= 1;
            ++ex;
        }
        if (ex > 127) return sign | 0x7F80u;                      // overflow -> Inf
        return (uint16_t)(sign | (uint16_t)((ex + 127) << 7) | (uint16_t)(keep & 0x7F));
    }
    // subnormal target: keep counts quanta of 2^-133; keep == 0x80 is the smallest normal,
    // whose encoding (exponent field 1, fraction 0) is the same bit pattern.
    return (uint16_t)(sign | (uint16_t)keep);
}

bool split_pairs(const double* in, float* out, int64_t n) {
    bool ok = true;
    for (int64_t i = 0; i < n; ++i) {
        const double a = in[i];
        const float h = (float)a;
        out[2 * i] = h;
        out[2 * i + 1] = (float)(a - (double)h);   // a - h is exact in FP64
        const double m = std::fabs(a);
        if (a != 0.0 && !(m >= 0x1p-39 && m <= 0x1p60)) ok = false;
    }
    return ok;
}

void narrow_bf16(const double* in, uint16_t* out, int64_t n) {
    for (int64_t i = 0; i < n; ++i) out[i] = f64_to_bf16(in[i]);
}

}  // namespace csrk
