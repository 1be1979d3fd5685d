"""Oracle Band-k ordering (TEST INFRASTRUCTURE).

Sec. 2.2 (Listing 2, Fig. 2) describes Band-k, the CSR-k ordering for SpMV: the matrix
graph is coarsened level by level, each coarse level is put in a weighted
bandwidth-limiting order, the coarse nodes are expanded again with the vertices inside
each coarse node reordered by a bandwidth-limiting order, and the coarse nodes of the
levels become the super-rows (and super-super-rows) of A.  The paper names neither the
coarsening scheme, nor the weights, nor the orders.  The reading used here (and by the
library) for k = 3 -- rows, super-rows (SR), super-super-rows (SSR):

  G0   graph of A + A^T without self-loops, every edge weight 1.
  Cuthill-McKee sequence CM(G): the reverse-Cuthill-McKee rules 1-4 of oracle.reorder
       (component starts, pseudo-peripheral search, neighbours by (degree, index)), not
       reversed.  degree = number of distinct neighbours at that level.
  1.   Coarsen G0 -> G1: walk CM(G0); each still unassigned vertex seeds a new aggregate,
       which grows one vertex at a time by the unassigned vertex adjacent to it with the
       fewest unassigned neighbours (the one most at risk of being stranded), then the
       largest edge weight into the aggregate, then the smallest index -- until it holds
       `sr` vertices or nothing unassigned touches it.  Aggregates are numbered in
       creation order.  G1 has an edge between two aggregates with weight = the number of
       G0 edges between them.
  2.   Coarsen G1 -> G2 the same way with CM(G1) and cap `ssr` (counted in G1 vertices).
  3.   Order G2 by weighted reverse Cuthill-McKee: CM with the dequeued vertex's neighbours
       taken by (edge weight descending, degree, index), then reversed.
  4.   Expand G2 -> G1: for each G2 vertex in that order, order its G1 members by a
       breadth-first walk inside the member set, neighbours by (edge weight descending,
       degree, index).  The walk starts at the member with the largest total edge weight
       to G1 vertices already placed (smallest index on ties).  When no member touches a
       placed vertex it starts at the member farthest, breadth-first inside the set, from
       the members with edges leaving the set (ties: smaller outside weight, then index)
       -- the end of the set away from its neighbours; a set with no edge leaving it
       starts at its pseudo-peripheral vertex (rules 2-3 of oracle.reorder, on the set's
       own edges).  A walk that runs out with members left restarts by the same rules.
  5.   Expand G1 -> G0 the same way (each G1 vertex's rows, edge weights 1).
  The rows in final order give perm (perm[new] = old); the member counts give the
  variable super-row sizes (sr_ptr, each <= sr) and super-super-row sizes (ssr_ptr, each
  <= ssr SRs).

Pins (tests/test_oracle_bandk.py): hand-worked examples (tests/golden/bandk_hand.txt);
perm is a bijection, SR / SSR sizes respect the caps, every SR's rows and every SSR's
super-rows form connected subgraphs; a scrambled path gets bandwidth 1; the library's
C++ version agrees exactly.
"""
from __future__ import annotations

import numpy as np

from .reorder import _levels, sym_graph


def _cm_sequence(n, adj, deg, nb_key):
    """Cuthill-McKee sequence over all components (rules 2-4 of oracle.reorder), the
    dequeued vertex v appending its unvisited neighbours u sorted by nb_key(v, u)."""
    visited = [False] * n
    seq = []
    while len(seq) < n:
        s = min((v for v in range(n) if not visited[v]), key=lambda v: (deg[v], v))
        lev = _levels(s, adj, visited)
        for _ in range(8):
            c = min(lev[-1], key=lambda v: (deg[v], v))
            lev_c = _levels(c, adj, visited)
            if len(lev_c) > len(lev):
                s, lev = c, lev_c
            else:
                break
        head = len(seq)
        seq.append(s)
        visited[s] = True
        while head < len(seq):
            v = seq[head]
            head += 1
            kids = sorted((u for u in adj[v] if not visited[u]), key=lambda u: nb_key(v, u))
            for u in kids:
                visited[u] = True
                seq.append(u)
    return seq


def _aggregate(n, nbw, seeds, cap):
    """Steps 1 / 2: aggregates of at most cap vertices, seeded in order; each grows by the
    adjacent unassigned vertex with the fewest unassigned neighbours, then the largest edge
    weight into the aggregate, then the smallest index."""
    agg = [-1] * n
    free = [len(d) for d in nbw]          # unassigned neighbours of each vertex
    groups = []

    def take(v, g, conn):
        agg[v] = g
        conn.pop(v, None)
        for u, w in nbw[v].items():
            free[u] -= 1
            if agg[u] < 0:
                conn[u] = conn.get(u, 0) + w

    for s in seeds:
        if agg[s] >= 0:
            continue
        g = len(groups)
        members = [s]
        conn = {}
        take(s, g, conn)
        while len(members) < cap and conn:
            v = min(conn, key=lambda u: (free[u], -conn[u], u))
            members.append(v)
            take(v, g, conn)
        groups.append(members)
    return agg, groups


def _coarse_graph(nbw, agg, ng):
    """Edge weights between aggregates: the summed weights of the fine edges between them."""
    cw = [dict() for _ in range(ng)]
    for v, nbrs in enumerate(nbw):
        a = agg[v]
        for u, w in nbrs.items():
            b = agg[u]
            if a != b:
                cw[a][b] = cw[a].get(b, 0) + w
    return cw


def _far_start(cand, remaining, inset, nbw, deg):
    """Start of a walk that touches nothing placed: the member farthest (breadth-first,
    inside the remaining members) from the members with edges leaving the set -- ties by
    smaller outside weight, then index; with no such edge at all, the pseudo-peripheral
    vertex of the remaining members (rules 2-3 of oracle.reorder)."""
    outside = {v: sum(w for u, w in nbw[v].items() if u not in inset) for v in cand}
    frontier = [v for v in cand if outside[v] > 0]
    if frontier:
        dist = {v: 0 for v in frontier}
        head = 0
        while head < len(frontier):
            v = frontier[head]
            head += 1
            for u in nbw[v]:
                if u in remaining and u not in dist:
                    dist[u] = dist[v] + 1
                    frontier.append(u)
        far = len(cand) + 1   # members the walk cannot reach count as farthest
        return min(cand, key=lambda v: (-dist.get(v, far), outside[v], v))
    ideg = {v: sum(1 for u in nbw[v] if u in remaining) for v in cand}
    sub = {v: [u for u in nbw[v] if u in remaining] for v in cand}

    def levels(root):
        seen, lev = {root}, [[root]]
        while True:
            nxt = [u for v in lev[-1] for u in sub[v] if u not in seen and not seen.add(u)]
            if not nxt:
                return lev
            lev.append(nxt)

    s = min(cand, key=lambda v: (ideg[v], v))
    lev = levels(s)
    for _ in range(8):
        c = min(lev[-1], key=lambda v: (ideg[v], v))
        lev_c = levels(c)
        if len(lev_c) > len(lev):
            s, lev = c, lev_c
        else:
            break
    return s


def _inner_order(members, nbw, deg, placed):
    """Steps 4 / 5: the members of one coarse node, in order (marks them placed)."""
    inset = set(members)
    remaining = set(members)
    out = []
    while remaining:
        cand = sorted(remaining)
        to_placed = {v: sum(w for u, w in nbw[v].items() if placed[u]) for v in cand}
        if max(to_placed.values()) > 0:
            s = min(cand, key=lambda v: (-to_placed[v], v))
        else:
            s = _far_start(cand, remaining, inset, nbw, deg)
        remaining.discard(s)
        placed[s] = True
        out.append(s)
        queue = [s]
        head = 0
        while head < len(queue):
            v = queue[head]
            head += 1
            kids = sorted((u for u in nbw[v] if u in remaining), key=lambda u: (-nbw[v][u], deg[u], u))
            for u in kids:
                remaining.discard(u)
                placed[u] = True
                out.append(u)
                queue.append(u)
    return out


def bandk_py(n, rowptr, colidx, sr, ssr):
    """Band-k for k = 3 (reading above), pure Python.  Returns (perm, sr_ptr, ssr_ptr)."""
    if sr < 1 or ssr < 1:
        raise ValueError("sr and ssr must be >= 1")
    if n == 0:
        z = np.zeros(1, dtype=np.int32)
        return np.zeros(0, dtype=np.int32), z, z.copy()
    adj0 = sym_graph(n, rowptr, colidx)
    deg0 = [len(a) for a in adj0]
    nbw0 = [{u: 1 for u in a} for a in adj0]
    seeds0 = _cm_sequence(n, adj0, deg0, lambda v, u: (deg0[u], u))
    agg1, groups1 = _aggregate(n, nbw0, seeds0, sr)
    n1 = len(groups1)
    nbw1 = _coarse_graph(nbw0, agg1, n1)
    adj1 = [sorted(d) for d in nbw1]
    deg1 = [len(a) for a in adj1]
    seeds1 = _cm_sequence(n1, adj1, deg1, lambda v, u: (deg1[u], u))
    agg2, groups2 = _aggregate(n1, nbw1, seeds1, ssr)
    n2 = len(groups2)
    nbw2 = _coarse_graph(nbw1, agg2, n2)
    adj2 = [sorted(d) for d in nbw2]
    deg2 = [len(a) for a in adj2]
    order2 = _cm_sequence(n2, adj2, deg2, lambda v, u: (-nbw2[v][u], deg2[u], u))[::-1]
    placed1 = [False] * n1
    order1, ssr_sizes = [], []
    for g in order2:
        inner = _inner_order(groups2[g], nbw1, deg1, placed1)
        order1 += inner
        ssr_sizes.append(len(inner))
    placed0 = [False] * n
    perm, sr_sizes = [], []
    for a in order1:
        inner = _inner_order(groups1[a], nbw0, deg0, placed0)
        perm += inner
        sr_sizes.append(len(inner))
    sr_ptr = np.concatenate([[0], np.cumsum(sr_sizes)]).astype(np.int32)
    ssr_ptr = np.concatenate([[0], np.cumsum(ssr_sizes)]).astype(np.int32)
    return np.array(perm, dtype=np.int32), sr_ptr, ssr_ptr
