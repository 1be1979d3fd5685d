"""Oracle reordering (TEST INFRASTRUCTURE).

Sec. 2.1 names reverse Cuthill-McKee (RCM) as a bandwidth-limiting ordering that pulls
nonzeros toward the diagonal; Sec. 5.3 feeds RCM-ordered matrices to the CSR-based
comparison libraries, and the reordering is what gives neighbouring rows of a super-row
their shared x entries (Sec. 2.2).  The paper leaves the RCM details open; the reading
used here (and by the library) is:

  1. Graph of the symmetrised pattern A + A^T without self-loops; degree = number of
     distinct neighbours.
  2. Each component starts at the unvisited vertex of least degree (smallest index on
     ties).
  3. George-Liu pseudo-peripheral search: from the start, take the least-degree vertex of
     the deepest BFS level (smallest index on ties); move there while that strictly
     deepens the level structure; at most 8 moves.
  4. Cuthill-McKee breadth-first order; a dequeued vertex appends its unvisited
     neighbours sorted by (degree, index).
  5. Components concatenated, the whole sequence reversed: perm[new] = old.

The permuted matrix is B = P A P^T with B[i, j] = A[perm[i], perm[j]]; each row's
columns ascend in the new numbering.

Pins (tests/test_oracle_reorder.py): a hand-worked 8-vertex example
(tests/golden/rcm_hand.txt); ``check_cm_order`` re-derives the Cuthill-McKee rules from
the sequence alone; perm is a bijection; scrambled path -> bandwidth 1; scrambled 64x64
grid -> bandwidth <= 2*64; bandwidth within 1.1x of scipy's reverse_cuthill_mckee; the
Python and C versions agree exactly; B built by scipy fancy indexing and by a plain loop
agree, and B[i, j] = A[perm i, perm j] on dense copies.
"""
from __future__ import annotations

import numpy as np

from . import native


def sym_graph(n, rowptr, colidx):
    """Sorted neighbour lists of A + A^T without self-loops (pure Python)."""
    nb = [set() for _ in range(n)]
    for i in range(n):
        for p in range(int(rowptr[i]), int(rowptr[i + 1])):
            j = int(colidx[p])
            if j != i:
                nb[i].add(j)
                nb[j].add(i)
    return [sorted(s) for s in nb]


def _levels(root, adj, visited):
    """BFS level structure restricted to unvisited vertices: list of levels."""
    seen = {root}
    levels = [[root]]
    while True:
        nxt = []
        for v in levels[-1]:
            for u in adj[v]:
                if not visited[u] and u not in seen:
                    seen.add(u)
                    nxt.append(u)
        if not nxt:
            return levels
        levels.append(nxt)


def rcm_py(n, rowptr, colidx):
    """Reverse Cuthill-McKee, reading above, pure Python (small graphs)."""
    adj = sym_graph(n, rowptr, colidx)
    deg = [len(a) for a in adj]
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
            kids = sorted((u for u in adj[v] if not visited[u]), key=lambda u: (deg[u], u))
            for u in kids:
                visited[u] = True
                seq.append(u)
    return np.array(seq[::-1], dtype=np.int32)


def rcm(n, rowptr, colidx):
    """Same ordering from the C twin (any size)."""
    perm = np.empty(n, dtype=np.int32)
    rc = native.lib().oracle_rcm(int(n), np.ascontiguousarray(rowptr, np.int32),
                                 np.ascontiguousarray(colidx, np.int32), perm)
    if rc != 0:
        raise MemoryError("oracle_rcm failed")
    return perm


def check_cm_order(n, rowptr, colidx, perm):
    """Independent check that reversed(perm) is a Cuthill-McKee sequence under the reading
    (steps 2 and 4; the choice of start vertex in step 3 is checked separately by
    re-running the pseudo-peripheral search).  Returns a list of violations."""
    adj = sym_graph(n, rowptr, colidx)
    deg = [len(a) for a in adj]
    seq = [int(v) for v in np.asarray(perm)[::-1]]
    errs = []
    if sorted(seq) != list(range(n)):
        return ["not a permutation"]
    pos = {v: i for i, v in enumerate(seq)}
    # Each vertex's parent is the earliest-placed neighbour placed before it; a vertex
    # with none starts a component.  Children of one parent must appear contiguously, in
    # (degree, index) order, and parents must be served in sequence order.
    last_parent_pos = -1
    i = 0
    while i < n:
        v = seq[i]
        earlier = [pos[u] for u in adj[v] if pos[u] < i]
        if not earlier:
            i += 1
            continue
        par = seq[min(earlier)]
        if pos[par] <= last_parent_pos:
            errs.append(f"parent {par} served out of breadth-first order")
        last_parent_pos = pos[par]
        block = []
        j = i
        while j < n:
            w = seq[j]
            e = [pos[u] for u in adj[w] if pos[u] < i]
            if not e or seq[min(e)] != par:
                break
            block.append(w)
            j += 1
        keys = [(deg[w], w) for w in block]
        if keys != sorted(keys):
            errs.append(f"children of {par} not in (degree, index) order: {block}")
        unplaced = sorted((u for u in adj[par] if pos[u] >= i), key=lambda u: (deg[u], u))
        if unplaced[:len(block)] != block or len(unplaced) != len(block):
            errs.append(f"vertex {par} did not enqueue exactly its unvisited neighbours")
        i = j
    return errs


def bandwidth(n, rowptr, colidx):
    """max |i - j| over stored entries (0 for an empty or diagonal matrix)."""
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(np.asarray(rowptr, np.int64)))
    if rows.size == 0:
        return 0
    return int(np.max(np.abs(rows - np.asarray(colidx, np.int64))))


def permute_scipy(n, rowptr, colidx, vals, perm):
    """B = P A P^T via scipy.sparse fancy indexing (library route), columns sorted."""
    import scipy.sparse as sp
    a = sp.csr_matrix((np.asarray(vals, np.float64), np.asarray(colidx, np.int64),
                       np.asarray(rowptr, np.int64)), shape=(n, n))
    p = np.asarray(perm, dtype=np.int64)
    b = a[p, :][:, p].tocsr()
    b.sort_indices()
    return (b.indptr.astype(np.int32), b.indices.astype(np.int32),
            b.data.astype(np.float64))


def permute_loop(n, rowptr, colidx, vals, perm):
    """B = P A P^T by the definition, in plain loops (small inputs)."""
    iperm = [0] * n
    for new, old in enumerate(perm):
        iperm[int(old)] = new
    brp = [0]
    bci, bv = [], []
    for i in range(n):
        old = int(perm[i])
        row = sorted((iperm[int(colidx[p])], float(vals[p]))
                     for p in range(int(rowptr[old]), int(rowptr[old + 1])))
        bci += [c for c, _ in row]
        bv += [v for _, v in row]
        brp.append(len(bci))
    return (np.array(brp, np.int32), np.array(bci, np.int32), np.array(bv, np.float64))


def inverse(perm):
    perm = np.asarray(perm, dtype=np.int64)
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(perm.size)
    return iperm
