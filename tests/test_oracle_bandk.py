"""Pins for the oracle's Band-k ordering (reading of Sec. 2.2, Listing 2)."""
import numpy as np
import pytest

import synth
from oracle import bandk, reorder
from tests.conftest import read_golden


def csr_from_edges(n, edges):
    rows = [{i} for i in range(n)]
    for a, b in edges:
        rows[a].add(b)
        rows[b].add(a)
    rp, ci = [0], []
    for r in rows:
        ci += sorted(r)
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32)


def parse_edges(s):
    return [tuple(int(v) for v in e.split("-")) for e in s.split()]


@pytest.mark.parametrize("case", read_golden("bandk_hand.txt"), ids=lambda c: c[0].split()[0])
def test_hand_worked_examples(case):
    name, n, sr, ssr, perm, sr_ptr, ssr_ptr = case[0].split()
    rp, ci = csr_from_edges(int(n), parse_edges(case[1]))
    p, s1, s2 = bandk.bandk_py(int(n), rp, ci, int(sr), int(ssr))
    assert p.tolist() == [int(v) for v in perm.split(",")]
    assert s1.tolist() == [int(v) for v in sr_ptr.split(",")]
    assert s2.tolist() == [int(v) for v in ssr_ptr.split(",")]


def connected(members, adj):
    members = set(members)
    if not members:
        return True
    start = next(iter(members))
    seen, stack = {start}, [start]
    while stack:
        v = stack.pop()
        for u in adj[v]:
            if u in members and u not in seen:
                seen.add(u)
                stack.append(u)
    return seen == members


CASES = [
    ("grid2d_scrambled", lambda: synth.relabel(synth.stencil_2d_5pt(17, 13), synth.vectors.permutation(221, 5)), 8, 4),
    ("stencil3d_27", lambda: synth.stencil_3d(7, 6, 5, 27, "random_dd", 2, labels=synth.vectors.permutation(210, 2)), 16, 3),
    ("fem", lambda: synth.fem_like(6, 3), 32, 2),
    ("random_components", lambda: synth.random_pattern(300, 0.01, 4, symmetric=True, empty_rows=7), 4, 5),
]


@pytest.mark.parametrize("name,make,sr,ssr", CASES, ids=[c[0] for c in CASES])
def test_invariants(name, make, sr, ssr):
    a = make()
    perm, sr_ptr, ssr_ptr = bandk.bandk_py(a.n, a.rowptr, a.colidx, sr, ssr)
    assert sorted(perm.tolist()) == list(range(a.n))                       # a bijection
    assert sr_ptr[0] == 0 and sr_ptr[-1] == a.n and np.all(np.diff(sr_ptr) >= 1)
    assert np.all(np.diff(sr_ptr) <= sr)                                    # SR cap
    nsr = len(sr_ptr) - 1
    assert ssr_ptr[0] == 0 and ssr_ptr[-1] == nsr and np.all(np.diff(ssr_ptr) >= 1)
    assert np.all(np.diff(ssr_ptr) <= ssr)                                  # SSR cap
    adj = reorder.sym_graph(a.n, a.rowptr, a.colidx)
    for s in range(nsr):                                                    # SRs are connected
        assert connected(perm[sr_ptr[s]:sr_ptr[s + 1]].tolist(), adj)
    for t in range(len(ssr_ptr) - 1):                                       # and so are SSRs
        rows = perm[sr_ptr[ssr_ptr[t]]:sr_ptr[ssr_ptr[t + 1]]].tolist()
        assert connected(rows, adj)


@pytest.mark.parametrize("sr,ssr", [(1, 1), (2, 3), (4, 2), (32, 8)])
def test_scrambled_path_gets_bandwidth_one(sr, ssr):
    n = 97
    lab = synth.vectors.permutation(n, 11)
    edges = [(int(lab[i]), int(lab[i + 1])) for i in range(n - 1)]
    rp, ci = csr_from_edges(n, edges)
    perm, _, _ = bandk.bandk_py(n, rp, ci, sr, ssr)
    pos = np.empty(n, np.int64)
    pos[perm] = np.arange(n)
    assert max(abs(pos[a] - pos[b]) for a, b in edges) == 1


def test_rows_of_one_sr_and_singletons():
    """sr = 1: every row its own SR; the row order is then the inner order of the SSRs."""
    a = synth.stencil_2d_5pt(6, 5)
    perm, sr_ptr, ssr_ptr = bandk.bandk_py(a.n, a.rowptr, a.colidx, 1, 4)
    assert sr_ptr.tolist() == list(range(a.n + 1))
    assert np.all(np.diff(ssr_ptr) <= 4)


def test_empty_matrix():
    perm, s1, s2 = bandk.bandk_py(0, np.zeros(1, np.int32), np.zeros(0, np.int32), 4, 4)
    assert perm.size == 0 and s1.tolist() == [0] and s2.tolist() == [0]
