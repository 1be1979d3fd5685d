"""The library's host-side CSR-k builder is bit-exact with the oracle: RCM permutation,
B = P A P^T, super-row pointers, value narrowing, and the tuning model."""
import numpy as np
import pytest

import synth
from oracle import csrk as ocsrk
from oracle import precision, reorder, tuning
from paper_2203_05096_gb300 import csrk
from tests.conftest import read_golden


def build(a, sr=32, ssr=8, method="rcm", dtype="f64"):
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals, dtype)
    perm = csrk.reorder(h, method)
    csrk.set_sizes(h, sr, ssr)
    return h, perm


def check_against_oracle(a, sr=32, ssr=8):
    h, perm = build(a, sr, ssr)
    e = csrk.export(h)
    ref_perm = reorder.rcm(a.n, a.rowptr, a.colidx)
    assert np.array_equal(perm, ref_perm)
    assert np.array_equal(e["perm"], ref_perm)
    rp, ci, v = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, ref_perm)
    assert np.array_equal(e["rowptr"], rp)
    assert np.array_equal(e["colidx"], ci)
    assert np.array_equal(e["vals"].view(np.uint64), v.view(np.uint64))
    srp, ssrp = ocsrk.fixed_pointers(a.n, sr, ssr)
    assert np.array_equal(e["sr_ptr"], srp) and np.array_equal(e["ssr_ptr"], ssrp)
    csrk.destroy(h)


@pytest.mark.parametrize("seed", range(8))
def test_random_patterns(seed):
    a = synth.random_pattern(90, 0.03 + 0.01 * seed, seed, symmetric=seed % 2 == 0, empty_rows=seed)
    check_against_oracle(a, sr=1 + seed, ssr=1 + seed % 3)


def test_scrambled_grids_and_fem():
    check_against_oracle(synth.stencil_2d_5pt(64, 64, labels=synth.vectors.permutation(4096, 1)))
    check_against_oracle(synth.stencil_3d(20, 17, 15, 27, "random_dd", 3,
                                          labels=synth.vectors.permutation(5100, 3)), sr=16, ssr=4)
    check_against_oracle(synth.fem_like(14, 4), sr=32, ssr=4)


def test_hand_worked_rcm():
    from tests.test_oracle_reorder import csr_from_edges, golden_cases
    for name, n, perm, edges in golden_cases():
        a = csr_from_edges(n, edges)
        h, p = build(a, 2, 2)
        assert p.tolist() == perm, name
        csrk.destroy(h)


@pytest.mark.slow
def test_full_size_7pt_128_rcm_bit_exact():
    n = 128 ** 3
    a = synth.stencil_3d(128, 128, 128, 7, "random_dd", 3, labels=synth.vectors.permutation(n, 3))
    check_against_oracle(a, 32, 8)


def test_second_reorder_composes():
    a = synth.stencil_2d_5pt(10, 10, labels=synth.vectors.permutation(100, 2))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    p1 = csrk.reorder(h)
    p2 = csrk.reorder(h)
    e = csrk.export(h, with_pointers=False)
    rp, ci, v = reorder.permute_scipy(a.n, a.rowptr, a.colidx, a.vals, p2)
    assert np.array_equal(e["colidx"], ci) and np.array_equal(e["vals"], v)
    csrk.destroy(h)


def test_explicit_pointers_fig1():
    a = synth.random_pattern(9, 0.4, 12)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.set_pointers(h, [0, 2, 5, 7, 9], [0, 2, 4])
    e = csrk.export(h)
    assert e["sr_ptr"].tolist() == [0, 2, 5, 7, 9] and e["ssr_ptr"].tolist() == [0, 2, 4]
    assert csrk.info(h)["nssr"] == 2
    csrk.destroy(h)


def test_narrowing_bit_exact():
    rng = np.random.default_rng(5)
    cases = []
    for expr, _bits, _why in read_golden("bf16_cases.txt"):
        cases.append(eval(expr, {"float": float}))
    vals = np.concatenate([np.array(cases), rng.standard_normal(3000), rng.standard_normal(500) * 1e-39,
                           rng.standard_normal(500) * 1e38, rng.uniform(-1, 0, 1000)])
    n = vals.size
    rowptr = np.arange(n + 1, dtype=np.int32)
    colidx = np.zeros(n, np.int32)
    h = csrk.create(n, rowptr, np.arange(n, dtype=np.int32) * 0 + np.arange(n, dtype=np.int32) % n, vals)
    got16 = csrk.export_values(h, "bf16")
    assert np.array_equal(got16, precision.to_bf16_bits(vals))
    got32 = csrk.export_values(h, "f32")
    ref32 = precision.to_f32(vals)
    same = (got32.view(np.uint32) == ref32.view(np.uint32)) | (np.isnan(got32) & np.isnan(ref32))
    assert np.all(same)
    csrk.destroy(h)


def test_model_sizes_hand_worked():
    for head, expect, _ in read_golden("tuning_model.txt"):
        arch, r = head.split()
        assert csrk.model_sizes(float(r), arch) == tuple(int(v) for v in expect.split()), head
        assert csrk.model_sizes(float(r), arch) == tuning.model_sizes(float(r), arch)


# ------------------------------------------------------------------ Band-k
BANDK_CASES = [
    ("grid2d", lambda: synth.stencil_2d_5pt(17, 13)),
    ("grid2d_scrambled", lambda: synth.relabel(synth.stencil_2d_5pt(17, 13), synth.vectors.permutation(221, 5))),
    ("stencil27", lambda: synth.stencil_3d(7, 6, 5, 27, "random_dd", 2, labels=synth.vectors.permutation(210, 2))),
    ("fem", lambda: synth.fem_like(6, 3)),
    ("components", lambda: synth.random_pattern(300, 0.01, 4, symmetric=True, empty_rows=7)),
    ("nonsymmetric", lambda: synth.random_pattern(200, 0.02, 9, symmetric=False)),
]


@pytest.mark.parametrize("name,make", BANDK_CASES, ids=[c[0] for c in BANDK_CASES])
@pytest.mark.parametrize("sr,ssr", [(8, 4), (32, 8), (1, 1), (5, 3)])
def test_bandk_bit_exact_against_oracle(name, make, sr, ssr):
    from oracle import bandk
    a = make()
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    perm = csrk.reorder_bandk(h, sr, ssr)
    e = csrk.export(h)
    p_ref, sr_ref, ssr_ref = bandk.bandk_py(a.n, a.rowptr, a.colidx, sr, ssr)
    assert np.array_equal(perm, p_ref) and np.array_equal(e["perm"], p_ref)
    assert np.array_equal(e["sr_ptr"], sr_ref) and np.array_equal(e["ssr_ptr"], ssr_ref)
    # the matrix is B = P A P^T under that permutation
    rp, ci, v = reorder.permute_loop(a.n, a.rowptr, a.colidx, a.vals, p_ref)
    assert np.array_equal(e["rowptr"], rp) and np.array_equal(e["colidx"], ci) and np.array_equal(e["vals"], v)
    csrk.destroy(h)


def test_bandk_state_and_arguments():
    a = synth.stencil_2d_5pt(8, 8)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    for sr, ssr in [(0, 4), (4, 0), (-1, 2)]:
        with pytest.raises(csrk.CsrkError) as ei:
            csrk.reorder_bandk(h, sr, ssr)
        assert ei.value.status == "ERR_ARG"
    csrk.reorder(h)                                   # composes with an earlier RCM
    p_rcm = csrk.export(h, with_pointers=False)["perm"].copy()
    perm = csrk.reorder_bandk(h, 8, 2)
    rcm_form = csrk.create(a.n, *reorder.permute_loop(a.n, a.rowptr, a.colidx, a.vals, p_rcm))
    from oracle import bandk
    local, _, _ = bandk.bandk_py(a.n, *reorder.permute_loop(a.n, a.rowptr, a.colidx, a.vals, p_rcm)[:2], 8, 2)
    assert np.array_equal(perm, p_rcm[local])
    with pytest.raises(csrk.CsrkError) as ei:        # pointers exist: no further reorder
        csrk.reorder_bandk(h, 8, 2)
    assert ei.value.status == "ERR_STATE"
    csrk.destroy(rcm_form)
    csrk.destroy(h)


def test_bandk_large_stencil_invariants():
    a = synth.stencil_3d(40, 40, 40, 7, "random_dd", 9, labels=synth.vectors.permutation(64000, 9))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    perm = csrk.reorder_bandk(h, 32, 4)
    e = csrk.export(h)
    assert np.array_equal(np.sort(perm), np.arange(a.n))
    assert np.all(np.diff(e["sr_ptr"]) >= 1) and np.all(np.diff(e["sr_ptr"]) <= 32)
    assert np.all(np.diff(e["ssr_ptr"]) >= 1) and np.all(np.diff(e["ssr_ptr"]) <= 4)
    # most super-rows are full: the aggregates pack the grid
    assert np.mean(np.diff(e["sr_ptr"])) > 24
    csrk.destroy(h)


# ------------------------------------------------------------------ 16-bit column offsets
def test_index_bits_follow_the_ssr_column_span():
    a = synth.stencil_3d(40, 40, 40, 27, "random_dd", 4, labels=synth.vectors.permutation(64000, 4))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.index_bits(h)
    assert ei.value.status == "ERR_STATE"
    csrk.reorder(h)
    csrk.set_sizes(h, 32, 8)
    assert csrk.index_bits(h) == 16                  # RCM: steps within a row of ~1.7K at most
    csrk.destroy(h)
    # without reordering, random labels put steps of up to ~125K columns inside rows
    a = synth.stencil_3d(50, 50, 50, 7, "random_dd", 4, labels=synth.vectors.permutation(125000, 4))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.set_sizes(h, 32, 8)
    assert csrk.index_bits(h) == 32
    csrk.destroy(h)
    # a step of 65,535 between two columns of a row fits, 65,536 does not
    for far, bits in [(65535, 16), (65536, 32)]:
        n = 70000
        rows = [[i] for i in range(n)]
        rows[0].append(far)
        rows[far].append(0)
        rp = np.array([0] + list(np.cumsum([len(r) for r in rows])), np.int32)
        ci = np.array([c for r in rows for c in sorted(r)], np.int32)
        h = csrk.create(n, rp, ci, np.ones(ci.size))
        csrk.set_sizes(h, 32, 8)
        assert csrk.index_bits(h) == bits, far
        csrk.destroy(h)


def decode_col16(e, codes, cbase):
    """Columns rebuilt from kernel 4's codes, row by row: the first code is an offset from the
    row's super-super-row cbase, every further code the step from the previous column."""
    out = np.zeros(len(codes), np.int64)
    srp, ssrp, rp = e["sr_ptr"], e["ssr_ptr"], e["rowptr"]
    for t in range(len(ssrp) - 1):
        for r in range(int(srp[ssrp[t]]), int(srp[ssrp[t + 1]])):
            p0, p1 = int(rp[r]), int(rp[r + 1])
            if p1 > p0:
                c = codes[p0:p1].astype(np.int64)
                c[0] += int(cbase[t])
                out[p0:p1] = np.cumsum(c)
    return out


@pytest.mark.parametrize("case", ["27pt_rcm", "fem_rcm", "random_empty_rows", "split_long_rows"])
def test_col16_codes_decode_to_the_columns(case):
    """Kernel 4's host coding (csrk_col16_export) rebuilt with the definition gives back every
    column of every covered row; cbase is each SSR's smallest column; split long rows carry
    no codes."""
    split = 0
    if case == "27pt_rcm":
        a, sizes = synth.stencil_3d(14, 13, 12, 27, "random_dd", 8, labels=synth.vectors.permutation(2184, 8)), (32, 4)
    elif case == "fem_rcm":
        a, sizes = synth.fem_like(9, 4), (64, 2)
    elif case == "random_empty_rows":
        a, sizes = synth.random_pattern(3000, 0.002, 9, empty_rows=150, symmetric=True), (16, 8)
    else:
        a, sizes = synth.with_dense_rows(synth.stencil_3d(11, 10, 9, 7, "random_dd", 3), 2, 600, 4), (32, 2)
        split = 400
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    csrk.reorder(h)
    if split:
        csrk.split_long_rows(h, split)
    csrk.set_sizes(h, *sizes)
    e = csrk.export(h)
    got = csrk.col16_export(h)
    covered_nnz = int(e["rowptr"][e["sr_ptr"][-1]])
    assert np.array_equal(decode_col16(e, got["codes"], got["cbase"])[:covered_nnz], e["colidx"][:covered_nnz])
    assert not got["codes"][covered_nnz:].any()
    rp, srp, ssrp = e["rowptr"], e["sr_ptr"], e["ssr_ptr"]
    for t in range(len(ssrp) - 1):
        p0, p1 = int(rp[srp[ssrp[t]]]), int(rp[srp[ssrp[t + 1]]])
        assert got["cbase"][t] == (e["colidx"][p0:p1].min() if p1 > p0 else 0)
    csrk.destroy(h)


def test_col16_export_refused_when_the_coding_does_not_fit():
    a = synth.stencil_3d(50, 50, 50, 7, "random_dd", 4, labels=synth.vectors.permutation(125000, 4))
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.col16_export(h)
    assert ei.value.status == "ERR_STATE"
    csrk.set_sizes(h, 32, 8)
    assert csrk.index_bits(h) == 32
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.col16_export(h)
    assert ei.value.status == "ERR_UNSUPPORTED"
    csrk.destroy(h)


# ------------------------------------------------------------------ long rows
def test_split_long_rows_moves_them_last():
    base = synth.stencil_3d(12, 12, 12, 7, "random_dd", 1, labels=synth.vectors.permutation(1728, 1))
    a = synth.with_dense_rows(base, 3, 900, 2)
    long_rows = set(np.nonzero(a.row_lengths() >= 500)[0].tolist())
    assert len(long_rows) == 3
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    p_rcm = csrk.reorder(h)
    assert csrk.split_long_rows(h, 500) == 3
    with pytest.raises(csrk.CsrkError) as ei:             # reordering now would mix them again
        csrk.reorder(h)
    assert ei.value.status == "ERR_STATE"
    csrk.set_sizes(h, 32, 8)
    e = csrk.export(h)
    # short rows in RCM order, then the long rows in RCM order
    expect = [p for p in p_rcm if p not in long_rows] + [p for p in p_rcm if p in long_rows]
    assert e["perm"].tolist() == expect
    assert e["sr_ptr"][-1] == a.n - 3 and e["ssr_ptr"][-1] == len(e["sr_ptr"]) - 1
    rp, ci, v = reorder.permute_loop(a.n, a.rowptr, a.colidx, a.vals, e["perm"])
    assert np.array_equal(e["rowptr"], rp) and np.array_equal(e["colidx"], ci) and np.array_equal(e["vals"], v)
    with pytest.raises(csrk.CsrkError) as ei:             # explicit pointers must stop at n - n_long
        csrk.set_pointers(h, [0, a.n], [0, 1])
    assert ei.value.status == "ERR_ARG"
    csrk.set_pointers(h, [0, a.n - 3], [0, 1])
    csrk.destroy(h)


def test_split_long_rows_arguments_and_no_long_rows():
    a = synth.stencil_2d_5pt(10, 10)
    h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.split_long_rows(h, 0)
    assert ei.value.status == "ERR_ARG"
    assert csrk.split_long_rows(h, 6) == 0                 # 5-point rows: nothing moves
    csrk.set_sizes(h, 8, 2)
    assert np.array_equal(csrk.export(h)["perm"], np.arange(a.n))
    with pytest.raises(csrk.CsrkError) as ei:
        csrk.split_long_rows(h, 3)
    assert ei.value.status == "ERR_STATE"
    csrk.destroy(h)


def test_property_random_csr_against_oracle():
    """Property-based: random CSR inputs (any size up to 120, any density, columns given
    in any order, empty rows, disconnected and nonsymmetric patterns, any SR/SSR sizes) --
    the library's RCM permutation, B = P A P^T and pointers equal the oracle's bit for bit."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(n=st.integers(1, 120), density=st.floats(0.0, 0.25), seed=st.integers(0, 2 ** 31 - 1),
               sr=st.integers(1, 40), ssr=st.integers(1, 9), shuffle=st.booleans())
    def prop(n, density, seed, sr, ssr, shuffle):
        rng = np.random.default_rng(seed)
        mask = rng.random((n, n)) < density
        rows, cols = np.nonzero(mask)
        vals = rng.standard_normal(rows.size)
        rowptr = np.zeros(n + 1, np.int64)
        np.add.at(rowptr, rows + 1, 1)
        rowptr = np.cumsum(rowptr)
        colidx = cols.astype(np.int32)
        if shuffle:                       # columns of each row in a random order
            for i in range(n):
                sl = slice(rowptr[i], rowptr[i + 1])
                p = rng.permutation(rowptr[i + 1] - rowptr[i])
                colidx[sl], vals[sl] = colidx[sl][p], vals[sl][p]
        h = csrk.create(n, rowptr.astype(np.int32), colidx, vals)
        perm = csrk.reorder(h, "rcm")
        csrk.set_sizes(h, sr, ssr)
        e = csrk.export(h)
        # the oracle takes rows with ascending columns
        order = np.lexsort((colidx, np.repeat(np.arange(n), np.diff(rowptr))))
        rp = rowptr.astype(np.int32)
        ci, vv = colidx[order], vals[order]
        ref = reorder.rcm(n, rp, ci)
        assert np.array_equal(perm, ref)
        brp, bci, bv = reorder.permute_scipy(n, rp, ci, vv, ref)
        assert np.array_equal(e["rowptr"], brp) and np.array_equal(e["colidx"], bci)
        assert np.array_equal(e["vals"].view(np.uint64), bv.view(np.uint64))
        srp, ssrp = ocsrk.fixed_pointers(n, sr, ssr)
        assert np.array_equal(e["sr_ptr"], srp) and np.array_equal(e["ssr_ptr"], ssrp)
        csrk.destroy(h)

    prop()


def test_property_bandk_random_graphs_against_oracle():
    """Property-based: Band-k on random symmetric and nonsymmetric patterns (isolated
    vertices, several components, any caps) -- the library equals the oracle bit for bit,
    and every SR / SSR respects its cap."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")
    from oracle import bandk

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(n=st.integers(1, 90), density=st.floats(0.0, 0.12), seed=st.integers(0, 2 ** 31 - 1),
               sr=st.integers(1, 12), ssr=st.integers(1, 6), symmetric=st.booleans())
    def prop(n, density, seed, sr, ssr, symmetric):
        a = synth.random_pattern(n, density, seed % 100000, symmetric=symmetric)
        h = csrk.create(a.n, a.rowptr, a.colidx, a.vals)
        perm = csrk.reorder_bandk(h, sr, ssr)
        e = csrk.export(h)
        p_ref, sr_ref, ssr_ref = bandk.bandk_py(a.n, a.rowptr, a.colidx, sr, ssr)
        assert np.array_equal(perm, p_ref)
        assert np.array_equal(e["sr_ptr"], sr_ref) and np.array_equal(e["ssr_ptr"], ssr_ref)
        assert np.all(np.diff(sr_ref) >= 1) and np.all(np.diff(sr_ref) <= sr)
        assert np.all(np.diff(ssr_ref) >= 1) and np.all(np.diff(ssr_ref) <= ssr)
        csrk.destroy(h)

    prop()


@pytest.mark.parametrize("symmetric", [False, True])
def test_rcm_large_random_patterns_bit_exact(symmetric):
    """200,000 vertices, ~8 random entries per row: the start-vertex search expands its wide
    breadth-first levels with several threads; the permutation still equals the oracle's
    (sequential) one exactly."""
    n = 200_000
    rng = np.random.default_rng(3)
    r = np.repeat(np.arange(n), rng.integers(0, 17, n))
    c = rng.integers(0, n, r.size)
    if symmetric:
        r, c = np.concatenate([r, c]), np.concatenate([c, r])
    key = np.unique(r.astype(np.int64) * n + c)
    r, c = key // n, key % n
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    colidx = c.astype(np.int32)
    h = csrk.create(n, rowptr, colidx, np.ones(colidx.size))
    perm = csrk.reorder(h, "rcm")
    assert np.array_equal(perm, reorder.rcm(n, rowptr, colidx))
    csrk.destroy(h)
