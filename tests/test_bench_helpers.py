"""The benchmark's byte accounting and timing aggregation (host only): the algorithmic
bytes behind the reported roofline, worked out here by hand for the 128^3 stencils."""
import bench


def test_algorithmic_bytes_27pt_128cubed_by_hand():
    n, nnz = 128 ** 3, 55_742_968
    nsr = n // 32                     # SR = 32 rows
    nssr = nsr // 4                   # SSR = 4 SRs
    # FP64 values + int32 columns: 12 B per nonzero; rowptr n+1, sr_ptr nsr+1 (int32);
    # a 32-byte descriptor per SSR; x read and y written once (8 B each); the permutation
    # read once by the fused unpermute
    want = 12 * nnz + 4 * (n + 1) + 4 * (nsr + 1) + 32 * nssr + 16 * n + 4 * n
    assert bench.alg_bytes_spmv(n, nnz, nsr, nssr) == want == 720_033_704
    # kernel 4 stores a 2-byte code per nonzero instead of the 4-byte column
    k4 = bench.alg_bytes_spmv(n, nnz, nsr, nssr, col_bytes=bench.col_bytes_of({"kernel": 4}))
    assert k4 == want - 2 * nnz == 608_547_768
    # in the reordered numbering (no permutation read)
    assert bench.alg_bytes_spmv(n, nnz, nsr, nssr, fused_unpermute=False) == want - 4 * n


def test_algorithmic_bytes_7pt_and_fp32_values():
    n, nnz = 128 ** 3, 14_581_760
    nsr, nssr = n // 32, n // 256
    fp64 = bench.alg_bytes_spmv(n, nnz, nsr, nssr)
    fp32 = bench.alg_bytes_spmv(n, nnz, nsr, nssr, val_bytes=4)
    assert fp64 - fp32 == 4 * nnz
    fp32x = bench.alg_bytes_spmv(n, nnz, nsr, nssr, val_bytes=4, x_bytes=4)
    assert fp32 - fp32x == 8 * n            # x and y 4 bytes narrower each


def test_whole_job_rate_and_replicas():
    # N replicas each doing W units in the slowest rank's time t: N * W / t
    assert bench.whole_job_rate(4, 1.0e9, 2.0) == 4 * 1.0e9 / 2.0e-3
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_algorithmic_bytes_window_kernel_by_hand():
    # kernels 5 / 6: 2-byte window codes, plus the run table (8 bytes a run, 4 bytes of run
    # pointer per SSR and one more) and, when the rows' length order is staged, 2 bytes a row
    n, nnz = 128 ** 3, 55_742_968
    nsr, nssr = n // 32, n // 64
    base = bench.alg_bytes_spmv(n, nnz, nsr, nssr, col_bytes=2)
    assert bench.col_bytes_of({"kernel": 5}) == bench.col_bytes_of({"kernel": 6}) == 2
    assert bench.alg_bytes_spmv(n, nnz, nsr, nssr, col_bytes=2, runs=300_000) == base + 8 * 300_000 + 4 * (nssr + 1)
    assert bench.alg_bytes_spmv(n, nnz, nsr, nssr, col_bytes=2, runs=300_000, row_order=True) == \
        base + 8 * 300_000 + 4 * (nssr + 1) + 2 * n
