"""FP64 CPU oracle for CSR-k SpMV — TEST INFRASTRUCTURE, not part of the product.

Plain, slow, obviously correct implementations of what the CSR-k hot path computes, each
function citing the passage of Lane & Booth, "Heterogeneous Sparse Matrix-Vector
Multiplication via Compressed Sparse Row Format" (arXiv 2203.05096) that it follows.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library under ``paper_2203_05096_gb300/``,
and the product never calls it.

Modules
    spmv       y = alpha*A*x + beta*y (plain CSR, CSR-3 loop nest, SpMM, sampled rows)
    reorder    reverse Cuthill-McKee, B = P A P^T, bandwidth
    csrk       super-row / super-super-row pointer arrays
    precision  FP64 -> FP32 / BF16 round-to-nearest-even
    cg         FP64 and mixed-precision conjugate gradients
    tuning     the paper's constant-time super-row size model
    native     the plain C versions used at full problem sizes

Pin status (what fixes each function other than itself) is listed in each module's
docstring; every function here is pinned.
"""
