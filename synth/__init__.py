"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This package only *creates* inputs: sparsity patterns, matrix values, random vertex
labellings and vectors.  It holds none of the CSR-k method's arithmetic (no SpMV, no
reordering, no super-row construction, no precision conversion), so both sides of every
parity test can draw from it without sharing code.

The workloads stand in for the regular, symmetric-pattern matrices of the paper's
SuiteSparse suite (Sec. 5.3, Table 1: N of 1-6 M, row density 2-35, row-length variance
<= 10), which are not available here: finite-difference stencils on structured grids and
an unstructured finite-element-like point cloud.
"""
from .matrices import (CSR, stencil_2d_5pt, stencil_3d, fem_like, random_pattern, with_dense_rows,
                       relabel, batch_specs, batch_matrix)
from .vectors import uniform_vector, uniform_block

__all__ = ["CSR", "stencil_2d_5pt", "stencil_3d", "fem_like", "random_pattern", "with_dense_rows", "relabel",
           "batch_specs", "batch_matrix", "uniform_vector", "uniform_block"]
