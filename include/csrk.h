/*
 * csrk.h -- C ABI of the GB300 CSR-k sparse matrix-vector library.
 *
 * The library computes y = alpha*A*x + beta*y (and the k-right-hand-side form
 * Y = alpha*A*X + beta*Y) for a square sparse matrix A held in CSR-k form: plain CSR
 * (row_ptr, col_idx, vals), its rows renumbered by a bandwidth-reducing permutation, and
 * the rows grouped into super-rows and super-super-rows described by two extra pointer
 * arrays (Lane & Booth, arXiv 2203.05096: problem statement Sec. 1; CSR Sec. 2.1;
 * CSR-k / CSR-3 and its pointer arrays Sec. 2.2 and Fig. 1; the GPU mapping of
 * super-super-rows to thread blocks and super-rows to the next thread level Sec. 3).
 *
 * Conventions shared by every entry point
 *   - Every function returns a csrk_status.  CSRK_OK is 0.  csrk_last_error() returns a
 *     message for the calling thread's last failure (static storage, valid until that
 *     thread's next call).  No C++ exception crosses this boundary.
 *   - Host arrays passed in are copied; the caller keeps ownership and may free them as
 *     soon as the call returns.
 *   - Vector arguments of the compute calls are DEVICE pointers owned by the caller
 *     (e.g. PyTorch tensors), aligned to their element size, unless CSRK_HOST_VECTORS is
 *     given.  x and y (X and Y) must not overlap.
 *   - Device work is enqueued on the given CUDA stream (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream) without synchronising the host, except where a
 *     function says otherwise.  Errors found on the host are reported synchronously.
 *     Device-side failures (a bounded wait that ran out) set a status word on the device;
 *     csrk_device_status() reads it.
 *   - The library owns all device copies of A and its own scratch vectors.  It allocates
 *     them on first use (the first compute call after csrk_set_sizes / csrk_set_pointers,
 *     or the first call that needs a larger scratch size) on the device current at that
 *     time; later calls must be made with the same device current.
 *   - Life cycle: csrk_create -> [csrk_reorder | csrk_reorder_bandk] ->
 *     [csrk_split_long_rows] -> csrk_set_sizes or csrk_set_pointers (Band-k installs its
 *     own) -> compute calls ...; csrk_set_sizes may be called again (the pointer arrays
 *     and device copies are rebuilt); csrk_reorder after the pointers exist returns
 *     CSRK_ERR_STATE.  A handle is not thread-safe: one thread uses it at a time.
 *   - Environment: CSRK_TUNE_CACHE names a file that keeps the autotuner's choices across
 *     processes (read once per process, appended to after each new tuning; one line per
 *     choice: a whitespace-free key of the matrix shape, dtype and device, then SR, SSR,
 *     kernel, lanes, unroll, warps, stages, blocks per SM and the measured microseconds);
 *     CSRK_BATCH_ITEM_BYTES overrides the batched kernel's item size;
 *     CSRK_FAULT (tests) makes host-side steps fail as if their CUDA call had: "alloc"
 *     (device allocations, CSRK_ERR_ALLOC), "h2d" (matrix uploads, CSRK_ERR_CUDA), "tune"
 *     (the autotuner, CSRK_ERR_CUDA), comma-separated.
 *   - The host stages (create, reorder, pointers, upload, autotune, solvers) are marked
 *     with NVTX ranges named "csrk ...".
 */
#ifndef CSRK_H
#define CSRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct csrk_matrix* csrk_handle;
typedef struct csrk_batch* csrk_batch_handle;

/* Storage precision of A's values on the device.  Narrowing from the FP64 input rounds
 * to nearest, ties to even, once and directly from FP64 (BF16 never through FP32). */
typedef enum { CSRK_F64 = 0, CSRK_F32 = 1, CSRK_BF16 = 2 } csrk_dtype;

typedef enum {
    CSRK_OK = 0,
    CSRK_ERR_ARG = 1,          /* bad argument: NULL where not allowed, size out of range */
    CSRK_ERR_MATRIX = 2,       /* invalid CSR: rowptr not monotone or not starting at 0,
                                  column out of [0, n), repeated column in a row,
                                  nnz >= 2^31 */
    CSRK_ERR_STATE = 3,        /* call out of order for this handle's life cycle */
    CSRK_ERR_ALLOC = 4,        /* host or device allocation failed */
    CSRK_ERR_CUDA = 5,         /* a CUDA runtime call failed (message has the CUDA error) */
    CSRK_ERR_UNSUPPORTED = 6,  /* valid request this build does not implement */
    CSRK_ERR_TIMEOUT = 7,      /* a device-side bounded wait ran out (see csrk_device_status) */
    CSRK_ERR_NOT_CONVERGED = 8 /* an iterative solve stopped at maxit above its tolerance */
} csrk_status;

/* Flags of the compute calls (bitwise OR). */
#define CSRK_VEC_PERMUTED 1u  /* x/y already in the reordered numbering: skip the device
                                 permute of x and unpermute of y */
#define CSRK_ACC_F32      2u  /* accumulate row sums in FP32 (default FP64) */
#define CSRK_X_F32        4u  /* x and y are FP32 (default FP64) */
#define CSRK_HOST_VECTORS 8u  /* x and y are HOST pointers: the call copies x in and y out
                                 through its own device scratch and returns after the
                                 copy of y has completed (synchronous).  A page-locked x
                                 (cudaHostAlloc / cudaHostRegister, mapped) that needs
                                 permuting is read by the permute kernel directly over the
                                 host link, one pass instead of copy + permute; the library
                                 then keeps the inverse permutation on the device (4n bytes) */
#define CSRK_X_PERMUTED  16u  /* SpMV only: x is already in the reordered numbering (e.g.
                                 from csrk_permute), y is in the input numbering; the kernel
                                 writes row r's result to y[perm[r]] directly */

/* Reordering methods for csrk_reorder. */
#define CSRK_REORDER_NONE 0   /* keep the input numbering (perm = identity) */
#define CSRK_REORDER_RCM  1   /* reverse Cuthill-McKee of the symmetrised pattern */

/* ---------------------------------------------------------------------------------
 * csrk_create: take a square n x n CSR matrix (Sec. 2.1).
 *   n       rows = columns, 0 <= n < 2^31
 *   rowptr  host, n+1 entries, rowptr[0] == 0, non-decreasing; nnz = rowptr[n] < 2^31
 *   colidx  host, nnz column indices in [0, n); a row's columns may come in any order
 *           (they are sorted, carrying their values) but may not repeat
 *   vals    host, nnz FP64 values (NaN / Inf are stored as given)
 *   dtype   storage precision used by csrk_spmv / csrk_spmm
 *   out     receives the handle (NULL on failure)
 * Errors: CSRK_ERR_ARG, CSRK_ERR_MATRIX (with the first offending row in the message),
 * CSRK_ERR_ALLOC.  Host only; touches no GPU.
 * --------------------------------------------------------------------------------- */
int csrk_create(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                csrk_dtype dtype, csrk_handle* out);

/* csrk_reorder: renumber rows and columns by a bandwidth-reducing permutation so that a
 * super-row's rows share x entries (Sec. 2.1 RCM; for the paper's own Band-k ordering,
 * Listing 2, see csrk_reorder_bandk).  B = P A P^T with B[i][j] = A[perm[i]][perm[j]],
 * each row's columns ascending.
 *   method    CSRK_REORDER_NONE or CSRK_REORDER_RCM
 *   perm_out  optional host array of n entries receiving perm (perm[new] = old)
 * RCM reading: graph of A + A^T without self-loops; each component starts at the
 * unvisited vertex of least degree (smallest index on ties), moved by the George-Liu
 * pseudo-peripheral search (least-degree vertex of the last BFS level, smallest index on
 * ties, while the level structure deepens, at most 8 moves); Cuthill-McKee order with
 * children by (degree, index); the whole sequence reversed.
 * Errors: CSRK_ERR_STATE after the pointers exist, CSRK_ERR_ARG, CSRK_ERR_ALLOC.
 * Host only. */
int csrk_reorder(csrk_handle h, int method, int32_t* perm_out);

/* csrk_reorder_bandk: the Band-k ordering for k = 3 (Sec. 2.2, Listing 2, Fig. 2): the
 * rows are coarsened into super-rows of at most sr rows and those into super-super-rows
 * of at most ssr super-rows, the coarse levels are put in weighted bandwidth-limiting
 * order and expanded again; the renumbering and the (variable) pointer arrays are
 * installed together, so no csrk_set_sizes / csrk_set_pointers call is needed after it.
 *   sr, ssr   caps, >= 1
 *   perm_out  optional host array of n entries receiving perm (perm[new] = old),
 *             composed with any earlier csrk_reorder
 * Reading (the paper names neither coarsening nor weights): graph of A + A^T without
 * self-loops, edge weights 1.  Coarsen: walk the Cuthill-McKee sequence (csrk_reorder's
 * rules, not reversed); each unassigned vertex seeds an aggregate grown breadth-first
 * (neighbours by degree, index) to the cap; the coarse edge weight is the number of fine
 * edges between two aggregates.  The coarsest graph is ordered by weighted reverse
 * Cuthill-McKee (neighbours by weight descending, degree, index).  Expansion orders each
 * coarse node's members by a breadth-first walk inside the node (same neighbour key) from
 * the member most connected to what is already placed, else from the member farthest from
 * the node's boundary (ties: smaller outside weight, index), else from the node's
 * pseudo-peripheral vertex.  csrk_set_sizes(h, 0, 0) afterwards tunes the launch shape
 * only and keeps these pointers; csrk_set_sizes with explicit sizes replaces them (the
 * row order stays).
 * Errors: CSRK_ERR_STATE after the pointers exist, CSRK_ERR_ARG, CSRK_ERR_ALLOC.
 * Host only. */
int csrk_reorder_bandk(csrk_handle h, int32_t sr, int32_t ssr, int32_t* perm_out);

/* csrk_split_long_rows: the irregular-matrix path (Sec. 7 names the row mapping of
 * irregular matrices as future work).  Rows with at least min_len stored entries are moved
 * behind all other rows (a symmetric renumbering composed with any earlier reorder, each
 * group keeping its order) and left out of the super-rows: the pointer arrays built
 * afterwards cover the first n - n_long rows only.  Every SpMV / SpMM / CG launch then
 * also computes the long rows in segments of 2,048 entries, one warp per segment and
 * right-hand side, and sums each row's segment partials in segment order (deterministic).
 *   min_len   threshold, >= 1
 *   n_long    optional: receives the number of rows moved
 * Call after csrk_reorder (CSRK_ERR_STATE if the pointer arrays exist; csrk_reorder and
 * csrk_reorder_bandk refuse a handle with split rows).  Batches refuse such handles.
 * Host only. */
int csrk_split_long_rows(csrk_handle h, int32_t min_len, int32_t* n_long);

/* csrk_set_sizes: build sr_ptr / ssr_ptr for fixed sizes (Sec. 2.2): every super-row
 * holds sr rows and every super-super-row ssr super-rows, the last of each possibly
 * fewer.  sr = ssr = 0 asks the autotuner to choose (it times candidates on the GPU,
 * so that form needs a device; the choice is cached per matrix shape, see
 * csrk_tuned_config).  Any other non-positive size is CSRK_ERR_ARG.
 * Host only for explicit sizes. */
int csrk_set_sizes(csrk_handle h, int32_t sr, int32_t ssr);

/* csrk_index_bits: 16 when the columns fit kernel 4's delta coding -- within each row, the
 * first column minus its super-super-row's smallest column, and every step from one column
 * to the next, at most 65,535 -- then kernel 4 (csrk_set_config) reads 2 bytes per nonzero
 * instead of 4; else 32.  Needs the pointer arrays (CSRK_ERR_STATE before).  Host only. */
int csrk_index_bits(csrk_handle h, int32_t* bits);

/* csrk_col16_export: kernel 4's delta-coded columns for the current pointers, built on the
 * host (no device needed, nothing uploaded; for tests and inspection).
 *   codes  nnz entries (reordered matrix, csrk_export's order): a row's first entry holds
 *          its column minus its super-super-row's cbase, every further entry the step
 *          from the previous column; entries of split long rows are 0
 *   cbase  nssr entries: the smallest column of each super-super-row
 * Either may be NULL.  Errors: CSRK_ERR_ARG, CSRK_ERR_STATE (no pointers yet),
 * CSRK_ERR_UNSUPPORTED (csrk_index_bits would report 32), CSRK_ERR_ALLOC. */
int csrk_col16_export(csrk_handle h, uint16_t* codes, int32_t* cbase);

/* csrk_set_pointers: give the super-row and super-super-row pointer arrays explicitly
 * (variable sizes, e.g. Fig. 1: sr_ptr = {0,2,5,7,9}, ssr_ptr = {0,2,4}).
 *   nsr     number of super-rows; sr_ptr has nsr+1 entries, sr_ptr[0] = 0,
 *           sr_ptr[nsr] = n (n - n_long after csrk_split_long_rows), non-decreasing
 *   nssr    number of super-super-rows; ssr_ptr has nssr+1 entries, ssr_ptr[0] = 0,
 *           ssr_ptr[nssr] = nsr, non-decreasing
 * Errors: CSRK_ERR_ARG for arrays that break these rules.  Host only. */
int csrk_set_pointers(csrk_handle h, int32_t nsr, const int32_t* sr_ptr, int32_t nssr,
                      const int32_t* ssr_ptr);

/* csrk_spmv: y = alpha*A*x + beta*y with A's stored dtype -- the paper's problem
 * statement y = A x over the CSR-k arrays (Sec. 1; the CSR-3 loop nest of Listing 1, whose
 * GPU forms are Listings 3 and 4, Sec. 3), with the BLAS scaling by alpha and beta added.
 * Each row's result is its stored entries' products summed in stored order (FP64 kernels);
 * the row grouping into super-rows and super-super-rows only decides who computes it.
 *   x, y    n entries, FP64 (FP32 with CSRK_X_F32), in the input numbering unless
 *           CSRK_VEC_PERMUTED; device pointers unless CSRK_HOST_VECTORS
 *   beta    0 means y is write-only (its old contents, even NaN, are not read)
 *   flags   CSRK_VEC_PERMUTED | CSRK_ACC_F32 | CSRK_X_F32 | CSRK_HOST_VECTORS
 *   stream  cudaStream_t (NULL = default stream)
 * FP64 values with CSRK_X_F32 are CSRK_ERR_UNSUPPORTED.  Without CSRK_VEC_PERMUTED the
 * call permutes x into library scratch (x_p[i] = x[perm[i]]) and runs the CSR-k kernel,
 * which stores each row's result straight to its place in the input numbering,
 * y[perm[i]] (and reads y there when beta != 0).  Errors: CSRK_ERR_STATE before the pointers
 * exist, CSRK_ERR_ARG, CSRK_ERR_ALLOC, CSRK_ERR_CUDA. */
int csrk_spmv(csrk_handle h, double alpha, const void* x, double beta, void* y,
              unsigned flags, void* stream);

/* csrk_spmm: Y = alpha*A*X + beta*Y for k right-hand sides, 1 <= k <= 64: the product of
 * Sec. 1 applied to k vectors at once over the same CSR-k arrays (Listing 1's loop nest,
 * a row's k sums formed together so A is read once); not in the paper, which multiplies
 * one vector.
 *   X       n x k, row-major, leading dimension ldx >= k (entry (i,c) at X[i*ldx + c])
 *   Y       n x k, row-major, leading dimension ldy >= k
 * Same flags, dtypes, numbering and errors as csrk_spmv; column c of Y is exactly what
 * csrk_spmv would give for column c of X, up to the order of floating-point additions. */
int csrk_spmm(csrk_handle h, int32_t k, double alpha, const void* X, int64_t ldx,
              double beta, void* Y, int64_t ldy, unsigned flags, void* stream);

/* csrk_permute: move a dense n x k block between the input numbering and the reordered
 * numbering on the device (the permute / unpermute steps that csrk_spmv performs around
 * its kernel when CSRK_VEC_PERMUTED is absent).
 *   direction 0: out[i][c] = in[perm[i]][c]  (input numbering -> reordered)
 *   direction 1: out[perm[i]][c] = in[i][c]  (reordered -> input numbering)
 *   in, out    device pointers, row-major, leading dimensions ldi, ldo >= k; FP64, or FP32
 *              with CSRK_X_F32 in flags; they must not overlap
 * With no reordering (perm = identity) this is a plain strided copy.  Errors:
 * CSRK_ERR_STATE before the pointers exist, CSRK_ERR_ARG, CSRK_ERR_CUDA. */
int csrk_permute(csrk_handle h, int direction, int32_t k, const void* in, int64_t ldi,
                 void* out, int64_t ldo, unsigned flags, void* stream);

/* csrk_cg: solve A x = b for symmetric positive definite A by conjugate gradients on the
 * CSR-k form (the paper names CG as the SpMV's consumer: Sec. 1, 5.3, 8, 9), with
 * x0 = 0 and the Hestenes-Stiefel recurrences.
 *   b, x          DEVICE FP64 vectors of n entries, input numbering unless
 *                 CSRK_VEC_PERMUTED; x receives the solution
 *   rtol          stop when ||b - A x|| <= rtol ||b|| (the FP64 residual)
 *   maxit         iteration limit (>= 1)
 *   inner         CSRK_F64: plain FP64 CG (stops on the recursive residual, then checks
 *                 the true one and resumes from it if needed); CSRK_F32 / CSRK_BF16: mixed
 *                 precision -- q = A_lo p with values stored in that precision, p rounded to
 *                 FP32 and FP32 accumulation, while vectors, dot products, alpha and beta
 *                 stay FP64
 *   replace_every mixed mode: recompute r = b - A x in FP64 every this many iterations
 *                 (earlier once the recursive residual passes rtol/2)
 *   restart       mixed mode: 0 keeps the direction across a replacement (reliable update)
 *                 unless the recomputed residual exceeds twice the recursive one or the
 *                 cycle diverged; 1 always restarts p = r (defect correction)
 *   flags         0 or CSRK_VEC_PERMUTED
 *   iters, relres optional outputs: iterations done and the final true relative residual
 *   stream        cudaStream_t; the call returns after the solve (it reads a 64-byte state
 *                 block from the device once per cycle)
 * Iterations are recorded once into a CUDA graph (one cycle per graph) and replayed; all
 * scalars stay on the device.  The first call allocates the solver workspace (7 vectors).
 * Returns CSRK_OK when converged, CSRK_ERR_NOT_CONVERGED at maxit or on breakdown
 * (p.q <= 0), with x holding the last iterate. */
int csrk_cg(csrk_handle h, const double* b, double* x, double rtol, int32_t maxit,
            csrk_dtype inner, int32_t replace_every, int32_t restart, unsigned flags,
            int32_t* iters, double* relres, void* stream);

/* ---------------------------------------------------------------- batches
 * Many matrices of uneven size handled by single launches (the library's batched mode;
 * the paper runs one matrix at a time).  A batch refers to its handles' device forms:
 * keep the handles alive and leave their sizes and pointers unchanged while the batch
 * exists.  All batched vectors are FP64, row-major n_i x k_i blocks (leading dimension
 * k_i), in each matrix's reordered numbering (csrk_permute moves vectors there). */

/* csrk_batch_create: build the work list of a batch.
 *   hs     count handles, each with its pointer arrays set (sizes or explicit); any
 *          value dtype; all on the current device
 *   k      right-hand sides per matrix, 1..64
 * Each matrix is cut into items, runs of whole super-rows holding at most 24 KB of
 * staged data (rowptr, colidx and value slices rounded out to 16 bytes, counted with 8-byte
 * values so that the FP64 operator of any matrix fits; at least one super-row each; the
 * environment variable CSRK_BATCH_ITEM_BYTES overrides the 24 KB),
 * grouped four to a tile; tiles are queued matrix by matrix (matrices by decreasing work,
 * each matrix's tiles in row order).  When two stages of the largest item do not fit a
 * block's shared memory (half an SM), the batch uses a direct-load kernel over tiles of
 * about 32K nonzeros (whole super-super-rows) instead.
 * Uploads the handles' device forms if needed.  Errors: CSRK_ERR_ARG, CSRK_ERR_STATE,
 * CSRK_ERR_ALLOC, CSRK_ERR_CUDA. */
int csrk_batch_create(const csrk_handle* hs, int32_t count, const int32_t* k,
                      csrk_batch_handle* out);

/* csrk_batch_spmm: Y_i = alpha A_i X_i + beta Y_i for every matrix of the batch in one
 * persistent launch (blocks take tiles from an atomic counter; no block waits on another;
 * in each block a producer warp stages the tiles' items into shared memory with bulk
 * copies while the other warps compute).  Every wait inside the kernel is bounded (2 s);
 * one that gives up sets a bit of the batch's status word (csrk_batch_device_status).
 *   X, Y    host arrays of count DEVICE pointers (X[i], Y[i]: n_i x k_i blocks, FP64, or
 *           FP32 with CSRK_X_F32)
 *   flags   CSRK_VEC_PERMUTED: FP64 vectors, FP64 accumulation, each matrix's stored values;
 *           CSRK_VEC_PERMUTED | CSRK_X_F32 | CSRK_ACC_F32: FP32 vectors and FP32
 *           accumulation, FP32 values (FP64-stored matrices use their values rounded to
 *           FP32; BF16 stays BF16) -- needs the staged kernel (else CSRK_ERR_UNSUPPORTED)
 * Blocks on 16-byte boundaries with a power-of-two k gather k/VW-lane groups of VW columns
 * with one vector load per nonzero (VW = 2 for FP64, 4 for FP32 with k >= 4).
 * A call with the same pointers as the previous one reuses the device-side table (one
 * launch, no copy); new pointers cost one small host-to-device copy first. */
int csrk_batch_spmm(csrk_batch_handle b, double alpha, const void* const* X, double beta,
                    void* const* Y, unsigned flags, void* stream);

/* csrk_batch_cg: independent CG solves A_i x = b for every (matrix, right-hand side) of the
 * batch, FP64 vectors and scalars, q = A_i p with each matrix's stored values (FP32-stored
 * matrices give FP32-valued operators).  Exactly `iters` iterations run, recorded once in
 * a CUDA graph (re-recorded when iters changes) and replayed; a system whose recursive
 * residual reaches rtol stops updating.
 *   B, X       host arrays of count DEVICE pointers (n_i x k_i FP64 blocks, reordered
 *              numbering); X receives the solutions (x0 = 0)
 *   k_i        must be a power of two <= 32
 *   relres     optional host array of (sum of k_i) FP64: final true ||b - A x|| / ||b||
 *              per system, systems ordered by matrix then column
 *   iters_done optional host array of (sum of k_i): iterations each system performed
 * Synchronous: returns when the results are on the host. */
int csrk_batch_cg(csrk_batch_handle b, const double* const* B, double* const* X,
                  int32_t iters, double rtol, double* relres, int32_t* iters_done,
                  void* stream);

/* csrk_batch_cg_solve: independent CG solves A_i x = b for every (matrix, right-hand side)
 * of the batch to a relative residual, in FP64 or mixed precision -- the batched
 * counterpart of csrk_cg.  The operator is each matrix's FP64 values (the handle's input
 * values, whatever its stored dtype).
 *   B, X          host arrays of count DEVICE pointers (n_i x k_i FP64 blocks, reordered
 *                 numbering); X receives the solutions (x0 = 0)
 *   rtol          a system has converged when ||b - A x|| <= rtol ||b||, A in FP64 (> 0)
 *   maxit         iteration limit per system, rounded up to whole cycles
 *   inner         CSRK_F64: plain FP64 CG, q = A p with FP64 values; a system whose
 *                 recursive residual meets rtol stops and is verified at the cycle's end.
 *                 CSRK_F32 / CSRK_BF16: mixed precision -- q = A_lo p32 with the values
 *                 rounded to that precision, p rounded to FP32 and FP32 accumulation, while
 *                 vectors, dot products, alpha and beta stay FP64; at every cycle's end
 *                 r = b - A x in FP64 (reliable update); a system whose recursive residual
 *                 passes rtol/2 waits for that check.  Needs the staged SpMM kernel.
 *   replace_every iterations per cycle (one CUDA graph, recorded once and replayed); the
 *                 true residual of every running system is computed at each cycle's end
 *   restart       mixed mode: 0 keeps p across a replacement unless the recomputed residual
 *                 exceeds twice the recursive one or the cycle diverged (recursive residual
 *                 up tenfold: the system stops until the cycle's end); 1 always restarts p = r
 *   relres        optional host array (sum k_i): last true relative residual per system
 *   iters_done    optional host array (sum k_i): iterations per system
 *   cycles        optional: cycles run (each reads one 4-byte counter back to the host)
 * Systems are ordered by matrix, then column.  Returns CSRK_OK when every system
 * converged, CSRK_ERR_NOT_CONVERGED otherwise (maxit reached or p.q <= 0), X holding the
 * last iterates.  k_i must be a power of two <= 32.  Synchronous. */
int csrk_batch_cg_solve(csrk_batch_handle b, const double* const* B, double* const* X,
                        double rtol, int32_t maxit, int inner, int32_t replace_every,
                        int restart, double* relres, int32_t* iters_done, int32_t* cycles,
                        void* stream);

/* csrk_batch_info: matrices, systems (sum of k_i), tiles, and elements of one
 * concatenated vector (sum of n_i k_i); any pointer may be NULL. */
int csrk_batch_info(csrk_batch_handle b, int32_t* nmat, int32_t* nsys, int32_t* ntiles,
                    int64_t* total);

/* csrk_batch_plan: the staged kernel's plan -- items (0 when the direct-load kernel is
 * used), shared-memory stages per block (0 likewise) and bytes per stage; any pointer may
 * be NULL. */
int csrk_batch_plan(csrk_batch_handle b, int32_t* items, int32_t* stages, int32_t* stage_bytes);

/* csrk_batch_device_status: read the batch's device status word (synchronous copy):
 * 0 = no error; bit 0 = a bounded wait in the batched SpMM kernel gave up (the launch's
 * results are incomplete); bit 1 = an item larger than a stage was skipped.  Sticky. */
int csrk_batch_device_status(csrk_batch_handle b, int32_t* status);

/* csrk_batch_destroy: free the batch (not its handles) after synchronising the device.
 * NULL is a no-op. */
int csrk_batch_destroy(csrk_batch_handle b);

/* csrk_destroy: free the handle and every host and device buffer it owns, after
 * synchronising the device.  NULL is a no-op. */
int csrk_destroy(csrk_handle h);

/* ---------------------------------------------------------------- inspection */

/* csrk_info: sizes of the current form; any output pointer may be NULL.
 *   n, nnz; nsr / nssr (0 before the pointers exist); sr / ssr the fixed sizes
 *   (0 after csrk_set_pointers); dtype. */
int csrk_info(csrk_handle h, int32_t* n, int64_t* nnz, int32_t* nsr, int32_t* nssr,
              int32_t* sr, int32_t* ssr, int32_t* dtype);

/* csrk_export: copy the host form out (any pointer may be NULL; arrays sized from
 * csrk_info): perm (n), the reordered CSR rowptr (n+1) / colidx (nnz) / vals (nnz, FP64),
 * sr_ptr (nsr+1), ssr_ptr (nssr+1).  The reordered arrays are plain CSR (Sec. 2.2: a
 * CSR-k matrix stays readable by CSR consumers). */
int csrk_export(csrk_handle h, int32_t* perm, int32_t* rowptr, int32_t* colidx,
                double* vals, int32_t* sr_ptr, int32_t* ssr_ptr);

/* csrk_export_values: the stored device-dtype values, in the reordered order, as the
 * host converts them: dtype CSRK_F64 -> double[nnz], CSRK_F32 -> float[nnz],
 * CSRK_BF16 -> uint16_t[nnz] bit patterns.  Host only. */
int csrk_export_values(csrk_handle h, csrk_dtype dtype, void* out);

/* csrk_model_sizes: the paper's constant-time size model (Sec. 4.1) for row density
 * rdensity = nnz / n: arch 0 = Volta, 1 = Ampere coefficients; outputs the
 * super-super-row size *ssrs and super-row size *srs after the rdensity case rules.
 * The library uses it only to seed its autotuner. */
int csrk_model_sizes(double rdensity, int arch, int32_t* ssrs, int32_t* srs);

/* csrk_xwin_info: the x windows of kernels 5 and 6 for the current pointers (built and
 * uploaded on this first ask if needed, on the current device).  *available = 1 when
 * every super-super-row's window fits the 16-bit window offsets (at most 65,536
 * elements), then *runs = the number of contiguous runs of x copied per SpMV over all
 * super-super-rows (each costs one 8-byte entry of the run table), *max_window = the
 * longest window in elements (a multiple of 4) and *row_order = 1 when the kernels hand
 * each super-super-row's rows to warp passes in order of length (built when that saves at
 * least 5 % of the passes' FP64 instruction slots: rows of unequal length; 2 bytes per row
 * more per SpMV).  Any output pointer may be NULL.  Errors: CSRK_ERR_ARG, CSRK_ERR_STATE
 * (no pointers yet), CSRK_ERR_CUDA. */
int csrk_xwin_info(csrk_handle h, int32_t* available, int64_t* runs, int32_t* max_window,
                   int32_t* row_order);

/* csrk_xwin_export: the x windows and the rows' length order that csrk_xwin_info
 * describes, built on the host for the current pointers (no device needed, nothing
 * uploaded; for tests and inspection).  Outputs (any may be NULL):
 *   *available  1 when every super-super-row's window fits the 16-bit offsets, else 0
 *               (then only ord and slots are written)
 *   *nruns      runs over all super-super-rows
 *   wptr        nssr + 1 entries: SSR t's runs are entries wptr[t] .. wptr[t+1]-1 of win
 *   win         2 * nruns entries: per run its first element of x (a multiple of 4, in the
 *               reordered numbering) and its offset in the window (runs of 4-element blocks
 *               of the SSR's columns; runs at most 2 blocks apart are merged)
 *   cover       nssr entries: elements of x the SSR's runs cover (its last run may end at n)
 *   codes       nnz entries: per stored entry (reordered matrix, csrk_export's order) the
 *               window offset of its column; entries of split long rows are 0
 *   ord         one entry per row the super-rows cover: position i of an SSR starting at
 *               row r0 holds row r0 + ord[i] (rows by decreasing length, ties in row order)
 *   slots       2 entries: FP64 issue slots of all warp passes (per pass: its longest row)
 *               in the natural and in the length order; the kernels use the order when it
 *               saves at least 5 %
 * Errors: CSRK_ERR_ARG, CSRK_ERR_STATE (no pointers yet), CSRK_ERR_ALLOC. */
int csrk_xwin_export(csrk_handle h, int32_t* available, int64_t* nruns, int32_t* wptr, int32_t* win,
                     int32_t* cover, uint16_t* codes, uint16_t* ord, int64_t* slots);

/* csrk_tuned_config: the launch configuration the handle will use (any pointer may be
 * NULL):
 *   kernel   0 = TMA-staged super-super-row kernel, 1 = direct-load kernel, 2 / 3 = the
 *            same for FP64 handles with the values stored as (hi, lo) FP32 pairs and the
 *            row sums kept as FP32 pairs: FP64 accuracy (per entry within ~7e-13 of
 *            sum |a_ij x_j| for rows up to 48 entries) on the FP32 pipes, which on GB300
 *            run 58x the FP64 FMA rate.  Available when every value is 0 or has magnitude
 *            in [2^-39, 2^60] and no row exceeds 48 entries; x entries outside that range
 *            are multiplied in FP64 individually.  SpMV only (SpMM uses 0 / 1);
 *            4 = TMA-staged with delta-coded 16-bit columns (csrk_index_bits = 16;
 *            lanes 1, unroll 4, 8 or 16; SpMV only, SpMM uses 0): 12 -> 10 bytes per FP64
 *            nonzero, results identical to kernel 0;
 *            5 = TMA-staged with each super-super-row's x window in shared memory: the
 *            producer warp also copies the runs of x (aligned blocks of 4 elements) that
 *            the SSR's columns fall in, and 16-bit column codes index that window, so the
 *            consumers read x from shared memory instead of gathering it from L2 (10 bytes
 *            per FP64 nonzero from HBM, results identical to kernel 0).  Available when
 *            every SSR's window holds at most 65,536 elements and the SSRs with their
 *            windows fit two shared-memory stages; needs a 16-byte aligned x (a tuned
 *            kernel 5 gives way to kernel 4 or 0 for a caller's x that is not); lanes 1,
 *            unroll 4, 8 or 16; SpMV only, SpMM uses 0;
 *            6 = kernel 5 for FP64 handles with kernel 2's arithmetic: values stored as
 *            (hi, lo) FP32 pairs, x split into FP32 pairs by a pass fused with its permute
 *            (or of its own for vectors already in the reordered numbering), the windows
 *            hold the split x and the row sums are FP32 pairs on the FP32 pipes, so a
 *            nonzero costs no FP64 instruction (GB300 issues FP64 at about 1/64 of the
 *            FP32 rate).  Same availability as kernels 2 and 5 together; per entry within
 *            ~7e-13 of sum |a_ij x_j|; a launch whose x has an element outside the pair
 *            range stages FP64 x and multiplies in FP64
 *   lanes    lanes cooperating on one row (SpMV): 1, 2, 4, 8 or 32
 *   unroll   x gathers a lane issues before consuming them; compiled (lanes, unroll)
 *            pairs: (1,4) (1,8) (1,16) (1,32) (2,8) (2,16) (4,8) (8,8) (32,4)
 *   warps    consumer warps per thread block (1..16)
 *   stages   shared-memory pipeline depth of the TMA kernel (0 = as many as fit)
 *   ctas     thread blocks per SM (TMA kernel), 1-8 (never more than fit at once); 0 = auto:
 *            2 when two stages fit, else 1
 * Once the pointer arrays exist and a device has been used, the values reported are the
 * ones the next launch resolves to (stages and ctas filled in, a TMA kernel that does not
 * fit replaced by the direct kernel). */
int csrk_tuned_config(csrk_handle h, int32_t* kernel, int32_t* lanes, int32_t* unroll,
                      int32_t* warps, int32_t* stages, int32_t* ctas);

/* csrk_set_config: force a launch configuration (same fields as csrk_tuned_config; a
 * negative field keeps the current value; a new lanes value without an unroll picks the
 * default unroll for it).  When kernel = 0 (or 2, 4, 5, 6) is given explicitly and the
 * super-super-rows do not fit two shared-memory stages, or kernel 2 / 4 / 5 / 6 is not
 * available for the matrix (or, for 5 and 6, the call's x is not 16-byte aligned), the
 * compute calls return CSRK_ERR_UNSUPPORTED; otherwise such a shape falls back (to the
 * direct kernel, from 6 to 5 or 2, from 5 to 4, from 4 to 0).  Used by the autotuner and
 * tests. */
int csrk_set_config(csrk_handle h, int32_t kernel, int32_t lanes, int32_t unroll,
                    int32_t warps, int32_t stages, int32_t ctas);

/* csrk_device_status: synchronise the handle's work on `stream` and return the device
 * status word (0 = clean; bit 0 = a pipeline wait ran out; bit 1 = in a bounds-checked
 * build, libcsrk_checks.so, a CSR-3 kernel met an index outside its array and skipped that
 * super-row or super-super-row) in *status, then clear it.
 * Returns CSRK_ERR_TIMEOUT when the word was non-zero.  A set bit means the launches since
 * the last check left some rows uncomputed (their results are invalid) and that a stage's
 * copies did not complete within two bounded waits; the blocks still ended, but treat the
 * CUDA context as suspect and re-create it before relying on later results. */
int csrk_device_status(csrk_handle h, void* stream, int32_t* status);

/* csrk_spmv_static_scratch: y = alpha*A*x + beta*y in the input numbering, for callers
 * that cannot allocate device memory -- for example a program whose arena allocator owns
 * all of the GPU's memory, a plugin held to a fixed memory budget by its host, or a
 * latency-critical loop that cannot afford an allocation's device synchronisation.  The
 * paper has no counterpart; this is a service of the library.  It allocates nothing: the
 * permuted x and result live in one static device array of 2 x 1,048,576 doubles
 * (16 MiB) that every GPU loading the library holds until the process exits.
 *   n        rows, at most 1,048,576 (larger n returns CSRK_ERR_ARG; use csrk_spmv)
 *   nssr, ssr_ptr, sr_ptr, rowptr, colidx, vals
 *            the reordered CSR-3 form in DEVICE memory, as csrk_export returns it
 *            (vals FP64; no padding needed: the kernels use plain loads).  Rows after the
 *            last super-row -- the long rows csrk_split_long_rows moves behind all others,
 *            which no super-row covers -- are computed as well, one warp per row
 *   perm     DEVICE array, perm[new] = old, or NULL when there is no reordering (then the
 *            kernels work on x and y directly and the static array is not touched)
 *   x, y     DEVICE vectors of n FP64 values in the input numbering; beta = 0 makes y
 *            write-only.  With perm given x and y may be the same vector (both are copied
 *            into the static array first); with perm NULL they must not overlap
 *   stream   cudaStream_t
 * The first call in a CUDA context (per device, and again after that device's context is
 * re-created, e.g. by cudaDeviceReset) looks up the static array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture.  Every call on a device shares the one array, which keeps the last
 * call's contents; nothing in it needs clearing, because each call writes every element
 * it later reads.  Calls whose work overlaps on the GPU (other streams, other threads)
 * race on the array: serialise them.  Errors: CSRK_ERR_ARG, CSRK_ERR_CUDA, message in
 * csrk_last_error(). */
int csrk_spmv_static_scratch(int32_t n, int32_t nssr, const int32_t* ssr_ptr,
                             const int32_t* sr_ptr, const int32_t* rowptr,
                             const int32_t* colidx, const double* vals, const int32_t* perm,
                             double alpha, const double* x, double beta, double* y,
                             void* stream);

/* csrk_selftest_bounded_wait: check the device-side timeout path.  Launches one block
 * that waits, with the same bounded wait the CSR-3 kernel uses, on an mbarrier that
 * nothing completes; the wait gives up after timeout_ns (at most 10 s), sets the handle's
 * status word and the kernel returns, leaving the context usable.  Synchronises `stream`
 * and returns the status read (and cleared) as csrk_device_status does: CSRK_ERR_TIMEOUT
 * with *status = 1 is the expected outcome. */
int csrk_selftest_bounded_wait(csrk_handle h, uint64_t timeout_ns, void* stream,
                               int32_t* status);

/* csrk_selftest_narrow: check the FP64 -> FP32 narrowing the solvers use to write their
 * FP32 copies of p (an integer rounding to nearest, ties to even: GB300 runs the
 * conversion instruction at the slow FP64 rate).  For i < n writes by_int[i] = that
 * narrowing of x[i] and by_cvt[i] = the conversion instruction's result; x, by_int, by_cvt
 * are device arrays of n (not overlapping), work enqueued on `stream`.  The two agree bit
 * for bit for every input but NaN (both NaN).  Errors: CSRK_ERR_ARG, CSRK_ERR_CUDA. */
int csrk_selftest_narrow(const double* x, int64_t n, float* by_int, float* by_cvt, void* stream);

/* csrk_selftest_stage_plan: the shared-memory stage layout the TMA kernels use for SSRs of
 * at most max_srs super-rows, max_rows rows and max_nnz nonzeros, values of val_bytes and
 * stored columns of col_bytes (2 = 16-bit codes), within max_smem bytes of shared memory
 * per block, at most want_stages stages (0 = as many as fit, up to 16), x_bytes of x
 * window per stage (kernels 5 / 6; 0 otherwise) and with_ord != 0 for the rows' length
 * order.  Host only, for tests.  out[10] receives the byte offsets inside a stage of the
 * sr_ptr, rowptr, column, value, x-window, permutation and length-order slices, the stage
 * size, the header size (mbarriers and descriptors) and the stage count; the kernels copy
 * each slice rounded out to 16-byte boundaries at both ends.  Errors: CSRK_ERR_ARG,
 * CSRK_ERR_UNSUPPORTED when two stages do not fit. */
int csrk_selftest_stage_plan(int32_t max_srs, int32_t max_rows, int64_t max_nnz, int32_t val_bytes,
                             int32_t col_bytes, int32_t max_smem, int32_t want_stages, int64_t x_bytes,
                             int32_t with_ord, uint32_t* out);

const char* csrk_last_error(void);

/* Library build description (static string): compiled architectures and options. */
const char* csrk_build_info(void);

#ifdef __cplusplus
}
#endif
#endif /* CSRK_H */
