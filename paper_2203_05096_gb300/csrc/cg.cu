// Conjugate gradients on the CSR-k form, FP64 or mixed precision, with iterations
// captured in CUDA graphs.
//
// The paper names CG on PDE matrices as the consumer of its SpMV (Sec. 1, Sec. 5.3, Sec. 8, Sec. 9).
// Recurrences (Hestenes-Stiefel): x0 = 0, r0 = b, p0 = r0;
//     q = A p;  alpha = r.r / p.q;  x += alpha p;  r -= alpha q;
//     beta = r'.r' / r.r;  p = r' + beta p.
// FP64 mode: every quantity in FP64; stop when the recursive ||r|| <= rtol ||b||.
// Mixed mode: vectors, dot products, alpha and beta stay FP64; q = A_lo p32 uses A's values
// stored in FP32 or BF16, p rounded to FP32 and FP32 accumulation.  Every `replace_every`
// iterations (earlier once the recursive residual passes rtol/2) the residual is
// recomputed in FP64, r = b - A x; the solve stops when that true residual meets rtol.
// After a replacement the direction p is kept (reliable update) unless `restart` is set,
// the recomputed residual norm exceeds twice the recursive one, or the recursive
// residual grew tenfold within the cycle -- then p = r.
//
// All scalars live on the device (CgState); reductions are deterministic (per-block
// partials summed in block order by the last block to finish).  One graph holds one cycle
// (FP64: 20 iterations); once converged, every kernel of the graph exits at entry, so
// the host reads the state once per replay.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "convert.cuh"
#include "kernels.cuh"
#include "runtime.h"

namespace {

constexpr int RED_THREADS = 256;
constexpr int MAX_RED_BLOCKS = 2048;
constexpr int ILP = 4;   // independent 16-byte accesses per thread per loop trip

// Element-pair loop: calls pair(j) for pairs j (elements 2j, 2j+1) = start, start +
// stride, ... < n/2, ILP pairs per trip with independent 16-byte loads, so each thread
// keeps several memory requests in flight; then odd(n-1) for an odd last element.
// Arrays are 256-byte aligned (cudaMalloc), so pairs are 16-byte aligned.
template <typename PairF, typename OddF>
__device__ __forceinline__ void for_pairs(int64_t n, PairF pair, OddF odd) {
    const int64_t np = n >> 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; j + (ILP - 1) * stride < np; j += ILP * stride) {
#pragma unroll
        for (int u = 0; u < ILP; ++u) pair(j + u * stride);
    }
    for (; j < np; j += stride) pair(j);
    if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) odd(n - 1);
}

__device__ __forceinline__ double2 ld2(const double* p, int64_t j) {
    return reinterpret_cast<const double2*>(p)[j];
}
__device__ __forceinline__ void st2(double* p, int64_t j, double a, double b) {
    reinterpret_cast<double2*>(p)[j] = make_double2(a, b);
}
__device__ __forceinline__ void ld2q(const double* q, int64_t j, double& a, double& b) {
    const double2 v = reinterpret_cast<const double2*>(q)[j];
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld2q(const float* q, int64_t j, double& a, double& b);
// part + a*b + c*d as two chained FMAs: GB300 issues FP64 at about one warp instruction
// per 20 clocks per SM whatever the active lanes, so the vector passes count FP64
// instructions as well as bytes (a*b + c*d + part would take three)
__device__ __forceinline__ double fma2(double part, double a, double b, double c, double d) {
    return fma(c, d, fma(a, b, part));
}
__device__ __forceinline__ void st2f(float* p, int64_t j, double a, double b) {
    reinterpret_cast<float2*>(p)[j] = make_float2(csrk::dev::f64_to_f32(a), csrk::dev::f64_to_f32(b));
}

struct CgState {
    double rr;        // r.r of the recursion
    double rr_start;  // r.r at the start of the current cycle
    double pq;        // p.q
    double alpha, beta;
    double bb;        // b.b
    double tol2;      // rtol^2 * b.b
    double rr_true;   // last recomputed ||b - A x||^2
    int32_t iters;
    int32_t done;     // 0 running, 1 converged, 2 breakdown, 3 iteration limit
    int32_t skip;     // rest of this cycle's iterations are no-ops
    int32_t restart;  // reset p = r at the replacement step
    int32_t maxit;
    int32_t keep_p;   // 1: reliable update (keep p when consistent); 0: always restart
    uint32_t counter; // blocks finished in the current reduction
    int32_t pad;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of v; the block total is returned to thread 0.  Warp 0 alone adds: each lane
// sums a fixed strided eighth of the block's values, then one shuffle tree -- 12 FP64 warp
// instructions per block instead of 45 for a shuffle tree in every warp (on GB300 an FP64
// instruction costs the same with one active lane as with 32).
__device__ double block_sum(double v) {
    __shared__ double vals[RED_THREADS];
    vals[threadIdx.x] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = vals[threadIdx.x];
#pragma unroll
        for (int i = 1; i < RED_THREADS / 32; ++i) t += vals[threadIdx.x + 32 * i];
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Store the block partial; returns true (for every thread of exactly one block) when every
// block has stored, after which partials[0..gridDim.x) are complete and visible.
__device__ bool last_block(double part, double* partials, uint32_t* counter) {
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = part;
        __threadfence();
        const uint32_t ticket = atomicAdd(counter, 1u);
        is_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    return is_last;
}

// Sum of the block partials by all threads of the last block (thread 0 gets the total):
// each thread adds a fixed strided subset, then the fixed block tree -- deterministic.
__device__ double sum_partials(const double* partials) {
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += ((volatile const double*)partials)[i];
    return block_sum(t);
}

// FP32 -> FP64 with integer instructions (a conversion instruction would occupy the FP64
// pipe, which the dot products and updates already load).
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return csrk::dev::x_f64(v); }

__device__ __forceinline__ void ld2q(const float* q, int64_t j, double& a, double& b) {
    const float2 v = reinterpret_cast<const float2*>(q)[j];
    a = as_f64(v.x);
    b = as_f64(v.y);
}

// r = b, p = r (and p32), x = 0; b.b -> state
__global__ void __launch_bounds__(RED_THREADS) cg_init(int32_t n, const double* __restrict__ b,
                                                       double* __restrict__ x, double* __restrict__ r,
                                                       double* __restrict__ p, float* __restrict__ p32,
                                                       double rtol, int32_t maxit, int32_t keep_p,
                                                       CgState* st, double* partials) {
    double part = 0.0;
    for_pairs(n, [&](int64_t j) {
        const double2 bv = ld2(b, j);
        st2(x, j, 0.0, 0.0);
        st2(r, j, bv.x, bv.y);
        st2(p, j, bv.x, bv.y);
        if (p32) st2f(p32, j, bv.x, bv.y);
        part = fma2(part, bv.x, bv.x, bv.y, bv.y);
    }, [&](int64_t i) {
        const double bi = b[i];
        x[i] = 0.0;
        r[i] = bi;
        p[i] = bi;
        if (p32) p32[i] = csrk::dev::f64_to_f32(bi);
        part += bi * bi;
    });
    part = block_sum(part);
    if (last_block(part, partials, &st->counter)) {
        const double bb = sum_partials(partials);
        if (threadIdx.x != 0) return;
        st->bb = bb;
        st->rr = bb;
        st->rr_start = bb;
        st->tol2 = rtol * rtol * bb;
        st->rr_true = bb;
        st->iters = 0;
        st->done = (bb == 0.0) ? 1 : 0;
        st->skip = st->done;
        st->restart = 0;
        st->maxit = maxit;
        st->keep_p = keep_p;
        st->counter = 0;
    }
}

// p.q -> alpha (breakdown when p.q <= 0 or not finite)
template <typename QT>
__global__ void __launch_bounds__(RED_THREADS) cg_dot_pq(int32_t n, const double* __restrict__ p,
                                                         const QT* __restrict__ q, CgState* st,
                                                         double* partials) {
    if (st->skip) return;
    double part = 0.0;
    for_pairs(n, [&](int64_t j) {
        const double2 pv = ld2(p, j);
        double q0, q1;
        ld2q(q, j, q0, q1);
        part = fma2(part, pv.x, q0, pv.y, q1);
    }, [&](int64_t i) { part += p[i] * as_f64(q[i]); });
    part = block_sum(part);
    if (last_block(part, partials, &st->counter)) {
        const double pq = sum_partials(partials);
        if (threadIdx.x != 0) return;
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->done = 2;
            st->skip = 1;
        } else {
            st->alpha = st->rr / pq;
        }
        st->counter = 0;
    }
}

// x += alpha p; r -= alpha q; r.r -> beta, convergence / cycle / divergence decisions
template <typename QT>
__global__ void __launch_bounds__(RED_THREADS) cg_update_xr(int32_t n, double* __restrict__ x,
                                                            double* __restrict__ r,
                                                            const double* __restrict__ p,
                                                            const QT* __restrict__ q, int32_t mixed,
                                                            CgState* st, double* partials) {
    if (st->skip) return;
    const double alpha = st->alpha;
    double part = 0.0;
    for_pairs(n, [&](int64_t j) {
        const double2 pv = ld2(p, j), xv = ld2(x, j), rv = ld2(r, j);
        double q0, q1;
        ld2q(q, j, q0, q1);
        const double r0 = rv.x - alpha * q0, r1 = rv.y - alpha * q1;
        st2(x, j, xv.x + alpha * pv.x, xv.y + alpha * pv.y);
        st2(r, j, r0, r1);
        part = fma2(part, r0, r0, r1, r1);
    }, [&](int64_t i) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * as_f64(q[i]);
        r[i] = ri;
        part += ri * ri;
    });
    part = block_sum(part);
    if (last_block(part, partials, &st->counter)) {
        const double rr_new = sum_partials(partials);
        if (threadIdx.x != 0) return;
        st->beta = rr_new / st->rr;
        st->rr = rr_new;
        st->iters += 1;
        if (!mixed) {
            if (rr_new <= st->tol2) {
                st->done = 1;
                st->skip = 1;
            }
        } else {
            if (rr_new <= 0.25 * st->tol2) st->skip = 1;   // go check the true residual
            if (rr_new > 100.0 * st->rr_start) {             // the cycle is diverging
                st->restart = 1;
                st->skip = 1;
            }
        }
        if (!st->done && st->iters >= st->maxit) {
            st->done = 3;
            st->skip = 1;
        }
        st->counter = 0;
    }
}

// p = r + beta p (and its FP32 copy)
__global__ void __launch_bounds__(RED_THREADS) cg_update_p(int32_t n, const double* __restrict__ r,
                                                           double* __restrict__ p, float* __restrict__ p32,
                                                           const CgState* st) {
    if (st->skip) return;
    const double beta = st->beta;
    for_pairs(n, [&](int64_t j) {
        const double2 rv = ld2(r, j), pv = ld2(p, j);
        const double p0 = rv.x + beta * pv.x, p1 = rv.y + beta * pv.y;
        st2(p, j, p0, p1);
        if (p32) st2f(p32, j, p0, p1);
    }, [&](int64_t i) {
        const double pi = r[i] + beta * p[i];
        p[i] = pi;
        if (p32) p32[i] = csrk::dev::f64_to_f32(pi);
    });
}

// Replacement, part 1: r = b (the FP64 SpMV then forms r = b - A x)
__global__ void __launch_bounds__(RED_THREADS) cg_copy_b(int32_t n, const double* __restrict__ b,
                                                         double* __restrict__ r, const CgState* st) {
    if (st->done) return;
    for_pairs(n, [&](int64_t j) {
        const double2 bv = ld2(b, j);
        st2(r, j, bv.x, bv.y);
    }, [&](int64_t i) { r[i] = b[i]; });
}

// Replacement, part 2: ||r||^2 of the recomputed residual; convergence test; decide
// whether the direction restarts; open the next cycle.
__global__ void __launch_bounds__(RED_THREADS) cg_replace_finish(int32_t n, const double* __restrict__ r,
                                                                 CgState* st, double* partials) {
    if (st->done) return;
    double part = 0.0;
    for_pairs(n, [&](int64_t j) {
        const double2 rv = ld2(r, j);
        part = fma2(part, rv.x, rv.x, rv.y, rv.y);
    }, [&](int64_t i) {
        const double ri = r[i];
        part += ri * ri;
    });
    part = block_sum(part);
    if (last_block(part, partials, &st->counter)) {
        const double rt = sum_partials(partials);
        if (threadIdx.x != 0) return;
        st->rr_true = rt;
        if (rt <= st->tol2) {
            st->done = 1;
            st->skip = 1;
        } else {
            if (!st->keep_p || rt > 4.0 * st->rr) st->restart = 1;
            st->rr = rt;
            st->rr_start = rt;
            st->skip = 0;
            if (!st->done && st->iters >= st->maxit) {
                st->done = 3;
                st->skip = 1;
            }
        }
        st->counter = 0;
    }
}

// Replacement, part 3: p = r when the direction restarts
__global__ void __launch_bounds__(RED_THREADS) cg_restart_p(int32_t n, const double* __restrict__ r,
                                                            double* __restrict__ p, float* __restrict__ p32,
                                                            CgState* st) {
    if (st->done || !st->restart) return;
    for_pairs(n, [&](int64_t j) {
        const double2 rv = ld2(r, j);
        st2(p, j, rv.x, rv.y);
        if (p32) st2f(p32, j, rv.x, rv.y);
    }, [&](int64_t i) {
        const double ri = r[i];
        p[i] = ri;
        if (p32) p32[i] = csrk::dev::f64_to_f32(ri);
    });
}

// the restart flag is consumed at the start of the next cycle
__global__ void cg_clear_restart(CgState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !st->done) st->restart = 0;
}

// ||r||^2 -> rr_true, whatever the state (final report)
__global__ void __launch_bounds__(RED_THREADS) cg_true_norm(int32_t n, const double* __restrict__ r,
                                                            CgState* st, double* partials) {
    double part = 0.0;
    for_pairs(n, [&](int64_t j) {
        const double2 rv = ld2(r, j);
        part = fma2(part, rv.x, rv.x, rv.y, rv.y);
    }, [&](int64_t i) {
        const double ri = r[i];
        part += ri * ri;
    });
    part = block_sum(part);
    if (last_block(part, partials, &st->counter)) {
        const double rt = sum_partials(partials);
        if (threadIdx.x != 0) return;
        st->rr_true = rt;
        st->counter = 0;
    }
}

// FP64 mode after a recursive stop whose true residual missed the tolerance: continue
// from the recomputed residual with a fresh direction.
__global__ void __launch_bounds__(RED_THREADS) cg_resume(int32_t n, const double* __restrict__ r,
                                                         double* __restrict__ p, CgState* st) {
    for_pairs(n, [&](int64_t j) {
        const double2 rv = ld2(r, j);
        st2(p, j, rv.x, rv.y);
    }, [&](int64_t i) { p[i] = r[i]; });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rr = st->rr_true;
        st->rr_start = st->rr_true;
        st->done = 0;
        st->skip = 0;
    }
}

}  // namespace

// Workspace of the solver, owned by the handle.
struct CgWork {
    int32_t n = 0;
    double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    float *p32 = nullptr, *q32 = nullptr;
    double* partials = nullptr;
    CgState* st = nullptr;
    CgState* host_st = nullptr;   // pinned mirror for the per-replay read
    cudaStream_t cap = nullptr;   // private stream for graph capture
    cudaGraphExec_t exec = nullptr;
    int exec_vt = -1, exec_every = 0;
    unsigned long long exec_gen = 0;
    int grid = 0;
};

namespace csrk {
namespace rt {

void free_cg(csrk_matrix* h) {
    CgWork* w = h->cg;
    if (!w) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    cudaFree(w->b);
    cudaFree(w->x);
    cudaFree(w->r);
    cudaFree(w->p);
    cudaFree(w->q);
    cudaFree(w->p32);
    cudaFree(w->q32);
    cudaFree(w->partials);
    cudaFree(w->st);
    cudaFreeHost(w->host_st);
    if (w->cap) cudaStreamDestroy(w->cap);
    delete w;
    h->cg = nullptr;
}

namespace {

int alloc_cg(csrk_matrix* h) {
    const int32_t n = h->m.n;
    if (h->cg && h->cg->n == n) return CSRK_OK;
    free_cg(h);
    CgWork* w = new (std::nothrow) CgWork();
    if (!w) return fail(CSRK_ERR_ALLOC, "out of host memory");
    h->cg = w;
    w->n = n;
    const size_t d = (size_t)std::max(n, 1) * 8, f = (size_t)std::max(n, 1) * 4;
    cudaError_t e = cudaSuccess;
    if (fault_injected("alloc")) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMalloc(&w->b, d);
    if (e == cudaSuccess) e = cudaMalloc(&w->x, d);
    if (e == cudaSuccess) e = cudaMalloc(&w->r, d);
    if (e == cudaSuccess) e = cudaMalloc(&w->p, d);
    if (e == cudaSuccess) e = cudaMalloc(&w->q, d);
    if (e == cudaSuccess) e = cudaMalloc(&w->p32, f);
    if (e == cudaSuccess) e = cudaMalloc(&w->q32, f);
    if (e == cudaSuccess) e = cudaMalloc(&w->partials, MAX_RED_BLOCKS * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&w->st, sizeof(CgState));
    if (e == cudaSuccess) e = cudaMemset(w->st, 0, sizeof(CgState));
    if (e == cudaSuccess) e = cudaMallocHost(&w->host_st, sizeof(CgState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_cg(h);
        return fail(CSRK_ERR_ALLOC, std::string("CG workspace: ") + cudaGetErrorString(e));
    }
    // 4 blocks of 256 per SM, each thread keeping ILP 16-byte loads per array in flight;
    // for n up to ~4.9M every thread runs at most one full ILP trip plus a short tail
    w->grid = std::min(MAX_RED_BLOCKS, std::max(1, h->num_sms * 4));
    return CSRK_OK;
}

// Enqueue one cycle: `every` iterations, then (mixed) the FP64 residual replacement.
int enqueue_cycle(csrk_matrix* h, int vt, int every, cudaStream_t s) {
    CgWork* w = h->cg;
    const int32_t n = w->n;
    const int g = w->grid;
    const bool mixed = vt != VAL_F64;
    int rc;
    for (int it = 0; it < every; ++it) {
        if (mixed) {
            if ((rc = launch_spmv_dev(h, vt, w->p32, w->q32, 1.0, 0.0, true, true, &w->st->skip, s))) return rc;
            cg_dot_pq<float><<<g, RED_THREADS, 0, s>>>(n, w->p, w->q32, w->st, w->partials);
            cg_update_xr<float><<<g, RED_THREADS, 0, s>>>(n, w->x, w->r, w->p, w->q32, 1, w->st, w->partials);
        } else {
            if ((rc = launch_spmv_dev(h, VAL_F64, w->p, w->q, 1.0, 0.0, false, false, &w->st->skip, s))) return rc;
            cg_dot_pq<double><<<g, RED_THREADS, 0, s>>>(n, w->p, w->q, w->st, w->partials);
            cg_update_xr<double><<<g, RED_THREADS, 0, s>>>(n, w->x, w->r, w->p, w->q, 0, w->st, w->partials);
        }
        cg_update_p<<<g, RED_THREADS, 0, s>>>(n, w->r, w->p, mixed ? w->p32 : nullptr, w->st);
    }
    if (mixed) {
        cg_copy_b<<<g, RED_THREADS, 0, s>>>(n, w->b, w->r, w->st);
        if ((rc = launch_spmv_dev(h, VAL_F64, w->x, w->r, -1.0, 1.0, false, false, &w->st->done, s))) return rc;
        cg_replace_finish<<<g, RED_THREADS, 0, s>>>(n, w->r, w->st, w->partials);
        cg_restart_p<<<g, RED_THREADS, 0, s>>>(n, w->r, w->p, w->p32, w->st);
        cg_clear_restart<<<1, 32, 0, s>>>(w->st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CG kernel launch");
    return CSRK_OK;
}

}  // namespace

int cg_solve(csrk_matrix* h, const double* b, double* x, double rtol, int32_t maxit, int vt,
             int32_t every, int32_t restart, unsigned flags, int32_t* iters, double* relres,
             cudaStream_t s) {
    int rc;
    NvtxRange range("csrk cg");
    if ((rc = ensure_context(h)) || (rc = ensure_struct(h)) || (rc = ensure_vals(h, VAL_F64))) return rc;
    if (vt != VAL_F64 && (rc = ensure_vals(h, vt))) return rc;
    if ((rc = alloc_cg(h))) return rc;
    CgWork* w = h->cg;
    const int32_t n = h->m.n;
    const bool permuted = (flags & CSRK_VEC_PERMUTED) || h->perm.empty();
    // b into the reordered numbering
    if (permuted)
        CK_CUDA(cudaMemcpyAsync(w->b, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
    else if ((rc = launch_gather_rows(b, 1, w->b, 1, h->d_perm, n, 1, 8, s)))
        return cuda_fail((cudaError_t)rc, "permute b");
    const bool mixed = vt != VAL_F64;
    const int g = w->grid;
    cg_init<<<g, RED_THREADS, 0, s>>>(n, w->b, w->x, w->r, w->p, mixed ? w->p32 : nullptr, rtol, maxit,
                                      restart ? 0 : 1, w->st, w->partials);
    CK_CUDA(cudaGetLastError(), "cg_init");

    // (Re)capture the cycle graph when the shape of the solve or the handle changed.
    if (!w->exec || w->exec_vt != vt || w->exec_every != every || w->exec_gen != h->generation) {
        if (w->exec) {
            cudaGraphExecDestroy(w->exec);
            w->exec = nullptr;
        }
        // one eager cycle on the capture stream first, so every kernel's attributes are set
        // and nothing but launches is recorded; its effect is undone by re-initialising
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
        // the inner product's launch shape, timed on these pointers at the first mixed solve
        if (mixed && h->inner_gen[vt] != h->generation && (rc = tune_inner(h, vt, w->p32, w->q32))) return rc;
        if ((rc = enqueue_cycle(h, vt, 1, w->cap))) return rc;
        CK_CUDA(cudaStreamSynchronize(w->cap), "synchronise");
        cg_init<<<g, RED_THREADS, 0, w->cap>>>(n, w->b, w->x, w->r, w->p, mixed ? w->p32 : nullptr, rtol,
                                               maxit, restart ? 0 : 1, w->st, w->partials);
        CK_CUDA(cudaStreamSynchronize(w->cap), "synchronise");
        CK_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        rc = enqueue_cycle(h, vt, every, w->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(w->cap, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&w->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        w->exec_vt = vt;
        w->exec_every = every;
        w->exec_gen = h->generation;
        CK_CUDA(cudaStreamSynchronize(w->cap), "synchronise");
    }
    // replay cycles until the device reports an end state; then recompute the true FP64
    // residual (mixed mode already has it from its last replacement)
    CgState hs{};
    for (int round = 0;; ++round) {
        for (;;) {
            CK_CUDA(cudaGraphLaunch(w->exec, s), "graph launch");
            CK_CUDA(cudaMemcpyAsync(w->host_st, w->st, sizeof(CgState), cudaMemcpyDeviceToHost, s),
                    "read state");
            CK_CUDA(cudaStreamSynchronize(s), "synchronise");
            if (w->host_st->done) break;
        }
        hs = *w->host_st;
        if (mixed && hs.done == 1) break;
        CK_CUDA(cudaMemcpyAsync(w->r, w->b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
        if ((rc = launch_spmv_dev(h, VAL_F64, w->x, w->r, -1.0, 1.0, false, false, nullptr, s))) return rc;
        cg_true_norm<<<g, RED_THREADS, 0, s>>>(n, w->r, w->st, w->partials);
        CK_CUDA(cudaMemcpyAsync(w->host_st, w->st, sizeof(CgState), cudaMemcpyDeviceToHost, s), "read state");
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
        hs = *w->host_st;
        const bool met = hs.rr_true <= hs.tol2;
        if (met || mixed || hs.done != 1 || hs.iters >= maxit || round >= 3) break;
        cg_resume<<<g, RED_THREADS, 0, s>>>(n, w->r, w->p, w->st);
        CK_CUDA(cudaGetLastError(), "cg_resume");
    }
    const double rr_true = hs.rr_true;
    if (iters) *iters = hs.iters;
    const double rel = hs.bb > 0 ? std::sqrt(rr_true / hs.bb) : 0.0;
    if (relres) *relres = rel;
    // x back to the input numbering
    if (permuted)
        CK_CUDA(cudaMemcpyAsync(x, w->x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s), "copy x");
    else if ((rc = launch_scatter_rows(w->x, 1, x, 1, h->d_perm, n, 1, 8, s)))
        return cuda_fail((cudaError_t)rc, "unpermute x");
    if (hs.done == 2) return fail(CSRK_ERR_NOT_CONVERGED, "CG breakdown (p.q <= 0)");
    if (!(rel <= rtol)) return fail(CSRK_ERR_NOT_CONVERGED, "CG stopped above the tolerance");
    return CSRK_OK;
}

}  // namespace rt
}  // namespace csrk

extern "C" int csrk_cg(csrk_handle h, const double* b, double* x, double rtol, int32_t maxit,
                       csrk_dtype inner, int32_t replace_every, int32_t restart, unsigned flags,
                       int32_t* iters, double* relres, void* stream) {
    using namespace csrk::rt;
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    if (inner != CSRK_F64 && inner != CSRK_F32 && inner != CSRK_BF16) return fail(CSRK_ERR_ARG, "unknown inner dtype");
    if (!(rtol > 0.0) || maxit < 1) return fail(CSRK_ERR_ARG, "rtol must be > 0 and maxit >= 1");
    if (inner != CSRK_F64 && replace_every < 1) return fail(CSRK_ERR_ARG, "replace_every must be >= 1");
    if (flags & ~(unsigned)CSRK_VEC_PERMUTED) return fail(CSRK_ERR_UNSUPPORTED, "csrk_cg takes only CSRK_VEC_PERMUTED");
    if (h->m.n > 0 && (!b || !x || b == x)) return fail(CSRK_ERR_ARG, "bad b / x");
    if (h->m.n == 0) {
        if (iters) *iters = 0;
        if (relres) *relres = 0.0;
        return CSRK_OK;
    }
    const int every = inner == CSRK_F64 ? 20 : replace_every;
    try {
        return cg_solve(h, b, x, rtol, maxit, (int)inner, every, restart, flags, iters, relres,
                        (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
}
