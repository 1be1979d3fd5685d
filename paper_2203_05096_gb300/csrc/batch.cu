// Batched work over many CSR-k matrices of uneven size.
//
// csrk_batch_spmm: Y_i = alpha A_i X_i + beta Y_i for every matrix i of a batch in ONE
// persistent launch.  The batch cuts each matrix into items -- runs of whole super-rows
// of at most 24 KB of matrix data, the batch's own super-super-rows sized to a shared-memory
// stage -- and queues tiles of a few items matrix by matrix (matrices by decreasing work,
// each matrix's items in row order, so the blocks running at any moment share one x
// window in L2).  In each block a producer warp takes the next tile from an atomic
// counter and streams its items' rowptr / colidx / value slices into a ring of shared
// memory stages with bulk copies (cp.async.bulk, mbarrier completion); the consumer warps
// split every staged item into row groups of one warp pass each (32 rows for k = 1, 32/G
// rows with G >= k lanes per row otherwise) and gather x from global memory.  No block
// ever waits for another, and no block-wide barrier is taken after the start.  The last
// producer to finish resets the counter, so the launch can be replayed from a CUDA graph.
// Batches whose super-rows do not fit two stages use a direct-load kernel instead.
//
// csrk_batch_cg: independent conjugate-gradient solves for every (matrix, right-hand side)
// pair, FP64 vectors and scalars, each step one batched SpMM launch plus batched vector
// kernels; a fixed number of iterations is recorded once into a CUDA graph and replayed.
// A system whose recursive residual reaches rtol freezes (alpha = 0).  Reductions are
// deterministic: per-chunk partials, then one warp per system summing its chunks in order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "convert.cuh"
#include "kernels.cuh"
#include "runtime.h"

namespace {

using csrk::dev::bf16_t;

struct BatchMat {
    const int32_t* rowptr;
    const int32_t* colidx;
    const void* vals;
    const int32_t* sr_ptr;
    const SsrDesc* desc;
    const void* X;   // FP64 (xt = 0) or FP32 (xt = 1) n x k block
    void* Y;
    int32_t n, k, vt;
    int32_t xt;      // 1: FP32 vectors and FP32 accumulation (FP32 / BF16 values only)
    int32_t vec;     // X and Y blocks 16-byte aligned: power-of-two k use vector loads
    int32_t pad;
};

struct BatchTile {
    int32_t mat, t0, t1, pad;
};

struct Chunk {   // contiguous rows of one matrix for the batched vector kernels
    int32_t mat, row0, row1, pad;
    int64_t off;  // element offset of row0 in the concatenated vectors
};

constexpr int BW = 8;   // warps per block of the persistent SpMM

// One super-row of a batch matrix, for one (value type, right-hand-side count) class.  Kept
// out of line: each class gets its own register allocation instead of one kernel body
// holding every variant at once.
template <typename VT, int G, int CPL>
__device__ __noinline__ void sr_rows(const BatchMat* m, int rb, int re, double alpha, double beta, int epi,
                                     int lane) {
    using namespace csrk::dev;
    const VT* vals = static_cast<const VT*>(m->vals);
    const double* X = static_cast<const double*>(m->X);
    double* Y = static_cast<double*>(m->Y);
    if constexpr (G == 1)
        spmv_rows<VT, double, double, 1, 8>(rb, re, m->rowptr, m->colidx, vals, X, Y, alpha, beta, epi, lane);
    else
        spmm_rows<VT, double, double, G, CPL>(rb, re, m->rowptr, m->colidx, vals, X, m->k, Y, m->k, m->k,
                                              alpha, beta, epi, lane);
}

template <typename VT>
__device__ __forceinline__ void tile_rows(const BatchMat* m, int rb, int re, double alpha, double beta,
                                          int epi, int lane) {
    const int k = m->k;
    if (k == 1) sr_rows<VT, 1, 1>(m, rb, re, alpha, beta, epi, lane);
    else if (k == 2) sr_rows<VT, 2, 1>(m, rb, re, alpha, beta, epi, lane);
    else if (k <= 4) sr_rows<VT, 4, 1>(m, rb, re, alpha, beta, epi, lane);
    else if (k <= 8) sr_rows<VT, 8, 1>(m, rb, re, alpha, beta, epi, lane);
    else if (k <= 16) sr_rows<VT, 16, 1>(m, rb, re, alpha, beta, epi, lane);
    else if (k <= 32) sr_rows<VT, 32, 1>(m, rb, re, alpha, beta, epi, lane);
    else sr_rows<VT, 32, 2>(m, rb, re, alpha, beta, epi, lane);
}

__global__ void __launch_bounds__(BW * 32, 4) batch_spmm_kernel(const BatchMat* __restrict__ mats,
                                                             const BatchTile* __restrict__ tiles,
                                                             int32_t ntiles, uint32_t* counters,
                                                             double alpha, double beta, int epi) {
    __shared__ int32_t tile_id;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) tile_id = (int32_t)atomicAdd(&counters[0], 1u);
        __syncthreads();
        const int32_t t = tile_id;
        __syncthreads();
        if (t >= ntiles) break;
        const BatchTile tl = tiles[t];
        const BatchMat* m = &mats[tl.mat];
        const SsrDesc* desc = m->desc;
        const int32_t* sr_ptr = m->sr_ptr;
        const int vt = m->vt;
        for (int32_t q = tl.t0; q < tl.t1; ++q) {
            const SsrDesc d = desc[q];
            for (int sr = d.s0 + warp; sr < d.s1; sr += BW) {
                const int rb = sr_ptr[sr], re = sr_ptr[sr + 1];
                if (vt == csrk::VAL_F64) tile_rows<double>(m, rb, re, alpha, beta, epi, lane);
                else if (vt == csrk::VAL_F32) tile_rows<float>(m, rb, re, alpha, beta, epi, lane);
                else tile_rows<bf16_t>(m, rb, re, alpha, beta, epi, lane);
            }
        }
    }
    // the last block out resets the tile counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&counters[1], 1u) == gridDim.x - 1) {
            atomicExch(&counters[0], 0u);
            atomicExch(&counters[1], 0u);
        }
    }
}

// ---------------------------------------------------------------- staged SpMM kernel
// A run of whole super-rows of one matrix, staged into shared memory as one unit.
struct BatchItem {
    int32_t mat, r0, r1, p0, p1, pad0, pad1, pad2;
};
struct ItemTile {   // items [i0, i1) of one matrix, handed out by the atomic counter
    int32_t i0, i1;
};
struct StageHdr {   // written by the producer before the stage's copies, read by consumers
    int32_t mat;     // -1: no more work; -2: item skipped (did not fit; status bit 2 set)
    int32_t r0, r1, p0;
    uint32_t off_col, off_val;
    int32_t pad0, pad1;
};

constexpr int TW = 16;                  // consumer warps per block (+1 producer warp)
constexpr int MAX_STAGES = 16;
constexpr int HDR_BYTES = MAX_STAGES * (2 * 8 + (int)sizeof(StageHdr));   // 768
constexpr int64_t ITEM_BYTES_DEFAULT = 24576;
constexpr size_t ITEMS_PER_TILE = 4;

// Element slice [first, last) rounded out to 16-byte boundaries, element size esz.
__host__ __device__ inline void slice16_rt(int64_t first, int64_t last, int esz, int64_t& a0, uint32_t& bytes) {
    const int64_t per = 16 / esz;
    a0 = first & ~(per - 1);
    const int64_t a1 = (last + per - 1) & ~(per - 1);
    bytes = (uint32_t)((a1 - a0) * esz);
}

__host__ __device__ inline int val_bytes_of(int vt) { return vt == csrk::VAL_F64 ? 8 : vt == csrk::VAL_F32 ? 4 : 2; }

// Rows one warp pass covers for k right-hand sides: the lane mapping of item_rows, or of
// item_rows_vec (VW columns per lane) for aligned power-of-two k.
__device__ __forceinline__ int rows_per_pass(int k, bool vec, int xbytes) {
    if (vec && k >= 2 && k <= 32 && (k & (k - 1)) == 0) {
        const int vw = xbytes == 4 ? (k == 2 ? 2 : 4) : 2;
        return 32 / (k / vw);
    }
    return k == 1 ? 32 : k == 2 ? 16 : k <= 4 ? 8 : k <= 8 ? 4 : k <= 16 ? 2 : 1;
}

// The row groups first, first + TW, ... of a staged item for one (value type, k) class.
// rp / col / vb point into the stage; out of line like sr_rows.
template <typename VT, typename XT, typename AT, int G, int CPL>
__device__ __noinline__ void item_rows(const XT* X, XT* Y, int k, int r0, int r1, int p0, int first,
                                       const int32_t* rp, const int32_t* col, const unsigned char* vb,
                                       double alpha, double beta, int epi, int lane) {
    using namespace csrk::dev;
    constexpr int VPER = 16 / (int)sizeof(VT);
    const VT* val = reinterpret_cast<const VT*>(vb) - (p0 & ~(VPER - 1));
    constexpr int RPP = G == 1 ? 32 : 32 / G;
    const int ng = (r1 - r0 + RPP - 1) / RPP;
    for (int g = first; g < ng; g += TW) {
        const int rb = r0 + g * RPP, re = min(rb + RPP, r1);
        if constexpr (G == 1)
            spmv_rows<VT, XT, AT, 1, 8>(rb, re, rp, col, val, X, Y, alpha, beta, epi, lane);
        else
            spmm_rows<VT, XT, AT, G, CPL>(rb, re, rp, col, val, X, k, Y, k, k, alpha, beta, epi, lane);
    }
}

template <typename XT, int VW> struct VecT;
template <> struct VecT<float, 2> { using T = float2; };
template <> struct VecT<float, 4> { using T = float4; };
template <> struct VecT<double, 2> { using T = double2; };

// As item_rows for k = G * VW right-hand sides with 16-byte aligned X / Y blocks: each lane
// owns VW consecutive columns and gathers them with one vector load per nonzero (a 16-byte
// request instead of VW separate ones), chunks of 4 nonzeros in flight per lane.
template <typename VT, typename XT, typename AT, int G, int VW>
__device__ __noinline__ void item_rows_vec(const XT* X, XT* Y, int k, int r0, int r1, int p0, int first,
                                           const int32_t* rp, const int32_t* col, const unsigned char* vb,
                                           double alpha, double beta, int epi, int lane) {
    using namespace csrk::dev;
    using V = typename VecT<XT, VW>::T;
    constexpr int VPER = 16 / (int)sizeof(VT);
    const VT* val = reinterpret_cast<const VT*>(vb) - (p0 & ~(VPER - 1));
    constexpr int RPP = 32 / G;
    constexpr int U = 4;
    const int c0 = (lane % G) * VW;
    const int ng = (r1 - r0 + RPP - 1) / RPP;
    for (int g = first; g < ng; g += TW) {
        const int r = r0 + g * RPP + lane / G;
        if (r >= r1) continue;
        AT acc[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) acc[j] = 0;
        const int pe = rp[r + 1];
        int p = rp[r];
        for (; p + U <= pe; p += U) {
            V xv[U];
#pragma unroll
            for (int t = 0; t < U; ++t) xv[t] = __ldg(reinterpret_cast<const V*>(X + (int64_t)col[p + t] * k + c0));
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const VT v = val[p + t];
                const XT* e = reinterpret_cast<const XT*>(&xv[t]);
#pragma unroll
                for (int j = 0; j < VW; ++j) acc[j] = Acc<AT>::fma(v, e[j], acc[j]);
            }
        }
        if (p < pe) {   // the last 1..3 nonzeros
            V xv[U];
#pragma unroll
            for (int t = 0; t < U; ++t)
                if (p + t < pe) xv[t] = __ldg(reinterpret_cast<const V*>(X + (int64_t)col[p + t] * k + c0));
#pragma unroll
            for (int t = 0; t < U; ++t)
                if (p + t < pe) {
                    const VT v = val[p + t];
                    const XT* e = reinterpret_cast<const XT*>(&xv[t]);
#pragma unroll
                    for (int j = 0; j < VW; ++j) acc[j] = Acc<AT>::fma(v, e[j], acc[j]);
                }
        }
        XT* yr = Y + (int64_t)r * k + c0;
        if (epi == 0) {
            V out;
            XT* o = reinterpret_cast<XT*>(&out);
#pragma unroll
            for (int j = 0; j < VW; ++j) o[j] = (XT)acc[j];
            *reinterpret_cast<V*>(yr) = out;
        } else {
#pragma unroll
            for (int j = 0; j < VW; ++j) store_y<XT, AT>(yr, j, acc[j], alpha, beta, epi);
        }
    }
}

template <typename VT, typename XT, typename AT>
__device__ __forceinline__ void item_dispatch(const BatchMat* m, int r0, int r1, int p0, int first,
                                              const int32_t* rp, const int32_t* col, const unsigned char* vb,
                                              double alpha, double beta, int epi, int lane) {
    const int k = m->k;
    const XT* X = static_cast<const XT*>(m->X);
    XT* Y = static_cast<XT*>(m->Y);
    if (m->vec && k >= 2 && k <= 32 && (k & (k - 1)) == 0) {
#define CSRK_ITEMV(G, VW) \
    item_rows_vec<VT, XT, AT, G, VW>(X, Y, k, r0, r1, p0, first, rp, col, vb, alpha, beta, epi, lane)
        if constexpr (sizeof(XT) == 4) {   // float2 for k = 2, float4 otherwise
            if (k == 2) CSRK_ITEMV(1, 2);
            else if (k == 4) CSRK_ITEMV(1, 4);
            else if (k == 8) CSRK_ITEMV(2, 4);
            else if (k == 16) CSRK_ITEMV(4, 4);
            else CSRK_ITEMV(8, 4);
        } else {                           // double2
            if (k == 2) CSRK_ITEMV(1, 2);
            else if (k == 4) CSRK_ITEMV(2, 2);
            else if (k == 8) CSRK_ITEMV(4, 2);
            else if (k == 16) CSRK_ITEMV(8, 2);
            else CSRK_ITEMV(16, 2);
        }
#undef CSRK_ITEMV
        return;
    }
#define CSRK_ITEM(G, CPL) item_rows<VT, XT, AT, G, CPL>(X, Y, k, r0, r1, p0, first, rp, col, vb, alpha, beta, epi, lane)
    if (k == 1) CSRK_ITEM(1, 1);
    else if (k == 2) CSRK_ITEM(2, 1);
    else if (k <= 4) CSRK_ITEM(4, 1);
    else if (k <= 8) CSRK_ITEM(8, 1);
    else if (k <= 16) CSRK_ITEM(16, 1);
    else if (k <= 32) CSRK_ITEM(32, 1);
    else CSRK_ITEM(32, 2);
#undef CSRK_ITEM
}

// At most 60 registers per thread: two blocks of 17 warps per SM.
__global__ void __launch_bounds__((TW + 1) * 32, 2)
    batch_spmm_tma_kernel(const BatchMat* __restrict__ mats, const BatchItem* __restrict__ items,
                          const ItemTile* __restrict__ tiles, int32_t ntiles, uint32_t* counters, double alpha,
                          double beta, int epi, uint32_t stage_bytes, int32_t S, unsigned long long timeout_ns,
                          int32_t* status) {
    using namespace csrk::dev;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + MAX_STAGES;
    StageHdr* hdr = reinterpret_cast<StageHdr*>(smem + 16 * MAX_STAGES);
    unsigned char* stage0 = smem + HDR_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == TW) {
        // ---------------- producer: one elected lane fetches tiles and issues the copies
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            int i = 0;
            bool ok = true;
            for (;;) {
                const int32_t t = (int32_t)atomicAdd(&counters[0], 1u);
                if (t >= ntiles) break;
                const ItemTile tl = tiles[t];
                for (int32_t q = tl.i0; q < tl.i1; ++q, ++i) {
                    const int s = i % S;
                    if (i >= S && !mbar_wait_bounded(&empty[s], ((i / S) - 1) & 1, timeout_ns)) {
                        report(status, 1);
                        ok = false;
                        break;
                    }
                    const BatchItem it = items[q];
                    const BatchMat* m = &mats[it.mat];
                    const int esz = val_bytes_of(m->vt);
                    int64_t o_rp, o_col, o_val;
                    uint32_t b_rp, b_col, b_val;
                    slice16_rt(it.r0, (int64_t)it.r1 + 1, 4, o_rp, b_rp);
                    slice16_rt(it.p0, it.p1, 4, o_col, b_col);
                    slice16_rt(it.p0, it.p1, esz, o_val, b_val);
                    StageHdr h{it.mat, it.r0, it.r1, it.p0, b_rp, b_rp + b_col, 0, 0};
                    if (b_rp + b_col + b_val > stage_bytes) {   // cannot happen for a plan built on the host
                        report(status, 2);
                        h.mat = -2;
                        hdr[s] = h;
                        mbar_arrive(&full[s]);
                        continue;
                    }
                    hdr[s] = h;
                    unsigned char* st = stage0 + (size_t)s * stage_bytes;
                    mbar_arrive_expect_tx(&full[s], b_rp + b_col + b_val);
                    bulk_g2s(st, m->rowptr + o_rp, b_rp, &full[s], pol);
                    if (b_col) bulk_g2s(st + b_rp, m->colidx + o_col, b_col, &full[s], pol);
                    if (b_val)
                        bulk_g2s(st + b_rp + b_col, static_cast<const unsigned char*>(m->vals) + o_val * esz, b_val,
                                 &full[s], pol);
                }
                if (!ok) break;
            }
            if (ok) {   // the end marker
                const int s = i % S;
                if (i >= S && !mbar_wait_bounded(&empty[s], ((i / S) - 1) & 1, timeout_ns)) {
                    report(status, 1);
                } else {
                    hdr[s].mat = -1;
                    mbar_arrive(&full[s]);
                }
            }
            // the last producer out resets the tile counter for the next launch
            __threadfence();
            if (atomicAdd(&counters[1], 1u) == gridDim.x - 1) {
                atomicExch(&counters[0], 0u);
                atomicExch(&counters[1], 0u);
            }
        }
        return;
    }

    // ---------------- consumers
    int seq = 0;   // row groups of this block's stream so far, mod TW
    for (int i = 0;; ++i) {
        const int s = i % S;
        if (!mbar_wait_bounded(&full[s], (i / S) & 1, timeout_ns)) {
            report(status, 1);
            mbar_wait_bounded(&full[s], (i / S) & 1, timeout_ns);   // let copies in flight land
            return;
        }
        const StageHdr h = hdr[s];
        if (h.mat == -1) break;
        if (h.mat >= 0) {
            const BatchMat* m = &mats[h.mat];
            const unsigned char* st = stage0 + (size_t)s * stage_bytes;
            const int32_t* rp = reinterpret_cast<const int32_t*>(st) - (h.r0 & ~3);
            const int32_t* col = reinterpret_cast<const int32_t*>(st + h.off_col) - (h.p0 & ~3);
            const unsigned char* vb = st + h.off_val;
            const int rpp = rows_per_pass(m->k, m->vec != 0, m->xt ? 4 : 8);
            const int ng = (h.r1 - h.r0 + rpp - 1) / rpp;
            const int first = (warp - seq + TW) % TW;
            seq = (seq + ng) % TW;
            if (first < ng) {
                const int vt = m->vt;
#define CSRK_DISPATCH(VT, XT, AT) \
    item_dispatch<VT, XT, AT>(m, h.r0, h.r1, h.p0, first, rp, col, vb, alpha, beta, epi, lane)
                if (m->xt) {   // FP32 vectors and accumulation: the inner product of a mixed solve
                    if (vt == csrk::VAL_F32) CSRK_DISPATCH(float, float, float);
                    else CSRK_DISPATCH(bf16_t, float, float);
                } else if (vt == csrk::VAL_F64) {
                    CSRK_DISPATCH(double, double, double);
                } else if (vt == csrk::VAL_F32) {
                    CSRK_DISPATCH(float, double, double);
                } else {
                    CSRK_DISPATCH(bf16_t, double, double);
                }
#undef CSRK_DISPATCH
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ---------------------------------------------------------------- batched CG kernels
constexpr int VT_THREADS = 256;   // vector-kernel block; a multiple of every k (power of two <= 32)

struct SysState {   // per (matrix, right-hand side)
    double rr, pq, alpha, beta, bb, tol2;
    int32_t frozen, iters;
    // csrk_batch_cg_solve only
    double rr_start;   // r.r at the start of the current cycle
    double rr_true;    // last ||b - A64 x||^2
    int32_t done;      // 1 converged (true residual), 2 breakdown (p.q <= 0)
    int32_t replace;   // at the end of this cycle: r = the true residual
    int32_t restart;   //                            p = r
    int32_t pad;
};

// Per-chunk, per-column partial sums of a[i]*b[i] over the chunk's elements.  With k a
// power of two dividing the block size, thread t always sees column t % k.
__device__ void chunk_partial(double v, int k, double* out /* k entries */) {
    __shared__ double red[VT_THREADS / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off >= k && off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane < k) red[warp][lane] = v;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int w = 0; w < VT_THREADS / 32; ++w) t += red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ int sys_of(const int32_t* sys_off, int mat, int c) { return sys_off[mat] + c; }

// B -> R, P (and its FP32 copy P32 when given); X = 0; partial b.b
__global__ void __launch_bounds__(VT_THREADS) bcg_init(const Chunk* __restrict__ chunks, const BatchMat* mats,
                                                       const double* __restrict__ Bv, double* X, double* R,
                                                       double* P, float* P32, double* partials) {
    const Chunk ch = chunks[blockIdx.x];
    const int k = mats[ch.mat].k;
    const int64_t e0 = ch.off, e1 = ch.off + (int64_t)(ch.row1 - ch.row0) * k;
    double v = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += VT_THREADS) {
        const double b = Bv[e];
        X[e] = 0.0;
        R[e] = b;
        P[e] = b;
        if (P32) P32[e] = csrk::dev::f64_to_f32(b);
        v += b * b;
    }
    chunk_partial(v, k, partials + (int64_t)blockIdx.x * 32);
}

// FP32 -> FP64 with integer instructions (exact, like the conversion instruction, which
// would take a slot of GB300's narrow FP64 pipe)
__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return csrk::dev::x_f64(v); }

// The hot vector kernels walk a chunk CHUNK_ILP elements per thread per trip (e, e + 256,
// ...), issuing all of a trip's loads before any arithmetic, so each thread keeps several
// independent requests in flight.  Thread t still sees only column t % k.
constexpr int CHUNK_ILP = 4;

// partial A.B per system; B is FP64 or the FP32 product of a mixed solve
template <typename TB>
__global__ void __launch_bounds__(VT_THREADS) bcg_dot(const Chunk* __restrict__ chunks, const BatchMat* mats,
                                                      const double* __restrict__ A, const TB* __restrict__ Bv,
                                                      double* partials) {
    const Chunk ch = chunks[blockIdx.x];
    const int k = mats[ch.mat].k;
    const int64_t e0 = ch.off, e1 = ch.off + (int64_t)(ch.row1 - ch.row0) * k;
    double v = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += CHUNK_ILP * VT_THREADS) {
        double a[CHUNK_ILP], b[CHUNK_ILP];
#pragma unroll
        for (int u = 0; u < CHUNK_ILP; ++u) {
            const int64_t q = e + u * VT_THREADS;
            a[u] = q < e1 ? A[q] : 0.0;
            b[u] = q < e1 ? as_f64(Bv[q]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < CHUNK_ILP; ++u) v += a[u] * b[u];
    }
    chunk_partial(v, k, partials + (int64_t)blockIdx.x * 32);
}

// R -= alpha Q; partial r.r (X += alpha P is done by bcg_update_p, which reads P anyway,
// when X is NULL here)
template <typename TQ>
__global__ void __launch_bounds__(VT_THREADS) bcg_update_xr(const Chunk* __restrict__ chunks, const BatchMat* mats,
                                                            const int32_t* sys_off, const SysState* st,
                                                            double* __restrict__ X, double* __restrict__ R,
                                                            const double* __restrict__ P,
                                                            const TQ* __restrict__ Q, double* partials) {
    const Chunk ch = chunks[blockIdx.x];
    const int k = mats[ch.mat].k;
    const int64_t e0 = ch.off, e1 = ch.off + (int64_t)(ch.row1 - ch.row0) * k;
    const double alpha = st[sys_of(sys_off, ch.mat, threadIdx.x % k)].alpha;
    double v = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += CHUNK_ILP * VT_THREADS) {
        double x[CHUNK_ILP], r[CHUNK_ILP], p[CHUNK_ILP], q[CHUNK_ILP];
#pragma unroll
        for (int u = 0; u < CHUNK_ILP; ++u) {
            const int64_t i = e + u * VT_THREADS;
            if (i < e1) {
                if (X) {
                    x[u] = X[i];
                    p[u] = P[i];
                }
                r[u] = R[i];
                q[u] = as_f64(Q[i]);
            }
        }
#pragma unroll
        for (int u = 0; u < CHUNK_ILP; ++u) {
            const int64_t i = e + u * VT_THREADS;
            if (i < e1) {
                if (X) X[i] = x[u] + alpha * p[u];
                const double rn = r[u] - alpha * q[u];
                R[i] = rn;
                v += rn * rn;
            }
        }
    }
    chunk_partial(v, k, partials + (int64_t)blockIdx.x * 32);
}

// P = R + beta P (and P32 = P rounded to FP32 when given); with X given, first X += alpha P
// with the old P (the iteration's x update, moved here from bcg_update_xr so that P is read
// once per iteration instead of twice)
__global__ void __launch_bounds__(VT_THREADS) bcg_update_p(const Chunk* __restrict__ chunks, const BatchMat* mats,
                                                           const int32_t* sys_off, const SysState* st,
                                                           const double* __restrict__ R, double* __restrict__ P,
                                                           float* __restrict__ P32, double* __restrict__ X) {
    const Chunk ch = chunks[blockIdx.x];
    const int k = mats[ch.mat].k;
    const int64_t e0 = ch.off, e1 = ch.off + (int64_t)(ch.row1 - ch.row0) * k;
    const SysState& y = st[sys_of(sys_off, ch.mat, threadIdx.x % k)];
    const double beta = y.beta, alpha = y.alpha;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += CHUNK_ILP * VT_THREADS) {
        double r[CHUNK_ILP], p[CHUNK_ILP], x[CHUNK_ILP];
#pragma unroll
        for (int u = 0; u < CHUNK_ILP; ++u) {
            const int64_t i = e + u * VT_THREADS;
            if (i < e1) {
                r[u] = R[i];
                p[u] = P[i];
                if (X) x[u] = X[i];
            }
        }
#pragma unroll
        for (int u = 0; u < CHUNK_ILP; ++u) {
            const int64_t i = e + u * VT_THREADS;
            if (i < e1) {
                if (X) X[i] = x[u] + alpha * p[u];
                const double pn = r[u] + beta * p[u];
                P[i] = pn;
                if (P32) P32[i] = csrk::dev::f64_to_f32(pn);
            }
        }
    }
}

// End of a cycle of csrk_batch_cg_solve: per system, R = T (the true residual) when its
// `replace` flag is set, then P = R (and P32) when `restart` is set.
__global__ void __launch_bounds__(VT_THREADS) bcg_replace(const Chunk* __restrict__ chunks, const BatchMat* mats,
                                                          const int32_t* sys_off, const SysState* st,
                                                          const double* __restrict__ T, double* R, double* P,
                                                          float* P32) {
    const Chunk ch = chunks[blockIdx.x];
    const int k = mats[ch.mat].k;
    const int64_t e0 = ch.off, e1 = ch.off + (int64_t)(ch.row1 - ch.row0) * k;
    const SysState& y = st[sys_of(sys_off, ch.mat, threadIdx.x % k)];
    const bool rep = y.replace, rst = y.restart;
    if (!rep && !rst) return;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += VT_THREADS) {
        const double r = rep ? T[e] : R[e];
        if (rep) R[e] = r;
        if (rst) {
            P[e] = r;
            if (P32) P32[e] = csrk::dev::f64_to_f32(r);
        }
    }
}

// One warp per system: sum the system's chunk partials in chunk order (lanes stride, then
// a fixed shuffle tree), then apply `stage`:
//   0: b.b (init)   1: p.q -> alpha   2: r.r -> beta, freeze when r.r <= margin2 tol^2
//   3: true r.r -> relative residual   4: true r.r at the end of a solve cycle -> converged,
//   or (counted in *active) continue with r replaced / p restarted per the solve's rules
struct FinalizeOpts {
    double margin2;      // stage 2 freeze threshold, as a factor of tol^2
    int32_t mixed;       // stage 4: mixed-precision rules (always replace r)
    int32_t restart;     // stage 4, mixed: always restart p = r
    int32_t* active;     // stage 4: count of systems still running
};

__global__ void bcg_finalize(const int32_t* sys_mat, const int32_t* sys_col, const int32_t* mat_chunk0,
                             const int32_t* mat_chunk1, const double* partials, SysState* st, int32_t nsys,
                             int stage, double rtol, double* out_true, FinalizeOpts o) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nsys) return;
    const int m = sys_mat[s], c = sys_col[s];
    double t = 0.0;
    for (int q = mat_chunk0[m] + lane; q < mat_chunk1[m]; q += 32) t += partials[(int64_t)q * 32 + c];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane != 0) return;
    SysState& y = st[s];
    if (stage == 0) {
        y.bb = t;
        y.rr = t;
        y.rr_start = t;
        y.rr_true = t;
        y.tol2 = rtol * rtol * t;
        y.frozen = (t == 0.0);
        y.done = (t == 0.0);
        y.replace = 0;
        y.restart = 0;
        y.iters = 0;
        y.alpha = 0.0;
        y.beta = 0.0;
    } else if (stage == 1) {
        y.pq = t;
        y.alpha = (y.frozen || !(t > 0.0)) ? 0.0 : y.rr / t;
        if (!y.frozen && !(t > 0.0)) {   // breakdown: the system stops for good
            y.frozen = 1;
            y.done = 2;
        }
    } else if (stage == 2) {
        if (y.frozen) {
            y.beta = 0.0;
            return;
        }
        y.beta = t / y.rr;
        y.rr = t;
        y.iters += 1;
        // stop until the cycle's end: converged by the recursion, or (mixed) diverging --
        // the recursive residual up tenfold within the cycle
        if (t <= o.margin2 * y.tol2 || (o.mixed && t > 100.0 * y.rr_start)) {
            y.frozen = 1;
            y.beta = 0.0;
        }
    } else if (stage == 3) {
        out_true[s] = y.bb > 0.0 ? sqrt(t / y.bb) : 0.0;
    } else {
        y.replace = 0;
        y.restart = 0;
        if (y.done) return;
        y.rr_true = t;
        if (t <= y.tol2) {   // converged on the FP64 residual
            y.done = 1;
            y.frozen = 1;
            y.beta = 0.0;
            return;
        }
        atomicAdd(o.active, 1);
        const bool pending = y.frozen;   // stopped early in the cycle, and not converged
        if (o.mixed) {
            y.replace = 1;
            y.restart = o.restart || t > 4.0 * y.rr || y.rr > 100.0 * y.rr_start;
            y.rr = t;
        } else if (pending) {
            y.replace = 1;
            y.restart = 1;
            y.rr = t;
        }
        y.frozen = 0;
        y.rr_start = y.rr;
    }
}

// copy between the user's per-matrix blocks and the concatenated buffer
__global__ void bcg_gather(const double* const* src, const int64_t* moff, const int64_t* mlen, int32_t nmat,
                           double* dst) {
    for (int m = blockIdx.y; m < nmat; m += gridDim.y)
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mlen[m]; e += (int64_t)gridDim.x * blockDim.x)
            dst[moff[m] + e] = src[m][e];
}
__global__ void bcg_scatter(const double* src, const int64_t* moff, const int64_t* mlen, int32_t nmat,
                            double* const* dst) {
    for (int m = blockIdx.y; m < nmat; m += gridDim.y)
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mlen[m]; e += (int64_t)gridDim.x * blockDim.x)
            dst[m][e] = src[moff[m] + e];
}

}  // namespace

// ------------------------------------------------------------------ the batch object
struct csrk_batch {
    std::vector<csrk_handle> hs;
    std::vector<int32_t> k;
    int device = -1;
    int num_sms = 0;
    int32_t nmat = 0, ntiles = 0, nchunks = 0, nsys = 0;
    int64_t total = 0;               // elements of one concatenated vector block
    BatchMat* d_mats_user = nullptr; // tables: user-bound vectors / internal P,Q / internal X,R
    BatchMat* d_mats_pq = nullptr;
    BatchMat* d_mats_xr = nullptr;
    BatchTile* d_tiles = nullptr;    // direct-load kernel: tiles of whole SSRs
    BatchItem* d_items = nullptr;    // staged kernel: items and tiles of items
    ItemTile* d_itiles = nullptr;
    int32_t nitems = 0, nitiles = 0;
    uint32_t stage_bytes = 0;
    int32_t stages = 0;              // 0: the staged kernel is not used
    int32_t* d_status = nullptr;     // bit 0: a bounded wait gave up; bit 1: an item did not fit
    uint32_t* d_counters = nullptr;
    Chunk* d_chunks = nullptr;
    int32_t *d_sys_mat = nullptr, *d_sys_col = nullptr, *d_sys_off = nullptr;
    int32_t *d_mat_chunk0 = nullptr, *d_mat_chunk1 = nullptr;
    int64_t *d_moff = nullptr, *d_mlen = nullptr;
    std::vector<BatchMat> h_mats;
    std::vector<int64_t> h_moff;     // element offset of each matrix's block in the concatenated vectors
    std::vector<const void*> bound_x, bound_x32;
    std::vector<void*> bound_y, bound_y32;
    BatchMat* h_pinned_mats = nullptr;
    BatchMat* d_mats_user32 = nullptr;   // csrk_batch_spmm with FP32 vectors
    BatchMat* h_pinned_mats32 = nullptr;
    // CG buffers
    double *B = nullptr, *X = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr, *partials = nullptr;
    // csrk_batch_cg_solve: FP32 copies of P and of the inner product, operator tables
    // (inner FP64 P -> Q, inner low precision P32 -> Q32, true residual X -> Q), the
    // running-system counter and its pinned host copy, the per-cycle graph
    float *P32 = nullptr, *Q32 = nullptr;
    BatchMat* d_mats_pq64 = nullptr;
    BatchMat* d_mats_lo = nullptr;
    BatchMat* d_mats_t64 = nullptr;
    int lo_vt = -1;
    int32_t* d_active = nullptr;
    int32_t* h_active = nullptr;
    cudaGraphExec_t sexec = nullptr;
    int sexec_key[3] = {-1, -1, -1};   // inner, replace_every, restart
    SysState* st = nullptr;
    double* d_true = nullptr;
    const double** d_ptrs_in = nullptr;
    double** d_ptrs_out = nullptr;
    unsigned long long timeout_ns = 2000000000ull;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t exec_iters = 0;
    double exec_rtol = 0.0;
};

namespace {
using namespace csrk::rt;

template <typename T>
int dmalloc(T** p, size_t count) {
    if (fault_injected("alloc")) return fail(CSRK_ERR_ALLOC, "batch cudaMalloc: injected fault");
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    return e == cudaSuccess ? CSRK_OK : fail(CSRK_ERR_ALLOC, std::string("batch cudaMalloc: ") + cudaGetErrorString(e));
}
template <typename T>
int upload(T** p, const std::vector<T>& v) {
    int rc = dmalloc(p, v.size());
    if (rc) return rc;
    if (!v.empty()) CK_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "batch upload");
    return CSRK_OK;
}

void batch_free(csrk_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->sexec) cudaGraphExecDestroy(b->sexec);
    for (void* p : {(void*)b->P32, (void*)b->Q32, (void*)b->d_mats_pq64, (void*)b->d_mats_lo,
                    (void*)b->d_mats_t64, (void*)b->d_active, (void*)b->d_mats_user32})
        cudaFree(p);
    if (b->h_pinned_mats32) cudaFreeHost(b->h_pinned_mats32);
    if (b->h_active) cudaFreeHost(b->h_active);
    for (void* p : {(void*)b->d_mats_user, (void*)b->d_mats_pq, (void*)b->d_mats_xr, (void*)b->d_tiles,
                    (void*)b->d_items, (void*)b->d_itiles, (void*)b->d_status, (void*)b->d_counters, (void*)b->d_chunks, (void*)b->d_sys_mat, (void*)b->d_sys_col,
                    (void*)b->d_sys_off, (void*)b->d_mat_chunk0, (void*)b->d_mat_chunk1, (void*)b->d_moff,
                    (void*)b->d_mlen, (void*)b->B, (void*)b->X, (void*)b->R, (void*)b->P, (void*)b->Q,
                    (void*)b->partials, (void*)b->st, (void*)b->d_true, (void*)b->d_ptrs_in,
                    (void*)b->d_ptrs_out})
        cudaFree(p);
    if (b->h_pinned_mats) cudaFreeHost(b->h_pinned_mats);
    if (b->cap) cudaStreamDestroy(b->cap);
}

int launch_batch_spmm(csrk_batch* b, const BatchMat* table, double alpha, double beta, cudaStream_t s) {
    const int epi = (alpha != 1.0 ? csrk::dev::EPI_SCALE : 0) | (beta != 0.0 ? csrk::dev::EPI_ACCUM : 0);
    if (b->stages >= 2) {
        const int grid = std::min<int>(b->nitiles, std::max(1, b->num_sms * 2));
        if (grid == 0) return CSRK_OK;
        const size_t smem = HDR_BYTES + (size_t)b->stages * b->stage_bytes;
        batch_spmm_tma_kernel<<<grid, (TW + 1) * 32, smem, s>>>(table, b->d_items, b->d_itiles, b->nitiles,
                                                                b->d_counters, alpha, beta, epi, b->stage_bytes,
                                                                b->stages, b->timeout_ns, b->d_status);
    } else {
        const int grid = std::min<int>(b->ntiles, std::max(1, b->num_sms * 4));
        if (grid == 0) return CSRK_OK;
        batch_spmm_kernel<<<grid, BW * 32, 0, s>>>(table, b->d_tiles, b->ntiles, b->d_counters, alpha, beta, epi);
    }
    CK_CUDA(cudaGetLastError(), "batch SpMM launch");
    return CSRK_OK;
}

// A device table binding matrix i to the concatenated vectors at xbase / ybase (element
// offset sum_{j<i} n_j k_j), with value type vt (-1: each handle's stored type) and
// FP32 vectors when xt = 1.
int fill_table(csrk_batch* b, BatchMat* table, const void* xbase, void* ybase, int vt = -1, int xt = 0) {
    std::vector<BatchMat> t = b->h_mats;
    const size_t esz = xt ? sizeof(float) : sizeof(double);
    for (int32_t i = 0; i < b->nmat; ++i) {
        if (vt >= 0) {
            int rc = ensure_vals(b->hs[i], vt);
            if (rc) return rc;
            t[i].vals = b->hs[i]->d_vals[vt];
            t[i].vt = vt;
        }
        t[i].xt = xt;
        t[i].vec = 1;   // cudaMalloc'd base, block offsets multiples of 4 elements
        t[i].X = static_cast<const unsigned char*>(xbase) + b->h_moff[i] * esz;
        t[i].Y = static_cast<unsigned char*>(ybase) + b->h_moff[i] * esz;
    }
    CK_CUDA(cudaMemcpy(table, t.data(), t.size() * sizeof(BatchMat), cudaMemcpyHostToDevice), "batch table");
    return CSRK_OK;
}

}  // namespace

extern "C" {

int csrk_batch_create(const csrk_handle* hs, int32_t count, const int32_t* k, csrk_batch_handle* out) {
    if (!out || !hs || !k || count < 1) return fail(CSRK_ERR_ARG, "bad batch arguments");
    NvtxRange range("csrk batch create");
    *out = nullptr;
    csrk_batch* b = new (std::nothrow) csrk_batch();
    if (!b) return fail(CSRK_ERR_ALLOC, "out of host memory");
    int rc = CSRK_OK;
    try {
        b->nmat = count;
        b->hs.assign(hs, hs + count);
        b->k.assign(k, k + count);
        int dev = 0;
        cudaGetDevice(&dev);
        b->device = dev;
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
        std::vector<BatchTile> tiles;
        std::vector<double> weight;
        std::vector<BatchItem> items;
        std::vector<ItemTile> itiles;
        std::vector<int32_t> itile_mat;
        int64_t max_stage = 0;
        int64_t item_bytes = ITEM_BYTES_DEFAULT;
        if (const char* e = std::getenv("CSRK_BATCH_ITEM_BYTES")) item_bytes = std::max<int64_t>(1, std::atoll(e));
        std::vector<Chunk> chunks;
        std::vector<int32_t> sys_mat, sys_col, sys_off(count), mc0(count), mc1(count);
        std::vector<int64_t> moff(count), mlen(count);
        int64_t off = 0;
        for (int32_t i = 0; i < count && !rc; ++i) {
            csrk_matrix* h = hs[i];
            if (!h || !h->have_ptrs) { rc = fail(CSRK_ERR_STATE, "every batch matrix needs its pointer arrays"); break; }
            if (h->n_long > 0) { rc = fail(CSRK_ERR_UNSUPPORTED, "batched matrices take no split long rows"); break; }
            if (k[i] < 1 || k[i] > 64) { rc = fail(CSRK_ERR_ARG, "k must be in [1, 64]"); break; }
            if ((rc = ensure_context(h)) || (rc = ensure_struct(h)) || (rc = ensure_vals(h, (int)h->dtype))) break;
            if (h->device != dev) { rc = fail(CSRK_ERR_STATE, "batch matrices must live on the current device"); break; }
            BatchMat m{};
            m.rowptr = h->d_rowptr;
            m.colidx = h->d_colidx;
            m.vals = h->d_vals[(int)h->dtype];
            m.sr_ptr = h->d_sr_ptr;
            m.desc = h->d_desc;
            m.n = h->m.n;
            m.k = k[i];
            m.vt = (int)h->dtype;
            b->h_mats.push_back(m);
            // tiles of about 32K nonzeros (whole SSRs)
            const int32_t nssr = (int32_t)h->desc.size();
            int32_t t0 = 0;
            int64_t acc = 0;
            for (int32_t t = 0; t < nssr; ++t) {
                acc += h->desc[t].p1 - h->desc[t].p0;
                if (acc >= 32768 || t == nssr - 1) {
                    tiles.push_back({i, t0, t + 1, 0});
                    weight.push_back((double)acc * (k[i] == 1 ? 1.0 : 0.5 + 0.5 * k[i]));
                    t0 = t + 1;
                    acc = 0;
                }
            }
            // items: runs of whole super-rows with at most item_bytes of staged data (at
            // least one super-row each), in tiles of ITEMS_PER_TILE
            {
                const int esz = 8;   // sized for FP64 values, so every operator of a solve fits a stage
                const std::vector<int32_t>& srp = h->sr_ptr;
                const std::vector<int32_t>& rp = h->m.rowptr;
                const int32_t nsr = (int32_t)srp.size() - 1;
                auto staged = [&](int32_t r0, int32_t r1) {
                    int64_t a;
                    uint32_t b1, b2, b3;
                    slice16_rt(r0, (int64_t)r1 + 1, 4, a, b1);
                    slice16_rt(rp[r0], rp[r1], 4, a, b2);
                    slice16_rt(rp[r0], rp[r1], esz, a, b3);
                    return (int64_t)b1 + b2 + b3;
                };
                const size_t first = items.size();
                for (int32_t s0 = 0; s0 < nsr;) {
                    int32_t s1 = s0 + 1;
                    while (s1 < nsr && staged(srp[s0], srp[s1 + 1]) <= item_bytes) ++s1;
                    const int32_t r0 = srp[s0], r1 = srp[s1];
                    items.push_back({i, r0, r1, rp[r0], rp[r1], 0, 0, 0});
                    max_stage = std::max(max_stage, staged(r0, r1));
                    s0 = s1;
                }
                for (size_t q = first; q < items.size(); q += ITEMS_PER_TILE) {
                    itiles.push_back({(int32_t)q, (int32_t)std::min(items.size(), q + ITEMS_PER_TILE)});
                    itile_mat.push_back(i);
                }
            }
            // vector chunks of about 8K elements (whole rows)
            sys_off[i] = (int32_t)sys_mat.size();
            for (int c = 0; c < k[i]; ++c) {
                sys_mat.push_back(i);
                sys_col.push_back(c);
            }
            mc0[i] = (int32_t)chunks.size();
            const int32_t rows_per_chunk = std::max<int32_t>(1, 8192 / k[i]);
            for (int32_t r0 = 0; r0 < m.n; r0 += rows_per_chunk)
                chunks.push_back({i, r0, std::min(m.n, r0 + rows_per_chunk), 0, off + (int64_t)r0 * k[i]});
            mc1[i] = (int32_t)chunks.size();
            moff[i] = off;
            mlen[i] = (int64_t)m.n * k[i];
            off += (mlen[i] + 3) & ~int64_t(3);   // every block 16-byte aligned (FP32) / 32-byte (FP64)
        }
        if (!rc) {
            // Matrices in order of decreasing total work; within a matrix, tiles in SSR
            // order, so the blocks running at any moment cover neighbouring rows of one
            // matrix and share its x window in L2 (tiles sorted by work alone interleave
            // many matrices and overflow L2 with their x windows).
            std::vector<double> mwork(count, 0.0);
            for (size_t q = 0; q < tiles.size(); ++q) mwork[tiles[q].mat] += weight[q];
            std::vector<size_t> order(tiles.size());
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) {
                if (tiles[a].mat != tiles[c].mat) {
                    if (mwork[tiles[a].mat] != mwork[tiles[c].mat])
                        return mwork[tiles[a].mat] > mwork[tiles[c].mat];
                    return tiles[a].mat < tiles[c].mat;
                }
                return tiles[a].t0 < tiles[c].t0;
            });
            std::vector<BatchTile> sorted;
            for (size_t q : order) sorted.push_back(tiles[q]);
            // the staged kernel's tiles in the same matrix order (stable: row order within)
            std::vector<size_t> iorder(itiles.size());
            std::iota(iorder.begin(), iorder.end(), 0);
            std::stable_sort(iorder.begin(), iorder.end(), [&](size_t a, size_t c) {
                const int32_t ma = itile_mat[a], mc = itile_mat[c];
                if (ma == mc) return false;
                if (mwork[ma] != mwork[mc]) return mwork[ma] > mwork[mc];
                return ma < mc;
            });
            std::vector<ItemTile> isorted;
            for (size_t q : iorder) isorted.push_back(itiles[q]);
            b->nitems = (int32_t)items.size();
            b->nitiles = (int32_t)isorted.size();
            // stage plan: two blocks per SM, 2..16 stages of the largest item
            int smem_sm = 0, optin = 0;
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            const int64_t budget = std::min<int64_t>(smem_sm / 2 - 1024, optin);
            const int64_t stage = (max_stage + 127) & ~int64_t(127);
            const int64_t fit = stage > 0 ? (budget - HDR_BYTES) / stage : 0;
            if (fit >= 2 && stage <= (int64_t)UINT32_MAX) {
                b->stage_bytes = (uint32_t)stage;
                b->stages = (int32_t)std::min<int64_t>(fit, MAX_STAGES);
                // the device maximum, not this batch's need: a later batch with smaller
                // stages must not lower the limit under an earlier one
                if (cudaFuncSetAttribute(batch_spmm_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
                    cudaSuccess)
                    rc = fail(CSRK_ERR_CUDA, "batch kernel shared-memory attribute");
            }
            if (!rc) rc = upload(&b->d_items, items);
            if (!rc) rc = upload(&b->d_itiles, isorted);
            if (!rc) rc = dmalloc(&b->d_status, 1);
            if (!rc && cudaMemset(b->d_status, 0, sizeof(int32_t)) != cudaSuccess)
                rc = fail(CSRK_ERR_CUDA, "batch status word");
            b->ntiles = (int32_t)sorted.size();
            b->nchunks = (int32_t)chunks.size();
            b->nsys = (int32_t)sys_mat.size();
            b->total = off;
            if (!rc) rc = upload(&b->d_tiles, sorted);
            if (!rc) rc = upload(&b->d_chunks, chunks);
            if (!rc) rc = upload(&b->d_sys_mat, sys_mat);
            if (!rc) rc = upload(&b->d_sys_col, sys_col);
            if (!rc) rc = upload(&b->d_sys_off, sys_off);
            if (!rc) rc = upload(&b->d_mat_chunk0, mc0);
            if (!rc) rc = upload(&b->d_mat_chunk1, mc1);
            b->h_moff = moff;
            if (!rc) rc = upload(&b->d_moff, moff);
            if (!rc) rc = upload(&b->d_mlen, mlen);
            if (!rc) rc = dmalloc(&b->d_mats_user, count);
            if (!rc) rc = dmalloc(&b->d_mats_pq, count);
            if (!rc) rc = dmalloc(&b->d_mats_xr, count);
            if (!rc) rc = dmalloc(&b->d_counters, 2);
            if (!rc && cudaMemset(b->d_counters, 0, 2 * sizeof(uint32_t)) != cudaSuccess)
                rc = fail(CSRK_ERR_CUDA, "batch counters");
            if (!rc && cudaMallocHost(&b->h_pinned_mats, count * sizeof(BatchMat)) != cudaSuccess)
                rc = fail(CSRK_ERR_ALLOC, "batch pinned table");
        }
    } catch (const std::bad_alloc&) {
        rc = fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return CSRK_OK;
}

int csrk_batch_spmm(csrk_batch_handle b, double alpha, const void* const* X, double beta,
                    void* const* Y, unsigned flags, void* stream) {
    if (!b || !X || !Y) return fail(CSRK_ERR_ARG, "NULL argument");
    const unsigned f32 = CSRK_VEC_PERMUTED | CSRK_X_F32 | CSRK_ACC_F32;
    if (flags != CSRK_VEC_PERMUTED && flags != f32)
        return fail(CSRK_ERR_UNSUPPORTED, "batched SpMM takes vectors in the reordered numbering: flags = "
                                          "CSRK_VEC_PERMUTED (FP64), or with CSRK_X_F32 | CSRK_ACC_F32 (FP32)");
    const int xt = flags == f32 ? 1 : 0;
    if (xt && b->stages < 2)
        return fail(CSRK_ERR_UNSUPPORTED, "FP32 batched SpMM needs the staged kernel "
                                          "(super-rows too large for two shared-memory stages)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if (xt && !b->d_mats_user32) {
        if ((rc = dmalloc(&b->d_mats_user32, b->nmat))) return rc;
        if (cudaMallocHost(&b->h_pinned_mats32, b->nmat * sizeof(BatchMat)) != cudaSuccess)
            return fail(CSRK_ERR_ALLOC, "batch pinned table");
        for (int32_t i = 0; i < b->nmat; ++i)   // FP64-stored values are used rounded to FP32
            if (b->hs[i]->dtype == CSRK_F64 && (rc = ensure_vals(b->hs[i], csrk::VAL_F32))) return rc;
    }
    BatchMat* table = xt ? b->d_mats_user32 : b->d_mats_user;
    BatchMat* pinned = xt ? b->h_pinned_mats32 : b->h_pinned_mats;
    std::vector<const void*>& bx = xt ? b->bound_x32 : b->bound_x;
    std::vector<void*>& by = xt ? b->bound_y32 : b->bound_y;
    // re-bind the vectors only when they changed (the table lives on the device)
    bool same = bx.size() == (size_t)b->nmat;
    for (int32_t i = 0; same && i < b->nmat; ++i) same = bx[i] == X[i] && by[i] == Y[i];
    if (!same) {
        // the pinned staging table may still feed an earlier copy: wait for it first
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
        for (int32_t i = 0; i < b->nmat; ++i) {
            if (b->h_mats[i].n > 0 && (!X[i] || !Y[i] || X[i] == Y[i]))   // empty matrices may pass NULL
                return fail(CSRK_ERR_ARG, "bad vector pointer");
            pinned[i] = b->h_mats[i];
            if (xt && b->hs[i]->dtype == CSRK_F64) {
                pinned[i].vals = b->hs[i]->d_vals[csrk::VAL_F32];
                pinned[i].vt = csrk::VAL_F32;
            }
            pinned[i].xt = xt;
            pinned[i].X = X[i];
            pinned[i].Y = Y[i];
            pinned[i].vec = ((uintptr_t)X[i] % 16 == 0) && ((uintptr_t)Y[i] % 16 == 0);
        }
        CK_CUDA(cudaMemcpyAsync(table, pinned, b->nmat * sizeof(BatchMat), cudaMemcpyHostToDevice, s),
                "bind vectors");
        bx.assign(X, X + b->nmat);
        by.assign(Y, Y + b->nmat);
    }
    return launch_batch_spmm(b, table, alpha, beta, s);
}

}  // extern "C"

namespace {

void bcg_fin(csrk_batch* b, cudaStream_t s, int stage, double rtol = 0.0, double* out = nullptr,
                    FinalizeOpts o = FinalizeOpts{1.0, 0, 0, nullptr}) {
    const int fin_blocks = (b->nsys * 32 + 255) / 256;
    bcg_finalize<<<fin_blocks, 256, 0, s>>>(b->d_sys_mat, b->d_sys_col, b->d_mat_chunk0, b->d_mat_chunk1,
                                            b->partials, b->st, b->nsys, stage, rtol, out, o);
}

int bcg_enqueue_iteration(csrk_batch* b, cudaStream_t s) {
    const int gv = b->nchunks;
    int rc;
    if ((rc = launch_batch_spmm(b, b->d_mats_pq, 1.0, 0.0, s))) return rc;   // Q = A P
    bcg_dot<double><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->P, b->Q, b->partials);
    bcg_fin(b, s, 1);
    bcg_update_xr<double><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->d_sys_off, b->st, nullptr,
                                                    b->R, b->P, b->Q, b->partials);
    bcg_fin(b, s, 2);
    bcg_update_p<<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->d_sys_off, b->st, b->R, b->P, nullptr,
                                           b->X);
    CK_CUDA(cudaGetLastError(), "batched CG launch");
    return CSRK_OK;
}

// One cycle of csrk_batch_cg_solve: E iterations, then the true residual T = B - A64 X
// (into Q), the per-system decision, and r / p replacement where decided.
int bsolve_enqueue_cycle(csrk_batch* b, cudaStream_t s, bool mixed, int32_t E, int restart) {
    const int gv = b->nchunks;
    const FinalizeOpts o2{mixed ? 0.25 : 1.0, mixed ? 1 : 0, 0, nullptr};   // mixed: stop at rtol/2, then verify
    int rc;
    CK_CUDA(cudaMemsetAsync(b->d_active, 0, sizeof(int32_t), s), "reset counter");
    for (int32_t it = 0; it < E; ++it) {
        if (mixed) {
            if ((rc = launch_batch_spmm(b, b->d_mats_lo, 1.0, 0.0, s))) return rc;   // Q32 = A_lo P32
            bcg_dot<float><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->P, b->Q32, b->partials);
            bcg_fin(b, s, 1);
            bcg_update_xr<float><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->d_sys_off, b->st, nullptr,
                                                           b->R, b->P, b->Q32, b->partials);
        } else {
            if ((rc = launch_batch_spmm(b, b->d_mats_pq64, 1.0, 0.0, s))) return rc;   // Q = A64 P
            bcg_dot<double><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->P, b->Q, b->partials);
            bcg_fin(b, s, 1);
            bcg_update_xr<double><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->d_sys_off, b->st, nullptr,
                                                            b->R, b->P, b->Q, b->partials);
        }
        bcg_fin(b, s, 2, 0.0, nullptr, o2);
        bcg_update_p<<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->d_sys_off, b->st, b->R, b->P,
                                               mixed ? b->P32 : nullptr, b->X);
    }
    CK_CUDA(cudaMemcpyAsync(b->Q, b->B, (size_t)b->total * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy B");
    if ((rc = launch_batch_spmm(b, b->d_mats_t64, -1.0, 1.0, s))) return rc;   // Q = B - A64 X
    bcg_dot<double><<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->Q, b->Q, b->partials);
    bcg_fin(b, s, 4, 0.0, nullptr, FinalizeOpts{1.0, mixed ? 1 : 0, restart, b->d_active});
    bcg_replace<<<gv, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->d_sys_off, b->st, b->Q, b->R, b->P,
                                          mixed ? b->P32 : nullptr);
    CK_CUDA(cudaGetLastError(), "batched CG cycle");
    return CSRK_OK;
}

// CG workspace shared by csrk_batch_cg and csrk_batch_cg_solve.
int bcg_workspace(csrk_batch* b) {
    if (b->B) return CSRK_OK;
    const size_t tot = (size_t)b->total;
    int rc;
    if ((rc = dmalloc(&b->B, tot)) || (rc = dmalloc(&b->X, tot)) || (rc = dmalloc(&b->R, tot)) ||
        (rc = dmalloc(&b->P, tot)) || (rc = dmalloc(&b->Q, tot)) ||
        (rc = dmalloc(&b->partials, (size_t)b->nchunks * 32)) || (rc = dmalloc(&b->st, (size_t)b->nsys)) ||
        (rc = dmalloc(&b->d_true, (size_t)b->nsys)) || (rc = dmalloc(&b->d_ptrs_in, (size_t)b->nmat)) ||
        (rc = dmalloc(&b->d_ptrs_out, (size_t)b->nmat)))
        return rc;
    if ((rc = fill_table(b, b->d_mats_pq, b->P, b->Q)) || (rc = fill_table(b, b->d_mats_xr, b->X, b->R)))
        return rc;
    CK_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batch stream");
    return CSRK_OK;
}

// Record `enqueue` on the capture stream into a graph and instantiate it.
template <typename F>
int bcg_capture(csrk_batch* b, cudaGraphExec_t* exec, F enqueue) {
    CK_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = enqueue(b->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    return CSRK_OK;
}

}  // namespace

extern "C" {

int csrk_batch_cg(csrk_batch_handle b, const double* const* B, double* const* Xout, int32_t iters,
                  double rtol, double* relres, int32_t* iters_done, void* stream) {
    if (!b || !B || !Xout || iters < 1 || !(rtol >= 0.0)) return fail(CSRK_ERR_ARG, "bad batched CG arguments");
    for (int32_t i = 0; i < b->nmat; ++i) {
        const int k = b->k[i];
        if (k & (k - 1) || k > 32) return fail(CSRK_ERR_UNSUPPORTED, "batched CG takes k in {1,2,4,8,16,32}");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if ((rc = bcg_workspace(b))) return rc;
    CK_CUDA(cudaMemcpyAsync(b->d_ptrs_in, B, b->nmat * sizeof(double*), cudaMemcpyHostToDevice, s), "B pointers");
    CK_CUDA(cudaMemcpyAsync(b->d_ptrs_out, Xout, b->nmat * sizeof(double*), cudaMemcpyHostToDevice, s), "X pointers");
    const dim3 cg_grid(64, std::min<int32_t>(b->nmat, 65535));
    bcg_gather<<<cg_grid, 256, 0, s>>>(b->d_ptrs_in, b->d_moff, b->d_mlen, b->nmat, b->B);
    bcg_init<<<b->nchunks, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->B, b->X, b->R, b->P, nullptr,
                                               b->partials);
    bcg_fin(b, s, 0, rtol);
    CK_CUDA(cudaGetLastError(), "batched CG init");
    if (!b->exec || b->exec_iters != iters) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
        rc = bcg_capture(b, &b->exec, [&](cudaStream_t cs) {
            int r = CSRK_OK;
            for (int32_t it = 0; it < iters && !r; ++it) r = bcg_enqueue_iteration(b, cs);
            return r;
        });
        if (rc) return rc;
        b->exec_iters = iters;
    }
    CK_CUDA(cudaGraphLaunch(b->exec, s), "graph launch");
    // true residuals: R = B - A X, then per-system norms
    CK_CUDA(cudaMemcpyAsync(b->R, b->B, (size_t)b->total * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy B");
    if ((rc = launch_batch_spmm(b, b->d_mats_xr, -1.0, 1.0, s))) return rc;   // R = B - A X
    bcg_dot<double><<<b->nchunks, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->R, b->R, b->partials);
    bcg_fin(b, s, 3, 0.0, b->d_true);
    bcg_scatter<<<cg_grid, 256, 0, s>>>(b->X, b->d_moff, b->d_mlen, b->nmat, b->d_ptrs_out);
    CK_CUDA(cudaGetLastError(), "batched CG finish");
    std::vector<SysState> hs(b->nsys);
    CK_CUDA(cudaMemcpyAsync(hs.data(), b->st, b->nsys * sizeof(SysState), cudaMemcpyDeviceToHost, s), "read state");
    if (relres)
        CK_CUDA(cudaMemcpyAsync(relres, b->d_true, b->nsys * sizeof(double), cudaMemcpyDeviceToHost, s), "read relres");
    CK_CUDA(cudaStreamSynchronize(s), "synchronise");
    if (iters_done)
        for (int32_t q = 0; q < b->nsys; ++q) iters_done[q] = hs[q].iters;
    return CSRK_OK;
}

int csrk_batch_cg_solve(csrk_batch_handle b, const double* const* B, double* const* Xout, double rtol,
                        int32_t maxit, int inner, int32_t replace_every, int restart, double* relres,
                        int32_t* iters_done, int32_t* cycles_out, void* stream) {
    if (!b || !B || !Xout || maxit < 1 || !(rtol > 0.0) || replace_every < 1 || (restart != 0 && restart != 1))
        return fail(CSRK_ERR_ARG, "bad batched CG arguments");
    if (inner != CSRK_F64 && inner != CSRK_F32 && inner != CSRK_BF16)
        return fail(CSRK_ERR_ARG, "inner must be CSRK_F64, CSRK_F32 or CSRK_BF16");
    for (int32_t i = 0; i < b->nmat; ++i) {
        const int k = b->k[i];
        if (k & (k - 1) || k > 32) return fail(CSRK_ERR_UNSUPPORTED, "batched CG takes k in {1,2,4,8,16,32}");
    }
    const bool mixed = inner != CSRK_F64;
    if (mixed && b->stages < 2)
        return fail(CSRK_ERR_UNSUPPORTED, "mixed-precision batched CG needs the staged SpMM kernel "
                                          "(super-rows too large for two shared-memory stages)");
    NvtxRange range("csrk batch cg solve");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc;
    if ((rc = bcg_workspace(b))) return rc;
    if (!b->d_mats_t64) {   // FP64 operator tables: inner P -> Q, true residual X -> Q
        if ((rc = dmalloc(&b->d_mats_pq64, b->nmat)) || (rc = dmalloc(&b->d_mats_t64, b->nmat)) ||
            (rc = dmalloc(&b->d_active, 1)))
            return rc;
        if (cudaMallocHost(&b->h_active, sizeof(int32_t)) != cudaSuccess)
            return fail(CSRK_ERR_ALLOC, "pinned counter");
        if ((rc = fill_table(b, b->d_mats_pq64, b->P, b->Q, csrk::VAL_F64)) ||
            (rc = fill_table(b, b->d_mats_t64, b->X, b->Q, csrk::VAL_F64)))
            return rc;
    }
    if (mixed) {
        const int lo = inner == CSRK_F32 ? csrk::VAL_F32 : csrk::VAL_BF16;
        if (!b->P32) {
            if ((rc = dmalloc(&b->P32, (size_t)b->total)) || (rc = dmalloc(&b->Q32, (size_t)b->total)) ||
                (rc = dmalloc(&b->d_mats_lo, b->nmat)))
                return rc;
        }
        if (b->lo_vt != lo) {
            if ((rc = fill_table(b, b->d_mats_lo, b->P32, b->Q32, lo, 1))) return rc;
            b->lo_vt = lo;
        }
    }
    const int key[3] = {inner, replace_every, restart};
    if (!b->sexec || std::memcmp(key, b->sexec_key, sizeof(key)) != 0) {
        if (b->sexec) {
            cudaGraphExecDestroy(b->sexec);
            b->sexec = nullptr;
        }
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
        rc = bcg_capture(b, &b->sexec,
                         [&](cudaStream_t cs) { return bsolve_enqueue_cycle(b, cs, mixed, replace_every, restart); });
        if (rc) return rc;
        std::memcpy(b->sexec_key, key, sizeof(key));
    }
    CK_CUDA(cudaMemcpyAsync(b->d_ptrs_in, B, b->nmat * sizeof(double*), cudaMemcpyHostToDevice, s), "B pointers");
    CK_CUDA(cudaMemcpyAsync(b->d_ptrs_out, Xout, b->nmat * sizeof(double*), cudaMemcpyHostToDevice, s), "X pointers");
    const dim3 cg_grid(64, std::min<int32_t>(b->nmat, 65535));
    bcg_gather<<<cg_grid, 256, 0, s>>>(b->d_ptrs_in, b->d_moff, b->d_mlen, b->nmat, b->B);
    bcg_init<<<b->nchunks, VT_THREADS, 0, s>>>(b->d_chunks, b->d_mats_pq, b->B, b->X, b->R, b->P,
                                               mixed ? b->P32 : nullptr, b->partials);
    bcg_fin(b, s, 0, rtol);
    CK_CUDA(cudaGetLastError(), "batched CG init");
    const int32_t max_cycles = (maxit + replace_every - 1) / replace_every;
    int32_t cycles = 0;
    for (; cycles < max_cycles;) {
        CK_CUDA(cudaGraphLaunch(b->sexec, s), "graph launch");
        ++cycles;
        CK_CUDA(cudaMemcpyAsync(b->h_active, b->d_active, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read counter");
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
        if (*b->h_active == 0) break;
    }
    bcg_scatter<<<cg_grid, 256, 0, s>>>(b->X, b->d_moff, b->d_mlen, b->nmat, b->d_ptrs_out);
    CK_CUDA(cudaGetLastError(), "batched CG finish");
    std::vector<SysState> hs(b->nsys);
    CK_CUDA(cudaMemcpyAsync(hs.data(), b->st, b->nsys * sizeof(SysState), cudaMemcpyDeviceToHost, s), "read state");
    CK_CUDA(cudaStreamSynchronize(s), "synchronise");
    bool all = true;
    for (int32_t q = 0; q < b->nsys; ++q) {
        if (relres) relres[q] = hs[q].bb > 0.0 ? std::sqrt(hs[q].rr_true / hs[q].bb) : 0.0;
        if (iters_done) iters_done[q] = hs[q].iters;
        all = all && hs[q].done == 1;
    }
    if (cycles_out) *cycles_out = cycles;
    if (!all) return fail(CSRK_ERR_NOT_CONVERGED, "some systems did not reach rtol (or broke down)");
    return CSRK_OK;
}

int csrk_batch_destroy(csrk_batch_handle b) {
    if (!b) return CSRK_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
    return CSRK_OK;
}

int csrk_batch_info(csrk_batch_handle b, int32_t* nmat, int32_t* nsys, int32_t* ntiles, int64_t* total) {
    if (!b) return fail(CSRK_ERR_ARG, "NULL batch");
    if (nmat) *nmat = b->nmat;
    if (nsys) *nsys = b->nsys;
    if (ntiles) *ntiles = b->stages >= 2 ? b->nitiles : b->ntiles;
    if (total) *total = b->total;
    return CSRK_OK;
}

int csrk_batch_plan(csrk_batch_handle b, int32_t* items, int32_t* stages, int32_t* stage_bytes) {
    if (!b) return fail(CSRK_ERR_ARG, "NULL batch");
    if (items) *items = b->stages >= 2 ? b->nitems : 0;
    if (stages) *stages = b->stages;
    if (stage_bytes) *stage_bytes = (int32_t)b->stage_bytes;
    return CSRK_OK;
}

int csrk_batch_device_status(csrk_batch_handle b, int32_t* status) {
    if (!b || !status) return fail(CSRK_ERR_ARG, "NULL argument");
    CK_CUDA(cudaMemcpy(status, b->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost), "read batch status");
    return CSRK_OK;
}

}  // extern "C"
