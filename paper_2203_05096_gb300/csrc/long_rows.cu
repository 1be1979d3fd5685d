// Rows too long for one warp: the irregular-matrix path.
//
// The paper leaves load imbalance on irregular matrices as future work (Sec. 7: choose
// the row mapping by the longest row rather than the mean).  Rows at least a threshold
// long are moved behind all others (csrk_split_long_rows) and left out of the super-rows;
// they are cut into segments of LSEG nonzeros and computed in two deterministic phases:
//   1. one warp per segment and right-hand side: the lanes stride the segment (coalesced
//      column and value loads, x gathered), then a fixed shuffle tree -> partial[s][c];
//   2. one thread per (long row, right-hand side): the row's segment partials summed in
//      segment order, then the alpha / beta epilogue, stored at y[yperm[r]] when the
//      unpermute is fused.
// So a row of a million entries occupies hundreds of warps instead of one.
#include <cuda_runtime.h>
#include <stdint.h>

#include "csrk_internal.h"
#include "kernels.cuh"

namespace csrk {
namespace {

using dev::Acc;
using dev::bf16_t;

constexpr int LR_WARPS = 8;   // warps per block in phase 1

template <typename VT, typename XT, typename AT>
__global__ void __launch_bounds__(LR_WARPS * 32) long_row_partials(
    const LongSeg* __restrict__ seg, int32_t nseg, const int32_t* __restrict__ colidx,
    const VT* __restrict__ vals, const XT* __restrict__ X, int64_t ldx, int32_t k, AT* __restrict__ partial,
    const int32_t* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * LR_WARPS + (threadIdx.x >> 5);
    if (w >= (int64_t)nseg * k) return;
    const int32_t s = (int32_t)(w / k), c = (int32_t)(w % k);
    const LongSeg g = seg[s];
    AT acc = 0;
    for (int64_t p = g.p0 + lane; p < g.p1; p += 32)
        acc = Acc<AT>::fma(vals[p], __ldg(&X[(int64_t)__ldg(&colidx[p]) * ldx + c]), acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) partial[(int64_t)s * k + c] = acc;
}

template <typename XT, typename AT>
__global__ void long_row_finish(const int32_t* __restrict__ seg_ptr, int32_t n_long, int32_t row0,
                                const AT* __restrict__ partial, int32_t k, XT* __restrict__ Y, int64_t ldy,
                                double alpha, double beta, int epi, const int32_t* __restrict__ yperm,
                                const int32_t* skip) {
    if (skip && *skip) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_long * k) return;
    const int32_t i = (int32_t)(t / k), c = (int32_t)(t % k);
    AT acc = 0;
    for (int32_t s = seg_ptr[i]; s < seg_ptr[i + 1]; ++s) acc += partial[(int64_t)s * k + c];
    const int32_t r = row0 + i;
    const int64_t yr = yperm ? __ldg(&yperm[r]) : r;
    dev::store_y<XT, AT>(Y + yr * ldy, c, acc, alpha, beta, epi);
}

template <typename VT, typename XT, typename AT>
int launch_pair(const LaunchArgs& a, cudaStream_t s) {
    const int epi = (a.alpha != 1.0 ? dev::EPI_SCALE : 0) | (a.beta != 0.0 ? dev::EPI_ACCUM : 0);
    const int64_t warps = (int64_t)a.nlseg * a.k;
    const int64_t blocks = (warps + LR_WARPS - 1) / LR_WARPS;
    if (blocks > 0x7fffffff) return (int)cudaErrorInvalidValue;
    AT* part = static_cast<AT*>(a.lpart);
    long_row_partials<VT, XT, AT><<<(unsigned)blocks, LR_WARPS * 32, 0, s>>>(
        a.lseg, a.nlseg, a.lcolidx, static_cast<const VT*>(a.lvals), static_cast<const XT*>(a.lx), a.ldx, a.k,
        part, a.skip);
    const int64_t threads = (int64_t)a.n_long * a.k;
    long_row_finish<XT, AT><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        a.lseg_ptr, a.n_long, a.row0_long, part, a.k, static_cast<XT*>(a.y), a.ldy, a.alpha, a.beta, epi, a.yperm,
        a.skip);
    return (int)cudaGetLastError();
}

}  // namespace

int launch_long_rows(const LaunchArgs& a, void* stream) {
    if (a.n_long == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    switch (a.lval_type) {
        case VAL_F64:
            return launch_pair<double, double, double>(a, s);
        case VAL_F32:
            if (!a.x_f32) return launch_pair<float, double, double>(a, s);
            return a.acc_f32 ? launch_pair<float, float, float>(a, s) : launch_pair<float, float, double>(a, s);
        default:
            if (!a.x_f32) return launch_pair<bf16_t, double, double>(a, s);
            return a.acc_f32 ? launch_pair<bf16_t, float, float>(a, s) : launch_pair<bf16_t, float, double>(a, s);
    }
}

}  // namespace csrk
