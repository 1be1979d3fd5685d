// Instantiation and launch of the CSR-3 kernels for one stored value type.  Each value
// type lives in its own translation unit (spmv_f64.cu, spmv_f32.cu, spmv_bf16.cu) so the
// template instances compile in parallel.
#pragma once

#include <algorithm>
#include <mutex>

#include "kernels.cuh"

namespace csrk {
namespace dev {

// Blocks of `kern` that fit on one SM at once with this block size and dynamic shared
// memory (at least 1), remembered per (device, threads, shared memory) for each kernel.
// When the query fails (e.g. while a stream is being captured into a graph) nothing is
// remembered and no limit is applied.
template <typename K>
static int resident_blocks(K kern, int dev, int threads, int smem) {
    struct Entry {
        int dev, threads, smem, blocks;
    };
    static Entry cache[16];
    static int used = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
        if (cache[i].dev == dev && cache[i].threads == threads && cache[i].smem == smem) return cache[i].blocks;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1 << 20;
    }
    blocks = std::max(blocks, 1);
    if (used < 16) cache[used++] = Entry{dev, threads, smem, blocks};
    return blocks;
}

template <typename VT, typename XT, typename AT, int LPR, int MODE, int U>
static int launch_one(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan,
                      cudaStream_t stream) {
    TmaParams P;
    P.desc = a.desc;
    P.sr_ptr = a.sr_ptr;
    P.rowptr = a.rowptr;
    P.colidx = a.colidx;
    P.vals = a.vals;
    P.x = a.x;
    P.y = a.y;
    P.ldx = a.ldx;
    P.ldy = a.ldy;
    P.k = a.k;
    P.nssr = a.nssr;
    P.alpha = a.alpha;
    P.beta = a.beta;
    P.epi = (a.alpha != 1.0 ? EPI_SCALE : 0) | (a.beta != 0.0 ? EPI_ACCUM : 0);
    P.skip = a.skip;
    P.x64 = a.x64;
    P.yperm = a.yperm;
    P.xflag = a.xflag;
    P.status = a.status;
    P.win = reinterpret_cast<const int2*>(a.win);
    P.wptr = a.wptr;
    P.n = a.n;
    P.nsr = a.nsr;
    P.nnz = a.nnz;
    P.off_x = plan.off_x;
    P.off_perm = plan.off_perm;
    P.off_ord = plan.off_ord;
    P.rord = a.rord;
    P.off_srp = plan.off_srp;
    P.off_rp = plan.off_rp;
    P.off_col = plan.off_col;
    P.off_val = plan.off_val;
    P.stage_bytes = plan.stage_bytes;
    P.header_bytes = plan.header_bytes;
    P.stages = plan.stages;
    P.timeout_ns = a.timeout_ns;
    if (a.nssr == 0) return 0;
    if (cfg.kernel == 0) {
        auto kern = csr3_tma_kernel<VT, XT, AT, LPR, MODE, U>;
        const int smem = (int)(plan.header_bytes + (size_t)plan.stages * plan.stage_bytes);
        // Raise the dynamic shared-memory limit to the device maximum once per device, so
        // that later launches (including ones recorded into a CUDA graph) only launch.
        static unsigned long long attr_set = 0;   // bit d: done on device d
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 64 || !(__atomic_load_n(&attr_set, __ATOMIC_ACQUIRE) >> dev & 1ull)) {
            int optin = 0;
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
            if (e != cudaSuccess) return (int)e;
            if (dev < 64) __atomic_fetch_or(&attr_set, 1ull << dev, __ATOMIC_ACQ_REL);
        }
        const int threads = 32 * (cfg.warps + 1);
        // persistent blocks: never more per SM than can be resident at once (registers,
        // shared memory, threads), or a second partial wave would trail the first
        const int ctas = std::min(cfg.ctas, resident_blocks(kern, dev, threads, smem));
        int grid = a.num_sms * ctas;
        if (grid > a.nssr) grid = a.nssr;
        kern<<<grid, threads, smem, stream>>>(P);
    } else if constexpr (MODE != 3 && MODE != 4 && MODE != 5) {   // 16-bit codes are staged only
        auto kern = csr3_direct_kernel<VT, XT, AT, LPR, MODE, U>;
        const int threads = 32 * cfg.warps;
        int grid = a.nssr;
        kern<<<grid, threads, 0, stream>>>(P);
    } else {
        return -1;
    }
    return (int)cudaGetLastError();
}

// SpMV (lanes, unroll) pairs compiled in: row per lane with gather chunks of 4..32, and
// 2..32 lanes per row for long rows.
#define CSRK_SPMV_CASE(L, UU) \
    if (cfg.lanes == L && cfg.unroll == UU) return launch_one<VT, XT, AT, L, 0, UU>(a, cfg, plan, s);

template <typename VT, typename XT, typename AT>
static int dispatch_lanes(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan,
                          cudaStream_t s) {
    if (cfg.kernel == 4) {   // 16-bit column offsets: TMA-staged SpMV, one row per lane
        if (a.spmm || cfg.lanes != 1) return -1;
        KernelConfig c = cfg;
        c.kernel = 0;
        switch (cfg.unroll) {
            case 4: return launch_one<VT, XT, AT, 1, 3, 4>(a, c, plan, s);
            case 8: return launch_one<VT, XT, AT, 1, 3, 8>(a, c, plan, s);
            case 16: return launch_one<VT, XT, AT, 1, 3, 16>(a, c, plan, s);
            default: return -1;
        }
    }
    if (cfg.kernel == 5) {   // x windows staged in shared memory: SpMV, one row per lane
        if (a.spmm || cfg.lanes != 1 || !a.win) return -1;
        KernelConfig c = cfg;
        c.kernel = 0;
        switch (cfg.unroll) {
            case 4: return launch_one<VT, XT, AT, 1, 4, 4>(a, c, plan, s);
            case 8: return launch_one<VT, XT, AT, 1, 4, 8>(a, c, plan, s);
            case 16: return launch_one<VT, XT, AT, 1, 4, 16>(a, c, plan, s);
            default: return -1;
        }
    }
    if (!a.spmm) {
        CSRK_SPMV_CASE(1, 4)
        CSRK_SPMV_CASE(1, 8)
        CSRK_SPMV_CASE(1, 16)
        CSRK_SPMV_CASE(1, 32)
        CSRK_SPMV_CASE(2, 8)
        CSRK_SPMV_CASE(2, 16)
        CSRK_SPMV_CASE(4, 8)
        CSRK_SPMV_CASE(8, 8)
        CSRK_SPMV_CASE(32, 4)
        return -1;
    }
    // SpMM: G lanes per row, columns split across them, at most 2 per lane.
    const int k = a.k;
    if (k <= 2) return launch_one<VT, XT, AT, 2, 1, 1>(a, cfg, plan, s);
    if (k <= 4) return launch_one<VT, XT, AT, 4, 1, 1>(a, cfg, plan, s);
    if (k <= 8) return launch_one<VT, XT, AT, 8, 1, 1>(a, cfg, plan, s);
    if (k <= 16) return launch_one<VT, XT, AT, 16, 1, 1>(a, cfg, plan, s);
    if (k <= 32) return launch_one<VT, XT, AT, 32, 1, 1>(a, cfg, plan, s);
    if (k <= 64) return launch_one<VT, XT, AT, 32, 1, 2>(a, cfg, plan, s);
    return -1;
}
#undef CSRK_SPMV_CASE

}  // namespace dev
}  // namespace csrk
