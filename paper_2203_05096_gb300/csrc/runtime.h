// Runtime internals shared by the C ABI (api.cu) and the solver (cg.cu): the handle and
// the helpers that build its device form.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "csrk_internal.h"

using csrk::CsrHost;
using csrk::KernelConfig;
using csrk::SsrDesc;
using csrk::StagePlan;
using csrk::TileStats;

// The handle behind csrk_handle.
struct csrk_matrix {
    CsrHost m;                     // current form (reordered after csrk_reorder)
    std::vector<int32_t> perm;     // perm[new] = old; empty = identity
    csrk_dtype dtype = CSRK_F64;
    bool have_ptrs = false;
    int32_t sr = 0, ssr = 0;       // fixed sizes (0 when given explicitly)
    int32_t bandk_sr = 0, bandk_ssr = 0;   // caps of the Band-k pointers in place (0: none)
    int32_t n_long = 0;            // rows moved behind the super-rows (csrk_split_long_rows)
    std::vector<csrk::LongSeg> lseg;      // their segments, row by row
    std::vector<int32_t> lseg_ptr;        // n_long + 1: segments of long row i
    csrk::LongSeg* d_lseg = nullptr;
    int32_t* d_lseg_ptr = nullptr;
    void* d_lpart = nullptr;              // per-segment partial sums (up to 64 columns)
    std::vector<int32_t> sr_ptr, ssr_ptr;
    std::vector<SsrDesc> desc;
    TileStats stats;
    KernelConfig cfg;
    bool cfg_set = false;
    bool kernel_forced = false;    // csrk_set_config asked for the TMA kernel explicitly
    unsigned long long timeout_ns = 2000000000ull;

    // device form
    int device = -1;
    int num_sms = 0;
    int smem_per_sm = 0, smem_optin = 0;
    bool dev_struct = false;       // rowptr/colidx/perm uploaded
    bool dev_ptrs = false;         // sr_ptr/desc uploaded
    int32_t* d_rowptr = nullptr;
    int32_t* d_colidx = nullptr;
    uint16_t* d_col16 = nullptr;   // 16-bit column offsets from each SSR's cbase (kernel 4)
    int col16_ok = -1;             // offsets usable with the current pointers; -1 unknown
    // kernel 5: per-SSR x windows (build_xwin), built and uploaded on first use
    SsrDesc* d_xdesc = nullptr;    // descriptors with the SSR's window runs in cbase / aux
    int32_t* d_win = nullptr;      // (start, offset) run pairs, SSR by SSR
    int32_t* d_wptr = nullptr;     // first run of each SSR in d_win (nssr + 1)
    uint16_t* d_colx = nullptr;    // window offset of each nonzero's column
    int xwin_ok = -1;              // windows usable with the current pointers; -1 unknown
    int32_t max_win = 0;           // longest window (elements, multiple of 4)
    int64_t xwin_runs = 0;         // runs over all SSRs
    uint16_t* d_rord = nullptr;    // rows of each SSR in length order (kernels 5 / 6), uploaded
                                   // only when it saves FP64 issue slots (irregular rows)
    void* d_vals[4] = {nullptr, nullptr, nullptr, nullptr};   // by ValType
    int pairs_ok = -1;             // FP32-pair path usable (values in range); -1 unknown
    int32_t* d_sr_ptr = nullptr;
    SsrDesc* d_desc = nullptr;
    int32_t* d_perm = nullptr;
    int32_t* d_iperm = nullptr;    // inverse permutation, uploaded on the first page-locked host x
    int32_t* d_status = nullptr;
    // scratch: permuted x / y, and device copies of host vectors
    // slots: 0 permuted x, 1 permuted y, 2/3 device copies of host x/y, 4 FP32-pair split
    // of x for the pair kernels, 5 the split's out-of-range flag
    void* d_scratch[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t scratch_bytes[6] = {0, 0, 0, 0, 0, 0};
    // conjugate-gradient workspace (cg.cu), allocated on the first solve
    struct CgWork* cg = nullptr;
    // bumped whenever pointers or the launch shape change (invalidates captured graphs)
    unsigned long long generation = 0;
    // launch shape of the inner SpMV of a mixed-precision solve, by value type (FP32 /
    // BF16 values, FP32 x and accumulation), timed on the current pointers at the first
    // solve of that precision (tune_inner); valid while generation is unchanged
    KernelConfig inner_cfg[4];
    unsigned long long inner_gen[4] = {~0ull, ~0ull, ~0ull, ~0ull};
};

namespace csrk {
namespace rt {

// Host-side fault injection for tests: CSRK_FAULT names steps that should fail as if the
// CUDA call behind them had ("alloc": device allocations -> CSRK_ERR_ALLOC; "h2d": uploads
// of the matrix -> CSRK_ERR_CUDA; "tune": the autotuner -> CSRK_ERR_CUDA).  Nothing is
// injected on the device.
bool fault_injected(const char* step);

// NVTX range around a host-side stage (visible in a profiler's timeline; a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
};

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
size_t val_size(int vt);
int ensure_context(csrk_matrix* h);
int ensure_struct(csrk_matrix* h);
int ensure_vals(csrk_matrix* h, int vt);
int ensure_scratch(csrk_matrix* h, int slot, size_t bytes);
KernelConfig default_config(const csrk_matrix* h);
bool pairs_available(csrk_matrix* h);
bool col16_available(csrk_matrix* h);
bool xwin_available(csrk_matrix* h);
bool mode3_compiled(int lanes, int unroll);
// xsz: bytes per x element of the launch (kernel 5 stages x); x: the launch's x, or NULL
// when unknown (kernel 5 copies x by TMA and needs it 16-byte aligned); spmm: the launch
// is an SpMM (kernels 2-5 are SpMV only and give way to kernel 0)
int resolve_config(csrk_matrix* h, int vt, KernelConfig& cfg, StagePlan& plan, int xsz = 8,
                   const void* x = nullptr, bool spmm = false);
int compute(csrk_matrix* h, int32_t k, bool spmm, double alpha, const void* X, int64_t ldx,
            double beta, void* Y, int64_t ldy, unsigned flags, void* stream);
// The CSR-3 kernel alone on device vectors in the reordered numbering, with value type vt;
// when skip is non-NULL and *skip != 0 at launch time on the device, the kernel exits at
// once (used by captured solver iterations after convergence).
void free_cg(csrk_matrix* h);
int launch_spmv_dev(csrk_matrix* h, int vt, const void* x, void* y, double alpha, double beta,
                    bool x_f32, bool acc_f32, const int32_t* skip, cudaStream_t s);
// Time launch shapes of the vt-valued SpMV with FP32 x and accumulation (the inner product
// of a mixed-precision solve) on the current pointers and keep the fastest for vt.  x, y:
// device FP32 vectors of n (contents irrelevant).  Runs on a private stream, synchronously.
int tune_inner(csrk_matrix* h, int vt, const void* x, void* y);

}  // namespace rt
}  // namespace csrk

#define CK_CUDA(call, what)                                                  \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return csrk::rt::cuda_fail(e_, what);         \
    } while (0)
