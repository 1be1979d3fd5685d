// Internal declarations of the CSR-k library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "csrk.h"

namespace csrk {

// ------------------------------------------------------------------ host CSR
struct CsrHost {
    int32_t n = 0;
    std::vector<int32_t> rowptr;   // n + 1
    std::vector<int32_t> colidx;   // nnz
    std::vector<double> vals;      // nnz
    int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// Per super-super-row work descriptor, derived from ssr_ptr / sr_ptr / rowptr so that a
// kernel learns an SSR's super-row, row and nonzero ranges with one 32-byte load instead
// of three dependent ones.  Not part of the CSR-k format itself.
struct alignas(16) SsrDesc {
    int32_t s0, s1;   // super-rows [s0, s1)
    int32_t r0, r1;   // rows [r0, r1)
    int32_t p0, p1;   // nonzeros [p0, p1)
    int32_t cbase;    // smallest column of the SSR (base of its 16-bit column coding); in
                      // kernels 5 / 6's copy of the descriptors: the elements its x window's
                      // runs cover
    int32_t aux;      // kernels 5 / 6's copy: the number of runs of its x window
};

struct TileStats {
    int32_t max_srs = 0;    // most super-rows in one SSR
    int32_t max_rows = 0;   // most rows in one SSR
    int64_t max_nnz = 0;    // most nonzeros in one SSR
    int32_t max_sr_rows = 0;
    int32_t max_row_len = 0;
};

// host_builder.cpp -------------------------------------------------------------
// Validate a CSR matrix and copy it with each row's columns ascending.  Returns
// CSRK_OK or CSRK_ERR_MATRIX / CSRK_ERR_ARG with a message in err.
int ingest_csr(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
               CsrHost& out, std::string& err);
// Reverse Cuthill-McKee permutation, perm[new] = old.
void rcm_permutation(const CsrHost& a, std::vector<int32_t>& perm);
// Band-k (k = 3) ordering and its variable super-row / super-super-row pointers.
void bandk_permutation(const CsrHost& a, int32_t sr, int32_t ssr, std::vector<int32_t>& perm,
                       std::vector<int32_t>& sr_ptr, std::vector<int32_t>& ssr_ptr);
// B = P A P^T, rows' columns ascending.
void permute_symmetric(const CsrHost& a, const std::vector<int32_t>& perm, CsrHost& b);
void fixed_pointers(int32_t n, int32_t sr, int32_t ssr, std::vector<int32_t>& sr_ptr,
                    std::vector<int32_t>& ssr_ptr);
bool check_pointers(int32_t n, const std::vector<int32_t>& sr_ptr,
                    const std::vector<int32_t>& ssr_ptr, std::string& err);
// Delta-coded 16-bit columns (first entry of a row from the SSR's cbase, then steps);
// false when some code exceeds 65,535.
bool compress_columns(const CsrHost& b, const std::vector<SsrDesc>& desc, std::vector<uint16_t>& col16);
// x windows of kernels 5 and 6: x is staged per SSR in runs of aligned blocks of
// XWIN_ALIGN elements (runs at most XWIN_GAP blocks apart merged).  win holds the
// (start column, offset in the window) pairs of all runs, SSR by SSR, SSR t's from pair
// wptr[t] to wptr[t + 1] (plus one zero pair of padding at the end); xdesc is desc with
// cbase = the elements SSR t's runs cover (the last run may end at n) and aux = its run
// count; colx[p] = the window offset of nonzero p's column; max_win = the longest aligned
// window.  Returns false when some window exceeds 65,536 elements.
// Length order of each SSR's rows (kernels 5 and 6): ord[r0 + j] = offset from the SSR's
// first row r0 of its j-th longest row (ties in row order).  A warp pass then takes rows of
// similar length, so fewer of its FP64 instruction slots go to lanes that have finished.
// Returns the FP64 issue slots (over all warp passes of 32 positions within each super-row)
// of the natural order and of the length order.
void build_row_order(const CsrHost& b, const std::vector<int32_t>& sr_ptr, const std::vector<SsrDesc>& desc,
                     std::vector<uint16_t>& ord, int64_t& slots_natural, int64_t& slots_ordered);
constexpr int32_t XWIN_ALIGN = 4;
constexpr int32_t XWIN_GAP = 2;
bool build_xwin(const CsrHost& b, const std::vector<SsrDesc>& desc, std::vector<SsrDesc>& xdesc,
                std::vector<int32_t>& win, std::vector<int32_t>& wptr, std::vector<uint16_t>& colx,
                int32_t& max_win, int64_t& total_runs);
void build_descs(const CsrHost& b, const std::vector<int32_t>& sr_ptr,
                 const std::vector<int32_t>& ssr_ptr, std::vector<SsrDesc>& desc,
                 TileStats& st);
void narrow_f32(const double* in, float* out, int64_t n);
void narrow_bf16(const double* in, uint16_t* out, int64_t n);
// (hi, lo) FP32 pairs of FP64 values; returns true when every value is 0 or has magnitude
// in [2^-39, 2^60] (the range in which the pair arithmetic keeps FP64 accuracy).
bool split_pairs(const double* in, float* out, int64_t n);
uint16_t f64_to_bf16(double d);
void parallel_for(int64_t n, int64_t grain, void (*fn)(int64_t, int64_t, void*), void* ctx);

// ------------------------------------------------------------------ launches
// VAL_DS: FP64 values stored as (hi, lo) FP32 pairs for the FP32-pipe FP64 path.
enum ValType { VAL_F64 = 0, VAL_F32 = 1, VAL_BF16 = 2, VAL_DS = 3 };

struct KernelConfig {
    int kernel = 0;    // 0 TMA-staged, 1 direct loads; 2 / 3 the same with FP64 values as
                       // FP32 pairs and FP32-pipe arithmetic (FP64 handles only); 4 TMA-staged
                       // with delta-coded 16-bit columns (SpMV, one row per lane, when every
                       // code fits); 5 TMA-staged with each SSR's x window in shared memory
                       // and 16-bit window offsets (SpMV, one row per lane, when every window
                       // fits)
    int lanes = 1;     // lanes per row (SpMV)
    int unroll = 8;    // x gathers issued per lane before the FMAs consume them
    int warps = 8;     // consumer warps per CTA
    int stages = 0;    // 0 = as many as fit
    int ctas = 1;      // CTAs per SM
};

// A segment [p0, p1) of one long row's nonzeros (the irregular-matrix path).
struct LongSeg {
    int32_t p0, p1;
};
constexpr int32_t LSEG = 2048;   // nonzeros per long-row segment

// Arguments of one SpMV / SpMM launch over the device CSR-k form.
struct LaunchArgs {
    const SsrDesc* desc;
    const int32_t* sr_ptr;
    const int32_t* rowptr;
    const void* colidx;   // int32 columns, or uint16 offsets when col16
    const void* vals;
    const void* x;
    void* y;
    int64_t ldx, ldy;
    int32_t k;          // right-hand sides (1 for SpMV)
    int32_t nssr;
    double alpha, beta;
    const int32_t* skip;  // optional device flag: non-zero makes the launch a no-op
    const double* x64;    // pair kernels: the FP64 x (x then holds the FP32-pair split)
    const int32_t* yperm; // SpMV: row r's result goes to y[yperm[r]] (fused unpermute)
    const int32_t* xflag; // pair kernels: split found an out-of-range element
    int32_t* status;
    const int32_t* win = nullptr;   // kernels 5 / 6: x-window runs (pairs), see build_xwin
    const int32_t* wptr = nullptr;  // kernels 5 / 6: first run of each SSR in win
    const uint16_t* rord = nullptr; // kernels 5 / 6 (optional): rows of each SSR in length order
    int32_t n = 0, nsr = 0;         // rows, super-rows (bounds checks of a CSRK_CHECKS build)
    int64_t nnz = 0;                // stored entries (the same)
    TileStats stats;
    int val_type;       // ValType
    bool x_f32;
    bool acc_f32;
    bool spmm;
    int num_sms;
    unsigned long long timeout_ns;
    // rows left out of the super-rows (csrk_split_long_rows): rows row0_long .. +n_long,
    // computed by launch_long_rows from int32 columns, values of lval_type and x = lx
    int32_t n_long = 0, row0_long = 0, nlseg = 0;
    const LongSeg* lseg = nullptr;
    const int32_t* lseg_ptr = nullptr;
    void* lpart = nullptr;
    const int32_t* lcolidx = nullptr;
    const void* lvals = nullptr;
    const void* lx = nullptr;
    int lval_type = 0;
};

// Shared-memory plan of the TMA kernel for one value type.
struct StagePlan {
    uint32_t off_srp, off_rp, off_col, off_val, off_x, off_perm, off_ord, stage_bytes, header_bytes;
    int stages;
};
// x_bytes: room for the x window per stage (kernels 5 / 6; 0 otherwise), with_ord: room for
// the SSR's slice of the rows' length order (kernels 5 / 6).  The 16-bit-column kernels
// (col_bytes 2: kernels 4 to 6) also stage the SSR's slice of the permutation.
bool plan_stages(const TileStats& st, int val_bytes, int max_smem, int want_stages, int col_bytes,
                 StagePlan& plan, int64_t x_bytes = 0, bool with_ord = false);

// spmv_*.cu: launch on `stream`; returns a cudaError_t value (0 = success) or -1 when the
// combination is not compiled in.
int launch_csr3(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan,
                void* stream);
int launch_csr3_f64(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream);
int launch_csr3_f32(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream);
int launch_csr3_bf16(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream);
int launch_csr3_ds(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream);
// The long rows of a launch (no-op when a.n_long == 0); long_rows.cu.
int launch_long_rows(const LaunchArgs& a, void* stream);

// api.cu: message returned by csrk_last_error() for the calling thread.
void set_last_error(const std::string& msg);

// vec_kernels.cu
int launch_gather_rows(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm,
                       int32_t n, int32_t k, int elem_bytes, void* stream);
// Split FP64 x (gathered through perm when given) into FP32 pairs for the pair kernels;
// also writes the gathered FP64 values to x64 when non-NULL; *flag = 1 when any element is
// outside the pair range (the flag is cleared first, on the same stream).
int launch_split_pairs(const double* in, const int32_t* perm, int32_t n, double* x64, void* pairs,
                       int32_t* flag, void* stream);
int launch_bounded_wait_probe(unsigned long long timeout_ns, int32_t* status, void* stream);
// by_int[i] = the solvers' integer FP64 -> FP32 narrowing of in[i], by_cvt[i] = the
// conversion instruction's (device arrays of n)
int launch_narrow_pair(const double* in, int64_t n, float* by_int, float* by_cvt, void* stream);
int launch_scatter_rows(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm,
                        int32_t n, int32_t k, int elem_bytes, void* stream);

}  // namespace csrk
