// C ABI entry points and the device runtime behind them: handle life cycle, one-time
// upload of the CSR-k form, library-owned scratch vectors, launch configuration and the
// permute -> CSR-3 kernel -> unpermute sequence of a compute call.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>

#include "runtime.h"

using namespace csrk;

namespace csrk {
namespace rt {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    return fail(CSRK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t val_size(int vt) { return vt == VAL_F64 ? 8 : (vt == VAL_F32 ? 4 : 2); }

}  // namespace rt
}  // namespace csrk

void csrk::set_last_error(const std::string& msg) { csrk::rt::g_last_error = msg; }

namespace csrk {
namespace rt {

bool fault_injected(const char* step) {
    const char* f = std::getenv("CSRK_FAULT");
    if (!f || !*f) return false;
    const std::string list = std::string(",") + f + ",";
    return list.find(std::string(",") + step + ",") != std::string::npos;
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

void free_xwin(csrk_matrix* h) {
    cudaFree(h->d_xdesc);
    cudaFree(h->d_win);
    cudaFree(h->d_wptr);
    cudaFree(h->d_colx);
    cudaFree(h->d_rord);
    h->d_xdesc = nullptr;
    h->d_win = nullptr;
    h->d_wptr = nullptr;
    h->d_colx = nullptr;
    h->d_rord = nullptr;
    h->xwin_ok = -1;
    h->max_win = 0;
}

void free_ptrs(csrk_matrix* h) {
    free_xwin(h);
    cudaFree(h->d_sr_ptr);
    cudaFree(h->d_desc);
    cudaFree(h->d_lseg);
    cudaFree(h->d_lseg_ptr);
    cudaFree(h->d_lpart);
    h->d_sr_ptr = nullptr;
    h->d_desc = nullptr;
    h->d_lseg = nullptr;
    h->d_lseg_ptr = nullptr;
    h->d_lpart = nullptr;
    h->dev_ptrs = false;
}

void free_struct(csrk_matrix* h) {
    free_ptrs(h);
    cudaFree(h->d_rowptr);
    cudaFree(h->d_colidx);
    cudaFree(h->d_col16);
    h->d_col16 = nullptr;
    h->col16_ok = -1;
    cudaFree(h->d_perm);
    cudaFree(h->d_iperm);
    h->d_rowptr = h->d_colidx = h->d_perm = h->d_iperm = nullptr;
    h->dev_struct = false;
}

void free_device(csrk_matrix* h) {
    if (h->device < 0) return;
    free_cg(h);
    free_struct(h);
    for (auto& v : h->d_vals) {
        cudaFree(v);
        v = nullptr;
    }
    for (int i = 0; i < 6; ++i) {
        cudaFree(h->d_scratch[i]);
        h->d_scratch[i] = nullptr;
        h->scratch_bytes[i] = 0;
    }
    cudaFree(h->d_status);
    h->d_status = nullptr;
}

// Allocate `count` elements of `esz` bytes plus 16 elements of zeroed padding (the TMA
// kernel rounds slices out to 16-byte boundaries) and copy `count` elements from host.
template <typename T>
int upload_padded(T** dst, const void* src, size_t count, size_t esz, const char* what) {
    const size_t bytes = (count + 16) * esz;
    void* p = nullptr;
    if (fault_injected("alloc")) return fail(CSRK_ERR_ALLOC, std::string("cudaMalloc ") + what + ": injected fault");
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(CSRK_ERR_ALLOC, std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
    e = cudaMemset(p, 0, bytes);
    if (e == cudaSuccess && count) e = cudaMemcpy(p, src, count * esz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && fault_injected("h2d")) {
        cudaFree(p);
        return fail(CSRK_ERR_CUDA, std::string(what) + ": injected copy fault");
    }
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(e, what);
    }
    *dst = static_cast<T*>(p);
    return CSRK_OK;
}

int ensure_context(csrk_matrix* h) {
    int dev = 0;
    CK_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (h->device >= 0 && h->device != dev)
        return fail(CSRK_ERR_STATE, "handle's device copies live on device " + std::to_string(h->device) +
                                        " but device " + std::to_string(dev) + " is current");
    if (h->device < 0) {
        h->device = dev;
        CK_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev), "attr");
        CK_CUDA(cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev), "attr");
        CK_CUDA(cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attr");
        void* p = nullptr;
        CK_CUDA(cudaMalloc(&p, 16), "cudaMalloc status");
        CK_CUDA(cudaMemset(p, 0, 16), "cudaMemset status");
        h->d_status = static_cast<int32_t*>(p);
    }
    return CSRK_OK;
}

int ensure_struct(csrk_matrix* h) {
    const CsrHost& m = h->m;
    int rc;
    if (!h->dev_struct) {
        NvtxRange range("csrk upload");
        if ((rc = upload_padded(&h->d_rowptr, m.rowptr.data(), m.rowptr.size(), 4, "rowptr"))) return rc;
        if ((rc = upload_padded(&h->d_colidx, m.colidx.data(), m.colidx.size(), 4, "colidx"))) return rc;
        if (!h->perm.empty())
            if ((rc = upload_padded(&h->d_perm, h->perm.data(), h->perm.size(), 4, "perm"))) return rc;
        h->dev_struct = true;
    }
    if (!h->dev_ptrs) {
        if ((rc = upload_padded(&h->d_sr_ptr, h->sr_ptr.data(), h->sr_ptr.size(), 4, "sr_ptr"))) return rc;
        if ((rc = upload_padded(&h->d_desc, h->desc.data(), h->desc.size(), sizeof(SsrDesc), "desc"))) return rc;
        if (h->n_long > 0) {
            if ((rc = upload_padded(&h->d_lseg, h->lseg.data(), h->lseg.size(), sizeof(LongSeg), "long segments")) ||
                (rc = upload_padded(&h->d_lseg_ptr, h->lseg_ptr.data(), h->lseg_ptr.size(), 4, "long rows")))
                return rc;
            CK_CUDA(cudaMalloc(&h->d_lpart, h->lseg.size() * 64 * sizeof(double)), "long-row partials");
        }
        h->dev_ptrs = true;
    }
    return CSRK_OK;
}

int ensure_vals(csrk_matrix* h, int vt) {
    if (h->d_vals[vt]) return CSRK_OK;
    const CsrHost& m = h->m;
    const size_t nnz = m.vals.size();
    if (vt == VAL_F64) return upload_padded(reinterpret_cast<double**>(&h->d_vals[vt]), m.vals.data(), nnz, 8, "vals");
    if (vt == VAL_DS) {
        std::vector<float> tmp(2 * nnz);
        h->pairs_ok = split_pairs(m.vals.data(), tmp.data(), (int64_t)nnz) ? 1 : 0;
        return upload_padded(reinterpret_cast<uint64_t**>(&h->d_vals[vt]), tmp.data(), nnz, 8, "vals pairs");
    }
    if (vt == VAL_F32) {
        std::vector<float> tmp(nnz);
        narrow_f32(m.vals.data(), tmp.data(), (int64_t)nnz);
        return upload_padded(reinterpret_cast<float**>(&h->d_vals[vt]), tmp.data(), nnz, 4, "vals f32");
    }
    std::vector<uint16_t> tmp(nnz);
    narrow_bf16(m.vals.data(), tmp.data(), (int64_t)nnz);
    return upload_padded(reinterpret_cast<uint16_t**>(&h->d_vals[vt]), tmp.data(), nnz, 2, "vals bf16");
}

int ensure_scratch(csrk_matrix* h, int slot, size_t bytes) {
    if (h->scratch_bytes[slot] >= bytes) return CSRK_OK;
    cudaFree(h->d_scratch[slot]);
    h->d_scratch[slot] = nullptr;
    h->scratch_bytes[slot] = 0;
    if (fault_injected("alloc")) return fail(CSRK_ERR_ALLOC, "cudaMalloc scratch: injected fault");
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(CSRK_ERR_ALLOC, std::string("cudaMalloc scratch: ") + cudaGetErrorString(e));
    h->d_scratch[slot] = p;
    h->scratch_bytes[slot] = bytes;
    return CSRK_OK;
}

// Inverse of perm (iperm[old] = new) on the device, for the permute that reads a
// page-locked host x in its own order and scatters it into the reordered numbering.
int ensure_iperm(csrk_matrix* h) {
    if (h->d_iperm || h->perm.empty()) return CSRK_OK;
    std::vector<int32_t> inv(h->perm.size());
    for (size_t i = 0; i < h->perm.size(); ++i) inv[(size_t)h->perm[i]] = (int32_t)i;
    return upload_padded(&h->d_iperm, inv.data(), inv.size(), 4, "inverse permutation");
}

// Device address of a page-locked, mapped host pointer (cudaHostAlloc, cudaHostRegister);
// NULL for pageable memory, whose contents go through cudaMemcpyAsync instead.
const void* mapped_host_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int default_lanes(const csrk_matrix* h) {
    const double mean = h->m.n ? (double)h->m.nnz() / h->m.n : 0.0;
    if (mean <= 32) return 1;
    if (mean <= 64) return 2;
    if (mean <= 128) return 4;
    if (mean <= 256) return 8;
    return 32;
}

// (lanes, unroll) pairs compiled into the kernels.
bool pair_compiled(int lanes, int unroll) {
    static const int pairs[][2] = {{1, 4}, {1, 8}, {1, 16}, {1, 32}, {2, 8}, {2, 16}, {4, 8}, {8, 8}, {32, 4}};
    for (auto& p : pairs)
        if (p[0] == lanes && p[1] == unroll) return true;
    return false;
}

// Gather chunk for a lane count: 8 (or 4 for rows of at most 4 entries per lane).  A
// chunk of 8 keeps the TMA kernel at 56 registers, so two blocks of 16 consumer warps fit
// on an SM; longer chunks only pay when a single block per SM is wanted.
int default_unroll(int lanes, int max_row_len) {
    const int share = (max_row_len + lanes - 1) / std::max(1, lanes);
    if (lanes == 32) return 4;
    if (lanes == 1 && share <= 4) return 4;
    return 8;
}

KernelConfig default_config(const csrk_matrix* h) {
    KernelConfig c;
    c.lanes = default_lanes(h);
    c.unroll = default_unroll(c.lanes, h->have_ptrs ? h->stats.max_row_len : 32);
    c.warps = 16;
    c.ctas = 0;   // auto: 2 blocks per SM when two stages fit, else 1
    return c;
}

// The FP32-pair FP64 path needs FP64 storage, every value in [2^-39, 2^60] (or 0) and rows
// of at most 48 entries (its error bound grows with the row length).
bool pairs_available(csrk_matrix* h) {
    if (h->dtype != CSRK_F64 || h->stats.max_row_len > 48) return false;
    if (h->pairs_ok < 0) {
        std::vector<float> tmp(2 * h->m.vals.size());
        h->pairs_ok = split_pairs(h->m.vals.data(), tmp.data(), (int64_t)h->m.vals.size()) ? 1 : 0;
    }
    return h->pairs_ok == 1;
}

// (lanes, unroll) pairs compiled with 16-bit column offsets (kernel 4).
bool mode3_compiled(int lanes, int unroll) { return lanes == 1 && (unroll == 4 || unroll == 8 || unroll == 16); }

// Delta-coded 16-bit columns (kernel 4) need every code to fit 16 bits; the coded array is
// built and uploaded on the first ask for the current pointers.
bool col16_available(csrk_matrix* h) {
    if (h->col16_ok < 0) {
        h->col16_ok = 0;
        std::vector<uint16_t> tmp;
        if (h->have_ptrs && compress_columns(h->m, h->desc, tmp) &&
            upload_padded(&h->d_col16, tmp.data(), tmp.size(), 2, "col16") == CSRK_OK)
            h->col16_ok = 1;
    }
    return h->col16_ok == 1;
}

// Kernel 5's x windows (build_xwin) need every window within 65,536 elements; the
// descriptors, runs and window codes are built and uploaded on the first ask for the
// current pointers.
bool xwin_available(csrk_matrix* h) {
    if (h->xwin_ok < 0) {
        h->xwin_ok = 0;
        if (!h->have_ptrs || h->desc.empty()) return false;
        NvtxRange range("csrk x windows");
        std::vector<SsrDesc> xdesc;
        std::vector<int32_t> win, wptr;
        std::vector<uint16_t> colx;
        int32_t mw = 0;
        int64_t runs = 0;
        if (build_xwin(h->m, h->desc, xdesc, win, wptr, colx, mw, runs) &&
            upload_padded(&h->d_xdesc, xdesc.data(), xdesc.size(), sizeof(SsrDesc), "x-window descriptors") == CSRK_OK &&
            upload_padded(&h->d_win, win.data(), win.size(), 4, "x-window runs") == CSRK_OK &&
            upload_padded(&h->d_wptr, wptr.data(), wptr.size(), 4, "x-window run pointers") == CSRK_OK &&
            upload_padded(&h->d_colx, colx.data(), colx.size(), 2, "x-window codes") == CSRK_OK) {
            h->xwin_ok = 1;
            h->max_win = mw;
            h->xwin_runs = runs;
            // rows of unequal length: hand them to warp passes in length order when that
            // saves at least 5 % of the passes' FP64 issue slots
            std::vector<uint16_t> ord;
            int64_t nat = 0, srt = 0;
            build_row_order(h->m, h->sr_ptr, h->desc, ord, nat, srt);
            if (srt < nat - nat / 20 && upload_padded(&h->d_rord, ord.data(), ord.size(), 2, "row order") != CSRK_OK)
                h->d_rord = nullptr;   // the natural order still works
        } else {
            free_xwin(h);
            h->xwin_ok = 0;
        }
    }
    return h->xwin_ok == 1;
}

// (lanes, unroll) pairs compiled with x windows (kernel 5).
bool mode4_compiled(int lanes, int unroll) { return lanes == 1 && (unroll == 4 || unroll == 8 || unroll == 16); }

int smem_budget(const csrk_matrix* h, int ctas) {
    int per_cta = h->smem_per_sm / std::max(1, ctas) - 1024;
    return std::min(per_cta, h->smem_optin);
}

}  // namespace rt
}  // namespace csrk

bool csrk::plan_stages(const TileStats& st, int val_bytes, int max_smem, int want_stages, int col_bytes,
                       StagePlan& plan, int64_t x_bytes, bool with_ord) {
    auto r16 = [](int64_t v) { return (v + 15) & ~int64_t(15); };
    // each slice is rounded out to 16-byte boundaries at both ends: room for the largest
    // slice plus up to 16 bytes' worth of elements
    const int64_t srp = r16((int64_t)(st.max_srs + 8) * 4);
    const int64_t rp = r16((int64_t)(st.max_rows + 8) * 4);
    const int64_t col = r16((st.max_nnz + 32 / col_bytes) * col_bytes);
    const int64_t val = r16((st.max_nnz + 32 / val_bytes) * val_bytes);
    const int64_t xw = r16(x_bytes);
    // kernels 4 to 6 also stage the SSR's slice of the permutation (the fused unpermute)
    const int64_t pm = x_bytes > 0 || col_bytes == 2 ? rp : 0;
    // ... and, for irregular rows, the SSR's slice of the rows' length order
    const int64_t od = x_bytes > 0 && with_ord ? r16((int64_t)(st.max_rows + 16) * 2) : 0;
    int64_t stage = srp + rp + col + val + xw + pm + od;
    stage = (stage + 127) & ~int64_t(127);
    // header: per stage two mbarriers and one 32-byte descriptor
    int64_t s = std::min<int64_t>(max_smem / (stage + 48), 16);
    if (want_stages > 0) s = std::min<int64_t>(s, want_stages);
    const int64_t header = r16(48 * std::max<int64_t>(s, 1));
    if (s < 2 || s * stage + header > max_smem || stage > (int64_t)UINT32_MAX) return false;
    plan.off_srp = 0;
    plan.off_rp = (uint32_t)srp;
    plan.off_col = (uint32_t)(srp + rp);
    plan.off_val = (uint32_t)(srp + rp + col);
    plan.off_x = (uint32_t)(srp + rp + col + val);
    plan.off_perm = (uint32_t)(srp + rp + col + val + xw);
    plan.off_ord = (uint32_t)(srp + rp + col + val + xw + pm);
    plan.stage_bytes = (uint32_t)stage;
    plan.header_bytes = (uint32_t)header;
    plan.stages = (int)s;
    return true;
}

int csrk::launch_csr3(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan,
                      void* stream) {
    int e;
    if (cfg.kernel == 2 || cfg.kernel == 3 || cfg.kernel == 6) e = launch_csr3_ds(a, cfg, plan, stream);
    else if (a.val_type == VAL_F64) e = launch_csr3_f64(a, cfg, plan, stream);
    else if (a.val_type == VAL_F32) e = launch_csr3_f32(a, cfg, plan, stream);
    else e = launch_csr3_bf16(a, cfg, plan, stream);
    if (e == 0 && a.n_long > 0) e = launch_long_rows(a, stream);
    return e;
}

namespace csrk {
namespace rt {

// The long rows of a launch (csrk_split_long_rows): int32 columns, and for the pair path
// the FP64 values and x.
void fill_long_rows(const csrk_matrix* h, LaunchArgs& a, bool pairs) {
    if (h->n_long == 0) return;
    a.n_long = h->n_long;
    a.row0_long = h->m.n - h->n_long;
    a.nlseg = (int32_t)h->lseg.size();
    a.lseg = h->d_lseg;
    a.lseg_ptr = h->d_lseg_ptr;
    a.lpart = h->d_lpart;
    a.lcolidx = h->d_colidx;
    a.lvals = pairs ? h->d_vals[VAL_F64] : a.vals;
    a.lval_type = pairs ? (int)VAL_F64 : a.val_type;
    a.lx = pairs ? static_cast<const void*>(a.x64) : a.x;
}

// The matrix arrays a launch of kernel cfg.kernel reads: the SSR descriptors, pointers and
// column form (int32, 16-bit delta codes, or 16-bit window offsets with the windows' own
// descriptors and runs).
void fill_matrix_args(const csrk_matrix* h, const KernelConfig& cfg, LaunchArgs& a) {
    a.sr_ptr = h->d_sr_ptr;
    a.rowptr = h->d_rowptr;
    const bool win = cfg.kernel == 5 || cfg.kernel == 6;
    a.desc = win ? h->d_xdesc : h->d_desc;
    a.colidx = win ? (const void*)h->d_colx : (cfg.kernel == 4 ? (const void*)h->d_col16 : (const void*)h->d_colidx);
    a.win = win ? h->d_win : nullptr;
    a.wptr = win ? h->d_wptr : nullptr;
    a.rord = win ? h->d_rord : nullptr;
    a.n = h->m.n;
    a.nsr = (int32_t)h->sr_ptr.size() - 1;
    a.nnz = h->m.nnz();
}

// Resolve the launch configuration and stage plan for this handle and value type.
int resolve_config(csrk_matrix* h, int vt, KernelConfig& cfg, StagePlan& plan, int xsz, const void* x,
                   bool spmm) {
    // the tuned / forced shape belongs to the handle's own value type; other value types
    // (the inner SpMV of a mixed-precision solve) start from the default shape
    cfg = (h->cfg_set && vt == (int)h->dtype) ? h->cfg : default_config(h);
    plan = StagePlan{};
    if (spmm) {   // the pair, 16-bit-column and x-window kernels are SpMV only
        if (cfg.kernel == 2 || cfg.kernel == 3) cfg.kernel -= 2;
        else if (cfg.kernel >= 4) cfg.kernel = 0;   // 4, 5, 6
    }
    const bool forced = h->kernel_forced && vt == (int)h->dtype && !spmm;
    // other value types (a mixed solve's inner product) take the shape timed for them on
    // these pointers (tune_inner), else the 16-bit column coding whenever it fits: their
    // bytes are mostly indices
    if (vt != (int)h->dtype && !spmm && vt < 4 && h->inner_gen[vt] == h->generation) {
        cfg = h->inner_cfg[vt];
    } else if (vt != (int)h->dtype && cfg.kernel == 0 && mode3_compiled(cfg.lanes, cfg.unroll) &&
               col16_available(h)) {
        cfg.kernel = 4;
    }
    if ((cfg.kernel == 2 || cfg.kernel == 3 || cfg.kernel == 6) && (vt != VAL_F64 || !pairs_available(h))) {
        if (forced)
            return fail(CSRK_ERR_UNSUPPORTED, "the FP32-pair FP64 path needs FP64 values in [2^-39, 2^60] "
                                              "and rows of at most 48 entries");
        cfg.kernel = cfg.kernel == 6 ? 5 : cfg.kernel - 2;
    }
    if (cfg.kernel == 6 && (!mode4_compiled(cfg.lanes, cfg.unroll) || !xwin_available(h) ||
                            (x && (reinterpret_cast<uintptr_t>(x) & 15u)))) {
        if (forced)
            return fail(CSRK_ERR_UNSUPPORTED, "x windows need every super-super-row's window within 65,536 "
                                              "elements, lanes 1, unroll 4, 8 or 16 and a 16-byte aligned x");
        cfg.kernel = 2;
    }
    if (cfg.kernel == 5 && (!mode4_compiled(cfg.lanes, cfg.unroll) || !xwin_available(h) ||
                            (x && (reinterpret_cast<uintptr_t>(x) & 15u)))) {
        if (forced)
            return fail(CSRK_ERR_UNSUPPORTED, "x windows need every super-super-row's window within 65,536 "
                                              "elements, lanes 1, unroll 4, 8 or 16 and a 16-byte aligned x");
        cfg.kernel = 4;
    }
    if (cfg.kernel == 4 && (!col16_available(h) || !mode3_compiled(cfg.lanes, cfg.unroll))) {
        if (forced)
            return fail(CSRK_ERR_UNSUPPORTED, "16-bit columns need every row's first column within 65,535 "
                                              "of its SSR's smallest and every step between a row's columns "
                                              "at most 65,535; lanes 1 and unroll 4, 8 or 16");
        cfg.kernel = 0;
    }
    if ((cfg.kernel == 2 || cfg.kernel == 3) && cfg.unroll != 4 && cfg.unroll != 8 && cfg.unroll != 16)
        cfg.unroll = 8;
    if (cfg.kernel == 5 || cfg.kernel == 6) {   // the windows must fit the stages as well
        const int64_t xb = (int64_t)h->max_win * xsz;
        const bool ord = h->d_rord != nullptr;
        if (cfg.ctas == 0)
            cfg.ctas = plan_stages(h->stats, (int)val_size(vt), smem_budget(h, 2), cfg.stages, 2, plan, xb, ord) ? 2 : 1;
        if (plan_stages(h->stats, (int)val_size(vt), smem_budget(h, cfg.ctas), cfg.stages, 2, plan, xb, ord))
            return CSRK_OK;
        if (forced)
            return fail(CSRK_ERR_UNSUPPORTED, "super-super-rows and their x windows too large for two "
                                              "shared-memory stages; choose smaller sizes");
        if (cfg.kernel == 6) {
            cfg.kernel = 2;
        } else {
            cfg.kernel = 4;
            if (!col16_available(h) || !mode3_compiled(cfg.lanes, cfg.unroll)) cfg.kernel = 0;
        }
    }
    const bool staged = cfg.kernel == 0 || cfg.kernel == 2 || cfg.kernel == 4;
    const int cb = cfg.kernel == 4 ? 2 : 4;
    if (cfg.ctas == 0)
        cfg.ctas = (staged && plan_stages(h->stats, (int)val_size(vt), smem_budget(h, 2), cfg.stages, cb, plan)) ? 2 : 1;
    if (staged) {
        if (!plan_stages(h->stats, (int)val_size(vt), smem_budget(h, cfg.ctas), cfg.stages, cb, plan)) {
            if (forced)
                return fail(CSRK_ERR_UNSUPPORTED, "super-super-rows too large for two shared-memory stages; "
                                                  "choose smaller sizes or the direct kernel");
            cfg.kernel = cfg.kernel == 2 ? 3 : 1;   // the SSRs do not fit: fall back to direct loads
        }
    }
    return CSRK_OK;
}

int compute(csrk_matrix* h, int32_t k, bool spmm, double alpha, const void* X, int64_t ldx,
            double beta, void* Y, int64_t ldy, unsigned flags, void* stream) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    const int32_t n = h->m.n;
    if (n > 0 && (!X || !Y)) return fail(CSRK_ERR_ARG, "x / y is NULL");
    if (X == Y && n > 0) return fail(CSRK_ERR_ARG, "x and y must not overlap");
    if (k < 1 || k > 64) return fail(CSRK_ERR_ARG, "k must be in [1, 64]");
    if (ldx < k || ldy < k) return fail(CSRK_ERR_ARG, "leading dimension smaller than k");
    const bool x_f32 = flags & CSRK_X_F32;
    const bool acc_f32 = flags & CSRK_ACC_F32;
    const int vt = (int)h->dtype;
    if (vt == VAL_F64 && (x_f32 || acc_f32))
        return fail(CSRK_ERR_UNSUPPORTED, "FP64 values take FP64 vectors and FP64 accumulation");
    if (acc_f32 && !x_f32)
        return fail(CSRK_ERR_UNSUPPORTED, "FP32 accumulation needs FP32 vectors (CSRK_X_F32)");
    int rc;
    if ((rc = ensure_context(h))) return rc;
    if ((rc = ensure_struct(h))) return rc;
    if ((rc = ensure_vals(h, vt))) return rc;
    if (n == 0) return CSRK_OK;

    const size_t esz = x_f32 ? 4 : 8;
    const bool host_vec = flags & CSRK_HOST_VECTORS;
    const bool x_only = (flags & CSRK_X_PERMUTED) && !(flags & CSRK_VEC_PERMUTED) && !h->perm.empty();
    if (x_only && spmm) return fail(CSRK_ERR_UNSUPPORTED, "CSRK_X_PERMUTED is for csrk_spmv");
    const bool permuted = (flags & CSRK_VEC_PERMUTED) || h->perm.empty();
    cudaStream_t s = (cudaStream_t)stream;
    KernelConfig cfg;
    StagePlan plan;
    if ((rc = resolve_config(h, vt, cfg, plan, (int)esz, nullptr, spmm))) return rc;
    const bool pairs = cfg.kernel == 2 || cfg.kernel == 3 || cfg.kernel == 6;
    if (pairs) {
        if ((rc = ensure_vals(h, VAL_DS)) || (rc = ensure_scratch(h, 4, (size_t)n * 8)) ||
            (rc = ensure_scratch(h, 5, 16)))
            return rc;
    }
    const void* xin = X;
    void* yout = Y;
    int64_t ldxin = ldx, ldyout = ldy;
    // a page-locked host x that needs permuting is read by the permute kernel itself over
    // the host link (in x's own order, scattered through the inverse permutation), so the
    // copy and the permute are one pass instead of two
    const void* x_mapped = nullptr;
    if (host_vec) {
        const size_t xb = (size_t)n * ldx * esz, yb = (size_t)n * ldy * esz;
        if (!permuted && !x_only && !pairs) x_mapped = mapped_host_ptr(X);
        if (x_mapped && (rc = ensure_iperm(h))) return rc;
        if (!x_mapped && (rc = ensure_scratch(h, 2, xb))) return rc;
        if ((rc = ensure_scratch(h, 3, yb))) return rc;
        if (!x_mapped) {
            CK_CUDA(cudaMemcpyAsync(h->d_scratch[2], X, xb, cudaMemcpyHostToDevice, s), "copy x to device");
            xin = h->d_scratch[2];
        }
        if (beta != 0.0)
            CK_CUDA(cudaMemcpyAsync(h->d_scratch[3], Y, yb, cudaMemcpyHostToDevice, s), "copy y to device");
        yout = h->d_scratch[3];
    }
    const void* xk = xin;
    void* yk = yout;
    int64_t ldxk = ldxin, ldyk = ldyout;
    // SpMV in the input numbering stores row r's result straight to y[perm[r]] (the kernel
    // reads y there too when beta != 0): no permuted copy of y, no separate unpermute
    const bool fuse_y = !permuted && !spmm;
    if (!permuted && !x_only) {
        const size_t b = (size_t)n * k * esz;
        if ((rc = ensure_scratch(h, 0, b))) return rc;
        if (!fuse_y && (rc = ensure_scratch(h, 1, b))) return rc;
        if (x_mapped) {
            int e = launch_scatter_rows(x_mapped, ldxin, h->d_scratch[0], k, h->d_iperm, n, k, (int)esz, s);
            if (e) return cuda_fail((cudaError_t)e, "permute host x");
        } else if (!pairs) {
            int e = launch_gather_rows(xin, ldxin, h->d_scratch[0], k, h->d_perm, n, k, (int)esz, s);
            if (e) return cuda_fail((cudaError_t)e, "permute x");
        }
        if (beta != 0.0 && !fuse_y) {
            int e = launch_gather_rows(yout, ldyout, h->d_scratch[1], k, h->d_perm, n, k, (int)esz, s);
            if (e) return cuda_fail((cudaError_t)e, "permute y");
        }
        xk = h->d_scratch[0];
        ldxk = k;
        if (!fuse_y) {
            yk = h->d_scratch[1];
            ldyk = k;
        }
    }
    const void* xkern = xk;
    if (pairs) {   // permute (when needed) and split x in one pass
        const bool gather = !permuted && !x_only;
        int e = launch_split_pairs(static_cast<const double*>(xin), gather ? h->d_perm : nullptr, n,
                                   gather ? static_cast<double*>(h->d_scratch[0]) : nullptr,
                                   h->d_scratch[4], static_cast<int32_t*>(h->d_scratch[5]), s);
        if (e) return cuda_fail((cudaError_t)e, "split x");
        xkern = h->d_scratch[4];
    }
    // kernels 5 and 6 copy x by TMA (kernel 6: the FP64 x when the split flags an
    // element): a caller's x off a 16-byte boundary takes another kernel
    if ((cfg.kernel == 5 && (reinterpret_cast<uintptr_t>(xkern) & 15u)) ||
        (cfg.kernel == 6 && (reinterpret_cast<uintptr_t>(xk) & 15u))) {
        if ((rc = resolve_config(h, vt, cfg, plan, (int)esz, cfg.kernel == 6 ? xk : xkern, spmm))) return rc;
    }
    LaunchArgs a{};
    fill_matrix_args(h, cfg, a);
    a.vals = h->d_vals[pairs ? (int)VAL_DS : vt];
    a.x = xkern;
    a.x64 = static_cast<const double*>(xk);
    a.xflag = static_cast<const int32_t*>(h->d_scratch[5]);
    a.y = yk;
    a.ldx = ldxk;
    a.ldy = ldyk;
    a.k = k;
    a.nssr = (int32_t)h->desc.size();
    a.alpha = alpha;
    a.beta = beta;
    a.skip = nullptr;
    a.yperm = fuse_y ? h->d_perm : nullptr;
    a.status = h->d_status;
    a.stats = h->stats;
    a.val_type = vt;
    a.x_f32 = x_f32;
    a.acc_f32 = acc_f32;
    a.spmm = spmm;
    a.num_sms = h->num_sms;
    a.timeout_ns = h->timeout_ns;
    fill_long_rows(h, a, pairs);
    int e = launch_csr3(a, cfg, plan, s);
    if (e == -1) return fail(CSRK_ERR_UNSUPPORTED, "kernel variant not compiled for this configuration");
    if (e) return cuda_fail((cudaError_t)e, "CSR-3 kernel launch");
    if (!permuted && !fuse_y) {
        e = launch_scatter_rows(h->d_scratch[1], k, yout, ldyout, h->d_perm, n, k, (int)esz, s);
        if (e) return cuda_fail((cudaError_t)e, "unpermute y");
    }
    if (host_vec) {
        CK_CUDA(cudaMemcpyAsync(Y, h->d_scratch[3], (size_t)n * ldy * esz, cudaMemcpyDeviceToHost, s),
                "copy y to host");
        CK_CUDA(cudaStreamSynchronize(s), "synchronise");
    }
    return CSRK_OK;
}

int launch_spmv_dev(csrk_matrix* h, int vt, const void* x, void* y, double alpha, double beta,
                    bool x_f32, bool acc_f32, const int32_t* skip, cudaStream_t s) {
    KernelConfig cfg;
    StagePlan plan;
    int rc;
    if ((rc = resolve_config(h, vt, cfg, plan, x_f32 ? 4 : 8, x))) return rc;
    const void* xkern = x;
    const bool pairs = cfg.kernel == 2 || cfg.kernel == 3 || cfg.kernel == 6;
    if (pairs) {
        if ((rc = ensure_vals(h, VAL_DS)) || (rc = ensure_scratch(h, 4, (size_t)h->m.n * 8)) ||
            (rc = ensure_scratch(h, 5, 16)))
            return rc;
        const int e = launch_split_pairs(static_cast<const double*>(x), nullptr, h->m.n, nullptr,
                                         h->d_scratch[4], static_cast<int32_t*>(h->d_scratch[5]), s);
        if (e) return cuda_fail((cudaError_t)e, "split x");
        xkern = h->d_scratch[4];
    }
    LaunchArgs a{};
    fill_matrix_args(h, cfg, a);
    a.vals = h->d_vals[pairs ? (int)VAL_DS : vt];
    a.x = xkern;
    a.x64 = static_cast<const double*>(x);
    a.xflag = static_cast<const int32_t*>(h->d_scratch[5]);
    a.y = y;
    a.ldx = a.ldy = 1;
    a.k = 1;
    a.nssr = (int32_t)h->desc.size();
    a.alpha = alpha;
    a.beta = beta;
    a.skip = skip;
    a.status = h->d_status;
    a.stats = h->stats;
    a.val_type = vt;
    a.x_f32 = x_f32;
    a.acc_f32 = acc_f32;
    a.spmm = false;
    a.num_sms = h->num_sms;
    a.timeout_ns = h->timeout_ns;
    fill_long_rows(h, a, pairs);
    int e = launch_csr3(a, cfg, plan, s);
    if (e == -1) return fail(CSRK_ERR_UNSUPPORTED, "kernel variant not compiled for this configuration");
    if (e) return cuda_fail((cudaError_t)e, "CSR-3 kernel launch");
    return CSRK_OK;
}

int tune_inner(csrk_matrix* h, int vt, const void* x, void* y) {
    if (vt == (int)h->dtype || vt >= 4) return CSRK_OK;
    NvtxRange range("csrk tune inner");
    cudaStream_t s;
    CK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "tune stream");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    KernelConfig best;
    float best_us = 1e30f;
    const bool win = xwin_available(h), c16 = col16_available(h);
    // small blocks in numbers as well: the narrow product's consumers are fast, so many
    // independent stage rings per SM keep more copies in flight
    for (int kernel : {4, 5})
        for (int unroll : {4, 8})
            for (int warps : {2, 4, 8, 16})
                for (int ctas : {2, 3, 4, 6, 8}) {
                    if ((kernel == 4 && !c16) || (kernel == 5 && !win)) continue;
                    if ((warps == 16 && ctas > 2) || (warps == 8 && ctas > 4) || (warps <= 4 && ctas < 4)) continue;
                    KernelConfig c;
                    c.kernel = kernel;
                    c.lanes = 1;
                    c.unroll = unroll;
                    c.warps = warps;
                    c.ctas = ctas;
                    c.stages = 0;
                    h->inner_cfg[vt] = c;
                    h->inner_gen[vt] = h->generation;
                    KernelConfig r;
                    StagePlan plan;
                    if (resolve_config(h, vt, r, plan, 4, x) || r.kernel != kernel) continue;   // does not fit
                    bool ok = launch_spmv_dev(h, vt, x, y, 1.0, 0.0, true, true, nullptr, s) == CSRK_OK;
                    cudaEventRecord(e0, s);
                    for (int i = 0; ok && i < 5; ++i) ok = launch_spmv_dev(h, vt, x, y, 1.0, 0.0, true, true, nullptr, s) == CSRK_OK;
                    cudaEventRecord(e1, s);
                    if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms * 200.f < best_us) {
                        best_us = ms * 200.f;
                        best = c;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaGetLastError();
    if (best_us >= 1e29f) {   // nothing timed: leave the default shape to resolve_config
        h->inner_gen[vt] = ~0ull;
        return CSRK_OK;
    }
    h->inner_cfg[vt] = best;
    h->inner_gen[vt] = h->generation;
    return CSRK_OK;
}

}  // namespace rt
}  // namespace csrk

using namespace csrk::rt;

// ================================================================== autotuner
// Chooses super-row / super-super-row sizes and the launch shape by timing candidates on
// the handle's own matrix (replacing the paper's constant-time model of Sec. 4.1, whose
// Ampere-coefficient answer is one of the candidates).  Phase 1 times fixed size pairs
// under the default launch shape; phase 2 times launch shapes on the three fastest size
// pairs.  Results are cached per (n, nnz, longest row, dtype, device) in-process and, when
// CSRK_TUNE_CACHE names a file, in that file.
namespace {

struct TunedChoice {
    int32_t sr = 0, ssr = 0;
    KernelConfig cfg;
    float us = 0.f;
};

std::mutex g_tune_mu;
std::vector<std::pair<std::string, TunedChoice>> g_tune_cache;
bool g_tune_file_loaded = false;

int install_pointers_impl(csrk_handle h, std::vector<int32_t>&& srp, std::vector<int32_t>&& ssrp);

int set_fixed(csrk_matrix* h, int32_t sr, int32_t ssr) {
    std::vector<int32_t> srp, ssrp;
    fixed_pointers(h->m.n - h->n_long, sr, ssr, srp, ssrp);
    int rc = install_pointers_impl(h, std::move(srp), std::move(ssrp));
    if (rc) return rc;
    h->sr = sr;
    h->ssr = ssr;
    return CSRK_OK;
}

// The key of a tuned choice, one whitespace-free token (as the cache file stores it).
std::string tune_key(const csrk_matrix* h) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, h->device);
    std::string name(prop.name);
    for (auto& ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    return std::to_string(h->m.n) + ":" + std::to_string(h->m.nnz()) + ":" +
           std::to_string(h->stats.max_row_len) + ":" + std::to_string((int)h->dtype) + ":" +
           std::to_string(h->num_sms) + ":" + name +
           (h->n_long ? ":long" + std::to_string(h->n_long) : std::string());
}

void load_tune_file() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char* path = std::getenv("CSRK_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char key[512];
    TunedChoice c;
    while (std::fscanf(f, "%511s %d %d %d %d %d %d %d %d %f", key, &c.sr, &c.ssr, &c.cfg.kernel,
                       &c.cfg.lanes, &c.cfg.unroll, &c.cfg.warps, &c.cfg.stages, &c.cfg.ctas, &c.us) == 10)
        g_tune_cache.emplace_back(key, c);
    std::fclose(f);
}

void save_tune_entry(const std::string& key, const TunedChoice& c) {
    const char* path = std::getenv("CSRK_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d %d %d %d %.3f\n", key.c_str(), c.sr, c.ssr, c.cfg.kernel,
                 c.cfg.lanes, c.cfg.unroll, c.cfg.warps, c.cfg.stages, c.cfg.ctas, c.us);
    std::fclose(f);
}

float time_launches(csrk_matrix* h, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps) {
    // a reordered handle is timed as its natural-numbering call runs: x already permuted,
    // y stored through the permutation by the kernel (the fused unpermute)
    const unsigned fl = h->perm.empty() ? CSRK_VEC_PERMUTED : CSRK_X_PERMUTED;
    for (int i = 0; i < 2; ++i)
        if (compute(h, 1, false, 1.0, h->d_scratch[0], 1, 0.0, h->d_scratch[1], 1, fl, s)) return 1e30f;
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i)
        if (compute(h, 1, false, 1.0, h->d_scratch[0], 1, 0.0, h->d_scratch[1], 1, fl, s)) return 1e30f;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms * 1000.f / reps;
}

int autotune(csrk_matrix* h) {
    int rc;
    NvtxRange range("csrk autotune");
    if (fault_injected("tune")) return fail(CSRK_ERR_CUDA, "autotuning: injected fault");
    // Band-k pointers in place: tune the launch shape only, on those pointers
    const bool bandk = h->have_ptrs && h->bandk_sr > 0;
    if (h->m.n == 0) return bandk ? CSRK_OK : set_fixed(h, 32, 8);
    if ((rc = ensure_context(h))) return rc;
    // sizes first so that the key can see the longest row
    if (!bandk && (rc = set_fixed(h, 32, 8))) return rc;
    const std::string key = tune_key(h) + (bandk ? ":bandk" + std::to_string(h->bandk_sr) + "x" +
                                                       std::to_string(h->bandk_ssr)
                                                 : std::string());
    // (re)install the chosen sizes; Band-k keeps its own pointers
    auto install = [&](int32_t sr, int32_t ssr) { return bandk ? CSRK_OK : set_fixed(h, sr, ssr); };
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        load_tune_file();
        for (auto& e : g_tune_cache)
            if (e.first == key) {
                if ((rc = install(e.second.sr, e.second.ssr))) return rc;
                h->cfg = e.second.cfg;
                h->cfg_set = true;
                h->kernel_forced = false;
                h->generation++;
                return CSRK_OK;
            }
    }
    const int vt = (int)h->dtype;
    if ((rc = ensure_struct(h)) || (rc = ensure_vals(h, vt))) return rc;
    const size_t vb = (size_t)h->m.n * 8;
    if ((rc = ensure_scratch(h, 0, vb)) || (rc = ensure_scratch(h, 1, vb))) return rc;
    CK_CUDA(cudaMemset(h->d_scratch[0], 0, vb), "tune memset");
    cudaStream_t s;
    CK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "tune stream");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int reps = 10;

    std::vector<std::pair<int32_t, int32_t>> sizes = {{32, 1}, {32, 2}, {32, 4}, {32, 8}, {32, 16},
                                                      {64, 1}, {64, 2}, {64, 4}, {64, 8}, {128, 1},
                                                      {128, 2}, {16, 4}, {16, 8}, {16, 16}};
    int32_t model_ssrs = 0, model_srs = 0;
    // mean row length over the rows the super-rows cover (split long rows excluded)
    const int32_t n_cov = h->m.n - h->n_long;
    const double rdens = n_cov > 0 ? (double)h->m.rowptr[n_cov] / n_cov : 0.0;
    if (rdens > 0 && csrk_model_sizes(rdens, 1, &model_ssrs, &model_srs) == CSRK_OK && model_srs > 0 &&
        model_ssrs > 0)
        sizes.emplace_back(model_srs, model_ssrs);

    std::vector<TunedChoice> phase1;
    h->cfg_set = false;
    h->kernel_forced = false;
    if (bandk) sizes.assign(1, {0, 0});
    // the x-window kernel's default shape, timed beside the default shape on size pairs
    // whose super-super-rows are small enough for its windows to fit the stages
    KernelConfig win_cfg;
    win_cfg.kernel = 5;
    win_cfg.lanes = 1;
    win_cfg.unroll = 4;
    win_cfg.warps = 8;
    win_cfg.ctas = 3;
    for (auto& sz : sizes) {
        if ((rc = install(sz.first, sz.second))) break;
        if ((rc = ensure_struct(h))) break;
        TunedChoice c;
        c.sr = sz.first;
        c.ssr = sz.second;
        c.us = time_launches(h, s, e0, e1, reps);
        StagePlan plan;
        if (resolve_config(h, vt, c.cfg, plan)) continue;   // the shape the timing ran with
        phase1.push_back(c);
        if (!bandk && (int64_t)sz.first * sz.second > 256) continue;
        if (rdens <= 48 && xwin_available(h)) {
            h->cfg = win_cfg;
            h->cfg_set = true;
            h->kernel_forced = false;
            TunedChoice w = c;
            w.us = time_launches(h, s, e0, e1, reps);
            if (resolve_config(h, vt, w.cfg, plan) == CSRK_OK && w.cfg.kernel == 5) phase1.push_back(w);
            h->cfg_set = false;
        }
    }
    std::sort(phase1.begin(), phase1.end(), [](auto& a, auto& b) { return a.us < b.us; });
    // distinct size pairs in order of their best phase-1 time
    {
        std::vector<TunedChoice> uniq;
        for (auto& c : phase1) {
            bool seen = false;
            for (auto& u : uniq) seen |= (u.sr == c.sr && u.ssr == c.ssr);
            if (!seen) uniq.push_back(c);
        }
        phase1.swap(uniq);
    }
    TunedChoice best = phase1.empty() ? TunedChoice{} : phase1.front();

    // lane counts for the mean row length, and -- for irregular matrices, whose longest
    // super-row row decides how long a warp pass takes -- for the longest row as well
    auto pairs_for = [](double len) -> std::vector<std::pair<int, int>> {
        if (len <= 32) return {{1, 4}, {1, 8}, {1, 16}, {2, 8}};
        if (len <= 64) return {{2, 8}, {2, 16}, {4, 8}};
        if (len <= 256) return {{4, 8}, {8, 8}, {32, 4}};
        return {{8, 8}, {32, 4}};
    };
    std::vector<std::pair<int, int>> pairs = pairs_for(rdens);
    if (h->stats.max_row_len > 4 * rdens)
        for (auto& p : pairs_for(h->stats.max_row_len))
            if (std::find(pairs.begin(), pairs.end(), p) == pairs.end()) pairs.push_back(p);
    const bool with_pairs = pairs_available(h);
    std::vector<TunedChoice> phase2;
    for (size_t b = 0; b < std::min<size_t>(3, phase1.size()) && rc == CSRK_OK; ++b) {
        if ((rc = install(phase1[b].sr, phase1[b].ssr)) || (rc = ensure_struct(h))) break;
        for (auto& pr : pairs)
            for (int warps : {4, 6, 8, 16})
                for (int kernel : {0, 1, 2, 3, 4, 5, 6})
                    for (int ctas : {1, 2, 3, 4}) {
                        if (warps < 8 && (kernel != 5 || ctas < 3)) continue;   // small blocks in numbers
                        if ((kernel == 1 || kernel == 3) && ctas >= 2) continue;
                        if (ctas >= 3 && (kernel < 4 || warps > 8)) continue;   // fits only small blocks
                        if (ctas == 4 && kernel != 5) continue;
                        if ((kernel == 2 || kernel == 3) && (!with_pairs || pr.first != 1 || pr.second > 16)) continue;
                        if (kernel == 4 && (!col16_available(h) || !mode3_compiled(pr.first, pr.second))) continue;
                        if (kernel == 5 && (!xwin_available(h) || !mode4_compiled(pr.first, pr.second))) continue;
                        if (kernel == 6 && (!with_pairs || !xwin_available(h) || !mode4_compiled(pr.first, pr.second)))
                            continue;
                        KernelConfig c;
                        c.kernel = kernel;
                        c.lanes = pr.first;
                        c.unroll = pr.second;
                        c.warps = warps;
                        c.ctas = ctas;
                        c.stages = 0;
                        h->cfg = c;
                        h->cfg_set = true;
                        h->kernel_forced = (kernel != 1);
                        const float us = time_launches(h, s, e0, e1, reps);
                        TunedChoice t;
                        t.sr = phase1[b].sr;
                        t.ssr = phase1[b].ssr;
                        t.cfg = c;
                        t.us = us;
                        phase2.push_back(t);
                    }
    }
    // phase 3: the four fastest shapes (and the best default-shape size pair) re-timed with
    // longer runs in two interleaved rounds, so that a lucky short timing does not decide
    if (rc == CSRK_OK) {
        std::sort(phase2.begin(), phase2.end(), [](auto& a, auto& b) { return a.us < b.us; });
        std::vector<TunedChoice> finalists(phase2.begin(), phase2.begin() + std::min<size_t>(4, phase2.size()));
        if (!phase1.empty()) finalists.push_back(phase1.front());   // its resolved default shape
        for (auto& f : finalists) f.us = 1e30f;
        for (int round = 0; round < 2 && rc == CSRK_OK; ++round)
            for (auto& f : finalists) {
                if ((rc = install(f.sr, f.ssr)) || (rc = ensure_struct(h))) break;
                h->cfg = f.cfg;
                h->cfg_set = true;
                h->kernel_forced = (f.cfg.kernel != 1);
                f.us = std::min(f.us, time_launches(h, s, e0, e1, 4 * reps));
            }
        if (!finalists.empty())
            best = *std::min_element(finalists.begin(), finalists.end(),
                                     [](auto& a, auto& b) { return a.us < b.us; });
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc) return rc;
    if (phase1.empty() || best.us >= 1e29f) return fail(CSRK_ERR_CUDA, "autotuning found no working configuration");
    if ((rc = install(best.sr, best.ssr))) return rc;
    h->cfg = best.cfg;
    h->cfg_set = true;
    h->kernel_forced = false;
    h->generation++;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.emplace_back(key, best);
    save_tune_entry(key, best);
    return CSRK_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

int csrk_create(int32_t n, const int32_t* rowptr, const int32_t* colidx, const double* vals,
                csrk_dtype dtype, csrk_handle* out) {
    if (!out) return fail(CSRK_ERR_ARG, "out is NULL");
    NvtxRange range("csrk create");
    *out = nullptr;
    if (dtype != CSRK_F64 && dtype != CSRK_F32 && dtype != CSRK_BF16)
        return fail(CSRK_ERR_ARG, "unknown dtype");
    csrk_matrix* h = new (std::nothrow) csrk_matrix();
    if (!h) return fail(CSRK_ERR_ALLOC, "out of host memory");
    try {
        std::string err;
        int rc = ingest_csr(n, rowptr, colidx, vals, h->m, err);
        if (rc) {
            delete h;
            return fail(rc, err);
        }
    } catch (const std::bad_alloc&) {
        delete h;
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    h->dtype = dtype;
    *out = h;
    return CSRK_OK;
}

int csrk_reorder(csrk_handle h, int method, int32_t* perm_out) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    NvtxRange range("csrk reorder");
    if (h->have_ptrs) return fail(CSRK_ERR_STATE, "reorder must come before csrk_set_sizes / csrk_set_pointers");
    if (h->n_long > 0) return fail(CSRK_ERR_STATE, "reorder must come before csrk_split_long_rows");
    if (method != CSRK_REORDER_NONE && method != CSRK_REORDER_RCM) return fail(CSRK_ERR_ARG, "unknown method");
    try {
        if (method == CSRK_REORDER_RCM) {
            std::vector<int32_t> local;   // permutation of the current form
            rcm_permutation(h->m, local);
            CsrHost b;
            permute_symmetric(h->m, local, b);
            h->m = std::move(b);
            // a second reorder composes with the first: new -> previous -> input numbering
            if (!h->perm.empty())
                for (auto& p : local) p = h->perm[p];
            h->perm = std::move(local);
        }
        if (perm_out) {
            if (h->perm.empty())
                for (int32_t i = 0; i < h->m.n; ++i) perm_out[i] = i;
            else
                std::memcpy(perm_out, h->perm.data(), sizeof(int32_t) * h->perm.size());
        }
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    return CSRK_OK;
}

int csrk_reorder_bandk(csrk_handle h, int32_t sr, int32_t ssr, int32_t* perm_out) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    NvtxRange range("csrk reorder band-k");
    if (h->have_ptrs) return fail(CSRK_ERR_STATE, "reorder must come before csrk_set_sizes / csrk_set_pointers");
    if (h->n_long > 0) return fail(CSRK_ERR_STATE, "Band-k does not take split long rows");
    if (sr < 1 || ssr < 1) return fail(CSRK_ERR_ARG, "sr and ssr must be >= 1");
    try {
        std::vector<int32_t> local, srp, ssrp;
        bandk_permutation(h->m, sr, ssr, local, srp, ssrp);
        CsrHost b;
        permute_symmetric(h->m, local, b);
        h->m = std::move(b);
        if (!h->perm.empty())
            for (auto& p : local) p = h->perm[p];
        h->perm = std::move(local);
        if (perm_out) {
            if (h->perm.empty())
                for (int32_t i = 0; i < h->m.n; ++i) perm_out[i] = i;
            else
                std::memcpy(perm_out, h->perm.data(), sizeof(int32_t) * h->perm.size());
        }
        int rc = install_pointers_impl(h, std::move(srp), std::move(ssrp));
        if (rc) return rc;
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    h->sr = h->ssr = 0;
    h->bandk_sr = sr;
    h->bandk_ssr = ssr;
    return CSRK_OK;
}

int csrk_split_long_rows(csrk_handle h, int32_t min_len, int32_t* n_long) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    NvtxRange range("csrk split long rows");
    if (h->have_ptrs) return fail(CSRK_ERR_STATE, "split long rows before csrk_set_sizes / csrk_set_pointers");
    if (min_len < 1) return fail(CSRK_ERR_ARG, "min_len must be >= 1");
    try {
        const int32_t n = h->m.n;
        std::vector<int32_t> local;   // short rows in order, then long rows in order
        local.reserve(n);
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t i = 0; i < n; ++i) {
                const bool is_long = h->m.rowptr[i + 1] - h->m.rowptr[i] >= min_len;
                if (is_long == (pass == 1)) local.push_back(i);
            }
        int32_t count = 0;
        for (int32_t i = 0; i < n; ++i) count += (h->m.rowptr[i + 1] - h->m.rowptr[i] >= min_len);
        if (count > 0) {
            CsrHost b;
            permute_symmetric(h->m, local, b);
            h->m = std::move(b);
            if (!h->perm.empty())
                for (auto& p : local) p = h->perm[p];
            h->perm = std::move(local);
            if (h->device >= 0) {   // the matrix changed: re-upload on next use
                free_struct(h);
                for (auto& v : h->d_vals) {
                    cudaFree(v);
                    v = nullptr;
                }
            }
            h->pairs_ok = -1;
        }
        h->n_long = count;
        if (n_long) *n_long = count;
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    return CSRK_OK;
}

}  // extern "C"

namespace {
int install_pointers_impl(csrk_handle h, std::vector<int32_t>&& srp, std::vector<int32_t>&& ssrp) {
    std::string err;
    NvtxRange range("csrk pointers");
    if (!check_pointers(h->m.n - h->n_long, srp, ssrp, err)) return fail(CSRK_ERR_ARG, err);
    h->sr_ptr = std::move(srp);
    h->ssr_ptr = std::move(ssrp);
    build_descs(h->m, h->sr_ptr, h->ssr_ptr, h->desc, h->stats);
    // the long rows' segments, row by row
    h->lseg.clear();
    h->lseg_ptr.assign(1, 0);
    for (int32_t r = h->m.n - h->n_long; r < h->m.n; ++r) {
        for (int64_t p = h->m.rowptr[r]; p < h->m.rowptr[r + 1]; p += LSEG)
            h->lseg.push_back({(int32_t)p, (int32_t)std::min<int64_t>(p + LSEG, h->m.rowptr[r + 1])});
        h->lseg_ptr.push_back((int32_t)h->lseg.size());
    }
    h->have_ptrs = true;
    if (h->dev_ptrs) free_ptrs(h);   // pointer arrays changed: re-upload on next use
    cudaFree(h->d_col16);            // the column bases moved with the SSRs
    h->d_col16 = nullptr;
    h->col16_ok = -1;
    h->generation++;
    return CSRK_OK;
}
}  // namespace

extern "C" {

int csrk_set_sizes(csrk_handle h, int32_t sr, int32_t ssr) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (sr == 0 && ssr == 0) {
        try {
            return autotune(h);
        } catch (const std::bad_alloc&) {
            return fail(CSRK_ERR_ALLOC, "out of host memory");
        }
    }
    if (sr <= 0 || ssr <= 0) return fail(CSRK_ERR_ARG, "sizes must be positive");
    try {
        std::vector<int32_t> srp, ssrp;
        fixed_pointers(h->m.n - h->n_long, sr, ssr, srp, ssrp);
        int rc = install_pointers_impl(h, std::move(srp), std::move(ssrp));
        if (rc) return rc;
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    h->sr = sr;
    h->ssr = ssr;
    h->bandk_sr = h->bandk_ssr = 0;
    return CSRK_OK;
}

int csrk_index_bits(csrk_handle h, int32_t* bits) {
    if (!h || !bits) return fail(CSRK_ERR_ARG, "NULL argument");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    std::vector<uint16_t> tmp;   // host only: the coding is checked, not uploaded
    if (h->col16_ok >= 0) *bits = h->col16_ok == 1 ? 16 : 32;
    else *bits = compress_columns(h->m, h->desc, tmp) ? 16 : 32;
    return CSRK_OK;
}

int csrk_col16_export(csrk_handle h, uint16_t* codes, int32_t* cbase) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    try {
        std::vector<uint16_t> tmp;
        if (!compress_columns(h->m, h->desc, tmp))
            return fail(CSRK_ERR_UNSUPPORTED, "a column step or first-column offset exceeds 65,535");
        if (codes && !tmp.empty()) std::memcpy(codes, tmp.data(), sizeof(uint16_t) * tmp.size());
        if (cbase)
            for (size_t t = 0; t < h->desc.size(); ++t) cbase[t] = h->desc[t].cbase;
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    return CSRK_OK;
}

int csrk_xwin_info(csrk_handle h, int32_t* available, int64_t* runs, int32_t* max_window,
                   int32_t* row_order) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    int rc;
    if ((rc = ensure_context(h))) return rc;
    const bool ok = xwin_available(h);
    if (available) *available = ok ? 1 : 0;
    if (runs) *runs = ok ? h->xwin_runs : 0;
    if (max_window) *max_window = ok ? h->max_win : 0;
    if (row_order) *row_order = ok && h->d_rord ? 1 : 0;
    return CSRK_OK;
}

int csrk_set_pointers(csrk_handle h, int32_t nsr, const int32_t* sr_ptr, int32_t nssr,
                      const int32_t* ssr_ptr) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (nsr < 0 || nssr < 0 || !sr_ptr || !ssr_ptr) return fail(CSRK_ERR_ARG, "bad pointer arrays");
    try {
        int rc = install_pointers_impl(h, std::vector<int32_t>(sr_ptr, sr_ptr + nsr + 1),
                                  std::vector<int32_t>(ssr_ptr, ssr_ptr + nssr + 1));
        if (rc) return rc;
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    h->sr = h->ssr = 0;
    h->bandk_sr = h->bandk_ssr = 0;
    return CSRK_OK;
}

int csrk_spmv(csrk_handle h, double alpha, const void* x, double beta, void* y, unsigned flags,
              void* stream) {
    return compute(h, 1, false, alpha, x, 1, beta, y, 1, flags, stream);
}

int csrk_spmm(csrk_handle h, int32_t k, double alpha, const void* X, int64_t ldx, double beta,
              void* Y, int64_t ldy, unsigned flags, void* stream) {
    if (k == 1 && ldx == 1 && ldy == 1) return compute(h, 1, false, alpha, X, 1, beta, Y, 1, flags, stream);
    return compute(h, k, true, alpha, X, ldx, beta, Y, ldy, flags, stream);
}

int csrk_permute(csrk_handle h, int direction, int32_t k, const void* in, int64_t ldi, void* out,
                 int64_t ldo, unsigned flags, void* stream) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    if (direction != 0 && direction != 1) return fail(CSRK_ERR_ARG, "direction must be 0 or 1");
    if (k < 1 || ldi < k || ldo < k) return fail(CSRK_ERR_ARG, "bad k or leading dimension");
    const int32_t n = h->m.n;
    if (n > 0 && (!in || !out || in == out)) return fail(CSRK_ERR_ARG, "bad vector pointers");
    int rc;
    if ((rc = ensure_context(h))) return rc;
    if ((rc = ensure_struct(h))) return rc;
    if (n == 0) return CSRK_OK;
    const int esz = (flags & CSRK_X_F32) ? 4 : 8;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->perm.empty()) {
        CK_CUDA(cudaMemcpy2DAsync(out, (size_t)ldo * esz, in, (size_t)ldi * esz, (size_t)k * esz, n,
                                  cudaMemcpyDeviceToDevice, s),
                "copy");
        return CSRK_OK;
    }
    int e = direction == 0 ? launch_gather_rows(in, ldi, out, ldo, h->d_perm, n, k, esz, s)
                           : launch_scatter_rows(in, ldi, out, ldo, h->d_perm, n, k, esz, s);
    if (e) return cuda_fail((cudaError_t)e, "permute");
    return CSRK_OK;
}

int csrk_destroy(csrk_handle h) {
    if (!h) return CSRK_OK;
    if (h->device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != h->device) cudaSetDevice(h->device);
        cudaDeviceSynchronize();
        free_device(h);
        if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
    }
    delete h;
    return CSRK_OK;
}

int csrk_info(csrk_handle h, int32_t* n, int64_t* nnz, int32_t* nsr, int32_t* nssr, int32_t* sr,
              int32_t* ssr, int32_t* dtype) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (n) *n = h->m.n;
    if (nnz) *nnz = h->m.nnz();
    if (nsr) *nsr = h->have_ptrs ? (int32_t)h->sr_ptr.size() - 1 : 0;
    if (nssr) *nssr = h->have_ptrs ? (int32_t)h->ssr_ptr.size() - 1 : 0;
    if (sr) *sr = h->sr;
    if (ssr) *ssr = h->ssr;
    if (dtype) *dtype = (int32_t)h->dtype;
    return CSRK_OK;
}

int csrk_export(csrk_handle h, int32_t* perm, int32_t* rowptr, int32_t* colidx, double* vals,
                int32_t* sr_ptr, int32_t* ssr_ptr) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    const CsrHost& m = h->m;
    if (perm) {
        if (h->perm.empty())
            for (int32_t i = 0; i < m.n; ++i) perm[i] = i;
        else
            std::memcpy(perm, h->perm.data(), sizeof(int32_t) * m.n);
    }
    if (rowptr) std::memcpy(rowptr, m.rowptr.data(), sizeof(int32_t) * m.rowptr.size());
    if (colidx && m.nnz()) std::memcpy(colidx, m.colidx.data(), sizeof(int32_t) * m.nnz());
    if (vals && m.nnz()) std::memcpy(vals, m.vals.data(), sizeof(double) * m.nnz());
    if ((sr_ptr || ssr_ptr) && !h->have_ptrs) return fail(CSRK_ERR_STATE, "pointer arrays not built yet");
    if (sr_ptr) std::memcpy(sr_ptr, h->sr_ptr.data(), sizeof(int32_t) * h->sr_ptr.size());
    if (ssr_ptr) std::memcpy(ssr_ptr, h->ssr_ptr.data(), sizeof(int32_t) * h->ssr_ptr.size());
    return CSRK_OK;
}

int csrk_xwin_export(csrk_handle h, int32_t* available, int64_t* nruns, int32_t* wptr, int32_t* win,
                     int32_t* cover, uint16_t* codes, uint16_t* ord, int64_t* slots) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    if (!h->have_ptrs) return fail(CSRK_ERR_STATE, "call csrk_set_sizes or csrk_set_pointers first");
    try {
        std::vector<SsrDesc> xdesc;
        std::vector<int32_t> w, wp;
        std::vector<uint16_t> colx;
        int32_t mw = 0;
        int64_t runs = 0;
        const bool ok = !h->desc.empty() && build_xwin(h->m, h->desc, xdesc, w, wp, colx, mw, runs);
        if (available) *available = ok ? 1 : 0;
        if (nruns) *nruns = ok ? runs : 0;
        if (ok) {
            if (wptr) std::memcpy(wptr, wp.data(), sizeof(int32_t) * wp.size());
            if (win && runs) std::memcpy(win, w.data(), sizeof(int32_t) * 2 * (size_t)runs);
            if (cover)
                for (size_t t = 0; t < xdesc.size(); ++t) cover[t] = xdesc[t].cbase;
            if (codes && !colx.empty()) std::memcpy(codes, colx.data(), sizeof(uint16_t) * colx.size());
        }
        if (ord || slots) {
            std::vector<uint16_t> o;
            int64_t nat = 0, srt = 0;
            build_row_order(h->m, h->sr_ptr, h->desc, o, nat, srt);
            if (ord && !o.empty()) std::memcpy(ord, o.data(), sizeof(uint16_t) * o.size());
            if (slots) {
                slots[0] = nat;
                slots[1] = srt;
            }
        }
    } catch (const std::bad_alloc&) {
        return fail(CSRK_ERR_ALLOC, "out of host memory");
    }
    return CSRK_OK;
}

int csrk_export_values(csrk_handle h, csrk_dtype dtype, void* out) {
    if (!h || !out) return fail(CSRK_ERR_ARG, "NULL argument");
    const int64_t nnz = h->m.nnz();
    switch (dtype) {
        case CSRK_F64: std::memcpy(out, h->m.vals.data(), sizeof(double) * nnz); return CSRK_OK;
        case CSRK_F32: narrow_f32(h->m.vals.data(), static_cast<float*>(out), nnz); return CSRK_OK;
        case CSRK_BF16: narrow_bf16(h->m.vals.data(), static_cast<uint16_t*>(out), nnz); return CSRK_OK;
    }
    return fail(CSRK_ERR_ARG, "unknown dtype");
}

int csrk_model_sizes(double rdensity, int arch, int32_t* ssrs, int32_t* srs) {
    if (!(rdensity > 0) || !ssrs || !srs || (arch != 0 && arch != 1)) return fail(CSRK_ERR_ARG, "bad arguments");
    // Sec. 4.1: log fit rounded half toward +infinity, then the rdensity case rules.
    auto rnd = [](double v) { return (int32_t)std::floor(v + 0.5); };
    const double lr = std::log(rdensity);
    int32_t a, b;
    const int c = rdensity <= 8 ? 1 : (rdensity <= 16 ? 2 : (rdensity <= 32 ? 3 : 4));
    if (arch == 0) {
        a = rnd(8.900 - 1.25 * lr);
        b = rnd(10.146 - 1.50 * lr);
        if (c == 2) { a = rnd(a * 1.5); b = b * 2; }
        else if (c == 3) { a = a * 4; b = a / 2; }
        else if (c == 4) { a = a * 5; b = a / 2; }
    } else {
        a = rnd(9.175 - 1.32 * lr);
        b = rnd(20.500 - 3.50 * lr);
        if (c == 2) { b = b * 4; }
        else if (c == 3) { a = rnd(a * 2.5); b = a * 3; }
        else if (c == 4) { a = a * 2; b = a * 2; }
    }
    *ssrs = a;
    *srs = b;
    return CSRK_OK;
}

int csrk_tuned_config(csrk_handle h, int32_t* kernel, int32_t* lanes, int32_t* unroll,
                      int32_t* warps, int32_t* stages, int32_t* ctas) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    KernelConfig c = h->cfg_set ? h->cfg : default_config(h);
    if (h->have_ptrs && h->smem_per_sm > 0) {   // device known: report what a launch will use
        StagePlan plan;
        KernelConfig r;
        if (resolve_config(h, (int)h->dtype, r, plan) == CSRK_OK) {
            c = r;
            c.stages = (c.kernel == 0 || c.kernel == 2 || c.kernel >= 4) ? plan.stages : 0;
        }
    }
    if (kernel) *kernel = c.kernel;
    if (lanes) *lanes = c.lanes;
    if (unroll) *unroll = c.unroll;
    if (warps) *warps = c.warps;
    if (stages) *stages = c.stages;
    if (ctas) *ctas = c.ctas;
    return CSRK_OK;
}

int csrk_set_config(csrk_handle h, int32_t kernel, int32_t lanes, int32_t unroll, int32_t warps,
                    int32_t stages, int32_t ctas) {
    if (!h) return fail(CSRK_ERR_ARG, "handle is NULL");
    KernelConfig c = h->cfg_set ? h->cfg : default_config(h);
    if (kernel >= 0) {
        if (kernel > 6) return fail(CSRK_ERR_ARG, "kernel must be 0 to 6");
        c.kernel = kernel;
        h->kernel_forced = (kernel != 1);
    }
    if (lanes >= 0) {
        if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 32)
            return fail(CSRK_ERR_ARG, "lanes must be 1, 2, 4, 8 or 32");
        c.lanes = lanes;
        if (unroll < 0) c.unroll = default_unroll(lanes, h->have_ptrs ? h->stats.max_row_len : 32);
    }
    if (unroll >= 0) c.unroll = unroll;
    if (c.kernel >= 2 && (c.lanes != 1 || (c.unroll != 4 && c.unroll != 8 && c.unroll != 16)))
        return fail(CSRK_ERR_ARG, "kernels 2 to 6 take lanes 1 and unroll 4, 8 or 16");
    if (!pair_compiled(c.lanes, c.unroll))
        return fail(CSRK_ERR_ARG, "unsupported (lanes, unroll) pair; compiled: (1,4) (1,8) (1,16) "
                                  "(1,32) (2,8) (2,16) (4,8) (8,8) (32,4)");
    if (warps >= 0) {
        if (warps < 1 || warps > 16) return fail(CSRK_ERR_ARG, "warps must be in [1, 16]");
        c.warps = warps;
    }
    if (stages >= 0) {
        if (stages == 1 || stages > 16) return fail(CSRK_ERR_ARG, "stages must be 0 or in [2, 16]");
        c.stages = stages;
    }
    if (ctas >= 0) {
        if (ctas > 8) return fail(CSRK_ERR_ARG, "ctas must be 0 (auto) or in [1, 8]");
        c.ctas = ctas;
    }
    h->cfg = c;
    h->cfg_set = true;
    h->generation++;
    return CSRK_OK;
}

int csrk_device_status(csrk_handle h, void* stream, int32_t* status) {
    if (!h || !status) return fail(CSRK_ERR_ARG, "NULL argument");
    *status = 0;
    if (h->device < 0) return CSRK_OK;
    CK_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronise");
    CK_CUDA(cudaMemcpy(status, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost), "read status");
    CK_CUDA(cudaMemset(h->d_status, 0, sizeof(int32_t)), "clear status");
    if (*status) return fail(CSRK_ERR_TIMEOUT, "a device-side bounded wait ran out");
    return CSRK_OK;
}

int csrk_selftest_bounded_wait(csrk_handle h, uint64_t timeout_ns, void* stream, int32_t* status) {
    if (!h || !status || timeout_ns == 0 || timeout_ns > 10000000000ull)
        return fail(CSRK_ERR_ARG, "bad arguments (timeout_ns in (0, 1e10])");
    int rc;
    if ((rc = ensure_context(h))) return rc;
    const int e = launch_bounded_wait_probe(timeout_ns, h->d_status, stream);
    if (e) return cuda_fail((cudaError_t)e, "probe launch");
    return csrk_device_status(h, stream, status);
}

int csrk_selftest_narrow(const double* x, int64_t n, float* by_int, float* by_cvt, void* stream) {
    if (n < 0 || (n > 0 && (!x || !by_int || !by_cvt))) return fail(CSRK_ERR_ARG, "bad arguments");
    const int e = launch_narrow_pair(x, n, by_int, by_cvt, stream);
    if (e) return cuda_fail((cudaError_t)e, "narrowing self-test launch");
    return CSRK_OK;
}

int csrk_selftest_stage_plan(int32_t max_srs, int32_t max_rows, int64_t max_nnz, int32_t val_bytes,
                             int32_t col_bytes, int32_t max_smem, int32_t want_stages, int64_t x_bytes,
                             int32_t with_ord, uint32_t* out) {
    if (!out || max_srs < 0 || max_rows < 0 || max_nnz < 0 || x_bytes < 0 || max_smem <= 0 ||
        (val_bytes != 2 && val_bytes != 4 && val_bytes != 8) || (col_bytes != 2 && col_bytes != 4))
        return fail(CSRK_ERR_ARG, "bad arguments");
    TileStats st;
    st.max_srs = max_srs;
    st.max_rows = max_rows;
    st.max_nnz = max_nnz;
    StagePlan plan{};
    if (!plan_stages(st, val_bytes, max_smem, want_stages, col_bytes, plan, x_bytes, with_ord != 0))
        return fail(CSRK_ERR_UNSUPPORTED, "no two stages fit");
    const uint32_t v[10] = {plan.off_srp, plan.off_rp, plan.off_col, plan.off_val, plan.off_x,
                            plan.off_perm, plan.off_ord, plan.stage_bytes, plan.header_bytes,
                            (uint32_t)plan.stages};
    std::memcpy(out, v, sizeof v);
    return CSRK_OK;
}

const char* csrk_last_error(void) { return g_last_error.c_str(); }

const char* csrk_build_info(void) {
#ifdef CSRK_CHECKS
    return "csrk: sm_103a; CSR-3 TMA (cp.async.bulk + mbarrier) and direct kernels; "
           "values f64/f32/bf16; bounds checks on (status bit 1)";
#else
    return "csrk: sm_103a; CSR-3 TMA (cp.async.bulk + mbarrier) and direct kernels; "
           "values f64/f32/bf16";
#endif
}

}  // extern "C"
