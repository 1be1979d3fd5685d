// csrk_spmv_static_scratch: the natural-numbering SpMV path (permute x, CSR-3 kernel,
// unpermute y) for callers that must not allocate device memory.
//
// Who needs it: code whose device memory is owned by someone else and may not be grown
// behind the owner's back -- an application whose arena allocator has taken the GPU's
// memory up front, a plugin handed a fixed memory budget by its host program, or a
// latency-critical loop where an allocation (which may synchronise the device) is not
// acceptable.  The regular csrk_spmv allocates its permuted-vector scratch on first use;
// this entry point instead uses one file-scope device array, sized once for
// STATIC_MAX_ROWS rows, that every GPU loading the library holds until the process exits.
//
// The caller passes every input and output: the reordered CSR-k arrays (as csrk_export
// gives them), the permutation, x and y, all in device memory.  The matrix is read with
// plain loads (no TMA over-read), so the caller's arrays need no padding.  Rows after the
// last super-row (the long rows csrk_split_long_rows moves behind all others) are
// computed too, one warp per row.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.cuh"

namespace {

constexpr int64_t STATIC_MAX_ROWS = 1 << 20;   // 1,048,576 rows: 16 MiB of FP64 scratch

// First half: x in the reordered numbering; second half: the reordered result.
static __device__ __align__(256) double g_static_scratch[2 * STATIC_MAX_ROWS];

std::mutex g_scratch_mu;
// Device address of g_static_scratch per CUDA context (the primary context of a device
// gets a new identifier when it is re-created, e.g. after cudaDeviceReset, and the module
// holding the array may then load at another address).
struct ScratchAddr {
    unsigned long long ctx_id;
    double* addr;
};
constexpr int MAX_CONTEXTS = 64;
ScratchAddr g_scratch_addr[MAX_CONTEXTS] = {};
int g_scratch_count = 0;

// One block per super-super-row, warps across its super-rows, one row per lane.  The
// SSR and SR bounds come straight from ssr_ptr / sr_ptr.
__global__ void __launch_bounds__(256) csr3_static_kernel(
    int32_t nssr, const int32_t* __restrict__ ssr_ptr, const int32_t* __restrict__ sr_ptr,
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
    const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
    double alpha, double beta, int epi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nssr; t += gridDim.x) {
        const int s0 = __ldg(&ssr_ptr[t]), s1 = __ldg(&ssr_ptr[t + 1]);
        for (int sr = s0 + warp; sr < s1; sr += W) {
            const int rb = __ldg(&sr_ptr[sr]), re = __ldg(&sr_ptr[sr + 1]);
            csrk::dev::spmv_rows<double, double, double, 1, 8>(rb, re, rowptr, colidx, vals, x, y,
                                                              alpha, beta, epi, lane);
        }
    }
}

// Rows [sr_ptr[ssr_ptr[nssr]], n): the rows no super-row covers (long rows moved behind
// the others), one warp per row, lanes striding the row's nonzeros, a fixed shuffle tree.
__global__ void __launch_bounds__(256) tail_rows_kernel(
    int32_t n, int32_t nssr, const int32_t* __restrict__ ssr_ptr, const int32_t* __restrict__ sr_ptr,
    const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
    const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
    double alpha, double beta, int epi) {
    const int32_t first = __ldg(&sr_ptr[__ldg(&ssr_ptr[nssr])]);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = first + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        double acc = 0.0;
        for (int32_t p = __ldg(&rowptr[r]) + lane; p < __ldg(&rowptr[r + 1]); p += 32)
            acc = fma(__ldg(&vals[p]), __ldg(&x[__ldg(&colidx[p])]), acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) csrk::dev::store_y<double, double>(y, r, acc, alpha, beta, epi);
    }
}

int err(int code, const std::string& m) {
    csrk::set_last_error(m);
    return code;
}

// Identifier of the calling thread's current CUDA context (0 when none is current yet),
// through the driver entry points the runtime exposes.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the static scratch in the current context: looked up (with the device
// current) on the first call in each context, then reused.
int scratch_on_current_device(double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = current_context_id();
    for (int i = 0; id && i < g_scratch_count; ++i)
        if (g_scratch_addr[i].ctx_id == id) {
            *out = g_scratch_addr[i].addr;
            return CSRK_OK;
        }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
        return err(CSRK_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    id = current_context_id();   // the lookup makes the device's context current if none was
    if (id) {
        int slot = g_scratch_count < MAX_CONTEXTS ? g_scratch_count++ : (int)(id % MAX_CONTEXTS);
        g_scratch_addr[slot] = ScratchAddr{id, static_cast<double*>(p)};
    }
    *out = static_cast<double*>(p);
    return CSRK_OK;
}

bool overlap(const double* a, const double* b, int64_t n) {
    const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    const uintptr_t len = (uintptr_t)n * sizeof(double);
    return pa < pb + len && pb < pa + len;
}

}  // namespace

extern "C" {

int csrk_spmv_static_scratch(int32_t n, int32_t nssr, const int32_t* ssr_ptr,
                             const int32_t* sr_ptr, const int32_t* rowptr,
                             const int32_t* colidx, const double* vals, const int32_t* perm,
                             double alpha, const double* x, double beta, double* y,
                             void* stream) {
    if (n < 0 || nssr < 0) return err(CSRK_ERR_ARG, "n and nssr must be >= 0");
    if (n > STATIC_MAX_ROWS)
        return err(CSRK_ERR_ARG, "n = " + std::to_string(n) + " exceeds the static scratch capacity of " +
                                     std::to_string(STATIC_MAX_ROWS) + " rows; use csrk_spmv");
    if (n == 0) return CSRK_OK;
    if (!ssr_ptr || !sr_ptr || !rowptr || !colidx || !vals || !x || !y)
        return err(CSRK_ERR_ARG, "NULL array argument");
    // without a permutation the kernels read x while they write y; with one, x and y are
    // copied into the static array first, so they may alias
    if (!perm && overlap(x, y, n)) return err(CSRK_ERR_ARG, "x and y overlap (allowed only when perm is given)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int grid = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    grid = (int)std::min<int64_t>(nssr, (int64_t)sms * 8);
    const int epi = (alpha != 1.0 ? csrk::dev::EPI_SCALE : 0) | (beta != 0.0 ? csrk::dev::EPI_ACCUM : 0);
    auto run = [&](const double* xk, double* yk) -> int {
        if (grid > 0)
            csr3_static_kernel<<<grid, 256, 0, s>>>(nssr, ssr_ptr, sr_ptr, rowptr, colidx, vals, xk, yk, alpha,
                                                    beta, epi);
        tail_rows_kernel<<<sms, 256, 0, s>>>(n, nssr, ssr_ptr, sr_ptr, rowptr, colidx, vals, xk, yk, alpha, beta,
                                             epi);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? CSRK_OK : err(CSRK_ERR_CUDA, cudaGetErrorString(e));
    };
    if (!perm) return run(x, y);   // no reordering: the kernels work on the caller's vectors
    double* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc) return rc;
    double* xp = scratch;
    double* yp = scratch + STATIC_MAX_ROWS;
    // Every scratch element the kernel reads is written first in this call (x always; the
    // old y only when beta != 0), so nothing has to be cleared between calls.
    if ((rc = csrk::launch_gather_rows(x, 1, xp, 1, perm, n, 1, 8, s)))
        return err(CSRK_ERR_CUDA, "permute x");
    if (beta != 0.0 && (rc = csrk::launch_gather_rows(y, 1, yp, 1, perm, n, 1, 8, s)))
        return err(CSRK_ERR_CUDA, "permute y");
    if ((rc = run(xp, yp))) return rc;
    if ((rc = csrk::launch_scatter_rows(yp, 1, y, 1, perm, n, 1, 8, s)))
        return err(CSRK_ERR_CUDA, "unpermute y");
    return CSRK_OK;
}

}  // extern "C"
