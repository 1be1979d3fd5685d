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
// plain loads (no TMA over-read), so the caller's arrays need no padding.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.cuh"

namespace {

constexpr int64_t STATIC_MAX_ROWS = 1 << 20;   // 1,048,576 rows: 16 MiB of FP64 scratch

// First half: x in the reordered numbering; second half: the reordered result.
static __device__ __align__(256) double g_static_scratch[2 * STATIC_MAX_ROWS];

std::mutex g_scratch_mu;
constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {};   // device address of g_static_scratch per device

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

int err(int code, const std::string& m) {
    csrk::set_last_error(m);
    return code;
}

// Device address of the static scratch on the current device, looked up once per device.
int scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(CSRK_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return err(CSRK_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return err(CSRK_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return CSRK_OK;
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
    if (!ssr_ptr || !sr_ptr || !rowptr || !colidx || !vals || !x || !y || x == y)
        return err(CSRK_ERR_ARG, "NULL or overlapping array argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int grid = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (int)std::min<int64_t>(nssr, (int64_t)(sms > 0 ? sms : 1) * 8);
    const int epi = (alpha != 1.0 ? csrk::dev::EPI_SCALE : 0) | (beta != 0.0 ? csrk::dev::EPI_ACCUM : 0);
    if (!perm) {   // no reordering: the kernel works on the caller's vectors directly
        if (grid > 0)
            csr3_static_kernel<<<grid, 256, 0, s>>>(nssr, ssr_ptr, sr_ptr, rowptr, colidx, vals, x, y,
                                                    alpha, beta, epi);
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? CSRK_OK : err(CSRK_ERR_CUDA, cudaGetErrorString(e));
    }
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
    if (grid > 0)
        csr3_static_kernel<<<grid, 256, 0, s>>>(nssr, ssr_ptr, sr_ptr, rowptr, colidx, vals, xp, yp,
                                                alpha, beta, epi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(CSRK_ERR_CUDA, cudaGetErrorString(e));
    if ((rc = csrk::launch_scatter_rows(yp, 1, y, 1, perm, n, 1, 8, s)))
        return err(CSRK_ERR_CUDA, "unpermute y");
    return CSRK_OK;
}

}  // extern "C"
