// Device permutation of dense vectors between the input numbering and the CSR-k
// (reordered) numbering: x_p[i] = x[perm[i]] before the SpMV, y[perm[i]] = y_p[i] after.
// Rows of k contiguous entries move together (SpMM blocks).  Pure data movement.
#include <cuda_runtime.h>
#include <stdint.h>

#include "csrk_internal.h"
#include "kernels.cuh"

namespace csrk {
namespace {

template <typename T>
__global__ void gather_rows_kernel(const T* __restrict__ in, int64_t ldi, T* __restrict__ out,
                                   int64_t ldo, const int32_t* __restrict__ perm, int32_t n,
                                   int32_t k) {
    const int64_t total = (int64_t)n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, c = t - i * k;
        out[i * ldo + c] = __ldg(&in[(int64_t)__ldg(&perm[i]) * ldi + c]);
    }
}

template <typename T>
__global__ void scatter_rows_kernel(const T* __restrict__ in, int64_t ldi, T* __restrict__ out,
                                    int64_t ldo, const int32_t* __restrict__ perm, int32_t n,
                                    int32_t k) {
    const int64_t total = (int64_t)n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, c = t - i * k;
        out[(int64_t)__ldg(&perm[i]) * ldo + c] = __ldg(&in[i * ldi + c]);
    }
}

int grid_for(int64_t total) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (total + 255) / 256;
    int64_t cap = (int64_t)sms * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int launch_gather_rows(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm,
                       int32_t n, int32_t k, int elem_bytes, void* stream) {
    if ((int64_t)n * k == 0) return 0;
    const int grid = grid_for((int64_t)n * k);
    cudaStream_t s = (cudaStream_t)stream;
    if (elem_bytes == 8)
        gather_rows_kernel<double><<<grid, 256, 0, s>>>((const double*)in, ldi, (double*)out, ldo, perm, n, k);
    else
        gather_rows_kernel<float><<<grid, 256, 0, s>>>((const float*)in, ldi, (float*)out, ldo, perm, n, k);
    return (int)cudaGetLastError();
}

int launch_scatter_rows(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm,
                        int32_t n, int32_t k, int elem_bytes, void* stream) {
    if ((int64_t)n * k == 0) return 0;
    const int grid = grid_for((int64_t)n * k);
    cudaStream_t s = (cudaStream_t)stream;
    if (elem_bytes == 8)
        scatter_rows_kernel<double><<<grid, 256, 0, s>>>((const double*)in, ldi, (double*)out, ldo, perm, n, k);
    else
        scatter_rows_kernel<float><<<grid, 256, 0, s>>>((const float*)in, ldi, (float*)out, ldo, perm, n, k);
    return (int)cudaGetLastError();
}

namespace {
// One block: initialise an mbarrier that expects two arrivals, arrive once, and wait on
// it with the kernels' bounded wait.  Nothing ever completes the phase, so the wait must
// give up after timeout_ns and report through the status word.
__global__ void bounded_wait_probe(unsigned long long timeout_ns, int32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 2);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        dev::mbar_arrive(&bar);
        if (!dev::mbar_wait_bounded(&bar, 0, timeout_ns)) dev::report(status, 1);
    }
}
}  // namespace

int launch_bounded_wait_probe(unsigned long long timeout_ns, int32_t* status, void* stream) {
    bounded_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(timeout_ns, status);
    return (int)cudaGetLastError();
}

}  // namespace csrk
