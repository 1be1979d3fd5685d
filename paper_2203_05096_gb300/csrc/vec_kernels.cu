// Device permutation of dense vectors between the input numbering and the CSR-k
// (reordered) numbering: x_p[i] = x[perm[i]] before the SpMV, y[perm[i]] = y_p[i] after.
// Rows of k contiguous entries move together (SpMM blocks).  Pure data movement.
#include <cuda_runtime.h>
#include <stdint.h>

#include "csrk_internal.h"
#include "convert.cuh"
#include "kernels.cuh"

namespace csrk {
namespace {

// Each thread moves ILP elements per loop trip with independent loads (the perm lookups
// first, then the data), so several dependent perm -> data chains are in flight at once
// instead of one.
constexpr int PERM_ILP = 4;

// Element t of the n x k block is row t / k, column t % k; with K1 (k == 1) no division
// is done at all (a 64-bit division by a runtime k costs dozens of instructions), and for
// k > 1 the division is 32-bit (n * k < 2^32 is checked by the launcher).
template <typename T, bool SCATTER, bool K1>
__global__ void permute_rows_kernel(const T* __restrict__ in, int64_t ldi, T* __restrict__ out,
                                    int64_t ldo, const int32_t* __restrict__ perm, int32_t n,
                                    int32_t k) {
    const uint32_t total = (uint32_t)n * (uint32_t)k;
    const uint32_t stride = gridDim.x * blockDim.x;
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    auto split = [&](uint32_t e, int64_t& i, int64_t& c) {
        if (K1) {
            i = e;
            c = 0;
        } else {
            const uint32_t q = e / (uint32_t)k;
            i = q;
            c = e - q * (uint32_t)k;
        }
    };
    for (; t + (PERM_ILP - 1) * stride < total && t + (PERM_ILP - 1) * stride >= t; t += PERM_ILP * stride) {
        int64_t i[PERM_ILP], c[PERM_ILP], pi[PERM_ILP];
        T v[PERM_ILP];
#pragma unroll
        for (int u = 0; u < PERM_ILP; ++u) {
            split(t + u * stride, i[u], c[u]);
            pi[u] = __ldg(&perm[i[u]]);
        }
#pragma unroll
        for (int u = 0; u < PERM_ILP; ++u)
            v[u] = SCATTER ? __ldg(&in[i[u] * ldi + c[u]]) : __ldg(&in[pi[u] * ldi + c[u]]);
#pragma unroll
        for (int u = 0; u < PERM_ILP; ++u) {
            if (SCATTER) out[pi[u] * ldo + c[u]] = v[u];
            else out[i[u] * ldo + c[u]] = v[u];
        }
    }
    for (; t < total; t += stride) {
        int64_t i, c;
        split(t, i, c);
        const int64_t pi = __ldg(&perm[i]);
        if (SCATTER) out[pi * ldo + c] = __ldg(&in[i * ldi + c]);
        else out[i * ldo + c] = __ldg(&in[pi * ldi + c]);
    }
}

template <typename T, bool SCATTER>
int launch_permute(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm, int32_t n,
                   int32_t k, int grid, cudaStream_t s) {
    if ((uint64_t)n * (uint64_t)k >= (1ull << 32)) return (int)cudaErrorInvalidValue;
    if (k == 1)
        permute_rows_kernel<T, SCATTER, true><<<grid, 256, 0, s>>>((const T*)in, ldi, (T*)out, ldo, perm, n, k);
    else
        permute_rows_kernel<T, SCATTER, false><<<grid, 256, 0, s>>>((const T*)in, ldi, (T*)out, ldo, perm, n, k);
    return (int)cudaGetLastError();
}

// Enough blocks of 256 for one ILP trip per thread, at most 8 per SM.
int grid_for(int64_t total) {
    static int sms_by_dev[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = dev < 64 ? sms_by_dev[dev] : 0;
    if (sms <= 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (dev < 64) sms_by_dev[dev] = sms;
    }
    int64_t g = (total + 256 * 4 - 1) / (256 * 4);
    int64_t cap = (int64_t)sms * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

int launch_gather_rows(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm,
                       int32_t n, int32_t k, int elem_bytes, void* stream) {
    if ((int64_t)n * k == 0) return 0;
    const int grid = grid_for((int64_t)n * k);
    cudaStream_t s = (cudaStream_t)stream;
    return elem_bytes == 8 ? launch_permute<double, false>(in, ldi, out, ldo, perm, n, k, grid, s)
                           : launch_permute<float, false>(in, ldi, out, ldo, perm, n, k, grid, s);
}

int launch_scatter_rows(const void* in, int64_t ldi, void* out, int64_t ldo, const int32_t* perm,
                        int32_t n, int32_t k, int elem_bytes, void* stream) {
    if ((int64_t)n * k == 0) return 0;
    const int grid = grid_for((int64_t)n * k);
    cudaStream_t s = (cudaStream_t)stream;
    return elem_bytes == 8 ? launch_permute<double, true>(in, ldi, out, ldo, perm, n, k, grid, s)
                           : launch_permute<float, true>(in, ldi, out, ldo, perm, n, k, grid, s);
}

namespace {
// x_pairs[i] = split(x[perm[i]]) (or x[i] without perm), optionally also x64[i] = that
// FP64 value; any element outside the pair range sets *flag (reset by the caller).
__global__ void split_pairs_kernel(const double* __restrict__ in, const int32_t* __restrict__ perm,
                                   int32_t n, double* __restrict__ x64, float2* __restrict__ pairs,
                                   int32_t* flag) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = perm ? __ldg(&in[__ldg(&perm[i])]) : __ldg(&in[i]);
        if (x64) x64[i] = v;
        dev::xpair q;
        bad |= !dev::split_x(v, q);
        pairs[i] = make_float2(q.hi, q.lo);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

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

int launch_split_pairs(const double* in, const int32_t* perm, int32_t n, double* x64, void* pairs,
                       int32_t* flag, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return (int)e;
    if (n == 0) return 0;
    split_pairs_kernel<<<grid_for(n), 256, 0, s>>>(in, perm, n, x64, (float2*)pairs, flag);
    return (int)cudaGetLastError();
}

namespace {
// both narrowings of each input: the integer one the solvers use and the instruction's
__global__ void narrow_pair_kernel(const double* __restrict__ in, int64_t n, float* __restrict__ by_int,
                                   float* __restrict__ by_cvt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = in[i];
        by_int[i] = dev::f64_to_f32(d);
        by_cvt[i] = (float)d;
    }
}
}  // namespace

int launch_narrow_pair(const double* in, int64_t n, float* by_int, float* by_cvt, void* stream) {
    if (n <= 0) return 0;
    narrow_pair_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(in, n, by_int, by_cvt);
    return (int)cudaGetLastError();
}

int launch_bounded_wait_probe(unsigned long long timeout_ns, int32_t* status, void* stream) {
    bounded_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(timeout_ns, status);
    return (int)cudaGetLastError();
}

}  // namespace csrk
