// CSR-3 kernels with FP32 stored values: (x, accumulation) in (FP64, FP64), (FP32, FP64)
// or (FP32, FP32).
#include "launch_impl.cuh"

namespace csrk {
int launch_csr3_f32(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!a.x_f32) {
        if (a.acc_f32) return -1;
        return dev::dispatch_lanes<float, double, double>(a, cfg, plan, s);
    }
    if (a.acc_f32) return dev::dispatch_lanes<float, float, float>(a, cfg, plan, s);
    return dev::dispatch_lanes<float, float, double>(a, cfg, plan, s);
}
}  // namespace csrk
