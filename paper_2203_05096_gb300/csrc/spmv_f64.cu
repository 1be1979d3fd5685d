// CSR-3 kernels with FP64 stored values (FP64 x, FP64 accumulation).
#include "launch_impl.cuh"

namespace csrk {
int launch_csr3_f64(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream) {
    if (a.x_f32 || a.acc_f32) return -1;
    return dev::dispatch_lanes<double, double, double>(a, cfg, plan, (cudaStream_t)stream);
}
}  // namespace csrk
