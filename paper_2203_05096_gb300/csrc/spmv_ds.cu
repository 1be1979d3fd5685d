// CSR-3 SpMV with FP64 values stored as (hi, lo) FP32 pairs and FP64 x / y: FP64-accurate
// row sums computed on the FP32 pipes (see ds_accum in kernels.cuh); kernels 2 / 3 gather
// the split x from L2, kernel 6 stages each SSR's window of it in shared memory.
#include "launch_impl.cuh"

namespace csrk {
int launch_csr3_ds(const LaunchArgs& a, const KernelConfig& cfg, const StagePlan& plan, void* stream) {
    if (a.x_f32 || a.acc_f32 || a.spmm) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    KernelConfig c = cfg;
    if (cfg.kernel == 6) {   // x windows in shared memory
        if (!a.win) return -1;
        c.kernel = 0;
        switch (cfg.unroll) {
            case 4: return dev::launch_one<dev::ds_t, double, double, 1, 5, 4>(a, c, plan, s);
            case 8: return dev::launch_one<dev::ds_t, double, double, 1, 5, 8>(a, c, plan, s);
            case 16: return dev::launch_one<dev::ds_t, double, double, 1, 5, 16>(a, c, plan, s);
            default: return -1;
        }
    }
    c.kernel = cfg.kernel - 2;   // 2 -> TMA-staged, 3 -> direct loads
    switch (cfg.unroll) {
        case 4: return dev::launch_one<dev::ds_t, double, double, 1, 2, 4>(a, c, plan, s);
        case 8: return dev::launch_one<dev::ds_t, double, double, 1, 2, 8>(a, c, plan, s);
        case 16: return dev::launch_one<dev::ds_t, double, double, 1, 2, 16>(a, c, plan, s);
        default: return -1;
    }
}
}  // namespace csrk
