// ems_krylov_m32_f64.cu -- the reduced-model kernel for FP64 contexts with chunks
// of 32 nodes per thread; see ems_krylov_kernels.cuh.
#include "ems_krylov_kernels.cuh"

namespace ems {
template <>
ems_status kr_launch<32, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a) {
    return launch_kr<32, double>(c, b, a);
}
}  // namespace ems
