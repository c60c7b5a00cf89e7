// ems_krylov_m8_f64.cu -- the reduced-model kernel for FP64 contexts with chunks
// of 8 nodes per thread; see ems_krylov_kernels.cuh.
#include "ems_krylov_kernels.cuh"

namespace ems {
template <>
ems_status kr_launch<8, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a) {
    return launch_kr<8, double>(c, b, a);
}
}  // namespace ems
