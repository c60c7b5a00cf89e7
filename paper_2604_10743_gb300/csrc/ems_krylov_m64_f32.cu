// ems_krylov_m64_f32.cu -- the reduced-model kernel for FP32 contexts with chunks
// of 64 nodes per thread; see ems_krylov_kernels.cuh.
#include "ems_krylov_kernels.cuh"

namespace ems {
template <>
ems_status kr_launch<64, float>(ems_ctx *c, const Bucket &b, KrArgs<float> &a) {
    return launch_kr<64, float>(c, b, a);
}
}  // namespace ems
