// ems_chain_cl_f32s.cu -- FP32 cluster chain kernels with the chunk
// coefficients and thresholds in shared memory (20 bytes per node): 16 nodes
// per thread on clusters of 2, 4, 8 CTAs of <= 320 threads (<= 102 registers,
// two CTAs per SM) or 5, 6 CTAs of <= 256 (<= 128 registers, two per SM).
#include "ems_chain_cl.cuh"

namespace ems {

cudaError_t cluster_smem_init() {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {smem_limit<float, 16, 2, 320>(), smem_limit<float, 16, 4, 320>(),
                          smem_limit<float, 16, 5, 256>(), smem_limit<float, 16, 6, 256>(),
                          smem_limit<float, 16, 8, 320>()})
        if (r != cudaSuccess && e == cudaSuccess) e = r;
    return e;
}

cudaError_t launch_cluster_smem(int M, int CL, int T_cta, unsigned n_trees, int S, cudaStream_t st,
                                const ChainArgs<float> &a) {
    if (cluster_smem_max_threads(M, CL) < T_cta) return cudaErrorInvalidValue;
    if (M == 16) {
        switch (CL) {
            case 2: return launch_cl<float, 16, 2, 320, true>(T_cta, n_trees, S, st, a);
            case 4: return launch_cl<float, 16, 4, 320, true>(T_cta, n_trees, S, st, a);
            case 5: return launch_cl<float, 16, 5, 256, true>(T_cta, n_trees, S, st, a);
            case 6: return launch_cl<float, 16, 6, 256, true>(T_cta, n_trees, S, st, a);
            case 8: return launch_cl<float, 16, 8, 320, true>(T_cta, n_trees, S, st, a);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace ems
