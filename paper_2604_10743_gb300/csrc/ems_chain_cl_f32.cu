// ems_chain_cl_f32.cu -- FP32 (increment form, compensated sums) cluster
// chain kernels: 16 nodes per thread on clusters of 2, 4, 8 CTAs of <= 320
// threads or 5, 6 CTAs of <= 256 (all registers, no spill).  (8 nodes per
// thread stays off in FP32: on 10,235-node stripes it missed the 1e-4 bar
// against the oracle, 1.4e-4, and ran at half the speed.)
#include "ems_chain_cl.cuh"

namespace ems {

cudaError_t launch_cluster(int M, int CL, int T_cta, unsigned n_trees, int S, cudaStream_t st,
                           const ChainArgs<float> &a) {
    if (cluster_max_threads(EMS_F32, M, CL) < T_cta) return cudaErrorInvalidValue;
    if (M == 16) {
        switch (CL) {
            case 2: return launch_cl<float, 16, 2, 320>(T_cta, n_trees, S, st, a);
            case 4: return launch_cl<float, 16, 4, 320>(T_cta, n_trees, S, st, a);
            case 5: return launch_cl<float, 16, 5, 256>(T_cta, n_trees, S, st, a);
            case 6: return launch_cl<float, 16, 6, 256>(T_cta, n_trees, S, st, a);
            case 8: return launch_cl<float, 16, 8, 320>(T_cta, n_trees, S, st, a);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace ems
