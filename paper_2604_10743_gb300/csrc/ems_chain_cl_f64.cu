// ems_chain_cl_f64.cu -- FP64 (state form) cluster chain kernels: 8 nodes
// per thread on clusters of 2, 4, 8 CTAs of <= 320 threads.
#include "ems_chain_cl.cuh"

namespace ems {

cudaError_t launch_cluster(int M, int CL, int T_cta, unsigned n_trees, int S, cudaStream_t st,
                           const ChainArgs<double> &a) {
    if (cluster_max_threads(EMS_F64, M, CL) < T_cta) return cudaErrorInvalidValue;
    if (M == 8) {
        switch (CL) {
            case 2: return launch_cl<double, 8, 2, 320>(T_cta, n_trees, S, st, a);
            case 4: return launch_cl<double, 8, 4, 320>(T_cta, n_trees, S, st, a);
            case 8: return launch_cl<double, 8, 8, 320>(T_cta, n_trees, S, st, a);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace ems
