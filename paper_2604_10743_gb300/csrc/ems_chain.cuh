// ems_chain.cuh -- device-side definitions shared by the chain kernels
// (ems_stress.cu: one-CTA chains and branched trees; ems_chain_cl_*.cu: chains
// on a thread-block cluster): the launch arguments, the 2 x 2 product helpers
// of the parallel factorisation, the nucleation tests, and the cluster
// launchers' declarations.
#pragma once
#include <cuda_runtime.h>

#include "ems_device.cuh"
#include "ems_internal.cuh"

namespace ems {

constexpr int kStatusOverflow = 2;       // status word: a void slot list overflowed

template <typename R>
struct ChainArgs {
    const int32_t *trees;
    const int64_t *toff, *pbase;
    int64_t N, P;
    int n_trees, maxv, n_steps, refactor_all, n_bucket, S;
    double dt, t0, Binv;
    const double *V, *g, *leak, *f;
    double *thr;
    R *sig, *alpha, *beta, *gam, *uu, *Pf, *Pb, *dtg, *dtl;
    R *kc;                            // increment form, streaming kernel: compensation of the state sums
    double *pinv;
    int32_t *v_count, *v_node, *v_seg;
    double *v_vol, *v_tnuc;
    int32_t *dirty;
    const double *j;
    int n_seg;
    const int32_t *face_seg, *inc_ptr, *inc_seg, *gpar, *child_ptr, *child_gidx;
    int32_t *status, *counters;
    const int32_t *kr_mode, *kdone;   // trees the reduced model advances; steps already done
    int32_t *sched;                   // per-tree step schedule: <= 1 fine, r > 1 r-times coarser, < 0 frozen
    double *fdt;                      // step the tree's factors were built for
    double guard;                     // a coarse tree turns fine once sigma >= guard * its lowest sigma_crit
    unsigned long long *work;         // node-steps executed
    const double *t0p;                // when set, the aging-step start time is read here
};


// 2 x 2 matrix product helpers for the parallel pivot recurrence; products
// are rescaled by exact powers of two (only ratios of entries are used)
struct M2 { double a, b, c, d; };                 // [[a, b], [c, d]]
__device__ __forceinline__ M2 m2mul(const M2 &x, const M2 &y) {   // x * y, every rounding explicit
    M2 r{__fma_rn(x.a, y.a, __dmul_rn(x.b, y.c)), __fma_rn(x.a, y.b, __dmul_rn(x.b, y.d)),
         __fma_rn(x.c, y.a, __dmul_rn(x.d, y.c)), __fma_rn(x.c, y.b, __dmul_rn(x.d, y.d))};
    const double mx = fmax(fmax(fabs(r.a), fabs(r.b)), fmax(fabs(r.c), fabs(r.d)));
    if (mx > 0.0 && isfinite(mx)) {
        const int e = ilogb(mx);
        r.a = scalbn(r.a, -e); r.b = scalbn(r.b, -e); r.c = scalbn(r.c, -e); r.d = scalbn(r.d, -e);
    }
    return r;
}
__device__ __forceinline__ M2 m2shfl_up(const M2 &x, int d) {
    const unsigned full = 0xffffffffu;
    return M2{__shfl_up_sync(full, x.a, d), __shfl_up_sync(full, x.b, d), __shfl_up_sync(full, x.c, d),
              __shfl_up_sync(full, x.d, d)};
}


template <typename R>
__device__ __forceinline__ bool above(R s, long long tb, float tf);
template <>
__device__ __forceinline__ bool above<double>(double s, long long tb, float) {
    // sigma >= thr for thr > 0 by comparing IEEE bit patterns as integers
    return __double_as_longlong(s) >= tb;
}
template <>
__device__ __forceinline__ bool above<float>(float s, long long, float tf) { return s >= tf; }

// Segment a void at stress node v (tree-local) degrades: an interior node's
// own segment; at an IR node the incident tree segment with the larger |j|
// (lowest id on ties; the list is ascending).
template <typename R>
__device__ __forceinline__ int void_segment(const ChainArgs<R> &a, int s, int64_t gnode) {
    int best = a.inc_seg[a.inc_ptr[gnode]];
    double bj = fabs(a.j[(int64_t)s * a.n_seg + best]);
    for (int k = a.inc_ptr[gnode] + 1; k < a.inc_ptr[gnode + 1]; ++k) {
        const int sg = a.inc_seg[k];
        const double aj = fabs(a.j[(int64_t)s * a.n_seg + sg]);
        if (aj > bj) { bj = aj; best = sg; }
    }
    return best;
}

// true when any of this thread's stresses reaches the guard level
template <typename R, int M>
__device__ __forceinline__ bool near_guard(const R (&sg)[M], double gthr) {
    bool near = false;
#pragma unroll
    for (int k = 0; k < M; ++k) near |= above<R>(sg[k], __double_as_longlong(gthr), __double2float_rd(gthr));
    return near;
}


// One launch of the cluster chain kernel for a bucket: n_trees chains x S
// samples, CL CTAs of T_cta threads per chain, M nodes per thread.  Defined in
// ems_chain_cl_f32.cu / ems_chain_cl_f64.cu; cudaErrorInvalidValue for a
// shape with no compiled kernel.
cudaError_t launch_cluster(int M, int CL, int T_cta, unsigned n_trees, int S, cudaStream_t st,
                           const ChainArgs<float> &a);
cudaError_t launch_cluster(int M, int CL, int T_cta, unsigned n_trees, int S, cudaStream_t st,
                           const ChainArgs<double> &a);
// the same with the chunk coefficients in shared memory (FP32; ems_chain_cl_f32s.cu)
cudaError_t launch_cluster_smem(int M, int CL, int T_cta, unsigned n_trees, int S, cudaStream_t st,
                                const ChainArgs<float> &a);

}  // namespace ems
