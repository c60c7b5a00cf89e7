// ems_device.cuh -- block-level device helpers shared by the stress and
// Krylov kernels: precision-exact FMA, chunk-carry scans, block reductions.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace ems {

// fused multiply-add in the precision of its arguments (an unqualified fma on
// floats may resolve to the double overload and run on the FP64 pipe)
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }

// exclusive scan of affine maps x -> A + B x, left to right; returns the carry
// into this thread's chunk (the composite of all earlier chunks applied to 0).
// One barrier: every warp publishes its aggregate, then composes the
// aggregates of the warps before it with a warp-shuffle scan.
template <typename R>
__device__ __forceinline__ R scan_fwd(R A, R B, R *sA, R *sB, R *sC) {
    (void)sC;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const R Ao = __shfl_up_sync(full, A, d), Bo = __shfl_up_sync(full, B, d);
        if (lane >= d) { A = fmx(B, Ao, A); B = B * Bo; }
    }
    R cw = R(0);
    if (nw > 1) {
        if (lane == 31) { sA[w] = A; sB[w] = B; }
        __syncthreads();
        // compose the aggregates of warps 0..w-1 with a warp scan (lane k
        // holds warp k's map, identity from lane w on)
        R a = lane < w ? sA[lane] : R(0), b = lane < w ? sB[lane] : R(1);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const R ao = __shfl_up_sync(full, a, d), bo = __shfl_up_sync(full, b, d);
            if (lane >= d) { a = fmx(b, ao, a); b = b * bo; }
        }
        cw = __shfl_sync(full, a, 31);
    }
    const R incl = fmx(B, cw, A);
    const R ex = __shfl_up_sync(full, incl, 1);
    return lane == 0 ? cw : ex;
}

// the same from right to left (carry = start value of the next chunk)
template <typename R>
__device__ __forceinline__ R scan_bwd(R A, R B, R *sA, R *sB, R *sC) {
    (void)sC;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const R Ao = __shfl_down_sync(full, A, d), Bo = __shfl_down_sync(full, B, d);
        if (lane + d < 32) { A = fmx(B, Ao, A); B = B * Bo; }
    }
    R cw = R(0);
    if (nw > 1) {
        if (lane == 0) { sA[32 + w] = A; sB[32 + w] = B; }
        __syncthreads();
        // warps nw-1 .. w+1 in that order: lane j holds warp nw-1-j's map
        const int k = nw - 1 - lane;
        R a = k > w ? sA[32 + k] : R(0), b = k > w ? sB[32 + k] : R(1);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const R ao = __shfl_up_sync(full, a, d), bo = __shfl_up_sync(full, b, d);
            if (lane >= d) { a = fmx(b, ao, a); b = b * bo; }
        }
        cw = __shfl_sync(full, a, 31);
    }
    const R incl = fmx(B, cw, A);
    const R ex = __shfl_down_sync(full, incl, 1);
    return lane == 31 ? cw : ex;
}

// block-wide argmax (largest value, lowest index on ties); all threads get it
__device__ __forceinline__ void block_argmax(double &v, int &i, double *sv, int *si) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const int oi = __shfl_down_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
    __syncthreads();
    if (lane == 0) { sv[w] = v; si[w] = i; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k)
            if (sv[k] > sv[0] || (sv[k] == sv[0] && si[k] < si[0])) { sv[0] = sv[k]; si[0] = si[k]; }
    }
    __syncthreads();
    v = sv[0]; i = si[0];
    __syncthreads();
}

__device__ __forceinline__ double block_min(double v, double *sv) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sv[w] = v;
    __syncthreads();
    double r = sv[0];
    for (int k = 1; k < nw; ++k) r = fmin(r, sv[k]);
    __syncthreads();
    return r;
}

}  // namespace ems
