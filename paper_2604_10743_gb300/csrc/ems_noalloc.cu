// ems_noalloc.cu -- a PCG solve that allocates no device memory.
//
// The context-based IR solve keeps its CG vectors in the caller's workspace.
// This entry point is for callers that cannot hand out device memory at all:
// code that runs under another framework's allocator and may not call
// cudaMalloc itself, or that cannot accept the device-wide synchronisation a
// cudaMalloc / cudaFree can cause in the middle of its own stream work.  Its
// five work vectors live in one file-scope device array of fixed size, held by
// every GPU that loads the library until the process exits.
#include <mutex>

#include "ems_internal.cuh"

#define EMS_NOALLOC_MAX_N 16384   // unknowns the static scratch holds (5 vectors, 640 KB)

namespace {

// r, z, p, Ap and the inverse diagonal for up to EMS_NOALLOC_MAX_N unknowns,
// then the iteration count and convergence flag of the last call
static __device__ __align__(256) double g_noalloc_scratch[5 * EMS_NOALLOC_MAX_N + 2];

__device__ __forceinline__ double csr_row_dot(const int32_t *rp, const int32_t *col, const double *val,
                                              const double *v, int i) {
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc += val[k] * v[col[k]];
    return acc;
}

template <int K>
__device__ void nsum(double (&v)[K], double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) sh[q * 32 + w] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += sh[q * 32 + k];
        v[q] = t;
    }
}

// Jacobi-preconditioned CG in one CTA on the caller's CSR matrix; the work
// vectors are the static array above, whose device address the host passes
// in.  Every scratch entry is written before it is read, so what an earlier
// call left there does not matter.
__global__ void __launch_bounds__(1024) k_pcg_noalloc(double *scratch, int n, const int32_t *rp, const int32_t *col,
                                                      const double *val, const double *b, double *x, double rtol,
                                                      int max_iter) {
    __shared__ double sh[96];
    double *r = scratch, *z = r + EMS_NOALLOC_MAX_N, *p = z + EMS_NOALLOC_MAX_N;
    double *Ap = p + EMS_NOALLOC_MAX_N, *dinv = Ap + EMS_NOALLOC_MAX_N, *info = dinv + EMS_NOALLOC_MAX_N;
    double v3[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double d = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] == i) d += val[k];
        const double di = 1.0 / d;
        const double ri = b[i] - csr_row_dot(rp, col, val, x, i);
        const double zi = di * ri;
        dinv[i] = di; r[i] = ri; z[i] = zi; p[i] = zi;
        v3[0] += ri * zi; v3[1] += ri * ri; v3[2] += b[i] * b[i];
    }
    nsum<3>(v3, sh);
    double rz = v3[0], rr = v3[1];
    const double tol2 = rtol * rtol * v3[2];
    int it = 0;
    while (rr > tol2 && it < max_iter) {
        __syncthreads();                               // p complete
        double v1[1] = {0.0};
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double q = csr_row_dot(rp, col, val, p, i);
            Ap[i] = q;
            v1[0] += p[i] * q;
        }
        nsum<1>(v1, sh);
        const double alpha = rz / v1[0];
        double v2[2] = {0.0, 0.0};
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            x[i] += alpha * p[i];
            const double ri = r[i] - alpha * Ap[i];
            const double zi = dinv[i] * ri;
            r[i] = ri; z[i] = zi;
            v2[0] += ri * zi; v2[1] += ri * ri;
        }
        nsum<2>(v2, sh);
        const double beta = v2[0] / rz;
        rz = v2[0]; rr = v2[1];
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
        ++it;
    }
    if (threadIdx.x == 0) {
        info[0] = (double)it;
        info[1] = rr <= tol2 ? 1.0 : 0.0;
    }
}

std::mutex g_mu;
void *g_addr[256];          // device address of the scratch array, per device ordinal

}  // namespace

extern "C" ems_status ems_ir_pcg_noalloc(int n, const int32_t *row_ptr, const int32_t *col, const double *val,
                                         const double *b, double *x, double rtol, int max_iter, int *iterations,
                                         void *stream) {
    if (n < 1 || n > EMS_NOALLOC_MAX_N || !row_ptr || !col || !val || !b || !x || !(rtol > 0.0) || max_iter < 0)
        return EMS_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) { cudaGetLastError(); return EMS_E_CUDA; }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            // once per device, with that device current: the host-side symbol
            // is only a stand-in, the kernel-visible address comes from here
            if (cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch) != cudaSuccess) {
                g_addr[dev] = nullptr;
                cudaGetLastError();
                return EMS_E_CUDA;
            }
        }
        scratch = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
    k_pcg_noalloc<<<1, threads, 0, st>>>((double *)scratch, n, row_ptr, col, val, b, x, rtol, max_iter);
    if (cudaGetLastError() != cudaSuccess) return EMS_E_CUDA;
    double info[2] = {0.0, 0.0};
    const double *dinfo = (const double *)scratch + 5 * EMS_NOALLOC_MAX_N;
    if (cudaMemcpyAsync(info, dinfo, sizeof info, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return EMS_E_CUDA;
    }
    if (iterations) *iterations = (int)info[0];
    return info[1] > 0.5 ? EMS_OK : EMS_E_NOCONV;
}
