// ems_ir.cu -- IR-drop solve (Sec. III-C, Eq. ir_drop_mna) on the GPU.
//
// The conductance matrix of the non-pad nodes is assembled from the current
// segment resistances (each CSR entry gathers its segments in a fixed order,
// so assembly is deterministic) and solved by Jacobi-preconditioned CG in
// FP64.  Small systems run one CTA per Monte Carlo sample with block-level
// reductions; large ones run a cooperative grid over one sample at a time
// with a grid barrier (bounded spin, EMS_E_TIMEOUT on expiry) and
// fixed-order partial sums, so results are bitwise reproducible.
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

#include "ems_internal.cuh"

namespace ems {
namespace {

constexpr int kStatusNoConv = 0;     // status word indices
constexpr int kStatusTimeout = 1;
constexpr int kStatusOverflow = 2;

struct IRArgs {
    int nf, S;
    int64_t nnz;
    const int32_t *ptr, *col, *ent_ptr, *ent_seg, *rhs_ptr, *rhs_seg;
    const int8_t *ent_diag;
    const double *rhs_padV, *sink, *R;
    int n_seg;
    double *val, *b, *dinv, *x, *r, *p, *Ap, *z;
    float *val32, *dinv32, *r32, *p32, *Ap32, *z32, *d32;
    double rtol;
    int max_iter;
    int32_t *iters, *status;
    double *red;
    unsigned int *bar;
};

// val[s][k] = sum over the entry's segments of +-1/R; b = -I_sink + sum V_pad/R
__global__ void k_ir_assemble(IRArgs a) {
    const int s = blockIdx.y;
    const double *R = a.R + (size_t)s * a.n_seg;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nf; i += gridDim.x * blockDim.x) {
        double diag = 0.0;
        for (int k = a.ptr[i]; k < a.ptr[i + 1]; ++k) {
            double v = 0.0;
            for (int e = a.ent_ptr[k]; e < a.ent_ptr[k + 1]; ++e) v += 1.0 / R[a.ent_seg[e]];
            if (a.ent_diag[k]) diag = v; else v = -v;
            a.val[(size_t)s * a.nnz + k] = v;
        }
        double bb = -a.sink[i];
        for (int e = a.rhs_ptr[i]; e < a.rhs_ptr[i + 1]; ++e) bb += a.rhs_padV[e] / R[a.rhs_seg[e]];
        a.b[(size_t)s * a.nf + i] = bb;
        a.dinv[(size_t)s * a.nf + i] = 1.0 / diag;
        a.dinv32[(size_t)s * a.nf + i] = (float)(1.0 / diag);
        for (int k = a.ptr[i]; k < a.ptr[i + 1]; ++k) a.val32[(size_t)s * a.nnz + k] = (float)a.val[(size_t)s * a.nnz + k];
    }
}

// deterministic block sum of up to 3 values (all threads get the result)
template <int K>
__device__ void block_sum(double (&v)[K], double *sh /* [32*K] */) {
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

__device__ __forceinline__ double row_dot(const IRArgs &a, const double *val, const double *v, int i) {
    double acc = 0.0;
    for (int k = a.ptr[i]; k < a.ptr[i + 1]; ++k) acc += val[k] * v[a.col[k]];
    return acc;
}

// Mode A: one CTA per sample.
__global__ void __launch_bounds__(1024) k_pcg_block(IRArgs a) {
    __shared__ double sh[96];
    const int s = blockIdx.x, nf = a.nf;
    const double *val = a.val + (size_t)s * a.nnz, *b = a.b + (size_t)s * nf, *dinv = a.dinv + (size_t)s * nf;
    double *x = a.x + (size_t)s * nf, *r = a.r + (size_t)s * nf, *p = a.p + (size_t)s * nf;
    double *Ap = a.Ap + (size_t)s * nf, *z = a.z + (size_t)s * nf;
    double v3[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        double ri = b[i] - row_dot(a, val, x, i);
        double zi = dinv[i] * ri;
        r[i] = ri; z[i] = zi; p[i] = zi;
        v3[0] += ri * zi; v3[1] += ri * ri; v3[2] += b[i] * b[i];
    }
    block_sum<3>(v3, sh);
    double rz = v3[0], rr = v3[1];
    const double tol2 = a.rtol * a.rtol * v3[2];
    int it = 0;
    while (rr > tol2 && it < a.max_iter) {
        __syncthreads();
        double v1[1] = {0.0};
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            double q = row_dot(a, val, p, i);
            Ap[i] = q;
            v1[0] += p[i] * q;
        }
        block_sum<1>(v1, sh);
        const double alpha = rz / v1[0];
        double v2[2] = {0.0, 0.0};
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            x[i] += alpha * p[i];
            double ri = r[i] - alpha * Ap[i];
            double zi = dinv[i] * ri;
            r[i] = ri; z[i] = zi;
            v2[0] += ri * zi; v2[1] += ri * ri;
        }
        block_sum<2>(v2, sh);
        const double beta = v2[0] / rz;
        rz = v2[0]; rr = v2[1];
        for (int i = threadIdx.x; i < nf; i += blockDim.x) p[i] = z[i] + beta * p[i];
        ++it;
    }
    if (threadIdx.x == 0) {
        a.iters[s] = it;
        if (rr > tol2) atomicOr(&a.status[kStatusNoConv], 1);
    }
}

// Grid barrier for a cooperative launch: sense by generation counter, bounded
// spin.  Returns false (and sets the timeout status) if the wait expired.
__device__ bool grid_sync(unsigned int *bar, int32_t *status) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = bar + 1;
        const long long limit = *((volatile long long *)(bar + 2));   // polls before giving up
        const unsigned int gen = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long spins = 0;
            while (*vgen == gen) {
                if (++spins > limit || *((volatile int32_t *)&status[kStatusTimeout])) {
                    atomicOr(&status[kStatusTimeout], 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// grid-wide deterministic sum of K values: each block writes its partials to
// red[q*G + block], barrier, then one warp per block adds them in a fixed
// order (lane-strided sums, then a fixed shuffle tree) and broadcasts
template <int K>
__device__ bool grid_sum(double (&v)[K], double *sh, double *red, unsigned int *bar, int32_t *status) {
    __shared__ double bc[K];
    block_sum<K>(v, sh);
    const int G = gridDim.x;
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) red[q * G + blockIdx.x] = v[q];
    __threadfence();
    if (!grid_sync(bar, status)) return false;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double t = 0.0;
            for (int k = threadIdx.x; k < G; k += 32) t += __ldcg(red + q * G + k);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (threadIdx.x == 0) bc[q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = bc[q];
    return true;
}

__device__ __forceinline__ float row_dot32(const IRArgs &a, const float *val, const float *v, int i) {
    float acc = 0.0f;
    for (int k = a.ptr[i]; k < a.ptr[i + 1]; ++k) acc = fmaf(val[k], v[a.col[k]], acc);
    return acc;
}

// Mode P: pipelined Jacobi-PCG (the Ghysels-Vanroose recurrences) on a
// cooperative grid, one barrier per iteration: each iteration's dot
// products and the preconditioned vector m = D^-1 w are published before a
// single grid barrier, after which every block sums the partials (fixed
// order) and forms A m from its neighbours' m.  Each thread owns up to ROWS
// rows and keeps their CG vectors in registers; m is double-buffered in
// global memory.  The recurrences run in FP64 (in FP32 they stagnate on
// these systems); the true residual b - A x is recomputed after each pass
// and a new pass is started on the correction (iterative refinement) while
// it misses rtol, which also closes the residual gap of the pipelined form.
template <int ROWS>
__global__ void __launch_bounds__(512, 1) k_pcg_pipe(IRArgs a) {
    __shared__ double sh[96];
    const int nf = a.nf, G = gridDim.x;
    const int nt = G * blockDim.x, gid = blockIdx.x * blockDim.x + threadIdx.x;
    // red0 / red1 alternate between consecutive iterations; red2 serves the
    // one-off reductions, so no buffer is rewritten while a block still reads it
    double *red0 = a.red, *red1 = a.red + 4 * G, *red2 = a.red + 8 * G;
    for (int s = 0; s < a.S; ++s) {
        const double *val = a.val + (size_t)s * a.nnz, *b = a.b + (size_t)s * nf;
        const double *dinv = a.dinv + (size_t)s * nf;
        double *x = a.x + (size_t)s * nf;
        double *mb0 = a.r + (size_t)s * nf, *mb1 = a.p + (size_t)s * nf, *ub = a.z + (size_t)s * nf;
        int row[ROWS];
        double dv[ROWS];
#pragma unroll
        for (int k = 0; k < ROWS; ++k) {
            row[k] = gid + k * nt;
            dv[k] = row[k] < nf ? dinv[row[k]] : 0.0;
        }
        double vb[1] = {0.0};
#pragma unroll
        for (int k = 0; k < ROWS; ++k)
            if (row[k] < nf) vb[0] += b[row[k]] * b[row[k]];
        if (!grid_sum<1>(vb, sh, red0, a.bar, a.status)) return;   // next reduction uses red2
        const double tol2 = a.rtol * a.rtol * vb[0];
        int it = 0, parity = 0;
        double rr64 = 0.0;
        for (int round = 0; round < 8; ++round) {
            double r[ROWS], u[ROWS], w[ROWS], z[ROWS], q[ROWS], sv[ROWS], p[ROWS], d[ROWS];
            double v1[1] = {0.0};
#pragma unroll
            for (int k = 0; k < ROWS; ++k) {
                r[k] = row[k] < nf ? b[row[k]] - row_dot(a, val, x, row[k]) : 0.0;
                u[k] = dv[k] * r[k];
                z[k] = q[k] = sv[k] = p[k] = d[k] = 0.0;
                v1[0] += r[k] * r[k];
                if (row[k] < nf) ub[row[k]] = u[k];
            }
            if (!grid_sum<1>(v1, sh, red2, a.bar, a.status)) return;   // also publishes u
            rr64 = v1[0];
            if (rr64 <= tol2 || it >= a.max_iter) break;
#pragma unroll
            for (int k = 0; k < ROWS; ++k) w[k] = row[k] < nf ? row_dot(a, val, ub, row[k]) : 0.0;
            double gam_old = 1.0, alpha_old = 1.0;
            bool first = true;
            for (;;) {
                double *mb = parity ? mb1 : mb0;
                double *red = parity ? red1 : red0;
                double v3[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    v3[0] += r[k] * u[k];
                    v3[1] += w[k] * u[k];
                    v3[2] += r[k] * r[k];
                    if (row[k] < nf) mb[row[k]] = dv[k] * w[k];
                }
                if (!grid_sum<3>(v3, sh, red, a.bar, a.status)) return;
                parity ^= 1;
                const double gam = v3[0], del = v3[1], rr = v3[2];
                // a quarter of the target leaves room for the residual gap
                if (rr <= 0.0625 * tol2 || it >= a.max_iter || !(gam > 0.0)) break;
                double beta = 0.0, alpha = gam / del;
                if (!first) {
                    beta = gam / gam_old;
                    alpha = gam / (del - beta * gam / alpha_old);
                }
                first = false;
#pragma unroll
                for (int k = 0; k < ROWS; ++k) {
                    const double m = dv[k] * w[k];
                    const double nn = row[k] < nf ? row_dot(a, val, mb, row[k]) : 0.0;
                    z[k] = fma(beta, z[k], nn);
                    q[k] = fma(beta, q[k], m);
                    sv[k] = fma(beta, sv[k], w[k]);
                    p[k] = fma(beta, p[k], u[k]);
                    d[k] = fma(alpha, p[k], d[k]);
                    r[k] = fma(-alpha, sv[k], r[k]);
                    u[k] = fma(-alpha, q[k], u[k]);
                    w[k] = fma(-alpha, z[k], w[k]);
                }
                gam_old = gam; alpha_old = alpha;
                ++it;
            }
#pragma unroll
            for (int k = 0; k < ROWS; ++k)
                if (row[k] < nf) x[row[k]] += d[k];
            if (!grid_sync(a.bar, a.status)) return;                   // x complete
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.iters[s] = it;
            if (rr64 > tol2) atomicOr(&a.status[kStatusNoConv], 1);
        }
        if (!grid_sync(a.bar, a.status)) return;
    }
}

// Mode B: cooperative grid, samples one after another.
__global__ void __launch_bounds__(512) k_pcg_grid(IRArgs a) {
    __shared__ double sh[96];
    const int nf = a.nf, G = gridDim.x;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x, gstride = G * blockDim.x;
    double *redA = a.red, *redB = a.red + 3 * G;   // alternate partial buffers
    for (int s = 0; s < a.S; ++s) {
        const double *val = a.val + (size_t)s * a.nnz, *b = a.b + (size_t)s * nf;
        const double *dinv = a.dinv + (size_t)s * nf;
        double *x = a.x + (size_t)s * nf, *r = a.r + (size_t)s * nf, *p = a.p + (size_t)s * nf;
        double *Ap = a.Ap + (size_t)s * nf, *z = a.z + (size_t)s * nf;
        double v3[3] = {0.0, 0.0, 0.0};
        for (int i = gid; i < nf; i += gstride) {
            double ri = b[i] - row_dot(a, val, x, i);
            double zi = dinv[i] * ri;
            r[i] = ri; z[i] = zi; p[i] = zi;
            v3[0] += ri * zi; v3[1] += ri * ri; v3[2] += b[i] * b[i];
        }
        if (!grid_sum<3>(v3, sh, redA, a.bar, a.status)) return;
        double rz = v3[0], rr = v3[1];
        const double tol2 = a.rtol * a.rtol * v3[2];
        int it = 0;
        while (rr > tol2 && it < a.max_iter) {
            if (!grid_sync(a.bar, a.status)) return;       // p complete
            double v1[1] = {0.0};
            for (int i = gid; i < nf; i += gstride) {
                double q = row_dot(a, val, p, i);
                Ap[i] = q;
                v1[0] += p[i] * q;
            }
            if (!grid_sum<1>(v1, sh, redB, a.bar, a.status)) return;
            const double alpha = rz / v1[0];
            double v2[2] = {0.0, 0.0};
            for (int i = gid; i < nf; i += gstride) {
                x[i] += alpha * p[i];
                double ri = r[i] - alpha * Ap[i];
                double zi = dinv[i] * ri;
                r[i] = ri; z[i] = zi;
                v2[0] += ri * zi; v2[1] += ri * ri;
            }
            if (!grid_sum<2>(v2, sh, redA, a.bar, a.status)) return;
            const double beta = v2[0] / rz;
            rz = v2[0]; rr = v2[1];
            for (int i = gid; i < nf; i += gstride) p[i] = z[i] + beta * p[i];
            ++it;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.iters[s] = it;
            if (rr > tol2) atomicOr(&a.status[kStatusNoConv], 1);
        }
        if (!grid_sync(a.bar, a.status)) return;
    }
}

// a sample whose currents changed (its PCG iterated) invalidates its reduced
// models: their cache key includes the forcing

__global__ void k_scatter_u(int nf, int n_nodes, const int32_t *node_of_free, const double *x, double *u) {
    const int s = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x)
        u[(size_t)s * n_nodes + node_of_free[i]] = x[(size_t)s * nf + i];
}

// IR initial guess from the node voltages (Monte Carlo windows: the work
// vectors are rebuilt for every window, the voltages persist)
__global__ void k_gather_x(int nf, int n_nodes, const int32_t *node_of_free, const double *u, double *x) {
    const int s = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x)
        x[(size_t)s * nf + i] = u[(size_t)s * n_nodes + node_of_free[i]];
}

// j = (u_a - u_b) / (R W H) per segment
__global__ void k_currents(int n_seg, int n_nodes, const int32_t *sa, const int32_t *sb, const double *R,
                           const double *W, const double *H, const double *u, double *j) {
    const int s = blockIdx.y;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_seg; k += gridDim.x * blockDim.x) {
        const double *us = u + (size_t)s * n_nodes;
        j[(size_t)s * n_seg + k] = (us[sa[k]] - us[sb[k]]) / (R[(size_t)s * n_seg + k] * W[k] * H[k]);
    }
}

// max over nodes of (Vdd - u) / Vdd; pads sit at Vdd, so the maximum is >= 0
// and non-negative doubles order like their bit patterns (atomicMax on bits)
__global__ void k_drop(int n_nodes, double Vdd, const double *u, unsigned long long *drop_bits) {
    const int s = blockIdx.y;
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += gridDim.x * blockDim.x)
        m = fmax(m, (Vdd - u[(size_t)s * n_nodes + i]) / Vdd);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(drop_bits + s, (unsigned long long)__double_as_longlong(m));
}

IRArgs make_args(ems_ctx *c) {
    Dev &d = c->d;
    IRArgs a;
    a.nf = c->nf; a.S = c->S; a.nnz = c->nnz;
    a.ptr = d.csr_ptr; a.col = d.csr_col; a.ent_ptr = d.ent_ptr; a.ent_seg = d.ent_seg;
    a.rhs_ptr = d.rhs_ptr; a.rhs_seg = d.rhs_seg; a.ent_diag = d.ent_diag; a.rhs_padV = d.rhs_padV;
    a.sink = d.sink_of_free; a.R = d.R; a.n_seg = c->n_seg;
    a.val = d.csr_val; a.b = d.ir_b; a.dinv = d.ir_dinv; a.x = d.ir_x; a.r = d.ir_r; a.p = d.ir_p;
    a.Ap = d.ir_Ap; a.z = d.ir_z; a.rtol = c->prm.ir_rtol; a.max_iter = c->prm.ir_max_iter;
    a.val32 = d.val32; a.dinv32 = d.dinv32; a.r32 = d.r32; a.p32 = d.p32; a.Ap32 = d.Ap32; a.z32 = d.z32;
    a.d32 = d.d32;
    a.iters = d.ir_iters; a.status = d.status; a.red = d.red; a.bar = d.gbar;
    return a;
}


}  // namespace

// PCG dispatch: one CTA per sample up to 4,096 unknowns; the pipelined
// mixed-precision grid solver while one to four rows per thread cover the
// system (one 512-thread CTA per SM); the FP64 cooperative grid solver
// beyond that.
ems_status ir_assemble_and_solve(ems_ctx *c, bool warm) {
    (void)warm;
    IRArgs a = make_args(c);
    cudaStream_t st = c->stream;
    if (c->nf > 0) {
        dim3 g1((c->nf + 255) / 256 < 1024 ? (c->nf + 255) / 256 : 1024, c->S);
        k_ir_assemble<<<g1, 256, 0, st>>>(a);
        ++c->launches;
        EMS_CUDA(c, cudaGetLastError());
        int dev = 0, nsm = 0;
        EMS_CUDA(c, cudaGetDevice(&dev));
        EMS_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (c->mg.L >= 2) {
            EMS_TRY(mg_solve(c));
        } else if (c->nf <= 4096) {
            int threads = c->nf >= 1024 ? 1024 : ((c->nf + 31) / 32) * 32;
            k_pcg_block<<<c->S, threads, 0, st>>>(a);
            ++c->launches;
            EMS_CUDA(c, cudaGetLastError());
        } else if ((int64_t)c->nf <= (int64_t)4 * nsm * 512) {
            const int rows = (c->nf + nsm * 512 - 1) / (nsm * 512);
            const int G = (c->nf + rows * 512 - 1) / (rows * 512);
            EMS_CUDA(c, cudaMemsetAsync(c->d.gbar, 0, 2 * sizeof(unsigned int), st));
            void *args[] = {&a};
            void *fn = rows == 1 ? (void *)k_pcg_pipe<1> : rows == 2 ? (void *)k_pcg_pipe<2> : (void *)k_pcg_pipe<4>;
            EMS_CUDA(c, cudaLaunchCooperativeKernel(fn, dim3(G), dim3(512), args, 0, st));
            ++c->launches;
        } else {
            if (c->coop_blocks == 0) {
                int per = 0;
                EMS_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_grid, 512, 0));
                if (per < 1) return fail(c, EMS_E_CUDA, "cooperative PCG cannot be resident");
                int G = nsm * (per < 2 ? per : 2);
                int need = (c->nf + 511) / 512;
                c->coop_blocks = G < need ? G : need;
                if (c->coop_blocks > 680) c->coop_blocks = 680;   // red[] holds 2 x 3 partials per block
            }
            EMS_CUDA(c, cudaMemsetAsync(c->d.gbar, 0, 2 * sizeof(unsigned int), st));
            void *args[] = {&a};
            EMS_CUDA(c, cudaLaunchCooperativeKernel((void *)k_pcg_grid, dim3(c->coop_blocks), dim3(512),
                                                    args, 0, st));
            ++c->launches;
        }
        dim3 g2((c->nf + 255) / 256 < 1024 ? (c->nf + 255) / 256 : 1024, c->S);
        k_scatter_u<<<g2, 256, 0, st>>>(c->nf, c->n_nodes, c->d.ir_node_of_free, c->d.ir_x, c->d.u);
        ++c->launches;
        EMS_CUDA(c, cudaGetLastError());
    }
    c->have_u = true;
    return EMS_OK;
}

ems_status gather_x(ems_ctx *c) {
    if (c->nf == 0) return EMS_OK;
    dim3 g((c->nf + 255) / 256 < 1024 ? (c->nf + 255) / 256 : 1024, c->S);
    k_gather_x<<<g, 256, 0, c->stream>>>(c->nf, c->n_nodes, c->d.ir_node_of_free, c->d.u, c->d.ir_x);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status currents(ems_ctx *c) {
    Dev &d = c->d;
    dim3 g((c->n_seg + 255) / 256 < 2048 ? (c->n_seg + 255) / 256 : 2048, c->S);
    k_currents<<<g, 256, 0, c->stream>>>(c->n_seg, c->n_nodes, d.seg_a, d.seg_b, d.R, d.seg_W, d.seg_H, d.u, d.j);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

// per-node coefficients of the mapped window (with the full layout they
// persist and nothing is rebuilt)
ems_status window_derive(ems_ctx *c) {
    if (!windowed(c)) return EMS_OK;
    return sample_physics(c);
}

ems_status ir_currents_and_drop(ems_ctx *c) {
    cudaStream_t st = c->stream;
    Dev &d = c->d;
    dim3 g((c->n_seg + 255) / 256 < 2048 ? (c->n_seg + 255) / 256 : 2048, c->S);
    k_currents<<<g, 256, 0, st>>>(c->n_seg, c->n_nodes, d.seg_a, d.seg_b, d.R, d.seg_W, d.seg_H, d.u, d.j);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    EMS_CUDA(c, cudaMemsetAsync(d.drop, 0, sizeof(double) * c->S, st));
    dim3 gd((c->n_nodes + 255) / 256 < 256 ? (c->n_nodes + 255) / 256 : 256, c->S);
    k_drop<<<gd, 256, 0, st>>>(c->n_nodes, c->prm.Vdd, d.u, (unsigned long long *)d.drop);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status check_status(ems_ctx *c) {
    int32_t h[8];
    EMS_CUDA(c, cudaMemcpyAsync(h, c->d.status, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h[kStatusTimeout] || h[kStatusNoConv] || h[kStatusOverflow])
        EMS_CUDA(c, cudaMemsetAsync(c->d.status, 0, sizeof h, c->stream));
    if (h[kStatusTimeout]) return fail(c, EMS_E_TIMEOUT, "device wait ran out its iteration limit");
    if (h[kStatusNoConv]) return fail(c, EMS_E_NOCONV, "IR PCG did not converge within ir_max_iter");
    if (h[kStatusOverflow]) return fail(c, EMS_E_OVERFLOW, "more voids in a tree than max_voids_per_tree");
    return EMS_OK;
}

}  // namespace ems

extern "C" ems_status ems_ir_solve(ems_ctx *c, double *u_out, double *max_drop_frac) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return ems::fail(c, EMS_E_STATE, "no grid loaded");
    EMS_TRY(ems::each_window(c, [&](int, int) -> ems_status {
        if (ems::windowed(c)) EMS_TRY(ems::gather_x(c));
        EMS_TRY(ems::ir_assemble_and_solve(c, true));
        return ems::ir_currents_and_drop(c);
    }));
    if (u_out)
        EMS_CUDA(c, cudaMemcpyAsync(u_out, c->d.u, sizeof(double) * c->S * c->n_nodes,
                                    cudaMemcpyDeviceToHost, c->stream));
    if (max_drop_frac)
        EMS_CUDA(c, cudaMemcpyAsync(max_drop_frac, c->d.drop, sizeof(double) * c->S,
                                    cudaMemcpyDeviceToHost, c->stream));
    return ems::check_status(c);
}

extern "C" ems_status ems_ir_iterations(ems_ctx *c, int32_t *iters) {
    if (!c || !iters) return EMS_E_INVAL;
    if (!c->loaded) return ems::fail(c, EMS_E_STATE, "no grid loaded");
    EMS_CUDA(c, cudaMemcpyAsync(iters, c->d.ir_iters, sizeof(int32_t) * c->S, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}
