// ems_krylov_kernels.cuh -- device side of the rational Krylov reduced
// models (Sec. IV-E, Alg. 1); included by ems_krylov.cu (host driver) and
// by one small translation unit per chunk length (ems_krylov_m*.cu) that
// instantiates the kernel, so that the instantiations compile in parallel.
#pragma once
#include <climits>
#include <cmath>

#include "ems_device.cuh"
#include "ems_internal.cuh"


namespace ems {
ems_status check_status(ems_ctx *c);
ems_status launch_be(ems_ctx *c, double dt, int n_steps);

template <typename R>
struct KrArgs {
    const int32_t *trees;
    const int64_t *toff, *pbase;
    int64_t N, P;
    int n_trees, rmax, q, kc;
    double eta, eps_rel;
    const double *Vn, *g, *leak, *f, *kap_a, *dx, *area;   // Vn: node volumes (diagonal of C)
    double *thr;
    R *sig;
    double *sp, *sg, *su, *sPf, *sPb;       // [S][P] factors of C - t_s A
    R *Vb;                                  // [S][rmax][P] basis columns
    double *Ah, *Ch, *Lm, *Xs;              // [S nt][rmax^2] projections; Cholesky and solve scratch
    double *s0;
    int32_t *kr_r, *kr_state, *kr_mode, *kdone;
    double dt, t0, Binv;
    const double *t0p;                      // device start time of the aging step (graph replay), or null
    int n_steps, build_only;
    int32_t *v_count, *v_node, *v_seg;
    double *v_vol, *v_tnuc;
    int maxv;
    int32_t *dirty;
    const double *j;
    int n_seg;
    const int32_t *inc_ptr, *inc_seg;
    int32_t *status, *counters;
    unsigned long long *work;
};

// one launch of the reduced-model kernel for the chains of bucket b
// (defined per chunk length M in ems_krylov_m<M>.cu)
template <int M, typename R>
ems_status kr_launch(ems_ctx *c, const Bucket &b, KrArgs<R> &a);
template <> ems_status kr_launch<4, float>(ems_ctx *c, const Bucket &b, KrArgs<float> &a);
template <> ems_status kr_launch<4, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a);
template <> ems_status kr_launch<8, float>(ems_ctx *c, const Bucket &b, KrArgs<float> &a);
template <> ems_status kr_launch<8, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a);
template <> ems_status kr_launch<16, float>(ems_ctx *c, const Bucket &b, KrArgs<float> &a);
template <> ems_status kr_launch<16, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a);
template <> ems_status kr_launch<32, float>(ems_ctx *c, const Bucket &b, KrArgs<float> &a);
template <> ems_status kr_launch<32, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a);
template <> ems_status kr_launch<64, float>(ems_ctx *c, const Bucket &b, KrArgs<float> &a);
template <> ems_status kr_launch<64, double>(ems_ctx *c, const Bucket &b, KrArgs<double> &a);

namespace {

constexpr int kStatusOverflow = 2;
constexpr double kPi = 3.141592653589793;
constexpr int kRm = 96;                     // >= 2 q + 2 for q <= 40

template <typename R>
__host__ __device__ constexpr int kr_max_threads(int M) {
    return sizeof(R) == 4 ? (M <= 8 ? 1024 : M <= 32 ? 640 : 320)
                          : (M <= 4 ? 1024 : M == 8 ? 896 : M == 16 ? 640 : M == 32 ? 384 : 256);
}


// per-CTA constants of the (tree, sample)
struct Tr {
    int t, s, T, c, n;
    int64_t st, cb, cs, ps, P;
};

struct Sh {                                 // static shared scratch
    double *red, *out, *sA, *sB, *sL, *sR, *h, *h2;
    int *phase;                             // per-thread reduction buffer parity (local)
};

// block sums of K values, fixed order; every thread gets the sums in x.
// Per-thread values and the warp tree are in precision R, the sum over the
// warps in FP64 (FP64 shuffles cost 64x the FP32 ones on this part).  One
// barrier: every warp reads all warps' partials and adds them itself (lane
// q < K sums value q), alternating between two halves of `red` so that the
// next call cannot overwrite partials a slower warp still reads.
template <int K, typename R>
__device__ __forceinline__ void bsum(const R (&xin)[K], double (&x)[K], double *red, int &phase) {
    static_assert(K <= 16, "at most 16 values per reduction");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double *buf = red + (phase & 1) * (16 * 32);
    ++phase;
    R v[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        v[q] = xin[q];
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) buf[q * 32 + w] = (double)v[q];
    __syncthreads();
    double t = 0.0;
    if (lane < K)
        for (int k = 0; k < nw; ++k) t += buf[lane * 32 + k];
#pragma unroll
    for (int q = 0; q < K; ++q) x[q] = __shfl_sync(0xffffffffu, t, q);
}

// h[i] = column_i . x for i < m: per-thread partial sums in R over the
// thread's M nodes, FP64 across threads
template <int M, typename R>
__device__ void dots(const R *base, const Tr &z, int m, const R (&x)[M], double *h, const Sh &sh) {
    for (int g0 = 0; g0 < m; g0 += 16) {
        R p[16];
        double acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            p[q] = R(0);
            if (g0 + q < m) {
                const R *col = base + (int64_t)(g0 + q) * z.P + z.c;
#pragma unroll
                for (int k = 0; k < M; ++k) p[q] = fmx(col[(int64_t)k * z.T], x[k], p[q]);
            }
        }
        bsum<16, R>(p, acc, sh.red, *sh.phase);
        if (threadIdx.x == 0)
            for (int q = 0; q < 16 && g0 + q < m; ++q) h[g0 + q] = acc[q];
    }
    __syncthreads();                        // h complete for every thread
}

// h[i] = column_i . y1 and h2[i] = column_i . y2 for i < m, one reduction for both
template <int M, typename R>
__device__ void dots2(const R *base, const Tr &z, int m, const R (&y1)[M], const R (&y2)[M], double *h,
                      double *h2, const Sh &sh) {
    for (int g0 = 0; g0 < m; g0 += 8) {
        R p[16];
        double acc[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            p[q] = R(0);
            p[8 + q] = R(0);
            if (g0 + q < m) {
                const R *col = base + (int64_t)(g0 + q) * z.P + z.c;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const R v = col[(int64_t)k * z.T];
                    p[q] = fmx(v, y1[k], p[q]);
                    p[8 + q] = fmx(v, y2[k], p[8 + q]);
                }
            }
        }
        bsum<16, R>(p, acc, sh.red, *sh.phase);
        if (threadIdx.x == 0)
            for (int q = 0; q < 8 && g0 + q < m; ++q) { h[g0 + q] = acc[q]; h2[g0 + q] = acc[8 + q]; }
    }
    __syncthreads();
}

// x -= sum_i h_i column_i, twice (classical Gram-Schmidt with reorthogonalisation)
template <int M, typename R>
__device__ void orth(const R *base, const Tr &z, int m, R (&x)[M], const Sh &sh) {
    for (int pass = 0; pass < 2; ++pass) {
        dots<M, R>(base, z, m, x, sh.h, sh);
        for (int i = 0; i < m; ++i) {
            const R hi = (R)sh.h[i];
            const R *col = base + (int64_t)i * z.P + z.c;
#pragma unroll
            for (int k = 0; k < M; ++k) x[k] = fmx(-hi, col[(int64_t)k * z.T], x[k]);
        }
    }
}

template <int M, typename R>
__device__ __forceinline__ double norm2(const R (&x)[M], const Sh &sh) {
    R p[1] = {R(0)};
#pragma unroll
    for (int k = 0; k < M; ++k) p[0] = fmx(x[k], x[k], p[0]);
    double v[1];
    bsum<1, R>(p, v, sh.red, *sh.phase);
    return v[0];
}

// x <- (C - t_s A)^-1 x with the shifted factors (chunk scans, FP64)
template <int M, typename R>
__device__ void ksolve(const KrArgs<R> &a, const Tr &z, double (&x)[M], const Sh &sh) {
    const int T = z.T, c = z.c;
    const int64_t ps = z.ps;
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int64_t pk = ps + (int64_t)k * T + c;
        v = fma(-a.sg[pk], v, a.sp[pk] * x[k]);
        x[k] = v;
    }
    const double cf = scan_fwd<double>(v, a.sPf[ps + (int64_t)(M - 1) * T + c], sh.sA, sh.sB, nullptr);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = fma(a.sPf[ps + (int64_t)k * T + c], cf, x[k]);
    double y = 0.0;
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        y = fma(-a.su[ps + (int64_t)k * T + c], y, x[k]);
        x[k] = y;
    }
    const double cr = scan_bwd<double>(y, a.sPb[ps + c], sh.sA, sh.sB, nullptr);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = fma(a.sPb[ps + (int64_t)k * T + c], cr, x[k]);
}

// y = A x on the chain (face fluxes plus the Robin leak at voids)
template <int M, typename R>
__device__ void amul(const KrArgs<R> &a, const Tr &z, const R (&x)[M], R (&y)[M], const Sh &sh) {
    const unsigned full = 0xffffffffu;
    const int c = z.c, lane = c & 31, w = c >> 5, nw = z.T >> 5;
    R left = __shfl_up_sync(full, x[M - 1], 1);
    R right = __shfl_down_sync(full, x[0], 1);
    __syncthreads();                        // earlier readers of the halo slots are done
    if (nw > 1) {
        if (lane == 31) sh.sL[w] = (double)x[M - 1];
        if (lane == 0) sh.sR[w] = (double)x[0];
        __syncthreads();
        if (lane == 0 && w > 0) left = (R)sh.sL[w - 1];
        if (lane == 31 && w + 1 < nw) right = (R)sh.sR[w + 1];
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        R v = R(0);
        if (i < z.n) {
            const R xl = k > 0 ? x[k - 1] : left, xr = k + 1 < M ? x[k + 1] : right;
            if (i > 0) v = fmx((R)a.g[z.cs + i], xl - x[k], v);
            if (i + 1 < z.n) v = fmx((R)a.g[z.cs + i + 1], xr - x[k], v);
            if (isinf(a.thr[z.cs + i])) v = fmx(-(R)a.leak[z.cs + i], x[k], v);
        }
        y[k] = v;
    }
}

template <int M, typename R>
__device__ __forceinline__ void store_col(R *Vs, const Tr &z, int slot, const R (&x)[M], R scale) {
#pragma unroll
    for (int k = 0; k < M; ++k) Vs[(int64_t)slot * z.P + (int64_t)k * z.T + z.c] = x[k] * scale;
}

template <int M, typename R>
__device__ __forceinline__ void load_col(const R *Vs, const Tr &z, int slot, R (&x)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = Vs[(int64_t)slot * z.P + (int64_t)k * z.T + z.c];
}

// rows/columns jc in [j0, j1) of A_h and C_h against columns 0..jc (symmetric)
template <int M, typename R>
__device__ void project(const KrArgs<R> &a, const Tr &z, const R *Vs, int j0, int j1, double *Ahs, double *Chs,
                        const Sh &sh) {
    const int rm = a.rmax;
    R x[M], y[M], yc[M];
    for (int jc = j0; jc < j1; ++jc) {
        load_col<M, R>(Vs, z, jc, x);
        amul<M, R>(a, z, x, y, sh);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = z.c * M + k;
            yc[k] = i < z.n ? (R)a.Vn[z.cb + i] * x[k] : R(0);
        }
        dots2<M, R>(Vs, z, jc + 1, y, yc, sh.h, sh.h2, sh);
        for (int i = z.c; i <= jc; i += z.T) {
            Ahs[(int64_t)i * rm + jc] = Ahs[(int64_t)jc * rm + i] = sh.h[i];
            Chs[(int64_t)i * rm + jc] = Chs[(int64_t)jc * rm + i] = sh.h2[i];
        }
        __syncthreads();                    // h, h2 are rewritten by the next column
    }
}

// 2x2 matrices [[a, b], [c, d]] for the continuant scan, rescaled by powers
// of two (exact) to stay in range; only ratios of the continuants matter
struct M2 {
    double a, b, c, d;
};
__device__ __forceinline__ M2 m2mul(const M2 &x, const M2 &y) {
    return M2{fma(x.a, y.a, x.b * y.c), fma(x.a, y.b, x.b * y.d), fma(x.c, y.a, x.d * y.c),
              fma(x.c, y.b, x.d * y.d)};
}
__device__ __forceinline__ M2 m2norm(M2 x) {
    const double mx = fmax(fmax(fabs(x.a), fabs(x.b)), fmax(fabs(x.c), fabs(x.d)));
    if (mx > 0.0 && isfinite(mx)) {
        const int e = ilogb(mx);
        x.a = scalbn(x.a, -e); x.b = scalbn(x.b, -e); x.c = scalbn(x.c, -e); x.d = scalbn(x.d, -e);
    }
    return x;
}
__device__ __forceinline__ M2 m2shfl_up(const M2 &x, int d) {
    const unsigned full = 0xffffffffu;
    return M2{__shfl_up_sync(full, x.a, d), __shfl_up_sync(full, x.b, d), __shfl_up_sync(full, x.c, d),
              __shfl_up_sync(full, x.d, d)};
}

template <int M, typename R>
__device__ void factor_shift(const KrArgs<R> &a, const Tr &z, double ts, const Sh &sh) {
    const int T = z.T, c = z.c, n = z.n, lane = c & 31, w = c >> 5, nw = T >> 5;
    const M2 I{1.0, 0.0, 0.0, 1.0};
    M2 P = I;                                        // A_last ... A_first of this chunk
#pragma unroll 1
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= n) break;
        const double gl = i > 0 ? a.g[z.cs + i] : 0.0, gr = i + 1 < n ? a.g[z.cs + i + 1] : 0.0;
        double d = a.Vn[z.cb + i] + ts * (gl + gr);
        if (isinf(a.thr[z.cs + i])) d += ts * a.leak[z.cs + i];
        const double e2 = (ts * gl) * (ts * gl);
        P = m2norm(m2mul(M2{d, -e2, 1.0, 0.0}, P));
    }
    // inclusive scan over the warp (later chunks multiply from the left)
    M2 v = P;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const M2 o = m2shfl_up(v, dd);
        if (lane >= dd) v = m2norm(m2mul(v, o));
    }
    M2 pw = I;                                       // product of all earlier warps
    double *agg = sh.red;                            // 4 x 32 doubles
    if (nw > 1) {
        __syncthreads();
        if (lane == 31) { agg[w] = v.a; agg[32 + w] = v.b; agg[64 + w] = v.c; agg[96 + w] = v.d; }
        __syncthreads();
        M2 u = lane < w ? M2{agg[lane], agg[32 + lane], agg[64 + lane], agg[96 + lane]} : I;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const M2 o = m2shfl_up(u, dd);
            if (lane >= dd) u = m2norm(m2mul(u, o));
        }
        pw = M2{__shfl_sync(0xffffffffu, u.a, 31), __shfl_sync(0xffffffffu, u.b, 31),
                __shfl_sync(0xffffffffu, u.c, 31), __shfl_sync(0xffffffffu, u.d, 31)};
    }
    M2 ex = m2shfl_up(v, 1);
    if (lane == 0) ex = I;
    const M2 E = m2norm(m2mul(ex, pw));
    double qp = E.a, qpp = E.c;                      // (q_(i-1), q_(i-2)) from (q_-1, q_-2) = (1, 0)
#pragma unroll 1
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= n) break;
        const double gl = i > 0 ? a.g[z.cs + i] : 0.0, gr = i + 1 < n ? a.g[z.cs + i + 1] : 0.0;
        double d = a.Vn[z.cb + i] + ts * (gl + gr);
        if (isinf(a.thr[z.cs + i])) d += ts * a.leak[z.cs + i];
        const double em = -ts * gl, ep = -ts * gr;
        const double q = fma(d, qp, -(em * em) * qpp);
        const double p = qp / q;
        const int64_t pk = z.ps + (int64_t)k * T + c;
        a.sp[pk] = p; a.sg[pk] = p * em; a.su[pk] = p * ep;
        const int e = ilogb(fabs(q));
        qpp = scalbn(qp, -e);
        qp = scalbn(q, -e);
    }
    __syncthreads();
}

// Alg. 1 from the current stress and forcing: returns the base rank (> 0),
// 0 when there is nothing to reduce, -1 on rank deficiency
template <int M, typename R>
__device__ int build(const KrArgs<R> &a, const Tr &z, R *Vs, double *Ahs, double *Chs, const Sh &sh,
                     double &ts_out) {
    const int T = z.T, c = z.c, n = z.n;
    // shift time t_s = eta L^2 / (pi^2 kappa_bar), L the chain length
    double x3[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= 1 && i < n) {
            const double d = a.dx[z.cb + i];
            x3[0] += a.kap_a[z.cs + i] * d;
            x3[1] += a.area[z.cb + i] * d;
            x3[2] += d;
        }
    }
    bsum<3, double>(x3, x3, sh.red, *sh.phase);
    const double ts = a.eta * x3[2] * x3[2] / (kPi * kPi * (x3[0] / x3[1]));
    ts_out = ts;
    // factor C - t_s A = L D L^T: pivots p_i = 1/(d_i - e_i^2 p_(i-1)) from
    // the continuants q_i = d_i q_(i-1) - e_i^2 q_(i-2) (p_i = q_(i-1)/q_i),
    // a prefix product of 2x2 matrices across the chunks, then each chunk's
    // pivots in order from its carried (q_(i-1), q_(i-2))
    if (c == 0) a.s0[z.st] = 1.0 / ts;
    factor_shift<M, R>(a, z, ts, sh);
    {
        double acc = 1.0;
        for (int k = 0; k < M; ++k) {
            const int64_t pk = z.ps + (int64_t)k * T + c;
            acc *= -a.sg[pk];
            a.sPf[pk] = acc;
        }
        acc = 1.0;
        for (int k = M - 1; k >= 0; --k) {
            const int64_t pk = z.ps + (int64_t)k * T + c;
            acc *= -a.su[pk];
            a.sPb[pk] = acc;
        }
    }
    __syncthreads();

    // starting block F0 = [R C s, R f] (raw columns in slots 0, 1)
    double xd[M], n0[2];
    R x[M];
    for (int col = 0; col < 2; ++col) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = c * M + k;
            xd[k] = i < n ? (col == 0 ? a.Vn[z.cb + i] * (double)a.sig[z.ps + (int64_t)k * T + c] : a.f[z.cs + i])
                          : 0.0;
        }
        ksolve<M, R>(a, z, xd, sh);
#pragma unroll
        for (int k = 0; k < M; ++k) { xd[k] *= ts; x[k] = (R)xd[k]; }
        n0[col] = sqrt(norm2<M, R>(x, sh));
        store_col<M, R>(Vs, z, col, x, R(1));
    }
    const double eps0 = a.eps_rel * fmax(n0[0], n0[1]);
    int m = 0;
    for (int col = 0; col < 2; ++col) {
        if (!(n0[col] > 0.0)) continue;
        load_col<M, R>(Vs, z, col, x);
        __syncthreads();
        orth<M, R>(Vs, z, m, x, sh);
        const double nw = sqrt(norm2<M, R>(x, sh));
        if (nw >= a.eps_rel * n0[col] && nw >= eps0) {
            store_col<M, R>(Vs, z, m, x, (R)(1.0 / nw));
            ++m;
        }
        __syncthreads();
    }
    if (m == 0) return 0;
    const int rq = 2 * a.q;
    int pb0 = 0, pb1 = m;
    for (int blk = 1; blk < a.q && m + (pb1 - pb0) <= rq; ++blk) {
        const int nb = pb1 - pb0;
        double w2 = 0.0;
        for (int q = 0; q < nb; ++q) {             // raw W = R C V_j into slots m + q
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = c * M + k;
                xd[k] = i < n ? a.Vn[z.cb + i] * (double)Vs[(int64_t)(pb0 + q) * z.P + (int64_t)k * T + c] : 0.0;
            }
            ksolve<M, R>(a, z, xd, sh);
#pragma unroll
            for (int k = 0; k < M; ++k) { xd[k] *= ts; x[k] = (R)xd[k]; }
            w2 += norm2<M, R>(x, sh);
            store_col<M, R>(Vs, z, m + q, x, R(1));
        }
        const double epsj = a.eps_rel * sqrt(w2);
        int acc = 0;
        bool deficient = false;
        for (int q = 0; q < nb; ++q) {
            load_col<M, R>(Vs, z, m + q, x);
            __syncthreads();
            orth<M, R>(Vs, z, m + acc, x, sh);
            const double nw = sqrt(norm2<M, R>(x, sh));
            if (nw < epsj) {
                deficient = true;
            } else {
                store_col<M, R>(Vs, z, m + acc, x, (R)(1.0 / nw));
                ++acc;
            }
            __syncthreads();
        }
        if (acc == 0) break;                       // the space is invariant: done
        if (deficient) return -1;                  // rank deficiency: full BE
        pb0 = m; pb1 = m + acc; m += acc;
    }
    project<M, R>(a, z, Vs, 0, m, Ahs, Chs, sh);
    return m;
}

// the cached basis plus the current starting block [R C s, R f]; returns the
// total number of columns
template <int M, typename R>
__device__ int augment(const KrArgs<R> &a, const Tr &z, R *Vs, int rb, double *Ahs, double *Chs, const Sh &sh) {
    const int T = z.T, c = z.c, n = z.n;
    const double ts = 1.0 / a.s0[z.st];
    int m = rb;
    double xd[M];
    R x[M];
    for (int col = 0; col < 2; ++col) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = c * M + k;
            xd[k] = i < n ? (col == 0 ? a.Vn[z.cb + i] * (double)a.sig[z.ps + (int64_t)k * T + c] : a.f[z.cs + i])
                          : 0.0;
        }
        ksolve<M, R>(a, z, xd, sh);
#pragma unroll
        for (int k = 0; k < M; ++k) { xd[k] *= ts; x[k] = (R)xd[k]; }
        const double nx = sqrt(norm2<M, R>(x, sh));
        if (!(nx > 0.0)) continue;
        orth<M, R>(Vs, z, m, x, sh);
        const double nw = sqrt(norm2<M, R>(x, sh));
        if (nw >= a.eps_rel * nx) {
            store_col<M, R>(Vs, z, m, x, (R)(1.0 / nw));
            ++m;
        }
        __syncthreads();
    }
    project<M, R>(a, z, Vs, rb, m, Ahs, Chs, sh);
    return m;
}

// lifted stress of node slot `off` from reduced coordinates y (row of the table)
template <typename R>
__device__ __forceinline__ R lift(const R *Vs, int64_t P, int64_t off, int m, const R *y) {
    R v = R(0);
    for (int l = 0; l < m; ++l) v = fmx(Vs[(int64_t)l * P + off], y[l], v);
    return v;
}

template <int M, typename R>
__global__ void __launch_bounds__(kr_max_threads<R>(M)) k_kr_step(KrArgs<R> a) {
    extern __shared__ __align__(16) unsigned char kr_dsm[];
    __shared__ double red[2 * 16 * 32], out[16], sA[64], sB[64], sL[32], sR[32], sv[32];
    __shared__ double h[kRm], h2[kRm], fh[kRm], sd[kRm], ssum[kRm], bv[kRm];
    __shared__ R hi[kRm], lo[kRm], dl[2][kRm];
    __shared__ int si[32];
    __shared__ int s_fail;
    __shared__ double s_m0;
    int phase = 0;
    const Sh sh{red, out, sA, sB, sL, sR, h, h2, &phase};
    const int rm = a.rmax;
    R *Ft = (R *)kr_dsm;                               // [rm][rm]: Ft[j*rm + l] = F_lj
    R *tab = Ft + (size_t)rm * rm;                     // [(kc+1)][rm]: chunk trajectory

    Tr z;
    z.t = a.trees[blockIdx.x]; z.s = blockIdx.y; z.T = blockDim.x; z.c = threadIdx.x;
    z.st = (int64_t)z.s * a.n_trees + z.t;
    if (!a.kr_mode[z.st]) return;
    z.cb = a.toff[z.t];
    z.n = (int)(a.toff[z.t + 1] - z.cb);
    z.cs = (int64_t)z.s * a.N + z.cb;
    z.ps = (int64_t)z.s * a.P + a.pbase[z.t];
    z.P = a.P;
    const int T = z.T, c = z.c, n = z.n;
    R *Vs = a.Vb + (int64_t)z.s * rm * a.P + a.pbase[z.t];
    double *Ahs = a.Ah + z.st * rm * rm, *Chs = a.Ch + z.st * rm * rm;
    double *Lms = a.Lm + z.st * rm * rm, *Xs = a.Xs + z.st * rm * (rm + 1);
    const int K = a.n_steps;
    const double dt = a.dt;
    int k = a.kdone[z.st];
    int rb = a.kr_r[z.st];
    bool fresh = false;
    double ts_unused;
    auto fallback = [&](int kd) {
        if (c == 0) { a.kr_state[z.st] = 2; a.kr_mode[z.st] = 0; a.kdone[z.st] = kd; }
    };
    if (a.kr_state[z.st] != 1) {
        rb = build<M, R>(a, z, Vs, Ahs, Chs, sh, ts_unused);
        if (rb <= 0) { fallback(k); return; }
        if (c == 0) { a.kr_r[z.st] = rb; a.kr_state[z.st] = 1; }
        fresh = true;
    }
    if (a.build_only) return;
    const int64_t k_begin = k;
    R x[M];
    while (k < K) {
        const int m = fresh ? rb : augment<M, R>(a, z, Vs, rb, Ahs, Chs, sh);
        fresh = false;
        // reduced forcing f_h = V^T f and initial condition s_hat(0) = V^T s
#pragma unroll
        for (int kk = 0; kk < M; ++kk) {
            const int i = c * M + kk;
            x[kk] = i < n ? (R)a.f[z.cs + i] : R(0);
        }
        dots<M, R>(Vs, z, m, x, fh, sh);
#pragma unroll
        for (int kk = 0; kk < M; ++kk) x[kk] = a.sig[z.ps + (int64_t)kk * T + c];
        dots<M, R>(Vs, z, m, x, sd, sh);
        // M = C_h - dt A_h, lower triangle, then Cholesky by warp 0
        for (int idx = c; idx < m * m; idx += T) {
            const int i = idx / m, jx = idx % m;
            if (jx <= i) Lms[(int64_t)i * rm + jx] = Chs[(int64_t)i * rm + jx] - dt * Ahs[(int64_t)i * rm + jx];
        }
        // right-hand side of the first increment: dt (A_h s_hat(0) + f_h)
        for (int i = c; i < m; i += T) {
            double v = fh[i];
            for (int jx = 0; jx < m; ++jx) v = fma(Ahs[(int64_t)i * rm + jx], sd[jx], v);
            bv[i] = dt * v;
        }
        if (c == 0) s_fail = 0;
        __syncthreads();
        if (c < 32) {
            const int lane = c;
            for (int jx = 0; jx < m; ++jx) {
                double d = Lms[(int64_t)jx * rm + jx];
                __syncwarp();
                if (!(d > 0.0)) { if (lane == 0) s_fail = 1; d = 1.0; }
                d = sqrt(d);
                if (lane == 0) Lms[(int64_t)jx * rm + jx] = d;
                for (int i = jx + 1 + lane; i < m; i += 32) Lms[(int64_t)i * rm + jx] /= d;
                __syncwarp();
                for (int i = jx + 1 + lane; i < m; i += 32) {
                    const double lij = Lms[(int64_t)i * rm + jx];
                    for (int q2 = jx + 1; q2 <= i; ++q2) Lms[(int64_t)i * rm + q2] -= lij * Lms[(int64_t)q2 * rm + jx];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_fail) { fallback(k); return; }
        // F = M^-1 C_h (column jx by thread jx) and the first increment (thread m)
        for (int jx = c; jx <= m; jx += T) {
            double *xs = Xs + (int64_t)jx * rm;
            for (int i = 0; i < m; ++i) {
                double v = jx < m ? Chs[(int64_t)i * rm + jx] : bv[i];
                for (int q2 = 0; q2 < i; ++q2) v -= Lms[(int64_t)i * rm + q2] * xs[q2];
                xs[i] = v / Lms[(int64_t)i * rm + i];
            }
            for (int i = m - 1; i >= 0; --i) {
                double v = xs[i];
                for (int q2 = i + 1; q2 < m; ++q2) v -= Lms[(int64_t)q2 * rm + i] * xs[q2];
                xs[i] = v / Lms[(int64_t)i * rm + i];
            }
            if (jx < m)
                for (int i = 0; i < m; ++i) Ft[(size_t)jx * rm + i] = (R)xs[i];
            else
                for (int i = 0; i < m; ++i) dl[0][i] = (R)xs[i];
        }
        for (int l = c; l < m; l += T) tab[l] = (R)sd[l];
        __syncthreads();

        // chunks of the reduced trajectory
        int kseg = 0, cur = 0;
        bool nucleated = false;
        while (k + kseg < K) {
            const int kc = min(a.kc, K - k - kseg);
            for (int l = c; l < m; l += T) { hi[l] = (R)(-INFINITY); lo[l] = (R)INFINITY; }
            __syncthreads();
            if (c < 32) {                             // one warp steps the reduced system
                for (int kk = 1; kk <= kc; ++kk) {
                    for (int l = c; l < m; l += 32) {
                        const R d = dl[cur][l];
                        sd[l] += (double)d;
                        const R sv2 = (R)sd[l];
                        tab[(size_t)kk * rm + l] = sv2;
                        hi[l] = max(hi[l], sv2);
                        lo[l] = min(lo[l], sv2);
                        R acc = R(0);
                        for (int jx = 0; jx < m; ++jx) acc = fmx(Ft[(size_t)jx * rm + l], dl[cur][jx], acc);
                        dl[cur ^ 1][l] = acc;
                    }
                    cur ^= 1;
                    __syncwarp();
                }
            } else {
                cur ^= kc & 1;
            }
            __syncthreads();
            // candidates: nodes whose bound over the chunk reaches their
            // threshold; each is lifted step by step to its first crossing
            const R slack = sizeof(R) == 4 ? R(1e-5) : R(1e-12);
            unsigned long long cand = 0ull;
            int kf = INT_MAX;
#pragma unroll 1
            for (int kk = 0; kk < M; ++kk) {
                const int i = c * M + kk;
                if (i >= n) continue;
                const double th = a.thr[z.cs + i];
                if (isinf(th)) continue;
                const int64_t off = (int64_t)kk * T + c;
                R U = R(0), Aa = R(0);
                for (int l = 0; l < m; ++l) {
                    const R v = Vs[(int64_t)l * a.P + off];
                    U += max(v * hi[l], v * lo[l]);
                    Aa = fmx(fabs(v), max(fabs(hi[l]), fabs(lo[l])), Aa);
                }
                if ((double)(U + slack * Aa) < th) continue;
                cand |= 1ull << kk;
                for (int s2 = 1; s2 <= kc && s2 < kf; ++s2)
                    if ((double)lift<R>(Vs, a.P, off, m, tab + (size_t)s2 * rm) >= th) { kf = s2; break; }
            }
            const double kfm = block_min((double)kf, sv);
            const int kstar = kfm < (double)INT_MAX ? (int)kfm : INT_MAX;
            int kend = kc;
            double best = -INFINITY;
            int arg = 0x7fffffff;
            if (kstar != INT_MAX) {
                kend = kstar;
                for (int kk = 0; kk < M; ++kk) {
                    if (!((cand >> kk) & 1ull)) continue;
                    const int i = c * M + kk;
                    const double mg =
                        (double)lift<R>(Vs, a.P, (int64_t)kk * T + c, m, tab + (size_t)kstar * rm) - a.thr[z.cs + i];
                    if (mg > best) { best = mg; arg = i; }
                }
                block_argmax(best, arg, sv, si);
                nucleated = best >= 0.0;
                if (nucleated && arg / M == c) {    // stress of the new void one step earlier
                    const int64_t off = (int64_t)(arg % M) * T + c;
                    const double prev = (kseg == 0 && kstar == 1)
                                            ? (double)a.sig[z.ps + off]
                                            : (double)lift<R>(Vs, a.P, off, m, tab + (size_t)(kstar - 1) * rm);
                    s_m0 = prev - a.thr[z.cs + arg];
                }
            }
            // void growth over steps 1..kend of the chunk (existing voids)
            for (int l = c; l < m; l += T) {
                double sacc = 0.0;
                for (int s2 = 1; s2 <= kend; ++s2) sacc += (double)tab[(size_t)s2 * rm + l];
                ssum[l] = sacc;
            }
            __syncthreads();
            const int nv = a.v_count[z.st];
            for (int qv = 0; qv < nv; ++qv) {
                const int v = a.v_node[z.st * a.maxv + qv];
                if (v / M != c) continue;
                const int64_t off = (int64_t)(v % M) * T + c;
                double sacc = 0.0;
                for (int l = 0; l < m; ++l) sacc = fma((double)Vs[(int64_t)l * a.P + off], ssum[l], sacc);
                a.v_vol[z.st * a.maxv + qv] += dt * a.Binv * a.leak[z.cs + v] * sacc;
            }
            const bool last = nucleated || (k + kseg + kend == K);
            if (last) {                               // lift at kend
                const R *y = tab + (size_t)kend * rm;
#pragma unroll 1
                for (int kk = 0; kk < M; ++kk) {
                    const int i = c * M + kk;
                    const int64_t off = (int64_t)kk * T + c;
                    if (i < n) a.sig[z.ps + off] = lift<R>(Vs, a.P, off, m, y);
                }
            }
            __syncthreads();
            if (nucleated && c == 0) {
                const int v = arg;
                const double m0 = s_m0, m1 = best;
                const double frac = m0 < 0.0 ? -m0 / (m1 - m0) : 0.0;
                const int nvv = a.v_count[z.st];
                if (nvv < a.maxv) {
                    const int64_t e = z.st * a.maxv + nvv;
                    int best_s = a.inc_seg[a.inc_ptr[z.cb + v]];
                    double bj = fabs(a.j[(int64_t)z.s * a.n_seg + best_s]);
                    for (int kx = a.inc_ptr[z.cb + v] + 1; kx < a.inc_ptr[z.cb + v + 1]; ++kx) {
                        const double aj = fabs(a.j[(int64_t)z.s * a.n_seg + a.inc_seg[kx]]);
                        if (aj > bj) { bj = aj; best_s = a.inc_seg[kx]; }
                    }
                    a.v_node[e] = v; a.v_seg[e] = best_s; a.v_vol[e] = 0.0;
                    a.v_tnuc[e] = (a.t0p ? *a.t0p : a.t0) + ((double)(k + kseg + kstar - 1) + frac) * dt;
                    a.v_count[z.st] = nvv + 1;
                    atomicAdd(&a.counters[0], 1);
                } else {
                    atomicOr(&a.status[kStatusOverflow], 1);
                }
                a.thr[z.cs + v] = INFINITY;
                a.dirty[z.st] = 1;                  // BE factors are stale too
            }
            kseg += kend;
            if (nucleated) break;
            // next chunk starts from the last row
            for (int l = c; l < m; l += T) tab[l] = tab[(size_t)kend * rm + l];
            __syncthreads();
        }
        k += kseg;
        __syncthreads();
        if (!nucleated) break;
        // the void changed A: rebuild from the lifted stress and carry on
        rb = build<M, R>(a, z, Vs, Ahs, Chs, sh, ts_unused);
        if (rb <= 0) {
            if (c == 0) atomicAdd(a.work, (unsigned long long)n * (unsigned long long)(k - k_begin));
            fallback(k);
            return;
        }
        if (c == 0) { a.kr_r[z.st] = rb; a.kr_state[z.st] = 1; atomicAdd(&a.counters[2], 1); }
        fresh = true;
    }
    if (c == 0) {
        a.kdone[z.st] = K;
        atomicAdd(a.work, (unsigned long long)n * (unsigned long long)(K - k_begin));
    }
}

template <typename R>
KrArgs<R> kr_args(ems_ctx *c, double dt, int n_steps, int build_only) {
    Dev &d = c->d;
    KrArgs<R> a;
    a.toff = d.toff; a.pbase = d.pbase; a.N = c->N; a.P = c->P;
    a.n_trees = c->n_trees; a.rmax = c->rmax; a.q = c->kr_q; a.kc = c->kr_kc;
    a.eta = c->kr_eta; a.eps_rel = c->prm.krylov_eps > 0.0 ? c->prm.krylov_eps : 1e-10;
    a.Vn = d.V; a.g = d.g; a.leak = d.leak; a.f = d.f; a.kap_a = d.kap_a; a.dx = d.face_dx; a.area = d.face_area;
    a.thr = d.thr; a.sig = (R *)d.sig;
    a.sp = d.kr_sp; a.sg = d.kr_sg; a.su = d.kr_su; a.sPf = d.kr_sPf; a.sPb = d.kr_sPb;
    a.Vb = (R *)d.kr_V; a.Ah = d.kr_Ah; a.Ch = d.kr_Ch; a.Lm = d.kr_Lm; a.Xs = d.kr_Xs; a.s0 = d.kr_s0;
    a.kr_r = d.kr_r; a.kr_state = d.kr_state; a.kr_mode = d.kr_mode; a.kdone = d.kdone;
    a.dt = dt; a.t0 = c->t; a.Binv = 1.0 / c->prm.B_modulus; a.n_steps = n_steps; a.build_only = build_only;
    a.t0p = c->graph_capturing ? d.gtime : nullptr;
    a.v_count = d.v_count; a.v_node = d.v_node; a.v_seg = d.v_seg; a.v_vol = d.v_vol; a.v_tnuc = d.v_tnuc;
    a.maxv = c->maxv; a.dirty = d.dirty; a.j = d.j; a.n_seg = c->n_seg; a.inc_ptr = d.inc_ptr;
    a.inc_seg = d.inc_seg; a.status = d.status; a.counters = d.counters; a.work = d.work;
    return a;
}

template <int M, typename R>
ems_status launch_kr(ems_ctx *c, const Bucket &b, KrArgs<R> &a) {
    if (b.T > kr_max_threads<R>(M)) return fail(c, EMS_E_STATE, "chunk shape exceeds the Krylov kernel's limit");
    dim3 grid((unsigned)b.trees.size(), c->S);
    const size_t smem = sizeof(R) * ((size_t)c->rmax * c->rmax + (size_t)(c->kr_kc + 1) * c->rmax);
    if (smem > 48 * 1024)
        EMS_CUDA(c, cudaFuncSetAttribute(k_kr_step<M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_kr_step<M, R><<<grid, b.T, smem, c->stream>>>(a);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

}  // namespace
}  // namespace ems
