// ems_krylov.cu -- rational Krylov reduced models of the chain trees
// (Sec. IV-E, Alg. 1, Eq. rak_moment_recurrence .. rak_shift_time).
//
// Build (one CTA per (tree, sample), the chunk layout of the BE kernel):
//   t_s = eta L^2 / (pi^2 kappa_bar); K = C/t_s - A is factored as
//   C - t_s A (the BE matrix with dt = t_s), so K^-1 y = t_s (C - t_s A)^-1 y
//   reuses the chunk-parallel elimination; starting block [K^-1 C s0, K^-1 f];
//   block Arnoldi to order q with classical Gram-Schmidt applied twice (FP64
//   reorthogonalisation); A_h = V^T A V, C_h = V^T C V, f_h = V^T f; then the
//   symmetric-definite pencil A_h y = lambda C_h y (Cholesky + Jacobi) gives
//   the modal basis W = V Y with Y^T C_h Y = I.
// Advance: backward Euler in modal coordinates is exact in closed form,
//   z_j(k) = z*_j + (z_j(0) - z*_j) rho_j^k, rho_j = 1/(1 - dt lambda_j),
//   so the lifted stress at any step costs O(r) per node.  A per-node bound
//   over the whole aging step (each mode term is monotone in k) leaves only
//   candidate nodes to be checked step by step for nucleation; void volumes
//   take the closed-form geometric sums; the state is lifted once at the end.
// Breakdown and rank deficiency send the tree back to full backward Euler.
#include <climits>
#include <cmath>

#include "ems_device.cuh"
#include "ems_internal.cuh"

namespace ems {
ems_status check_status(ems_ctx *c);
ems_status launch_be(ems_ctx *c, double dt, int n_steps);

namespace {

constexpr int kStatusOverflow = 2;
constexpr double kPi = 3.141592653589793;

struct KrArgs {
    const int32_t *trees;
    const int64_t *toff, *pbase;
    int64_t N, P;
    int n_trees, S, rmax, q;
    double eta, eps_rel;
    const double *V, *g, *leak, *f, *kap_a, *dx, *area;
    double *thr;
    void *sig;
    int f32;
    double *sp, *sg, *su, *sPf, *sPb;
    double *Vb, *Wb, *lam, *Y, *Ch, *s0;
    int32_t *kr_r, *kr_state, *kr_mode, *kdone;
    double dt, t0, Binv;
    int n_steps;
    int32_t *v_count, *v_node, *v_seg;
    double *v_vol, *v_tnuc;
    int maxv;
    int32_t *dirty;
    const double *j;
    int n_seg;
    const int32_t *inc_ptr, *inc_seg;
    int32_t *status, *counters;
};

__device__ __forceinline__ double sig_at(const KrArgs &a, int64_t pk) {
    return a.f32 ? (double)((const float *)a.sig)[pk] : ((const double *)a.sig)[pk];
}
__device__ __forceinline__ void sig_set(const KrArgs &a, int64_t pk, double v) {
    if (a.f32) ((float *)a.sig)[pk] = (float)v;
    else ((double *)a.sig)[pk] = v;
}

// block sums of K values, fixed order; every thread gets the sums in x
template <int K>
__device__ __forceinline__ void bsum(double (&x)[K], double *red, double *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q)
        for (int o = 16; o > 0; o >>= 1) x[q] += __shfl_down_sync(0xffffffffu, x[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) red[q * 32 + w] = x[q];
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += red[threadIdx.x * 32 + k];
        out[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < K; ++q) x[q] = out[q];
}

// h[i] = column_i . x for i < m (columns at base + i P, chunk layout)
template <int M>
__device__ void dots(const double *base, int64_t P, int T, int c, int m, const double (&x)[M], double *h,
                     double *red, double *out) {
    for (int g0 = 0; g0 < m; g0 += 8) {
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            acc[q] = 0.0;
            if (g0 + q < m) {
                const double *col = base + (int64_t)(g0 + q) * P + c;
#pragma unroll
                for (int k = 0; k < M; ++k) acc[q] = fma(col[(int64_t)k * T], x[k], acc[q]);
            }
        }
        bsum<8>(acc, red, out);
        if (threadIdx.x == 0)
            for (int q = 0; q < 8 && g0 + q < m; ++q) h[g0 + q] = acc[q];
    }
    __syncthreads();
}

// x -= sum_i h_i column_i, twice (classical Gram-Schmidt with reorthogonalisation)
template <int M>
__device__ void orth(const double *base, int64_t P, int T, int c, int m, double (&x)[M], double *h, double *red,
                     double *out) {
    for (int pass = 0; pass < 2; ++pass) {
        dots<M>(base, P, T, c, m, x, h, red, out);
        for (int i = 0; i < m; ++i) {
            const double hi = h[i];
            const double *col = base + (int64_t)i * P + c;
#pragma unroll
            for (int k = 0; k < M; ++k) x[k] = fma(-hi, col[(int64_t)k * T], x[k]);
        }
    }
}

template <int M>
__device__ __forceinline__ double norm2(const double (&x)[M], double *red, double *out) {
    double v[1] = {0.0};
#pragma unroll
    for (int k = 0; k < M; ++k) v[0] = fma(x[k], x[k], v[0]);
    bsum<1>(v, red, out);
    return v[0];
}

// x <- (C - t_s A)^-1 x with the shifted factors (chunk scans, FP64)
template <int M>
__device__ void ksolve(const KrArgs &a, int64_t ps, int T, int c, double (&x)[M], double *sA, double *sB) {
    double z = 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int64_t pk = ps + (int64_t)k * T + c;
        z = fma(-a.sg[pk], z, a.sp[pk] * x[k]);
        x[k] = z;
    }
    const double cf = scan_fwd<double>(z, a.sPf[ps + (int64_t)(M - 1) * T + c], sA, sB, nullptr);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = fma(a.sPf[ps + (int64_t)k * T + c], cf, x[k]);
    double y = 0.0;
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        y = fma(-a.su[ps + (int64_t)k * T + c], y, x[k]);
        x[k] = y;
    }
    const double cr = scan_bwd<double>(y, a.sPb[ps + c], sA, sB, nullptr);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = fma(a.sPb[ps + (int64_t)k * T + c], cr, x[k]);
}

// y = A x on the chain (face fluxes plus the Robin leak at voids)
template <int M>
__device__ void amul(const KrArgs &a, int n, int64_t cs, int T, int c, const double (&x)[M], double (&y)[M],
                     double *sL, double *sR) {
    const unsigned full = 0xffffffffu;
    const int lane = c & 31, w = c >> 5, nw = T >> 5;
    double left = __shfl_up_sync(full, x[M - 1], 1);
    double right = __shfl_down_sync(full, x[0], 1);
    if (nw > 1) {
        if (lane == 31) sL[w] = x[M - 1];
        if (lane == 0) sR[w] = x[0];
        __syncthreads();
        if (lane == 0 && w > 0) left = sL[w - 1];
        if (lane == 31 && w + 1 < nw) right = sR[w + 1];
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        double v = 0.0;
        if (i < n) {
            const double xl = k > 0 ? x[k - 1] : left, xr = k + 1 < M ? x[k + 1] : right;
            if (i > 0) v += a.g[cs + i] * (xl - x[k]);
            if (i + 1 < n) v += a.g[cs + i + 1] * (xr - x[k]);
            if (isinf(a.thr[cs + i])) v -= a.leak[cs + i] * x[k];
        }
        y[k] = v;
    }
    __syncthreads();
}

template <int M>
__global__ void __launch_bounds__(1024) k_kr_build(KrArgs a) {
    extern __shared__ double dsm[];
    __shared__ double sA[64], sB[64], red[256], out[8], sL[32], sR[32];
    const int t = a.trees[blockIdx.x], s = blockIdx.y, T = blockDim.x, c = threadIdx.x;
    const int64_t st = (int64_t)s * a.n_trees + t;
    if (!a.kr_mode[st] || a.kr_state[st] == 1) return;
    const int64_t cb = a.toff[t];
    const int n = (int)(a.toff[t + 1] - cb);
    const int64_t cs = (int64_t)s * a.N + cb, ps = (int64_t)s * a.P + a.pbase[t];
    const int R = a.rmax;
    const int64_t P = a.P;
    double *Vs = a.Vb + (int64_t)s * R * P + a.pbase[t];
    double *Ws = a.Wb + (int64_t)s * R * P + a.pbase[t];
    double *Chs = dsm, *Ss = dsm + R * R, *Ls = dsm + 2 * R * R, *Qs = dsm + 3 * R * R, *h = dsm + 4 * R * R;
    double *fh = h + R;
    __shared__ int s_fail;

    // shift time t_s = eta L^2 / (pi^2 kappa_bar), L the chain length
    double x3[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= 1 && i < n) {
            const double d = a.dx[cb + i];
            x3[0] += a.kap_a[cs + i] * d;
            x3[1] += a.area[cb + i] * d;
            x3[2] += d;
        }
    }
    bsum<3>(x3, red, out);
    const double ts = a.eta * x3[2] * x3[2] / (kPi * kPi * (x3[0] / x3[1]));
    // factor C - t_s A (serial pass), then each chunk's carry products
    if (c == 0) {
        a.s0[st] = 1.0 / ts;
        s_fail = 0;
        double pprev = 0.0;
        for (int i = 0; i < n; ++i) {
            const double gl = i > 0 ? a.g[cs + i] : 0.0, gr = i + 1 < n ? a.g[cs + i + 1] : 0.0;
            double d = a.V[cb + i] + ts * (gl + gr);
            if (isinf(a.thr[cs + i])) d += ts * a.leak[cs + i];
            const double em = -ts * gl, ep = -ts * gr;
            const double p = 1.0 / (d - em * em * pprev);
            const int64_t pk = ps + (int64_t)(i % M) * T + i / M;
            a.sp[pk] = p; a.sg[pk] = p * em; a.su[pk] = p * ep;
            pprev = p;
        }
    }
    __syncthreads();
    {
        double acc = 1.0;
        for (int k = 0; k < M; ++k) {
            const int64_t pk = ps + (int64_t)k * T + c;
            acc *= -a.sg[pk];
            a.sPf[pk] = acc;
        }
        acc = 1.0;
        for (int k = M - 1; k >= 0; --k) {
            const int64_t pk = ps + (int64_t)k * T + c;
            acc *= -a.su[pk];
            a.sPb[pk] = acc;
        }
    }
    __syncthreads();

    // starting block F0 = [K^-1 C s0, K^-1 f] (raw columns in slots 0, 1)
    double x[M], n0[2];
    for (int col = 0; col < 2; ++col) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = c * M + k;
            x[k] = i < n ? (col == 0 ? a.V[cb + i] * sig_at(a, ps + (int64_t)k * T + c) : a.f[cs + i]) : 0.0;
        }
        ksolve<M>(a, ps, T, c, x, sA, sB);
#pragma unroll
        for (int k = 0; k < M; ++k) x[k] *= ts;
        n0[col] = sqrt(norm2<M>(x, red, out));
#pragma unroll
        for (int k = 0; k < M; ++k) Vs[(int64_t)col * P + (int64_t)k * T + c] = x[k];
    }
    const double eps0 = a.eps_rel * fmax(n0[0], n0[1]);
    int m = 0;
    for (int col = 0; col < 2; ++col) {
        if (!(n0[col] > 0.0)) continue;
#pragma unroll
        for (int k = 0; k < M; ++k) x[k] = Vs[(int64_t)col * P + (int64_t)k * T + c];
        __syncthreads();
        orth<M>(Vs, P, T, c, m, x, h, red, out);
        const double nw = sqrt(norm2<M>(x, red, out));
        if (nw >= a.eps_rel * n0[col] && nw >= eps0) {
#pragma unroll
            for (int k = 0; k < M; ++k) Vs[(int64_t)m * P + (int64_t)k * T + c] = x[k] / nw;
            ++m;
        }
        __syncthreads();
    }
    if (m == 0) {                                  // nothing to reduce: full BE
        if (c == 0) { a.kr_state[st] = 2; a.kr_mode[st] = 0; }
        return;
    }
    int pb0 = 0, pb1 = m;
    for (int blk = 1; blk < a.q && m + (pb1 - pb0) <= R; ++blk) {
        const int nb = pb1 - pb0;
        double w2 = 0.0;
        for (int q = 0; q < nb; ++q) {             // raw W = K^-1 C V_j into slots m + q
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = c * M + k;
                x[k] = i < n ? a.V[cb + i] * Vs[(int64_t)(pb0 + q) * P + (int64_t)k * T + c] : 0.0;
            }
            ksolve<M>(a, ps, T, c, x, sA, sB);
#pragma unroll
            for (int k = 0; k < M; ++k) x[k] *= ts;
            w2 += norm2<M>(x, red, out);
#pragma unroll
            for (int k = 0; k < M; ++k) Vs[(int64_t)(m + q) * P + (int64_t)k * T + c] = x[k];
        }
        const double epsj = a.eps_rel * sqrt(w2);
        int acc = 0;
        bool deficient = false;
        for (int q = 0; q < nb; ++q) {
#pragma unroll
            for (int k = 0; k < M; ++k) x[k] = Vs[(int64_t)(m + q) * P + (int64_t)k * T + c];
            __syncthreads();
            orth<M>(Vs, P, T, c, m + acc, x, h, red, out);
            const double nw = sqrt(norm2<M>(x, red, out));
            if (nw < epsj) {
                deficient = true;
            } else {
#pragma unroll
                for (int k = 0; k < M; ++k) Vs[(int64_t)(m + acc) * P + (int64_t)k * T + c] = x[k] / nw;
                ++acc;
            }
            __syncthreads();
        }
        if (acc == 0) break;                       // the space is invariant: done
        if (deficient) {                           // rank deficiency: full BE (Sec. IV-E.5)
            if (c == 0) { a.kr_state[st] = 2; a.kr_mode[st] = 0; }
            return;
        }
        pb0 = m; pb1 = m + acc; m += acc;
    }

    // projections C_h = V^T C V, A_h = V^T A V, f_h = V^T f
    double y[M];
    for (int jc = 0; jc < m; ++jc) {
#pragma unroll
        for (int k = 0; k < M; ++k) x[k] = Vs[(int64_t)jc * P + (int64_t)k * T + c];
        amul<M>(a, n, cs, T, c, x, y, sL, sR);
        dots<M>(Vs, P, T, c, m, y, h, red, out);
        if (c == 0)
            for (int i = 0; i < m; ++i) Ss[i * R + jc] = h[i];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = c * M + k;
            y[k] = i < n ? a.V[cb + i] * x[k] : 0.0;
        }
        dots<M>(Vs, P, T, c, m, y, h, red, out);
        if (c == 0)
            for (int i = 0; i < m; ++i) Chs[i * R + jc] = h[i];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        x[k] = i < n ? a.f[cs + i] : 0.0;
    }
    dots<M>(Vs, P, T, c, m, x, fh, red, out);

    // pencil A_h y = lambda C_h y: C_h = L L^T, S = L^-1 A_h L^-T, Jacobi on S
    if (c == 0) {
        for (int i = 0; i < m; ++i)                // symmetrise the projections
            for (int k = 0; k < i; ++k) {
                const double sa = 0.5 * (Ss[i * R + k] + Ss[k * R + i]);
                const double sc = 0.5 * (Chs[i * R + k] + Chs[k * R + i]);
                Ss[i * R + k] = Ss[k * R + i] = sa;
                Chs[i * R + k] = Chs[k * R + i] = sc;
            }
        for (int i = 0; i < m; ++i) {              // Cholesky
            for (int k = 0; k <= i; ++k) {
                double v = Chs[i * R + k];
                for (int l = 0; l < k; ++l) v -= Ls[i * R + l] * Ls[k * R + l];
                if (i == k) {
                    if (!(v > 0.0)) { s_fail = 1; v = 1.0; }
                    Ls[i * R + i] = sqrt(v);
                } else {
                    Ls[i * R + k] = v / Ls[k * R + k];
                }
            }
            for (int k = i + 1; k < m; ++k) Ls[i * R + k] = 0.0;
        }
        // S <- L^-1 S (columns), then S <- S L^-T (rows)
        for (int jc = 0; jc < m; ++jc)
            for (int i = 0; i < m; ++i) {
                double v = Ss[i * R + jc];
                for (int l = 0; l < i; ++l) v -= Ls[i * R + l] * Ss[l * R + jc];
                Ss[i * R + jc] = v / Ls[i * R + i];
            }
        for (int i = 0; i < m; ++i)
            for (int jc = 0; jc < m; ++jc) {
                double v = Ss[i * R + jc];
                for (int l = 0; l < jc; ++l) v -= Ss[i * R + l] * Ls[jc * R + l];
                Ss[i * R + jc] = v / Ls[jc * R + jc];
            }
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < m; ++k) Qs[i * R + k] = i == k ? 1.0 : 0.0;
        double fro = 0.0;
        for (int i = 0; i < m; ++i)
            for (int k = 0; k < m; ++k) fro += Ss[i * R + k] * Ss[i * R + k];
        for (int sweep = 0; sweep < 60; ++sweep) {
            double off = 0.0;
            for (int i = 0; i < m; ++i)
                for (int k = i + 1; k < m; ++k) off += Ss[i * R + k] * Ss[i * R + k];
            if (off <= 1e-30 * fro) break;
            for (int p = 0; p < m - 1; ++p)
                for (int qq = p + 1; qq < m; ++qq) {
                    const double apq = Ss[p * R + qq];
                    if (fabs(apq) <= 1e-300) continue;
                    const double th = (Ss[qq * R + qq] - Ss[p * R + p]) / (2.0 * apq);
                    const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    const double cc = 1.0 / sqrt(tt * tt + 1.0), sn = tt * cc;
                    for (int k = 0; k < m; ++k) {   // columns p, q
                        const double kp = Ss[k * R + p], kq = Ss[k * R + qq];
                        Ss[k * R + p] = cc * kp - sn * kq;
                        Ss[k * R + qq] = sn * kp + cc * kq;
                    }
                    for (int k = 0; k < m; ++k) {   // rows p, q
                        const double pk = Ss[p * R + k], qk = Ss[qq * R + k];
                        Ss[p * R + k] = cc * pk - sn * qk;
                        Ss[qq * R + k] = sn * pk + cc * qk;
                    }
                    for (int k = 0; k < m; ++k) {
                        const double kp = Qs[k * R + p], kq = Qs[k * R + qq];
                        Qs[k * R + p] = cc * kp - sn * kq;
                        Qs[k * R + qq] = sn * kp + cc * kq;
                    }
                }
        }
        // Y = L^-T Q (back substitution, column by column)
        double *Yg = a.Y + st * R * R, *Cg = a.Ch + st * R * R, *lg = a.lam + st * R;
        for (int jc = 0; jc < m; ++jc)
            for (int i = m - 1; i >= 0; --i) {
                double v = Qs[i * R + jc];
                for (int l = i + 1; l < m; ++l) v -= Ls[l * R + i] * Qs[l * R + jc];
                Qs[i * R + jc] = v / Ls[i * R + i];
            }
        for (int i = 0; i < m; ++i) {
            lg[i] = Ss[i * R + i];
            for (int k = 0; k < m; ++k) { Yg[i * R + k] = Qs[i * R + k]; Cg[i * R + k] = Chs[i * R + k]; }
        }
    }
    __syncthreads();
    if (s_fail) {
        if (c == 0) { a.kr_state[st] = 2; a.kr_mode[st] = 0; }
        return;
    }
    // modal basis W = V Y
    const double *Yg = a.Y + st * R * R;
    for (int jc = 0; jc < m; ++jc) {
#pragma unroll
        for (int k = 0; k < M; ++k) x[k] = 0.0;
        for (int i = 0; i < m; ++i) {
            const double yij = Yg[i * R + jc];
            const double *col = Vs + (int64_t)i * P + c;
#pragma unroll
            for (int k = 0; k < M; ++k) x[k] = fma(yij, col[(int64_t)k * T], x[k]);
        }
#pragma unroll
        for (int k = 0; k < M; ++k) Ws[(int64_t)jc * P + (int64_t)k * T + c] = x[k];
    }
    if (c == 0) { a.kr_r[st] = m; a.kr_state[st] = 1; }
}

// lifted stress at step k of node (chunk thread c, offset kk) from the modal form
__device__ __forceinline__ double modal_sigma(const double *Ws, int64_t P, int64_t off, int m, const double *zs,
                                              const double *cc, const double *rho, const double *z0,
                                              const double *phi, const int *lin, double dt, int k) {
    double v = 0.0;
    for (int j = 0; j < m; ++j) {
        const double w = Ws[(int64_t)j * P + off];
        const double zj = lin[j] ? z0[j] + k * dt * phi[j] : zs[j] + cc[j] * pow(rho[j], (double)k);
        v = fma(w, zj, v);
    }
    return v;
}

template <int M>
__global__ void __launch_bounds__(1024) k_kr_advance(KrArgs a) {
    __shared__ double red[256], out[8], sv[32];
    __shared__ int si[32];
    __shared__ double h[80], phi[80], z0[80], zs[80], cc[80], rho[80], rhoK[80];
    __shared__ int lin[80];
    const int t = a.trees[blockIdx.x], s = blockIdx.y, T = blockDim.x, c = threadIdx.x;
    const int64_t st = (int64_t)s * a.n_trees + t;
    if (!a.kr_mode[st] || a.kr_state[st] != 1) return;
    const int kd = a.kdone[st];
    if (kd >= a.n_steps) return;
    const int K = a.n_steps - kd;
    const double dt = a.dt, t0 = a.t0 + kd * dt;
    const int64_t cb = a.toff[t];
    const int n = (int)(a.toff[t + 1] - cb);
    const int64_t cs = (int64_t)s * a.N + cb, ps = (int64_t)s * a.P + a.pbase[t];
    const int R = a.rmax, m = a.kr_r[st];
    const int64_t P = a.P;
    const double *Vs = a.Vb + (int64_t)s * R * P + a.pbase[t];
    const double *Ws = a.Wb + (int64_t)s * R * P + a.pbase[t];

    // reduced initial condition (Eq. rak_reduced: s_hat(0) = V^T s0) and forcing
    double x[M];
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = sig_at(a, ps + (int64_t)k * T + c);
    dots<M>(Vs, P, T, c, m, x, h, red, out);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        x[k] = i < n ? a.f[cs + i] : 0.0;
    }
    dots<M>(Ws, P, T, c, m, x, phi, red, out);     // phi = W^T f = Y^T f_h
    if (c == 0) {
        const double *Yg = a.Y + st * R * R, *Cg = a.Ch + st * R * R, *lg = a.lam + st * R;
        for (int jm = 0; jm < m; ++jm) {           // z0 = Y^T C_h s_hat(0)
            double v = 0.0;
            for (int i = 0; i < m; ++i) {
                double chs = 0.0;
                for (int l = 0; l < m; ++l) chs += Cg[i * R + l] * h[l];
                v += Yg[i * R + jm] * chs;
            }
            z0[jm] = v;
            const double lam = lg[jm];
            if (fabs(dt * lam) < 1e-13) {
                lin[jm] = 1; zs[jm] = 0.0; cc[jm] = 0.0; rho[jm] = 1.0; rhoK[jm] = 1.0;
            } else {
                lin[jm] = 0;
                rho[jm] = 1.0 / (1.0 - dt * lam);
                zs[jm] = -phi[jm] / lam;
                cc[jm] = v - zs[jm];
                rhoK[jm] = pow(rho[jm], (double)K);
            }
        }
    }
    __syncthreads();

    // candidates: nodes whose bound over the whole step reaches their threshold;
    // each scans the steps for its first crossing
    int kf = INT_MAX;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= n) continue;
        const double th = a.thr[cs + i];
        if (isinf(th)) continue;
        const int64_t off = (int64_t)k * T + c;
        double U = 0.0;
        for (int j = 0; j < m; ++j) {
            const double w = Ws[(int64_t)j * P + off];
            double t1, tK;
            if (lin[j]) { t1 = w * (z0[j] + dt * phi[j]); tK = w * (z0[j] + K * dt * phi[j]); }
            else { t1 = w * (zs[j] + cc[j] * rho[j]); tK = w * (zs[j] + cc[j] * rhoK[j]); }
            U += fmax(t1, tK);
        }
        if (U < th - 1e-9 * fabs(th)) continue;
        for (int kk = 1; kk <= K && kk < kf; ++kk)
            if (modal_sigma(Ws, P, off, m, zs, cc, rho, z0, phi, lin, dt, kk) >= th) { kf = kk; break; }
    }
    const int kstar = (int)block_min((double)kf, sv);
    const int kend = kstar < INT_MAX ? kstar : K;
    double best = -INFINITY;
    int arg = 0x7fffffff;
    if (kstar < INT_MAX) {
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = c * M + k;
            if (i >= n) continue;
            const double th = a.thr[cs + i];
            if (isinf(th)) continue;
            const double mg = modal_sigma(Ws, P, (int64_t)k * T + c, m, zs, cc, rho, z0, phi, lin, dt, kstar) - th;
            if (mg > best) { best = mg; arg = i; }
        }
        block_argmax(best, arg, sv, si);
    }
    // void growth over steps 1..kend in closed form (existing voids only)
    const int nv = a.v_count[st];
    for (int q = 0; q < nv; ++q) {
        const int v = a.v_node[st * a.maxv + q];
        if (v / M != c) continue;
        const int64_t off = (int64_t)(v % M) * T + c;
        double ssum = 0.0;
        for (int j = 0; j < m; ++j) {
            const double w = Ws[(int64_t)j * P + off];
            double zsum;
            if (lin[j]) zsum = kend * z0[j] + dt * phi[j] * 0.5 * (double)kend * (kend + 1);
            else zsum = kend * zs[j] + cc[j] * rho[j] * (1.0 - pow(rho[j], (double)kend)) / (1.0 - rho[j]);
            ssum = fma(w, zsum, ssum);
        }
        a.v_vol[st * a.maxv + q] += dt * a.Binv * a.leak[cs + v] * ssum;
    }
    // lift at kend
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        const int64_t off = (int64_t)k * T + c;
        if (i < n) sig_set(a, ps + off, modal_sigma(Ws, P, off, m, zs, cc, rho, z0, phi, lin, dt, kend));
    }
    if (c == 0) {
        if (kstar < INT_MAX && best >= 0.0) {
            const int v = arg;
            const int64_t off = (int64_t)(v % M) * T + v / M;
            const double s1 = modal_sigma(Ws, P, off, m, zs, cc, rho, z0, phi, lin, dt, kstar);
            const double s0v = modal_sigma(Ws, P, off, m, zs, cc, rho, z0, phi, lin, dt, kstar - 1);
            const double th = a.thr[cs + v];
            const double m0 = s0v - th, m1 = s1 - th;
            const double frac = m0 < 0.0 ? -m0 / (m1 - m0) : 0.0;
            const int nvv = a.v_count[st];
            if (nvv < a.maxv) {
                const int64_t e = st * a.maxv + nvv;
                int best_s = a.inc_seg[a.inc_ptr[cb + v]];
                double bj = fabs(a.j[(int64_t)s * a.n_seg + best_s]);
                for (int kx = a.inc_ptr[cb + v] + 1; kx < a.inc_ptr[cb + v + 1]; ++kx) {
                    const double aj = fabs(a.j[(int64_t)s * a.n_seg + a.inc_seg[kx]]);
                    if (aj > bj) { bj = aj; best_s = a.inc_seg[kx]; }
                }
                a.v_node[e] = v; a.v_seg[e] = best_s; a.v_vol[e] = 0.0;
                a.v_tnuc[e] = t0 + ((double)(kstar - 1) + frac) * dt;
                a.v_count[st] = nvv + 1;
                atomicAdd(&a.counters[0], 1);
            } else {
                atomicOr(&a.status[kStatusOverflow], 1);
            }
            a.thr[cs + v] = INFINITY;
            a.dirty[st] = 1;                        // BE factors are stale too
            a.kr_state[st] = 0;                     // the matrix changed: rebuild
            atomicAdd(&a.counters[2], 1);
        }
        a.kdone[st] = kd + kend;
    }
}

KrArgs kr_args(ems_ctx *c, double dt, int n_steps) {
    Dev &d = c->d;
    KrArgs a;
    a.toff = d.toff; a.pbase = d.pbase; a.N = c->N; a.P = c->P;
    a.n_trees = c->n_trees; a.S = c->S; a.rmax = c->rmax; a.q = c->kr_q; a.eta = c->kr_eta; a.eps_rel = 1e-10;
    a.V = d.V; a.g = d.g; a.leak = d.leak; a.f = d.f; a.kap_a = d.kap_a; a.dx = d.face_dx; a.area = d.face_area;
    a.thr = d.thr; a.sig = d.sig; a.f32 = c->prm.precision == EMS_F32 ? 1 : 0;
    a.sp = d.kr_sp; a.sg = d.kr_sg; a.su = d.kr_su; a.sPf = d.kr_sPf; a.sPb = d.kr_sPb;
    a.Vb = d.kr_V; a.Wb = d.kr_W; a.lam = d.kr_lam; a.Y = d.kr_Y; a.Ch = d.kr_Ch; a.s0 = d.kr_s0;
    a.kr_r = d.kr_r; a.kr_state = d.kr_state; a.kr_mode = d.kr_mode; a.kdone = d.kdone;
    a.dt = dt; a.t0 = c->t; a.Binv = 1.0 / c->prm.B_modulus; a.n_steps = n_steps;
    a.v_count = d.v_count; a.v_node = d.v_node; a.v_seg = d.v_seg; a.v_vol = d.v_vol; a.v_tnuc = d.v_tnuc;
    a.maxv = c->maxv; a.dirty = d.dirty; a.j = d.j; a.n_seg = c->n_seg; a.inc_ptr = d.inc_ptr;
    a.inc_seg = d.inc_seg; a.status = d.status; a.counters = d.counters;
    return a;
}

template <int M>
ems_status launch_kr(ems_ctx *c, const Bucket &b, KrArgs &a, bool build) {
    dim3 grid((unsigned)b.trees.size(), c->S);
    if (build) {
        const size_t smem = sizeof(double) * (4 * (size_t)c->rmax * c->rmax + 2 * (size_t)c->rmax);
        if (smem > 48 * 1024)
            EMS_CUDA(c, cudaFuncSetAttribute(k_kr_build<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_kr_build<M><<<grid, b.T, smem, c->stream>>>(a);
    } else {
        k_kr_advance<M><<<grid, b.T, 0, c->stream>>>(a);
    }
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status kr_pass(ems_ctx *c, KrArgs &a, bool build) {
    for (auto &b : c->buckets) {
        if (!b.chain) continue;
        a.trees = b.d_trees;
        switch (b.M) {
            case 4: EMS_TRY(launch_kr<4>(c, b, a, build)); break;
            case 8: EMS_TRY(launch_kr<8>(c, b, a, build)); break;
            case 16: EMS_TRY(launch_kr<16>(c, b, a, build)); break;
            case 32: EMS_TRY(launch_kr<32>(c, b, a, build)); break;
            case 64: EMS_TRY(launch_kr<64>(c, b, a, build)); break;
            default: return fail(c, EMS_E_STATE, "unsupported chunk length");
        }
    }
    return EMS_OK;
}

// reduced-model eligibility (Eq. krylov_threshold): chains with n >= max(3q, 30)
ems_status set_modes(ems_ctx *c, int q) {
    const int S = c->S, nt = c->n_trees;
    std::vector<int32_t> mode((size_t)S * nt, 0);
    for (int t = 0; t < nt; ++t) {
        const int64_t n = c->trees.off[t + 1] - c->trees.off[t];
        const bool ok = c->pack[t].T > 1 && n >= (3 * q > 30 ? 3 * q : 30);
        for (int s = 0; s < S; ++s) mode[(size_t)s * nt + t] = ok ? 1 : 0;
    }
    EMS_CUDA(c, cudaMemcpyAsync(c->d.kr_mode, mode.data(), 4 * mode.size(), cudaMemcpyHostToDevice, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

ems_status ensure_q(ems_ctx *c, int q, double eta) {
    if (c->rmax == 0) return fail(c, EMS_E_STATE, "context created with method EMS_BE: no Krylov storage");
    if (q < 1 || 2 * q > c->rmax || !(eta > 0.0)) return fail(c, EMS_E_INVAL, "q must be 1..params.krylov_q, eta > 0");
    if (q != c->kr_q || eta != c->kr_eta) {
        c->kr_q = q;
        c->kr_eta = eta;
        EMS_CUDA(c, cudaMemsetAsync(c->d.kr_state, 0, sizeof(int32_t) * c->S * c->n_trees, c->stream));
    }
    return EMS_OK;
}

}  // namespace

ems_status krylov_advance(ems_ctx *c, double dt, int n_steps, int method, int *n_new) {
    (void)method;
    EMS_TRY(ensure_q(c, c->kr_q > 0 ? c->kr_q : c->prm.krylov_q, c->kr_q > 0 ? c->kr_eta : c->prm.krylov_eta));
    EMS_TRY(set_modes(c, c->kr_q));
    cudaStream_t st = c->stream;
    EMS_CUDA(c, cudaMemsetAsync(c->d.counters, 0, 3 * sizeof(int32_t), st));
    EMS_CUDA(c, cudaMemsetAsync(c->d.kdone, 0, sizeof(int32_t) * c->S * c->n_trees, st));
    KrArgs a = kr_args(c, dt, n_steps);
    for (int round = 0; round < 4 * EMS_MAX_VOIDS; ++round) {
        EMS_TRY(kr_pass(c, a, true));
        EMS_TRY(kr_pass(c, a, false));
        int32_t again = 0;
        EMS_CUDA(c, cudaMemcpyAsync(&again, c->d.counters + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        EMS_CUDA(c, cudaStreamSynchronize(st));
        if (again == 0) break;
        EMS_CUDA(c, cudaMemsetAsync(c->d.counters + 2, 0, sizeof(int32_t), st));
    }
    // trees without a reduced model (small, branched, fallen back) take BE
    EMS_TRY(launch_be(c, dt, n_steps));
    if (dt != c->factored_dt) c->factored_dt = dt;
    c->t += dt * n_steps;
    if (n_new) EMS_CUDA(c, cudaMemcpyAsync(n_new, c->d.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return EMS_OK;
}

}  // namespace ems

using namespace ems;

extern "C" ems_status ems_krylov_reduce(ems_ctx *c, int q, double eta, int *n_reduced, int *n_fallback) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "Krylov reduction before the first IR solve");
    EMS_TRY(ensure_q(c, q, eta));
    EMS_TRY(set_modes(c, q));
    EMS_TRY(forcing(c));
    KrArgs a = kr_args(c, 0.0, 0);
    EMS_TRY(kr_pass(c, a, true));
    const size_t ts = (size_t)c->S * c->n_trees;
    std::vector<int32_t> state(ts), mode(ts);
    EMS_CUDA(c, cudaMemcpyAsync(state.data(), c->d.kr_state, 4 * ts, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaMemcpyAsync(mode.data(), c->d.kr_mode, 4 * ts, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    int nr = 0, nf = 0;
    for (size_t k = 0; k < ts; ++k) {
        if (state[k] == 1) ++nr;
        if (state[k] == 2) ++nf;
    }
    if (n_reduced) *n_reduced = nr;
    if (n_fallback) *n_fallback = nf;
    return check_status(c);
}
