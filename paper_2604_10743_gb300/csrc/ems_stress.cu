// ems_stress.cu -- per-tree EM/TM stress path on the GPU.
//
//   node physics  T at every stress node (bilinear map sample), kappa and the
//                 TM term per face, node volume, Robin leak coefficient and
//                 critical stress per node (Sec. III-A, III-D.1)
//   forcing       f = B j - D of Eq. em_tm_ode per node from the currents
//   advance       backward-Euler steps (Sec. IV-B) with nucleation, Robin
//                 voids (Sec. IV-D) and void growth (Eq. void_volume_equation)
//   void update   resistance write-back (Sec. III-D.3, IV-C)
//   screen        steady-state immortality check (Sec. III-B)
//
// Chain trees (every stripe of a mesh) run one CTA of T threads per (tree,
// sample).  Thread c owns the contiguous chunk [c M, c M + M) of the chain
// and keeps its stress in registers for all inner steps of a launch.  The
// matrix M = C - dt A is factored once per (dt, void set) as
// M = L D L^T, written as the scaled recurrences
//     z_i = alpha_i s_i + beta_i - gamma_i z_{i-1},    x_i = z_i - u_i x_{i+1}
// with alpha = V/d', beta = dt f/d', gamma = e_{i-1}/d', u = e_i/d'.  Each
// first-order recurrence is solved chunk-parallel: a local sweep with zero
// carry, an exclusive scan of the chunk's affine transfer maps across the
// team (warp shuffles + one shared-memory level), and a correction with the
// precomputed carry products Pf / Pb.  Trees with branches run one thread
// per (tree, sample) with leaf-to-root elimination.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <map>
#include <vector>

#include "ems_chain.cuh"
#include "ems_device.cuh"
#include "ems_internal.cuh"

namespace ems {
ems_status check_status(ems_ctx *c);

namespace {

// ---------------------------------------------------------------------------
// Node physics
// ---------------------------------------------------------------------------
__global__ void k_temperature(int64_t N, const double *x, const double *y, const double *T, int nx, int ny,
                              double x0, double y0, double x1, double y1, double T0, double *Tn) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        if (nx == 0) { Tn[i] = T0; continue; }
        double fx = (x[i] - x0) / (x1 - x0) * (nx - 1);
        double fy = (y[i] - y0) / (y1 - y0) * (ny - 1);
        fx = fmin(fmax(fx, 0.0), (double)(nx - 1));
        fy = fmin(fmax(fy, 0.0), (double)(ny - 1));
        int ix = min((int)floor(fx), nx - 2), iy = min((int)floor(fy), ny - 2);
        double tx = fx - ix, ty = fy - iy;
        const double *r0 = T + (int64_t)iy * nx, *r1 = r0 + nx;
        Tn[i] = (1 - tx) * (1 - ty) * r0[ix] + tx * (1 - ty) * r0[ix + 1] + (1 - tx) * ty * r1[ix] +
                tx * ty * r1[ix + 1];
    }
}

struct PhysArgs {
    int64_t N;
    int n_seg;
    const int32_t *gpar, *face_seg, *owner_seg, *child_ptr, *child_gidx;
    const double *Tn, *dx, *area, *kfac, *sfac;
    const double *pert, *nx, *ny;      // per-sample perturbation rasters [S][EMS_MAX_PERT] (pnx = 0: none)
    int pnx, pny;
    double px0, py0, px1, py1;
    double D0, Ea, kB, B, Omega, Qs, delta, sigma_crit;
    double *kap_a, *g, *Mface, *V, *leak, *thr0, *thr;
    double *fb_ka, *fb_g, *fb_M;       // face terms without the sample factor (no perturbation)
};

// a sample's temperature perturbation at (x, y): bilinear over its raster,
// vertex-centred over the map's extent, clamped at the border
__device__ double pert_at(const PhysArgs &a, const double *r, double x, double y) {
    double fx = (x - a.px0) / (a.px1 - a.px0) * (a.pnx - 1);
    double fy = (y - a.py0) / (a.py1 - a.py0) * (a.pny - 1);
    fx = fmin(fmax(fx, 0.0), (double)(a.pnx - 1));
    fy = fmin(fmax(fy, 0.0), (double)(a.pny - 1));
    const int ix = min((int)floor(fx), a.pnx - 2), iy = min((int)floor(fy), a.pny - 2);
    const double tx = fx - ix, ty = fy - iy;
    const double *r0 = r + (int64_t)iy * a.pnx, *r1 = r0 + a.pnx;
    return (1 - tx) * (1 - ty) * r0[ix] + tx * (1 - ty) * r0[ix + 1] + (1 - tx) * ty * r1[ix] + tx * ty * r1[ix + 1];
}

// per face, from the node temperatures alone (Arrhenius kappa without the
// sample's factor, Eq. kappa; TM term): once per temperature change
__global__ void k_face_base(PhysArgs a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = a.gpar[i];
        if (q < 0) {
            a.fb_ka[i] = 0.0; a.fb_g[i] = 0.0; a.fb_M[i] = 0.0;
            continue;
        }
        const double Ti = a.Tn[i], Tq = a.Tn[q];
        const double Te = 0.5 * (Ti + Tq);
        const double ikT = 1.0 / (a.kB * Te);
        const double ka = a.area[i] * (a.D0 * exp(-a.Ea * ikT) * a.B * a.Omega * ikT);
        a.fb_ka[i] = ka;
        a.fb_g[i] = ka / a.dx[i];
        a.fb_M[i] = a.Qs / (a.Omega * Te) * (Ti - Tq) / a.dx[i];
    }
}

// per face (stored at the child node): a kappa, g = a kappa / dx, TM term M
// of each mapped sample: the temperature-only terms times the sample's kappa
// factor, or (a sample's perturbation raster adds to the node temperatures)
// evaluated per sample
__global__ void k_faces(PhysArgs a) {
    const int s = blockIdx.y;
    const double *pr = a.pert + (int64_t)s * EMS_MAX_PERT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t si = (int64_t)s * a.N + i;
        const int32_t q = a.gpar[i];
        if (q < 0) {
            a.kap_a[si] = 0.0; a.g[si] = 0.0;
            a.Mface[si] = 0.0;
            continue;
        }
        if (a.pnx == 0) {
            const double kf = a.kfac[(int64_t)s * a.n_seg + a.face_seg[i]];
            a.kap_a[si] = a.fb_ka[i] * kf;
            a.g[si] = a.fb_g[i] * kf;
            a.Mface[si] = a.fb_M[i];
            continue;
        }
        double Ti = a.Tn[i], Tq = a.Tn[q];
        if (a.pnx > 0) {
            Ti += pert_at(a, pr, a.nx[i], a.ny[i]);
            Tq += pert_at(a, pr, a.nx[q], a.ny[q]);
        }
        const double Te = 0.5 * (Ti + Tq);
        const double ikT = 1.0 / (a.kB * Te);
        const double kap = a.D0 * exp(-a.Ea * ikT) * a.B * a.Omega * ikT *
                           a.kfac[(int64_t)s * a.n_seg + a.face_seg[i]];
        const double ka = a.area[i] * kap;
        a.kap_a[si] = ka;
        a.g[si] = ka / a.dx[i];
        a.Mface[si] = a.Qs / (a.Omega * Te) * (Ti - Tq) / a.dx[i];
    }
}

// per node: V = sum of a dx / 2, leak = sum of a kappa / delta over faces at
// the node; critical stress from the owner segment's factor
__global__ void k_nodes(PhysArgs a) {
    const int s = blockIdx.y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t so = (int64_t)s * a.N;
        double vol = 0.0, lk = 0.0;
        if (a.gpar[i] >= 0) { vol += 0.5 * a.area[i] * a.dx[i]; lk += a.kap_a[so + i]; }
        for (int k = a.child_ptr[i]; k < a.child_ptr[i + 1]; ++k) {
            const int32_t ch = a.child_gidx[k];
            vol += 0.5 * a.area[ch] * a.dx[ch];
            lk += a.kap_a[so + ch];
        }
        if (s == 0) a.V[i] = vol;
        a.leak[so + i] = lk / a.delta;
        const double t0 = a.sigma_crit * a.sfac[(int64_t)s * a.n_seg + a.owner_seg[i]];
        a.thr0[so + i] = t0;
        a.thr[so + i] = t0;
    }
}

// voids exclude their node from nucleation (threshold +inf) and force a refactor
__global__ void k_apply_voids(int n_trees, int S, int maxv, int64_t N, const int64_t *toff,
                              const int32_t *v_count, const int32_t *v_node, double *thr, int32_t *dirty) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n_trees * S) return;
    const int s = (int)(k / n_trees), t = (int)(k % n_trees);
    for (int q = 0; q < v_count[k]; ++q) thr[(int64_t)s * N + toff[t] + v_node[k * maxv + q]] = INFINITY;
    dirty[k] = 1;
}

// f_i = q_i - sum over children q_c with q = a kappa G, G = S + M
__global__ void k_forcing(int64_t N, int n_seg, double sfac_em, const int32_t *gpar, const int32_t *face_seg,
                          const int8_t *sign, const int32_t *child_ptr, const int32_t *child_gidx,
                          const double *Mface, const double *kap_a, const double *j, double *f) {
    const int s = blockIdx.y;
    const double *js = j + (int64_t)s * n_seg, *ka = kap_a + (int64_t)s * N, *Ms = Mface + (int64_t)s * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        if (gpar[i] >= 0) acc = ka[i] * (sfac_em * sign[i] * js[face_seg[i]] + Ms[i]);
        for (int k = child_ptr[i]; k < child_ptr[i + 1]; ++k) {
            const int32_t ch = child_gidx[k];
            acc -= ka[ch] * (sfac_em * sign[ch] * js[face_seg[ch]] + Ms[ch]);
        }
        f[(int64_t)s * N + i] = acc;
    }
}

// ---------------------------------------------------------------------------
// Packed <-> canonical stress
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_pack(int n_trees, int64_t N, int64_t P, const int64_t *toff, const int64_t *pbase,
                       const int32_t *pT, const int32_t *pM, double *canon, R *packed, int dir, double fill) {
    // dir 1: canonical -> packed; 0: packed -> canonical; 2: packed := fill on real nodes
    const int t = blockIdx.x, s = blockIdx.y;
    const int64_t cb = toff[t], n = toff[t + 1] - cb;
    const int T = pT[t], M = pM[t];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t pk = (int64_t)s * P + pbase[t] + (T > 1 ? (i % M) * T + i / M : i);
        const int64_t ck = (int64_t)s * N + cb + i;
        if (dir == 1) packed[pk] = (R)canon[ck];
        else if (dir == 0) canon[ck] = (double)packed[pk];
        else packed[pk] = (R)fill;
    }
}

// ---------------------------------------------------------------------------
// Chain kernel
// ---------------------------------------------------------------------------
// Factor M = C - dt A of one chain, then every chunk's right-hand-side
// coefficients and carry products.  Must be called by the whole block.
// DELTA (increment form) stores p = 1/d', dt g, dt f, dt leak instead of
// alpha = V/d', beta = dt f/d'.
//
// The pivots d'_i = d_i - e_i^2 / d'_{i-1} follow from the linear recurrence
// q_i = d_i q_{i-1} - e_i^2 q_{i-2} (d'_i = q_i / q_{i-1}), i.e. from products
// of the matrices [[d_i, -e_i^2], [1, 0]].  Each thread multiplies its
// chunk's matrices, a block scan of the products gives the pivot entering
// every chunk, and each thread then runs the pivot recurrence on its own
// nodes: O(M + log T) per thread instead of O(n) on one thread.  One
// compiled copy per instantiation (not inlined) with every rounding written
// out, so a refactor after a nucleation and a refactor from a checkpoint
// give the same bits.
template <typename R, int M, bool DELTA>
__device__ __noinline__ void chain_factor(const ChainArgs<R> &a, double dt, int n, int T, int c, int64_t cb,
                                          int64_t cs, int64_t ps, int from) {
    (void)from;                       // the whole chain is refactored (cheap in parallel)
    __shared__ double sfm[4][32];
    const int lane = c & 31, w = c >> 5, nw = T >> 5;
    __syncthreads();
    auto node = [&](int i, double &d, double &em, double &ep, bool &is_void) {
        const double gl = i > 0 ? a.g[cs + i] : 0.0, gr = i + 1 < n ? a.g[cs + i + 1] : 0.0;
        is_void = isinf(a.thr[cs + i]);
        d = __fma_rn(dt, __dadd_rn(gl, gr), a.V[cb + i]);
        if (is_void) d = __fma_rn(dt, a.leak[cs + i], d);
        em = -__dmul_rn(dt, gl);
        ep = -__dmul_rn(dt, gr);
    };
    // this chunk's product (later nodes on the left)
    M2 P{1.0, 0.0, 0.0, 1.0};
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= n) break;
        double d, em, ep;
        bool v;
        node(i, d, em, ep, v);
        P = m2mul(M2{d, -__dmul_rn(em, em), 1.0, 0.0}, P);
    }
    // inclusive scan over the chunks, then the exclusive product entering c
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const M2 o = m2shfl_up(P, d);
        if (lane >= d) P = m2mul(P, o);
    }
    M2 Cw{1.0, 0.0, 0.0, 1.0};
    if (nw > 1) {
        if (lane == 31) { sfm[0][w] = P.a; sfm[1][w] = P.b; sfm[2][w] = P.c; sfm[3][w] = P.d; }
        __syncthreads();
        for (int k = 0; k < w; ++k) Cw = m2mul(M2{sfm[0][k], sfm[1][k], sfm[2][k], sfm[3][k]}, Cw);
    }
    const M2 incl = m2mul(P, Cw);
    const M2 prev = m2shfl_up(incl, 1);
    const M2 Q = lane == 0 ? Cw : prev;
    // state entering the chunk: (q_{cM-1}, q_{cM-2}) = Q (1, 0)^T
    double pprev = c == 0 ? 0.0 : __ddiv_rn(Q.c, Q.a);   // 1 / d'_{cM-1}
    for (int k = 0; k < M; ++k) {
        const int i = c * M + k;
        if (i >= n) break;
        double d, em, ep;
        bool is_void;
        node(i, d, em, ep, is_void);
        const double p = __drcp_rn(__fma_rn(-__dmul_rn(em, em), pprev, d));
        const int64_t pk = ps + (int64_t)k * T + c;
        a.pinv[pk] = p;
        if (DELTA) {
            a.alpha[pk] = (R)p;
            a.dtg[pk] = (R)(-em);
            a.dtl[pk] = is_void ? (R)(dt * a.leak[cs + i]) : R(0);
        } else {
            a.alpha[pk] = (R)(p * a.V[cb + i]);
        }
        a.gam[pk] = (R)(p * em);
        a.uu[pk] = (R)(p * ep);
        pprev = p;
    }
    __syncthreads();
    if (DELTA) {
        // increment form: gamma_k = -p_k dtg_k and u_k = -p_k dtg_{k+1} are
        // formed on the fly, so the carry products use the same products
        R acc = R(1);
        for (int k = 0; k < M; ++k) {
            const int64_t pk = ps + (int64_t)k * T + c;
            const int i = c * M + k;
            a.beta[pk] = i < n ? (R)(dt * a.f[cs + i]) : R(0);
            acc *= a.alpha[pk] * a.dtg[pk];
            a.Pf[pk] = acc;
        }
        acc = R(1);
        for (int k = M - 1; k >= 0; --k) {
            const int64_t pk = ps + (int64_t)k * T + c;
            const R gn = k + 1 < M ? a.dtg[pk + T] : (c + 1 < T ? a.dtg[ps + c + 1] : R(0));
            acc *= a.alpha[pk] * gn;
            a.Pb[pk] = acc;
        }
        return;
    }
    R acc = R(1);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int64_t pk = ps + (int64_t)k * T + c;
        const int i = c * M + k;
        a.beta[pk] = i < n ? (R)(a.pinv[pk] * dt * a.f[cs + i]) : R(0);
        acc *= -a.gam[pk];
        a.Pf[pk] = acc;
    }
    acc = R(1);
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        const int64_t pk = ps + (int64_t)k * T + c;
        acc *= -a.uu[pk];
        a.Pb[pk] = acc;
    }
}

// SMC (increment form only): the tree's per-node coefficients (p, dt g,
// dt f, carry products) are staged in shared memory once per factorisation
// instead of being re-read from L2 on every step, and the forward values stay
// in registers; the arithmetic is the same as with global coefficients.
template <typename R, int M, bool DELTA, bool SMC>
__global__ void __launch_bounds__(ChainMaxThreads<R, M>::value, SMC ? 1 : ChainMinBlocks<R, M>::value)
    k_chain(ChainArgs<R> a) {
    __shared__ R sA[64], sB[64], sC[32], sL[32], sR[32];
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int s_nv;
    __shared__ int s_node[EMS_MAX_VOIDS];
    __shared__ double s_vol[EMS_MAX_VOIDS], s_coef[EMS_MAX_VOIDS];

    extern __shared__ float2 zu[];      // increment form: [M][T] forward values (SMC: coefficients)
    const int t = a.trees[blockIdx.x], s = blockIdx.y;
    const int T = blockDim.x, c = threadIdx.x;
    R *scr = reinterpret_cast<R *>(zu);   // SMC: p, dt g, dt f, Pf, Pb, each [M][T]
    const int MT = M * T;
    const int64_t cb = a.toff[t];
    const int n = (int)(a.toff[t + 1] - cb);
    const int64_t cs = (int64_t)s * a.N + cb, ps = (int64_t)s * a.P + a.pbase[t];
    const int64_t st = (int64_t)s * a.n_trees + t;
    const int sm = a.sched[st];
    if (a.kr_mode[st] || sm < 0) return;           // reduced model / frozen by the schedule
    const int kd = a.kdone[st];                    // steps already done (reduced model fell back)

    double tm = INFINITY;
    for (int i = c; i < n; i += T) tm = fmin(tm, a.thr[cs + i]);
    double thrmin = block_min(tm, sv);
    long long thr_bits = __double_as_longlong(thrmin);
    float thr_f = __double2float_rd(thrmin);
    R sg[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        sg[k] = a.sig[ps + (int64_t)k * T + c];
        if (DELTA) a.kc[ps + (int64_t)k * T + c] = R(0);    // compensations start at 0 every launch
    }

    // Step schedule, block-uniform and kept in shared memory (read only on
    // rare branches): s_rs fine steps per step of length s_dt; the current
    // run of such steps began at step s_sbase, time s_tbase.  A coarse tree
    // whose stress already reaches the guard level steps finely from now on.
    __shared__ double s_dt, s_tbase, s_gthr;
    __shared__ int s_rs, s_sbase;
    int rs = sm > 1 ? sm : 1;
    if ((a.n_steps - kd) % rs) rs = 1;
    if (rs > 1 && __syncthreads_or(near_guard<R, M>(sg, a.guard * thrmin))) {
        rs = 1;
        if (c == 0) a.sched[st] = 0;
    }
    int n_steps = (a.n_steps - kd) / rs;

    __shared__ int s_refac;
    if (c == 0) {
        const double dt = a.dt * rs;
        s_dt = dt;
        s_rs = rs;
        s_gthr = a.guard * thrmin;
        s_sbase = 0;
        s_tbase = (a.t0p ? *a.t0p : a.t0) + kd * a.dt;
        const int nv = a.v_count[st];
        s_nv = nv;
        for (int q = 0; q < nv; ++q) {
            const int v = a.v_node[st * a.maxv + q];
            s_node[q] = v;
            s_vol[q] = a.v_vol[st * a.maxv + q];
            s_coef[q] = dt * a.Binv * a.leak[cs + v];
        }
        s_refac = (a.refactor_all || a.dirty[st] || a.fdt[st] != dt) ? 1 : 0;
        a.dirty[st] = 0;
        a.fdt[st] = dt;
    }
    __syncthreads();
    if (s_refac) {
        chain_factor<R, M, DELTA>(a, s_dt, n, T, c, cb, cs, ps, 0);
    } else {
        const double dt = s_dt;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int64_t pk = ps + (int64_t)k * T + c;
            const int i = c * M + k;
            if (DELTA) a.beta[pk] = i < n ? (R)(dt * a.f[cs + i]) : R(0);
            else a.beta[pk] = i < n ? (R)(a.pinv[pk] * dt * a.f[cs + i]) : R(0);
        }
    }
    // stage the coefficients in shared memory (after every factorisation)
    auto stage = [&]() {
        if constexpr (SMC) {
            __syncthreads();
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int64_t pk = ps + (int64_t)k * T + c;
                const int o = k * T + c;
                scr[o] = a.alpha[pk];
                scr[MT + o] = a.dtg[pk];
                scr[2 * MT + o] = a.beta[pk];
                scr[3 * MT + o] = a.Pf[pk];
                scr[4 * MT + o] = a.Pb[pk];
            }
            __syncthreads();
        }
    };
    stage();
    __syncthreads();
    unsigned long long vmask = 0ull;     // void nodes in this thread's chunk
    for (int q = 0; q < s_nv; ++q)
        if (s_node[q] / M == c) vmask |= 1ull << (s_node[q] % M);

    for (int step = 0; step < n_steps; ++step) {
        if (!DELTA) {
            // forward sweep z_i = alpha s_i + beta - gamma z_{i-1}
            R z = R(0);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int64_t pk = ps + (int64_t)k * T + c;
                const R av = fmx(a.alpha[pk], sg[k], a.beta[pk]);
                z = fmx(-a.gam[pk], z, av);
                sg[k] = z;
            }
            const R cf = scan_fwd<R>(z, a.Pf[ps + (int64_t)(M - 1) * T + c], sA, sB, sC);
#pragma unroll
            for (int k = 0; k < M; ++k) sg[k] = fmx(a.Pf[ps + (int64_t)k * T + c], cf, sg[k]);
            // backward sweep x_i = z_i - u_i x_{i+1}
            R x = R(0);
#pragma unroll
            for (int k = M - 1; k >= 0; --k) {
                x = fmx(-a.uu[ps + (int64_t)k * T + c], x, sg[k]);
                sg[k] = x;
            }
            const R cr = scan_bwd<R>(x, a.Pb[ps + c], sA, sB, sC);
#pragma unroll
            for (int k = 0; k < M; ++k) sg[k] = fmx(a.Pb[ps + (int64_t)k * T + c], cr, sg[k]);
        } else {
            // increment form: (C - dt A) d = dt (A s + f), s += d.  The
            // forward values z and the products u = p dtg_{k+1} go to shared
            // memory; the state chunk is the only array kept in registers.
            const unsigned full = 0xffffffffu;
            const int lane = c & 31, w = c >> 5, nw = T >> 5;
            R left = __shfl_up_sync(full, sg[M - 1], 1);
            R right = __shfl_down_sync(full, sg[0], 1);
            if (nw > 1) {
                if (lane == 31) sL[w] = sg[M - 1];
                if (lane == 0) sR[w] = sg[0];
                __syncthreads();
                if (lane == 0 && w > 0) left = sL[w - 1];
                if (lane == 31 && w + 1 < nw) right = sR[w + 1];
            }
            const R *pG = SMC ? scr + MT + c : a.dtg + ps + c;
            const R *pP = SMC ? scr + c : a.alpha + ps + c;
            const R *pB = SMC ? scr + 2 * MT + c : a.beta + ps + c;
            const R *pF = SMC ? scr + 3 * MT + c : a.Pf + ps + c;
            const R *pBk = SMC ? scr + 4 * MT + c : a.Pb + ps + c;
            const R g_next = c + 1 < T ? pG[1] : R(0);          // face to the next chunk
            R gk = pG[0];
            R qprev = gk * (left - sg[0]);
            R z = R(0);
            R zr[SMC ? M : 1];
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const R nxt = k + 1 < M ? sg[k + 1] : right;
                const R gk1 = k + 1 < M ? pG[(int64_t)(k + 1) * T] : g_next;
                const R pk = pP[(int64_t)k * T];
                const R qn = gk1 * (sg[k] - nxt);
                R r = qprev - qn + pB[(int64_t)k * T];
                if ((vmask >> k) & 1ull) r -= a.dtl[ps + (int64_t)k * T + c] * sg[k];
                z = pk * fmx(gk, z, r);
                if constexpr (SMC) zr[k] = z;
                else zu[k * T + c] = make_float2((float)z, (float)(pk * gk1));
                qprev = qn;
                gk = gk1;
            }
            const R cf = scan_fwd<R>(z, pF[(int64_t)(M - 1) * T], sA, sB, sC);
            R x = R(0);
            // this chunk's increments before the right carry replace the
            // forward values (registers with SMC, else shared memory)
#pragma unroll
            for (int k = M - 1; k >= 0; --k) {
                if constexpr (SMC) {
                    const R gk1 = k + 1 < M ? pG[(int64_t)(k + 1) * T] : g_next;
                    x = fmx(pP[(int64_t)k * T] * gk1, x, fmx(pF[(int64_t)k * T], cf, zr[k]));
                    zr[k] = x;
                } else {
                    const float2 e = zu[k * T + c];
                    x = fmx((R)e.y, x, fmx(pF[(int64_t)k * T], cf, (R)e.x));
                    zu[k * T + c].x = (float)x;
                }
            }
            const R cr = scan_bwd<R>(x, pBk[0], sA, sB, sC);
            // compensated (Kahan) state update, the compensation kept in a
            // global array (no register room for it at these chunk lengths)
#pragma unroll
            for (int k = 0; k < M; ++k) {
                R &ck = a.kc[ps + (int64_t)k * T + c];
                R xk;
                if constexpr (SMC) xk = zr[k];
                else xk = (R)zu[k * T + c].x;
                const R y = fmx(pBk[(int64_t)k * T], cr, xk) - ck;
                const R t = sg[k] + y;
                ck = (t - sg[k]) - y;
                sg[k] = t;
            }
        }

        // void growth by the Robin leak: the owner thread of a void node stores
        // it (compile-time register index under a bit mask) and reads it back
        if (vmask) {
#pragma unroll
            for (int k = 0; k < M; ++k)
                if ((vmask >> k) & 1ull) a.sig[ps + (int64_t)k * T + c] = sg[k];
            for (int q = 0; q < s_nv; ++q) {
                const int v = s_node[q];
                if (v / M == c) s_vol[q] += s_coef[q] * (double)a.sig[ps + (int64_t)(v % M) * T + c];
            }
        }
        // nucleation: cheap test against the tree's lowest threshold, exact on a hit
        bool hit = false;
#pragma unroll
        for (int k = 0; k < M; ++k) hit |= above<R>(sg[k], thr_bits, thr_f);
        int refac_from = -1;                        // block-uniform: refactor from this node
        if (__syncthreads_or(hit)) {
            double best = -INFINITY;
            int arg = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = c * M + k;
                if (i < n) {
                    const double m = (double)sg[k] - a.thr[cs + i];
                    if (m > best) { best = m; arg = i; }
                }
            }
            block_argmax(best, arg, sv, si);
            if (best >= 0.0) {
#pragma unroll
                for (int k = 0; k < M; ++k) a.sig[ps + (int64_t)k * T + c] = sg[k];
                __syncthreads();
                if (c == 0) {
                    const int v = arg;
                    const double dt = s_dt;
                    auto S_ = [&](int i) { return (double)a.sig[ps + (int64_t)(i % M) * T + i / M]; };
                    // previous-step stress at v from the BE relation M s^{k+1} = V s^k + dt f
                    const double gl = v > 0 ? a.g[cs + v] : 0.0, gr = v + 1 < n ? a.g[cs + v + 1] : 0.0;
                    double acc = (a.V[cb + v] + dt * (gl + gr)) * S_(v);
                    if (v > 0) acc -= dt * gl * S_(v - 1);
                    if (v + 1 < n) acc -= dt * gr * S_(v + 1);
                    const double s0 = (acc - dt * a.f[cs + v]) / a.V[cb + v];
                    const double m0 = s0 - a.thr[cs + v];
                    const double frac = m0 < 0.0 ? -m0 / (best - m0) : 0.0;
                    const int nv = s_nv;
                    if (nv < a.maxv) {
                        const int64_t e = st * a.maxv + nv;
                        a.v_node[e] = v;
                        a.v_seg[e] = void_segment<R>(a, s, cb + v);
                        a.v_tnuc[e] = s_tbase + ((double)(step - s_sbase) + frac) * dt;
                        a.v_vol[e] = 0.0;
                        s_node[nv] = v; s_vol[nv] = 0.0; s_coef[nv] = dt * a.Binv * a.leak[cs + v];
                        s_nv = nv + 1;
                        a.v_count[st] = nv + 1;
                        atomicAdd(&a.counters[0], 1);
                    } else {
                        atomicOr(&a.status[kStatusOverflow], 1);
                    }
                    a.thr[cs + v] = INFINITY;
                }
                if (arg / M == c) vmask |= 1ull << (arg % M);
                refac_from = arg;
            }
        }
        bool promoted = false;
        if (s_rs > 1 && __syncthreads_or(near_guard<R, M>(sg, s_gthr))) {
            // coarse tree near its critical stress: finish this call with
            // the plain solver's fine steps and keep them
            n_steps = step + 1 + (n_steps - step - 1) * s_rs;
            promoted = true;
            __syncthreads();
            if (c == 0) {
                s_tbase += (double)(step + 1 - s_sbase) * s_dt;
                s_sbase = step + 1;
                s_dt = a.dt;
                s_rs = 1;
                a.sched[st] = 0;
                a.fdt[st] = a.dt;
                for (int q = 0; q < s_nv; ++q) s_coef[q] = a.dt * a.Binv * a.leak[cs + s_node[q]];
            }
            refac_from = 0;
        }
        if (refac_from >= 0) {
            // the step is passed by value, so it must not be read from
            // shared memory that thread 0 may still be updating
            const double dtf = promoted ? a.dt : s_dt;
            chain_factor<R, M, DELTA>(a, dtf, n, T, c, cb, cs, ps, refac_from);
            stage();
            tm = INFINITY;
            for (int i = c; i < n; i += T) tm = fmin(tm, a.thr[cs + i]);
            thrmin = block_min(tm, sv);
            thr_bits = __double_as_longlong(thrmin);
            thr_f = __double2float_rd(thrmin);
            if (c == 0) s_gthr = a.guard * thrmin;
            __syncthreads();
        }
    }
#pragma unroll
    for (int k = 0; k < M; ++k) a.sig[ps + (int64_t)k * T + c] = sg[k];
    __syncthreads();
    if (c == 0) {
        for (int q = 0; q < s_nv; ++q) a.v_vol[st * a.maxv + q] = s_vol[q];
        atomicAdd(a.work, (unsigned long long)n * (unsigned long long)n_steps);
    }
}

// ---------------------------------------------------------------------------
// Register-resident FP32 chain kernel (increment form).  Thread c keeps, for
// its M nodes, the state, the forward values and every per-node coefficient
// of the factorisation (p = 1/d', dt g, dt f, the carry products Pf and Pb,
// and the nucleation threshold rounded down to FP32, or dt leak at a void
// node) in registers, so a BE step reads no memory but the two chunk scans.
// The nucleation test compares every node with its own threshold; void
// growth reads the void node's stress by compile-time register selection.
// The arithmetic of a step is the same as k_chain's increment form.
// ---------------------------------------------------------------------------
template <int M> struct RegMaxThreads;
template <> struct RegMaxThreads<4> { static constexpr int value = 896; };
template <> struct RegMaxThreads<8> { static constexpr int value = 576; };
template <> struct RegMaxThreads<16> { static constexpr int value = 320; };

template <int M>
__global__ void __launch_bounds__(RegMaxThreads<M>::value, 1) k_chain_reg(ChainArgs<float> a) {
    using R = float;
    __shared__ R sA[64], sB[64], sC[32], sL[32], sR[32];
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int s_nv, s_refac;
    __shared__ int s_node[EMS_MAX_VOIDS];
    __shared__ double s_vol[EMS_MAX_VOIDS], s_coef[EMS_MAX_VOIDS];
    __shared__ double s_dt, s_tbase, s_gthr;
    __shared__ int s_rs, s_sbase;

    const int t = a.trees[blockIdx.x], s = blockIdx.y;
    const int T = blockDim.x, c = threadIdx.x;
    const int lane = c & 31, w = c >> 5, nw = T >> 5;
    const int64_t cb = a.toff[t];
    const int n = (int)(a.toff[t + 1] - cb);
    const int64_t cs = (int64_t)s * a.N + cb, ps = (int64_t)s * a.P + a.pbase[t];
    const int64_t st = (int64_t)s * a.n_trees + t;
    const int sm = a.sched[st];
    if (a.kr_mode[st] || sm < 0) return;
    const int kd = a.kdone[st];

    double tm = INFINITY;
    for (int i = c; i < n; i += T) tm = fmin(tm, a.thr[cs + i]);
    double thrmin = block_min(tm, sv);
    // state and its compensation: every increment is added with Kahan's
    // compensated summation, so increments far below an ulp of the stress
    // (late, slow evolution) accumulate instead of being rounded away
    R sg[M], cc[M];
#pragma unroll
    for (int k = 0; k < M; ++k) { sg[k] = a.sig[ps + (int64_t)k * T + c]; cc[k] = R(0); }

    int rs = sm > 1 ? sm : 1;
    if ((a.n_steps - kd) % rs) rs = 1;
    if (rs > 1 && __syncthreads_or(near_guard<R, M>(sg, a.guard * thrmin))) {
        rs = 1;
        if (c == 0) a.sched[st] = 0;
    }
    int n_steps = (a.n_steps - kd) / rs;
    if (c == 0) {
        const double dt = a.dt * rs;
        s_dt = dt;
        s_rs = rs;
        s_gthr = a.guard * thrmin;
        s_sbase = 0;
        s_tbase = (a.t0p ? *a.t0p : a.t0) + kd * a.dt;
        const int nv = a.v_count[st];
        s_nv = nv;
        for (int q = 0; q < nv; ++q) {
            const int v = a.v_node[st * a.maxv + q];
            s_node[q] = v;
            s_vol[q] = a.v_vol[st * a.maxv + q];
            s_coef[q] = dt * a.Binv * a.leak[cs + v];
        }
        s_refac = (a.refactor_all || a.dirty[st] || a.fdt[st] != dt) ? 1 : 0;
        a.dirty[st] = 0;
        a.fdt[st] = dt;
    }
    __syncthreads();
    if (s_refac) {
        chain_factor<R, M, true>(a, s_dt, n, T, c, cb, cs, ps, 0);
    } else {
        const double dt = s_dt;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = c * M + k;
            a.beta[ps + (int64_t)k * T + c] = i < n ? (R)(dt * a.f[cs + i]) : R(0);
        }
    }

    R cp[M], cg[M], cbt[M], cpf[M], cpb[M], cth[M], g_next;
    unsigned vmask = 0u;
    auto load = [&]() {
        __syncthreads();
        vmask = 0u;
        for (int q = 0; q < s_nv; ++q)
            if (s_node[q] / M == c) vmask |= 1u << (s_node[q] % M);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int64_t pk = ps + (int64_t)k * T + c;
            const int i = c * M + k;
            cp[k] = a.alpha[pk];
            cg[k] = a.dtg[pk];
            cbt[k] = a.beta[pk];
            cpf[k] = a.Pf[pk];
            cpb[k] = a.Pb[pk];
            cth[k] = ((vmask >> k) & 1u) ? a.dtl[pk] : (i < n ? __double2float_rd(a.thr[cs + i]) : INFINITY);
        }
        g_next = c + 1 < T ? a.dtg[ps + c + 1] : R(0);
    };
    load();

    const unsigned full = 0xffffffffu;
    // warp-boundary stresses for the halo exchange are published before the
    // barrier that ends every step (and once here)
    if (lane == 31) sL[w] = sg[M - 1];
    if (lane == 0) sR[w] = sg[0];
    __syncthreads();
    for (int step = 0; step < n_steps; ++step) {
        // increment form: (C - dt A) d = dt (A s + f), s += d
        R left = __shfl_up_sync(full, sg[M - 1], 1);
        R right = __shfl_down_sync(full, sg[0], 1);
        if (lane == 0 && w > 0) left = sL[w - 1];
        if (lane == 31 && w + 1 < nw) right = sR[w + 1];
        R gk = cg[0];
        R qprev = gk * (left - sg[0]);
        R z = R(0);
        R zr[M];
        if (vmask == 0u) {                     // no void in this chunk (the common case)
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const R nxt = k + 1 < M ? sg[k + 1] : right;
                const R gk1 = k + 1 < M ? cg[k + 1] : g_next;
                const R qn = gk1 * (sg[k] - nxt);
                const R r = qprev - qn + cbt[k];
                z = cp[k] * fmx(gk, z, r);
                zr[k] = z;
                qprev = qn;
                gk = gk1;
            }
        } else {
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const R nxt = k + 1 < M ? sg[k + 1] : right;
                const R gk1 = k + 1 < M ? cg[k + 1] : g_next;
                const R qn = gk1 * (sg[k] - nxt);
                R r = qprev - qn + cbt[k];
                if ((vmask >> k) & 1u) r -= cth[k] * sg[k];
                z = cp[k] * fmx(gk, z, r);
                zr[k] = z;
                qprev = qn;
                gk = gk1;
            }
        }
        const R cf = scan_fwd<R>(z, cpf[M - 1], sA, sB, sC);
        R x = R(0);
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            const R gk1 = k + 1 < M ? cg[k + 1] : g_next;
            x = fmx(cp[k] * gk1, x, fmx(cpf[k], cf, zr[k]));
            zr[k] = x;
        }
        const R cr = scan_bwd<R>(x, cpb[0], sA, sB, sC);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const R y = fmx(cpb[k], cr, zr[k]) - cc[k];      // the step's increment, compensated
            const R t = sg[k] + y;
            cc[k] = (t - sg[k]) - y;
            sg[k] = t;
        }

        // void growth by the Robin leak
        if (vmask) {
            for (int q = 0; q < s_nv; ++q) {
                const int v = s_node[q];
                if (v / M == c) {
                    R val = R(0);
#pragma unroll
                    for (int k = 0; k < M; ++k)
                        if (v % M == k) val = sg[k];
                    s_vol[q] += s_coef[q] * (double)val;
                }
            }
        }
        // nucleation: every node against its own threshold (rounded down),
        // exact test in FP64 on a hit.  The barrier also publishes the
        // boundary stresses for the next step's halo.
        bool hit = false;
        if (vmask == 0u) {
#pragma unroll
            for (int k = 0; k < M; ++k) hit |= sg[k] >= cth[k];
        } else {
#pragma unroll
            for (int k = 0; k < M; ++k) hit |= !((vmask >> k) & 1u) && sg[k] >= cth[k];
        }
        if (lane == 31) sL[w] = sg[M - 1];
        if (lane == 0) sR[w] = sg[0];
        int refac_from = -1;
        if (__syncthreads_or(hit)) {
            double best = -INFINITY;
            int arg = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = c * M + k;
                if (i < n) {
                    const double m = (double)sg[k] - a.thr[cs + i];
                    if (m > best) { best = m; arg = i; }
                }
            }
            block_argmax(best, arg, sv, si);
            if (best >= 0.0) {
#pragma unroll
                for (int k = 0; k < M; ++k) a.sig[ps + (int64_t)k * T + c] = sg[k];
                __syncthreads();
                if (c == 0) {
                    const int v = arg;
                    const double dt = s_dt;
                    auto S_ = [&](int i) { return (double)a.sig[ps + (int64_t)(i % M) * T + i / M]; };
                    // previous-step stress at v from the BE relation M s^{k+1} = V s^k + dt f
                    const double gl = v > 0 ? a.g[cs + v] : 0.0, gr = v + 1 < n ? a.g[cs + v + 1] : 0.0;
                    double acc = (a.V[cb + v] + dt * (gl + gr)) * S_(v);
                    if (v > 0) acc -= dt * gl * S_(v - 1);
                    if (v + 1 < n) acc -= dt * gr * S_(v + 1);
                    const double s0 = (acc - dt * a.f[cs + v]) / a.V[cb + v];
                    const double m0 = s0 - a.thr[cs + v];
                    const double frac = m0 < 0.0 ? -m0 / (best - m0) : 0.0;
                    const int nv = s_nv;
                    if (nv < a.maxv) {
                        const int64_t e = st * a.maxv + nv;
                        a.v_node[e] = v;
                        a.v_seg[e] = void_segment<R>(a, s, cb + v);
                        a.v_tnuc[e] = s_tbase + ((double)(step - s_sbase) + frac) * dt;
                        a.v_vol[e] = 0.0;
                        s_node[nv] = v; s_vol[nv] = 0.0; s_coef[nv] = dt * a.Binv * a.leak[cs + v];
                        s_nv = nv + 1;
                        a.v_count[st] = nv + 1;
                        atomicAdd(&a.counters[0], 1);
                    } else {
                        atomicOr(&a.status[kStatusOverflow], 1);
                    }
                    a.thr[cs + v] = INFINITY;
                }
                refac_from = arg;
            }
        }
        bool promoted = false;
        if (s_rs > 1 && __syncthreads_or(near_guard<R, M>(sg, s_gthr))) {
            // coarse tree near its critical stress: finish this call with
            // the plain solver's fine steps and keep them
            n_steps = step + 1 + (n_steps - step - 1) * s_rs;
            promoted = true;
            __syncthreads();
            if (c == 0) {
                s_tbase += (double)(step + 1 - s_sbase) * s_dt;
                s_sbase = step + 1;
                s_dt = a.dt;
                s_rs = 1;
                a.sched[st] = 0;
                a.fdt[st] = a.dt;
                for (int q = 0; q < s_nv; ++q) s_coef[q] = a.dt * a.Binv * a.leak[cs + s_node[q]];
            }
            refac_from = 0;
        }
        if (refac_from >= 0) {
            const double dtf = promoted ? a.dt : s_dt;
            chain_factor<R, M, true>(a, dtf, n, T, c, cb, cs, ps, refac_from);
            tm = INFINITY;
            for (int i = c; i < n; i += T) tm = fmin(tm, a.thr[cs + i]);
            thrmin = block_min(tm, sv);
            if (c == 0) s_gthr = a.guard * thrmin;
            load();
        }
    }
#pragma unroll
    for (int k = 0; k < M; ++k) a.sig[ps + (int64_t)k * T + c] = sg[k];
    __syncthreads();
    if (c == 0) {
        for (int q = 0; q < s_nv; ++q) a.v_vol[st * a.maxv + q] = s_vol[q];
        atomicAdd(a.work, (unsigned long long)n * (unsigned long long)n_steps);
    }
}

// ---------------------------------------------------------------------------
// Branched trees: one thread per (tree, sample), leaf-to-root elimination.
// Packed layout == canonical order.  pinv holds 1/d', gam holds l = e/d',
// uu holds e, beta is the right-hand-side scratch.
// ---------------------------------------------------------------------------
template <typename R>
__device__ void tree_factor(const ChainArgs<R> &a, double dt, int n, int64_t cb, int64_t cs, int64_t ps) {
    for (int i = 0; i < n; ++i) {
        double d = a.V[cb + i] + (i > 0 ? dt * a.g[cs + i] : 0.0);
        if (isinf(a.thr[cs + i])) d += dt * a.leak[cs + i];
        a.pinv[ps + i] = d;
    }
    for (int i = 1; i < n; ++i) a.pinv[ps + (a.gpar[cb + i] - cb)] += dt * a.g[cs + i];
    for (int i = n - 1; i >= 1; --i) {
        const int q = (int)(a.gpar[cb + i] - cb);
        const double e = -dt * a.g[cs + i];
        const double l = e / a.pinv[ps + i];
        a.pinv[ps + q] -= l * e;
        a.gam[ps + i] = (R)l;
        a.uu[ps + i] = (R)e;
    }
    for (int i = 0; i < n; ++i) a.pinv[ps + i] = 1.0 / a.pinv[ps + i];
    if (sizeof(R) == 4) {
        // increment form: dt g of the face to the parent and dt leak at a void
        for (int i = 0; i < n; ++i) {
            a.dtg[ps + i] = i > 0 ? (R)(dt * a.g[cs + i]) : R(0);
            a.dtl[ps + i] = isinf(a.thr[cs + i]) ? (R)(dt * a.leak[cs + i]) : R(0);
        }
    }
}

template <typename R>
__global__ void k_tree(ChainArgs<R> a) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.n_bucket * a.S) return;
    const int t = a.trees[idx % a.n_bucket], s = (int)(idx / a.n_bucket);
    const int64_t cb = a.toff[t];
    const int n = (int)(a.toff[t + 1] - cb);
    const int64_t cs = (int64_t)s * a.N + cb, ps = (int64_t)s * a.P + a.pbase[t];
    const int64_t st = (int64_t)s * a.n_trees + t;
    const int sm = a.sched[st];
    if (a.kr_mode[st] || sm < 0) return;
    const int kd = a.kdone[st];
    double tcur = (a.t0p ? *a.t0p : a.t0) + kd * a.dt;
    double thrmin = INFINITY;
    for (int i = 0; i < n; ++i) thrmin = fmin(thrmin, a.thr[cs + i]);
    const double gthr = a.guard * thrmin;
    auto near = [&]() {
        for (int i = 0; i < n; ++i)
            if ((double)a.sig[ps + i] >= gthr) return true;
        return false;
    };
    int rs = sm > 1 ? sm : 1;
    if ((a.n_steps - kd) % rs) rs = 1;
    if (rs > 1 && near()) { rs = 1; a.sched[st] = 0; }
    double dt = a.dt * rs;
    int n_steps = (a.n_steps - kd) / rs;
    if (a.refactor_all || a.dirty[st] || a.fdt[st] != dt) {
        tree_factor<R>(a, dt, n, cb, cs, ps);
        a.dirty[st] = 0;
        a.fdt[st] = dt;
    }
    int nv = a.v_count[st];
    int step = 0;
    for (; step < n_steps; ++step) {
        R *r = a.beta + ps, *x = a.sig + ps;
        if constexpr (sizeof(R) == 4) {
            // increment form (C - dt A) d = dt (A s + f), s += d: the residual
            // from face fluxes (each face's flux added to one end and taken
            // from the other), so the rounding of the FP32 factors touches
            // only the increment and the conserved slow modes stay exact
            for (int i = 0; i < n; ++i) r[i] = (R)(dt * a.f[cs + i]) - a.dtl[ps + i] * x[i];
            for (int i = 1; i < n; ++i) {
                const int q = (int)(a.gpar[cb + i] - cb);
                const R fl = a.dtg[ps + i] * (x[q] - x[i]);
                r[i] += fl;
                r[q] -= fl;
            }
            for (int i = n - 1; i >= 1; --i) {
                const int q = (int)(a.gpar[cb + i] - cb);
                r[q] -= a.gam[ps + i] * r[i];
            }
            r[0] = (R)((double)r[0] * a.pinv[ps]);
            for (int i = 1; i < n; ++i) {
                const int q = (int)(a.gpar[cb + i] - cb);
                r[i] = (R)(((double)r[i] - (double)a.uu[ps + i] * (double)r[q]) * a.pinv[ps + i]);
            }
            for (int i = 0; i < n; ++i) x[i] += r[i];
        } else {
            for (int i = 0; i < n; ++i) r[i] = (R)(a.V[cb + i] * (double)x[i] + dt * a.f[cs + i]);
            for (int i = n - 1; i >= 1; --i) {
                const int q = (int)(a.gpar[cb + i] - cb);
                r[q] -= a.gam[ps + i] * r[i];
            }
            x[0] = (R)((double)r[0] * a.pinv[ps]);
            for (int i = 1; i < n; ++i) {
                const int q = (int)(a.gpar[cb + i] - cb);
                x[i] = (R)(((double)r[i] - (double)a.uu[ps + i] * (double)x[q]) * a.pinv[ps + i]);
            }
        }
        for (int q = 0; q < nv; ++q) {
            const int64_t e = st * a.maxv + q;
            const int v = a.v_node[e];
            a.v_vol[e] += dt * a.Binv * a.leak[cs + v] * (double)x[v];
        }
        double best = -INFINITY;
        int arg = -1;
        for (int i = 0; i < n; ++i) {
            const double m = (double)x[i] - a.thr[cs + i];
            if (m > best) { best = m; arg = i; }
        }
        if (arg >= 0 && best >= 0.0) {
            const int v = arg;
            // previous-step stress at v from the BE relation
            double diag = a.V[cb + v], acc = 0.0;
            if (v > 0) {
                const int q = (int)(a.gpar[cb + v] - cb);
                diag += dt * a.g[cs + v];
                acc -= dt * a.g[cs + v] * (double)x[q];
            }
            for (int k = a.child_ptr[cb + v]; k < a.child_ptr[cb + v + 1]; ++k) {
                const int ch = (int)(a.child_gidx[k] - cb);
                diag += dt * a.g[cs + ch];
                acc -= dt * a.g[cs + ch] * (double)x[ch];
            }
            acc += diag * (double)x[v];
            const double s0 = (acc - dt * a.f[cs + v]) / a.V[cb + v];
            const double m0 = s0 - a.thr[cs + v];
            const double frac = m0 < 0.0 ? -m0 / (best - m0) : 0.0;
            if (nv < a.maxv) {
                const int64_t e = st * a.maxv + nv;
                a.v_node[e] = v;
                a.v_seg[e] = void_segment<R>(a, s, cb + v);
                a.v_tnuc[e] = tcur + frac * dt;
                a.v_vol[e] = 0.0;
                ++nv;
                a.v_count[st] = nv;
                atomicAdd(&a.counters[0], 1);
            } else {
                atomicOr(&a.status[kStatusOverflow], 1);
            }
            a.thr[cs + v] = INFINITY;
            tree_factor<R>(a, dt, n, cb, cs, ps);
        }
        tcur += dt;
        if (rs > 1 && near()) {
            n_steps = step + 1 + (n_steps - step - 1) * rs;
            rs = 1;
            dt = a.dt;
            a.sched[st] = 0;
            a.fdt[st] = dt;
            tree_factor<R>(a, dt, n, cb, cs, ps);
        }
    }
    atomicAdd(a.work, (unsigned long long)n * (unsigned long long)step);
}

// ---------------------------------------------------------------------------
// Void growth resistance and the steady-state screen
// ---------------------------------------------------------------------------
__global__ void k_reset_R(int n_seg, int S, const double *R0, double *R) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)n_seg * S;
         k += (int64_t)gridDim.x * blockDim.x)
        R[k] = R0[k % n_seg];
}

// one thread per (sample, tree): a tree's voids degrade only its own segments
// (late failure); a void past the critical volume at an IR node with a via up
// to a higher layer also opens that via (early failure, explicit vias only)
__global__ void k_void_R(int n_trees, int S, int maxv, int n_seg, const int32_t *v_count, const int32_t *v_seg,
                         const int32_t *v_node, const double *v_vol, const double *W, const double *H,
                         double rho_Ta, double h_Ta, double rho_Cu, const int64_t *toff, const int32_t *ir_id,
                         const int32_t *up_via, double *R) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n_trees * S) return;
    const int s = (int)(k / n_trees), t = (int)(k % n_trees);
    for (int q = 0; q < v_count[k]; ++q) {
        const int sg = v_seg[k * maxv + q];
        const double w = W[sg], h = H[sg];
        const double coef = rho_Ta / (h_Ta * (2.0 * h + w)) - rho_Cu / (h * w);
        const double vol = v_vol[k * maxv + q];
        const double dR = (vol - w * w * h) / (w * h) * coef;
        if (dR > 0.0) R[(int64_t)s * n_seg + sg] += dR;
        const int irn = ir_id[toff[t] + v_node[k * maxv + q]];
        if (irn >= 0 && up_via[irn] >= 0 && vol > w * w * h) R[(int64_t)s * n_seg + up_via[irn]] = kOpenCircuit;
    }
}

__global__ void k_count_changed(int64_t n, const double *R, double *R_prev, int32_t *counter) {
    int local = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (R[k] != R_prev[k]) { ++local; R_prev[k] = R[k]; }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(counter, local);
}

// steady state per (sample, tree): sigma_child - sigma_parent = dx G, constant
// from sum V (sigma - sigma_T) = 0; mortal iff some sigma_ss > sigma_crit
__global__ void k_screen(int n_trees, int S, int64_t N, int n_seg, double sfac_em, double sigma_T,
                         const int64_t *toff, const int32_t *gpar, const int32_t *face_seg, const int8_t *sign,
                         const double *dx, const double *Mface, const double *V, const double *j,
                         const double *thr0, double *ss, uint8_t *mortal, double *ssmax) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n_trees * S) return;
    const int s = (int)(k / n_trees), t = (int)(k % n_trees);
    const int64_t cb = toff[t], n = toff[t + 1] - cb, cs = (int64_t)s * N + cb;
    const double *js = j + (int64_t)s * n_seg;
    double sv = V[cb], svp = 0.0;
    ss[cs] = 0.0;
    for (int64_t i = 1; i < n; ++i) {
        const int64_t gi = cb + i;
        const double G = sfac_em * sign[gi] * js[face_seg[gi]] + Mface[(int64_t)s * N + gi];
        const double Pi = ss[(int64_t)s * N + gpar[gi]] + dx[gi] * G;
        ss[cs + i] = Pi;
        sv += V[gi];
        svp += V[gi] * Pi;
    }
    const double mean = svp / sv;
    double mx = -INFINITY;
    uint8_t mort = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double v = sigma_T + ss[cs + i] - mean;
        ss[cs + i] = v;
        mx = fmax(mx, v);
        if (v > thr0[cs + i]) mort = 1;
    }
    mortal[k] = mort;
    ssmax[k] = mx;
}

template <typename R>
ChainArgs<R> chain_args(ems_ctx *c, double dt, int n_steps) {
    Dev &d = c->d;
    ChainArgs<R> a;
    a.toff = d.toff; a.pbase = d.pbase; a.N = c->N; a.P = c->P;
    a.n_trees = c->n_trees; a.maxv = c->maxv; a.n_steps = n_steps; a.S = c->S;
    a.refactor_all = (dt != c->factored_dt) ? 1 : 0;
    a.dt = dt; a.t0 = c->t; a.Binv = 1.0 / c->prm.B_modulus;
    a.V = d.V; a.g = d.g; a.leak = d.leak; a.f = d.f; a.thr = d.thr;
    a.sig = (R *)d.sig; a.alpha = (R *)d.alpha; a.beta = (R *)d.beta; a.gam = (R *)d.gam;
    a.uu = (R *)d.uu; a.Pf = (R *)d.Pf; a.Pb = (R *)d.Pb; a.pinv = (double *)d.pinv;
    a.dtg = (R *)d.dtg; a.dtl = (R *)d.dtl; a.kc = (R *)d.kc;
    a.v_count = d.v_count; a.v_node = d.v_node; a.v_seg = d.v_seg; a.v_vol = d.v_vol; a.v_tnuc = d.v_tnuc;
    a.dirty = d.dirty; a.j = d.j; a.n_seg = c->n_seg; a.face_seg = d.face_seg; a.inc_ptr = d.inc_ptr;
    a.inc_seg = d.inc_seg; a.gpar = d.par; a.child_ptr = d.child_ptr; a.child_gidx = d.child_idx;
    a.status = d.status; a.counters = d.counters;
    a.kr_mode = d.kr_mode; a.kdone = d.kdone; a.sched = d.sched; a.fdt = d.fdt;
    a.guard = c->sched_guard; a.work = d.work;
    a.t0p = c->graph_capturing ? d.gtime : nullptr;
    return a;
}

template <typename R, int M, bool D, bool SM>
cudaError_t launch_chain(dim3 grid, int T, size_t smem, cudaStream_t st, const ChainArgs<R> &a) {
    if constexpr (SM && !D) {
        return cudaErrorInvalidValue;                 // no shared-memory variant of the state form
    } else {
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(k_chain<R, M, D, SM>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_chain<R, M, D, SM><<<grid, T, smem, st>>>(a);
        return cudaGetLastError();
    }
}

// One bucket's launch over S samples: the kernel its shape names.  FP64
// solves the state directly; FP32 solves for the increment so that the
// rounding of its coefficients cannot drift the conserved slow modes.
template <typename R>
cudaError_t launch_bucket_raw(ems_ctx *c, const Bucket &b, ChainArgs<R> a, int S) {
    constexpr bool kDelta = sizeof(R) == 4;
    a.trees = b.d_trees;
    a.n_bucket = (int)b.trees.size();
    a.S = S;
    ++c->launches;
    if (!b.chain) {
        const int64_t items = (int64_t)b.trees.size() * S;   // (tree, sample) pairs
        k_tree<R><<<(unsigned)((items + 63) / 64), 64, 0, c->stream>>>(a);
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)b.trees.size(), S);
    cudaError_t e = cudaSuccess;
    switch (b.kind) {
        case EMS_CHAIN_CLUSTER:             // one thread-block cluster of CL CTAs per (tree, sample)
            if (b.CL < 2 || b.T % b.CL) return cudaErrorInvalidValue;
            e = launch_cluster(b.M, b.CL, b.T / b.CL, (unsigned)b.trees.size(), S, c->stream, a);
            break;
        case EMS_CHAIN_CLUSTER_SHARED:      // the same, coefficients in shared memory (FP32)
            if constexpr (kDelta) {
                if (b.CL < 2 || b.T % b.CL) return cudaErrorInvalidValue;
                e = launch_cluster_smem(b.M, b.CL, b.T / b.CL, (unsigned)b.trees.size(), S, c->stream, a);
                break;
            } else {
                return cudaErrorInvalidValue;
            }

        case EMS_CHAIN_REGISTER:
            if constexpr (kDelta) {
                if (b.T > reg_max_threads(b.M)) return cudaErrorInvalidValue;
                if (b.M == 4) k_chain_reg<4><<<grid, b.T, 0, c->stream>>>(a);
                else if (b.M == 8) k_chain_reg<8><<<grid, b.T, 0, c->stream>>>(a);
                else if (b.M == 16) k_chain_reg<16><<<grid, b.T, 0, c->stream>>>(a);
                else return cudaErrorInvalidValue;
                e = cudaGetLastError();
                break;
            } else {
                return cudaErrorInvalidValue;      // the register chain kernel is FP32 only
            }
        case EMS_CHAIN_SHARED:
        case EMS_CHAIN_GLOBAL: {
            // increment form: the chunk coefficients in shared memory (SHARED),
            // else the forward sweep staged there (8 bytes per node)
            const bool smc = b.kind == EMS_CHAIN_SHARED;
            if (smc && !kDelta) return cudaErrorInvalidValue;   // the shared-memory kernel is FP32 only
            const size_t smem = smc ? 5 * sizeof(R) * (size_t)b.T * b.M
                                    : (kDelta ? sizeof(float2) * (size_t)b.T * b.M : 0);
            if (smc && smem > kSharedCoefBytes) return cudaErrorInvalidValue;
            switch (b.M) {
                case 4: e = smc ? launch_chain<R, 4, kDelta, true>(grid, b.T, smem, c->stream, a)
                                : launch_chain<R, 4, kDelta, false>(grid, b.T, smem, c->stream, a); break;
                case 8: e = smc ? launch_chain<R, 8, kDelta, true>(grid, b.T, smem, c->stream, a)
                                : launch_chain<R, 8, kDelta, false>(grid, b.T, smem, c->stream, a); break;
                case 16: e = smc ? launch_chain<R, 16, kDelta, true>(grid, b.T, smem, c->stream, a)
                                 : launch_chain<R, 16, kDelta, false>(grid, b.T, smem, c->stream, a); break;
                case 32: e = smc ? launch_chain<R, 32, kDelta, true>(grid, b.T, smem, c->stream, a)
                                 : launch_chain<R, 32, kDelta, false>(grid, b.T, smem, c->stream, a); break;
                case 64: e = smc ? launch_chain<R, 64, kDelta, true>(grid, b.T, smem, c->stream, a)
                                 : launch_chain<R, 64, kDelta, false>(grid, b.T, smem, c->stream, a); break;
                default: return cudaErrorInvalidValue;
            }
            break;
        }
        default: return cudaErrorInvalidValue;
    }
    return e;
}

template <typename R>
ems_status launch_bucket(ems_ctx *c, const Bucket &b, ChainArgs<R> a, int S) {
    const cudaError_t e = launch_bucket_raw<R>(c, b, a, S);
    if (e != cudaSuccess) {
        char what[96];
        snprintf(what, sizeof what, "chain launch (kernel %d, M %d, T %d, CL %d)", b.kind, b.M, b.T, b.CL);
        return cuda_check(c, e, what);
    }
    return EMS_OK;
}

template <typename R>
ems_status launch_advance(ems_ctx *c, double dt, int n_steps) {
    for (auto &b : c->buckets) EMS_TRY(launch_bucket<R>(c, b, chain_args<R>(c, dt, n_steps), c->S));
    return EMS_OK;
}

inline dim3 grid_1d(int64_t n, int S) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return dim3((unsigned)b, (unsigned)S);
}

// ---------------------------------------------------------------------------
// Shape autotuner.  Each candidate shape of a bucket's chains runs on scratch
// copies (stress repacked into the candidate's layout; thresholds, voids and
// schedules copied), so the context's state is never touched.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_repack(const int32_t *trees, const int64_t *toff, const int64_t *pb_src, int T_src, int M_src,
                         int64_t P_src, const int64_t *pb_dst, const int32_t *T_dst, int M_dst, int64_t P_dst,
                         const R *src, R *dst) {
    const int t = trees[blockIdx.x];
    const int64_t s = blockIdx.y;
    const int64_t n = toff[t + 1] - toff[t];
    const int Td = T_dst[t];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        dst[s * P_dst + pb_dst[t] + (i % M_dst) * Td + i / M_dst] =
            src[s * P_src + pb_src[t] + (i % M_src) * T_src + i / M_src];
}

struct TuneShape { int kind, M, CL; };

// Time one shape on the bucket's chains over the first S mapped samples: a
// launch that factorises and runs n_steps steps, then n_steps more timed.
// *ms < 0: some chain of the bucket cannot take the shape.
template <typename R>
ems_status tune_time(ems_ctx *c, const Bucket &b, const TuneShape &sh, int S, double dt, int n_steps, double *ms) {
    const int nt = c->n_trees, maxv = c->maxv, prec = c->prm.precision;
    const int64_t N = c->N;
    std::vector<int64_t> pb(nt, 0);
    std::vector<int32_t> Tt(nt, 0);
    std::map<int, std::vector<int32_t>> groups;    // chains of equal team size launch together
    int64_t P = 0;
    for (int32_t t : b.trees) {
        const int64_t n = c->trees.off[t + 1] - c->trees.off[t];
        int T = 0;
        if (!shape_valid(n, prec, sh.kind, sh.M, sh.CL, &T)) { *ms = -1.0; return EMS_OK; }
        pb[t] = P; Tt[t] = T; P += (int64_t)T * sh.M;
        groups[T].push_back(t);
    }
    const size_t ts = (size_t)S * nt, L = (size_t)S * P;
    size_t bytes = 0;
    auto take = [&](size_t n) { const size_t o = bytes; bytes += (n + 255) / 256 * 256; return o; };
    const size_t o_pk = take(10 * L * sizeof(R)), o_pinv = take(L * 8), o_thr = take((size_t)S * N * 8);
    const size_t o_vc = take(ts * 4), o_vn = take(ts * maxv * 4), o_vs = take(ts * maxv * 4);
    const size_t o_vv = take(ts * maxv * 8), o_vt = take(ts * maxv * 8);
    const size_t o_dirty = take(ts * 4), o_sched = take(ts * 4), o_fdt = take(ts * 8), o_kr = take(ts * 4);
    const size_t o_kd = take(ts * 4), o_misc = take(64 * 4 + 8), o_pb = take((size_t)nt * 8), o_T = take((size_t)nt * 4);
    const size_t o_tr = take(b.trees.size() * 4);
    size_t fr = 0, tot = 0;
    EMS_CUDA(c, cudaMemGetInfo(&fr, &tot));
    if (bytes > fr / 10 * 9) return fail(c, EMS_E_NOMEM, "autotuner scratch does not fit: lower max_samples");
    char *base = nullptr;
    EMS_CUDA(c, cudaMalloc(&base, bytes));
    cudaStream_t st = c->stream;
    Dev &d = c->d;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ems_status rc = EMS_OK;
    auto run = [&]() -> ems_status {
        EMS_CUDA(c, cudaMemsetAsync(base, 0, bytes, st));
        const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice, hd = cudaMemcpyHostToDevice;
        EMS_CUDA(c, cudaMemcpyAsync(base + o_thr, d.thr, (size_t)S * N * 8, dd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_vc, d.v_count, ts * 4, dd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_vn, d.v_node, ts * maxv * 4, dd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_vs, d.v_seg, ts * maxv * 4, dd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_vv, d.v_vol, ts * maxv * 8, dd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_vt, d.v_tnuc, ts * maxv * 8, dd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_sched, d.sched, ts * 4, dd, st));
        const std::vector<int32_t> ones(ts, 1);
        const std::vector<double> nofdt(ts, -1.0);
        EMS_CUDA(c, cudaMemcpyAsync(base + o_dirty, ones.data(), ts * 4, hd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_fdt, nofdt.data(), ts * 8, hd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_pb, pb.data(), (size_t)nt * 8, hd, st));
        EMS_CUDA(c, cudaMemcpyAsync(base + o_T, Tt.data(), (size_t)nt * 4, hd, st));
        std::vector<Bucket> gb;
        std::vector<int32_t> order;
        for (auto &kv : groups) {
            Bucket g;
            g.chain = true; g.T = kv.first; g.M = sh.M; g.CL = sh.CL; g.kind = sh.kind; g.trees = kv.second;
            g.d_trees = (int32_t *)(base + o_tr) + order.size();
            order.insert(order.end(), kv.second.begin(), kv.second.end());
            gb.push_back(std::move(g));
        }
        EMS_CUDA(c, cudaMemcpyAsync(base + o_tr, order.data(), order.size() * 4, hd, st));
        R *pk = (R *)(base + o_pk);
        k_repack<R><<<dim3((unsigned)b.trees.size(), S), 256, 0, st>>>(
            b.d_trees, d.toff, d.pbase, b.T, b.M, c->P, (const int64_t *)(base + o_pb), (const int32_t *)(base + o_T),
            sh.M, P, (const R *)d.sig, pk);
        ++c->launches;
        EMS_CUDA(c, cudaGetLastError());
        ChainArgs<R> a = chain_args<R>(c, dt, n_steps);
        a.pbase = (const int64_t *)(base + o_pb); a.P = P;
        a.sig = pk; a.alpha = pk + L; a.beta = pk + 2 * L; a.gam = pk + 3 * L; a.uu = pk + 4 * L;
        a.Pf = pk + 5 * L; a.Pb = pk + 6 * L; a.dtg = pk + 7 * L; a.dtl = pk + 8 * L; a.kc = pk + 9 * L;
        a.pinv = (double *)(base + o_pinv);
        a.thr = (double *)(base + o_thr);
        a.v_count = (int32_t *)(base + o_vc); a.v_node = (int32_t *)(base + o_vn); a.v_seg = (int32_t *)(base + o_vs);
        a.v_vol = (double *)(base + o_vv); a.v_tnuc = (double *)(base + o_vt);
        a.dirty = (int32_t *)(base + o_dirty); a.sched = (int32_t *)(base + o_sched); a.fdt = (double *)(base + o_fdt);
        a.kr_mode = (const int32_t *)(base + o_kr); a.kdone = (const int32_t *)(base + o_kd);
        int32_t *misc = (int32_t *)(base + o_misc);
        a.status = misc; a.counters = misc + 32; a.work = (unsigned long long *)(misc + 64);
        a.refactor_all = 0;               // the first launch factorises every chain (dirty)
        a.t0p = nullptr;
        for (const Bucket &g : gb) {
            // a shape the device cannot launch (a configuration error; the
            // context stays usable) is skipped, not an error of the tuner
            const cudaError_t le = launch_bucket_raw<R>(c, g, a, S);
            if (le == cudaErrorInvalidValue || le == cudaErrorInvalidConfiguration ||
                le == cudaErrorLaunchOutOfResources || le == cudaErrorInvalidClusterSize) {
                (void)cudaGetLastError();
                *ms = -1.0;
                return EMS_OK;
            }
            EMS_CUDA(c, le);
        }
        EMS_CUDA(c, cudaEventCreate(&e0));
        EMS_CUDA(c, cudaEventCreate(&e1));
        EMS_CUDA(c, cudaEventRecord(e0, st));
        for (const Bucket &g : gb) EMS_TRY(launch_bucket<R>(c, g, a, S));
        EMS_CUDA(c, cudaEventRecord(e1, st));
        EMS_CUDA(c, cudaEventSynchronize(e1));
        float t = 0.f;
        EMS_CUDA(c, cudaEventElapsedTime(&t, e0, e1));
        *ms = t;
        return EMS_OK;
    };
    rc = run();
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(base);
    return rc;
}

template <typename R>
ems_status autotune_run(ems_ctx *c, int n_steps, int max_samples, ems_chain_rule *rules, double *ms,
                        double *ms_default, int cap, int *n_rules) {
    const double dt = c->prm.horizon / ((double)c->prm.n_outer * c->prm.n_inner);
    const int S = std::min(max_samples, c->S), prec = c->prm.precision;
    int k = 0;
    c->tune_log.clear();
    auto log = [&](const TuneShape &sh, int64_t lo, int64_t hi, double t_ms, int grp) {
        int T = 0;
        shape_valid(hi, prec, sh.kind, sh.M, sh.CL, &T);
        c->tune_log.push_back(ems_ctx::TuneRec{ems_chain_rule{lo, hi, sh.kind, sh.M, sh.CL, T}, t_ms, grp});
    };
    for (const Bucket &b : c->buckets) {
        if (!b.chain) continue;
        if (k >= cap) break;
        int64_t lo = LLONG_MAX, hi = 0;
        for (int32_t t : b.trees) {
            const int64_t n = c->trees.off[t + 1] - c->trees.off[t];
            lo = std::min(lo, n);
            hi = std::max(hi, n);
        }
        const TuneShape cur{b.kind, b.M, b.CL};
        double def_ms = -1.0;
        EMS_TRY(tune_time<R>(c, b, cur, S, dt, n_steps, &def_ms));
        log(cur, lo, hi, def_ms, k);
        TuneShape best = cur;
        double best_ms = def_ms;
        for (const ems_chain_rule &r : shape_candidates(hi, prec)) {
            if (r.kind == cur.kind && r.M == cur.M && r.CL == cur.CL) continue;
            double t_ms = -1.0;
            EMS_TRY(tune_time<R>(c, b, TuneShape{r.kind, r.M, r.CL}, S, dt, n_steps, &t_ms));
            log(TuneShape{r.kind, r.M, r.CL}, lo, hi, t_ms, k);
            if (t_ms >= 0.0 && t_ms < best_ms) { best = TuneShape{r.kind, r.M, r.CL}; best_ms = t_ms; }
        }
        // a change of shape has to beat the current one by 3 %, more than the timing noise
        if (best_ms > 0.97 * def_ms) { best = cur; best_ms = def_ms; }
        int T = 0;
        shape_valid(hi, prec, best.kind, best.M, best.CL, &T);
        rules[k] = ems_chain_rule{lo, hi, best.kind, best.M, best.CL, T};
        if (ms) ms[k] = best_ms;
        if (ms_default) ms_default[k] = def_ms;
        ++k;
    }
    *n_rules = k;
    return EMS_OK;
}

}  // namespace

ems_status node_physics(ems_ctx *c) {
    Dev &d = c->d;
    const ems_params &p = c->prm;
    cudaStream_t st = c->stream;
    if (!c->joule) {           // a Joule-heating profile, once set, stays until a new map
        k_temperature<<<grid_1d(c->N, 1), 256, 0, st>>>(c->N, d.nx_, d.ny_, d.raster, c->rnx, c->rny, c->rx0,
                                                        c->ry0, c->rx1, c->ry1, p.T0, d.Tn);
        ++c->launches;
        EMS_CUDA(c, cudaGetLastError());
    }
    EMS_TRY(face_base(c));
    return sample_physics(c);
}

namespace {
PhysArgs phys_args(ems_ctx *c) {
    Dev &d = c->d;
    const ems_params &p = c->prm;
    PhysArgs a;
    a.N = c->N; a.n_seg = c->n_seg; a.gpar = d.par; a.face_seg = d.face_seg; a.owner_seg = d.owner_seg;
    a.child_ptr = d.child_ptr; a.child_gidx = d.child_idx; a.Tn = d.Tn; a.dx = d.face_dx; a.area = d.face_area;
    a.kfac = d.kfac; a.sfac = d.sfac; a.D0 = p.D0;
    a.pert = d.pert; a.nx = d.nx_; a.ny = d.ny_; a.pnx = c->pnx; a.pny = c->pny;
    a.px0 = c->rx0; a.py0 = c->ry0; a.px1 = c->rx1; a.py1 = c->ry1; a.Ea = p.Ea; a.kB = p.k_B; a.B = p.B_modulus;
    a.Omega = p.Omega; a.Qs = p.Q_star; a.delta = p.delta; a.sigma_crit = p.sigma_crit;
    a.kap_a = d.kap_a; a.g = d.g; a.Mface = d.Mface; a.V = d.V; a.leak = d.leak; a.thr0 = d.thr0; a.thr = d.thr;
    a.fb_ka = d.fb_ka; a.fb_g = d.fb_g; a.fb_M = d.fb_M;
    return a;
}
}  // namespace

ems_status face_base(ems_ctx *c) {
    k_face_base<<<grid_1d(c->N, 1), 256, 0, c->stream>>>(phys_args(c));
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

// kappa a, conductances, TM term, volumes, leak and thresholds of the mapped
// samples from the node temperatures and the per-segment factors; voids
// raise their node's threshold to +inf and mark the tree for a refactor
ems_status sample_physics(ems_ctx *c) {
    Dev &d = c->d;
    cudaStream_t st = c->stream;
    const PhysArgs a = phys_args(c);
    k_faces<<<grid_1d(c->N, c->S), 256, 0, st>>>(a);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    k_nodes<<<grid_1d(c->N, c->S), 256, 0, st>>>(a);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    const int64_t ts = (int64_t)c->n_trees * c->S;
    k_apply_voids<<<(unsigned)((ts + 255) / 256), 256, 0, st>>>(c->n_trees, c->S, c->maxv, c->N, d.toff,
                                                                d.v_count, d.v_node, d.thr, d.dirty);
    if (d.kr_state) EMS_CUDA(c, cudaMemsetAsync(d.kr_state, 0, sizeof(int32_t) * ts, st));
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status forcing(ems_ctx *c) {
    Dev &d = c->d;
    const ems_params &p = c->prm;
    const double sem = p.e_charge * p.Z_star * p.rho_Cu / p.Omega;
    k_forcing<<<grid_1d(c->N, c->S), 256, 0, c->stream>>>(c->N, c->n_seg, sem, d.par, d.face_seg, d.face_sign,
                                                          d.child_ptr, d.child_idx, d.Mface, d.kap_a, d.j, d.f);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status launch_be(ems_ctx *c, double dt, int n_steps) {
    if (c->prm.precision == EMS_F32) {
        EMS_TRY(launch_advance<float>(c, dt, n_steps));
    } else {
        EMS_TRY(launch_advance<double>(c, dt, n_steps));
    }
    c->factored_dt = dt;
    return EMS_OK;
}

ems_status advance(ems_ctx *c, double dt, int n_steps, int *n_new, int method) {
    if (method != EMS_BE) return krylov_advance(c, dt, n_steps, method, n_new);
    EMS_CUDA(c, cudaMemsetAsync(c->d.counters, 0, sizeof(int32_t), c->stream));
    EMS_CUDA(c, cudaMemsetAsync(c->d.kr_mode, 0, sizeof(int32_t) * c->S * c->n_trees, c->stream));
    EMS_CUDA(c, cudaMemsetAsync(c->d.kdone, 0, sizeof(int32_t) * c->S * c->n_trees, c->stream));
    EMS_TRY(launch_be(c, dt, n_steps));
    c->t += dt * n_steps;
    if (n_new) {
        EMS_CUDA(c, cudaMemcpyAsync(n_new, c->d.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    }
    return EMS_OK;
}

ems_status void_update(ems_ctx *c, int *n_changed) {
    Dev &d = c->d;
    const ems_params &p = c->prm;
    cudaStream_t st = c->stream;
    const int64_t nsS = (int64_t)c->n_seg * c->S;
    k_reset_R<<<grid_1d(nsS, 1), 256, 0, st>>>(c->n_seg, c->S, d.seg_R0, d.R);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    const int64_t ts = (int64_t)c->n_trees * c->S;
    k_void_R<<<(unsigned)((ts + 255) / 256), 256, 0, st>>>(c->n_trees, c->S, c->maxv, c->n_seg, d.v_count,
                                                           d.v_seg, d.v_node, d.v_vol, d.seg_W, d.seg_H, p.rho_Ta,
                                                           p.h_Ta, p.rho_Cu, d.toff, d.ir_id, d.up_via, d.R);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    EMS_CUDA(c, cudaMemsetAsync(d.counters + 1, 0, sizeof(int32_t), st));
    k_count_changed<<<grid_1d(nsS, 1), 256, 0, st>>>(nsS, d.R, d.R_prev, d.counters + 1);
    EMS_CUDA(c, cudaGetLastError());
    if (n_changed)
        EMS_CUDA(c, cudaMemcpyAsync(n_changed, d.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return EMS_OK;
}

ems_status screen(ems_ctx *c) {
    Dev &d = c->d;
    const ems_params &p = c->prm;
    const double sem = p.e_charge * p.Z_star * p.rho_Cu / p.Omega;
    const int64_t ts = (int64_t)c->n_trees * c->S;
    k_screen<<<(unsigned)((ts + 63) / 64), 64, 0, c->stream>>>(c->n_trees, c->S, c->N, c->n_seg, sem, p.sigma_T,
                                                               d.toff, d.par, d.face_seg, d.face_sign, d.face_dx,
                                                               d.Mface, d.V, d.j, d.thr0, d.sig_ss, d.mortal,
                                                               d.ssmax);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status pack_sigma(ems_ctx *c, bool to_packed) {
    Dev &d = c->d;
    dim3 grid(c->n_trees, c->S);
    if (c->prm.precision == EMS_F32)
        k_pack<float><<<grid, 256, 0, c->stream>>>(c->n_trees, c->N, c->P, d.toff, d.pbase, d.pT, d.pM, d.sig_ss,
                                                   (float *)d.sig, to_packed ? 1 : 0, 0.0);
    else
        k_pack<double><<<grid, 256, 0, c->stream>>>(c->n_trees, c->N, c->P, d.toff, d.pbase, d.pT, d.pM, d.sig_ss,
                                                    (double *)d.sig, to_packed ? 1 : 0, 0.0);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

ems_status init_sigma(ems_ctx *c) {
    Dev &d = c->d;
    dim3 grid(c->n_trees, c->S);
    if (c->prm.precision == EMS_F32)
        k_pack<float><<<grid, 256, 0, c->stream>>>(c->n_trees, c->N, c->P, d.toff, d.pbase, d.pT, d.pM, d.sig_ss,
                                                   (float *)d.sig, 2, c->prm.sigma_T);
    else
        k_pack<double><<<grid, 256, 0, c->stream>>>(c->n_trees, c->N, c->P, d.toff, d.pbase, d.pT, d.pM, d.sig_ss,
                                                    (double *)d.sig, 2, c->prm.sigma_T);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

}  // namespace ems

using namespace ems;

extern "C" ems_status ems_set_thermal_map(ems_ctx *c, const double *T, int nx, int ny, double x0, double y0,
                                          double x1, double y1) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (T) {
        if (nx < 2 || ny < 2 || (int64_t)nx * ny > EMS_MAX_RASTER || !(x1 > x0) || !(y1 > y0))
            return fail(c, EMS_E_INVAL, "thermal raster must be 2x2..1024x1024 over a positive extent");
        for (int64_t k = 0; k < (int64_t)nx * ny; ++k)
            if (!(std::isfinite(T[k]) && T[k] > 0.0)) return fail(c, EMS_E_INVAL, "non-positive temperature");
        EMS_CUDA(c, cudaMemcpyAsync(c->d.raster, T, sizeof(double) * nx * ny, cudaMemcpyHostToDevice, c->stream));
        c->rnx = nx; c->rny = ny; c->rx0 = x0; c->ry0 = y0; c->rx1 = x1; c->ry1 = y1;
    } else {
        c->rnx = 0; c->rny = 0;
        c->pnx = c->pny = 0;                    // perturbations live on the map's extent
    }
    c->joule = false;
    if (windowed(c)) {
        // the per-node coefficients are rebuilt for every window before use;
        // here the temperatures, and the first window's coefficients
        map_window(c, 0, c->W);
        ems_status s = node_physics(c);
        map_all(c);
        EMS_TRY(s);
    } else {
        EMS_TRY(node_physics(c));
    }
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_stress_advance(ems_ctx *c, double dt, int n_steps, int method, int *n_new_voids) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "stress advance before the first IR solve");
    if (!(dt > 0.0) || n_steps < 0) return fail(c, EMS_E_INVAL, "dt must be > 0 and n_steps >= 0");
    if (method != EMS_BE && method != EMS_KRYLOV && method != EMS_AUTO)
        return fail(c, EMS_E_INVAL, "unknown method");
    if (method != EMS_BE && c->rmax == 0)
        return fail(c, EMS_E_STATE, "Krylov method needs a context created with method EMS_KRYLOV or EMS_AUTO");
    if (windowed(c) && method != EMS_BE)
        return fail(c, EMS_E_STATE, "the reduced models need every sample's coefficients (window_samples 0)");
    const double t0 = c->t;
    std::vector<int> nn((size_t)(c->S_all + c->W - 1) / c->W, 0);
    EMS_TRY(each_window(c, [&](int s0, int) -> ems_status {
        c->t = t0;
        EMS_TRY(window_derive(c));
        EMS_TRY(forcing(c));
        return advance(c, dt, n_steps, &nn[(size_t)s0 / c->W], method);
    }));
    EMS_TRY(check_status(c));
    if (n_new_voids) {
        int tot = 0;
        for (int v : nn) tot += v;
        *n_new_voids = tot;
    }
    return EMS_OK;
}

extern "C" ems_status ems_void_update(ems_ctx *c, int *n_segments_changed) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    int nc = 0;
    EMS_TRY(void_update(c, &nc));
    EMS_TRY(check_status(c));
    if (n_segments_changed) *n_segments_changed = nc;
    return EMS_OK;
}

extern "C" ems_status ems_immortality_check(ems_ctx *c, uint8_t *mortal, double *sigma_ss_max, double *sigma_ss) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "screen before the first IR solve");
    EMS_TRY(each_window(c, [&](int s0, int ns) -> ems_status {
        EMS_TRY(window_derive(c));
        EMS_TRY(screen(c));
        if (sigma_ss)
            EMS_CUDA(c, cudaMemcpyAsync(sigma_ss + (size_t)s0 * c->N, c->d.sig_ss, sizeof(double) * ns * c->N,
                                        cudaMemcpyDeviceToHost, c->stream));
        if (windowed(c)) EMS_CUDA(c, cudaStreamSynchronize(c->stream));   // the window's scratch is reused
        return EMS_OK;
    }));
    const size_t ts = (size_t)c->n_trees * c->S;
    if (mortal) EMS_CUDA(c, cudaMemcpyAsync(mortal, c->d.mortal, ts, cudaMemcpyDeviceToHost, c->stream));
    if (sigma_ss_max)
        EMS_CUDA(c, cudaMemcpyAsync(sigma_ss_max, c->d.ssmax, ts * 8, cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

extern "C" ems_status ems_set_thermal_perturbation(ems_ctx *c, const double *dT, int nx, int ny) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (dT) {
        if (c->rnx == 0) return fail(c, EMS_E_STATE, "a perturbation needs a thermal map (its extent)");
        if (nx < 2 || ny < 2 || nx * ny > EMS_MAX_PERT)
            return fail(c, EMS_E_INVAL, "perturbation raster must be 2x2 .. 4,096 values");
        for (int64_t k = 0; k < (int64_t)c->S_all * nx * ny; ++k)
            if (!std::isfinite(dT[k])) return fail(c, EMS_E_INVAL, "non-finite temperature perturbation");
        for (int s = 0; s < c->S_all; ++s)
            EMS_CUDA(c, cudaMemcpyAsync(c->d_all.pert + (size_t)s * EMS_MAX_PERT, dT + (size_t)s * nx * ny,
                                        sizeof(double) * nx * ny, cudaMemcpyHostToDevice, c->stream));
        c->pnx = nx; c->pny = ny;
    } else {
        c->pnx = c->pny = 0;
    }
    if (windowed(c)) {
        map_window(c, 0, c->W);
        ems_status s = sample_physics(c);
        map_all(c);
        EMS_TRY(s);
    } else {
        EMS_TRY(sample_physics(c));
    }
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_autotune(ems_ctx *c, int n_steps, int max_samples, ems_chain_rule *rules, double *ms,
                                   double *ms_default, int cap, int *n_rules) {
    if (!c || n_steps < 1 || max_samples < 1 || cap < 0 || (cap > 0 && !rules) || !n_rules) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "autotune before the first IR solve (the forcing needs the currents)");
    if (c->prm.method != EMS_BE) return fail(c, EMS_E_STATE, "the autotuner picks backward-Euler shapes");
    *n_rules = 0;
    if (windowed(c)) map_window(c, 0, c->W);
    ems_status s = window_derive(c);
    if (s == EMS_OK) s = forcing(c);
    if (s == EMS_OK)
        s = c->prm.precision == EMS_F32 ? autotune_run<float>(c, n_steps, max_samples, rules, ms, ms_default, cap, n_rules)
                                        : autotune_run<double>(c, n_steps, max_samples, rules, ms, ms_default, cap, n_rules);
    if (windowed(c)) map_all(c);
    EMS_TRY(s);
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_autotune_log(const ems_ctx *c, int cap, ems_chain_rule *shapes, double *ms, int32_t *group,
                                       int *count) {
    if (!c || cap < 0 || !count || (cap > 0 && (!shapes || !ms || !group))) return EMS_E_INVAL;
    const int k = (int)std::min<size_t>(c->tune_log.size(), (size_t)cap);
    for (int i = 0; i < k; ++i) {
        shapes[i] = c->tune_log[i].shape;
        ms[i] = c->tune_log[i].ms;
        group[i] = c->tune_log[i].group;
    }
    *count = cap > 0 ? k : (int)c->tune_log.size();
    return EMS_OK;
}
