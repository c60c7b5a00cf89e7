// ems_chain_cl.cuh -- chains on a thread-block cluster (Sec. IV-B's
// backward-Euler chain solve for chains longer than one CTA holds).
//
// A chain is split over CL CTAs of one cluster: team thread g = rank T + c
// owns nodes [M g, M g + M) in the chunk layout of the one-CTA kernels (team
// size CL T).  State, compensation and the per-node coefficients stay in
// registers for all steps of a launch; thresholds (dt leak at a void node)
// in shared memory.  Each step every CTA solves its part with no carry from
// the other CTAs; the increment is affine in the two carries crossing its
// ends with responses fixed by the factorisation, so one exchange per step
// through distributed shared memory -- each rank's forward aggregate and
// first-node increment, its end stresses (halos) and the previous step's
// flags, pushed into every peer's slot before one cluster barrier -- gives
// every CTA all carries.  A nucleation's cluster-wide argmax, the threshold
// minimum and the factorisation's 2 x 2 product scan go the same way.  Every
// CTA keeps an identical copy of the tree's void list; a void's volume is
// accumulated and stored by the CTA that owns its node.  All CTAs of a
// cluster execute the same sequence of cluster barriers (every branch
// between them depends on cluster-wide values only).
#pragma once
#include <cooperative_groups.h>

#include "ems_chain.cuh"

namespace ems {
namespace {

namespace cg = cooperative_groups;

// component j (0..3) of a float4; j is a constant after unrolling
__device__ __forceinline__ float f4at(const float4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

template <typename R>
struct ClSlots {                      // written by the other CTAs of the cluster (push), read locally
    // every step, two buffers by step parity
    R fA[2][8];                       // each rank's forward aggregate (no carry into it)
    R bA[2][8];                       // each rank's first-node increment (no carries into it)
    R first[2][8], last[2][8];        // each rank's stress at its first / last node (halos)
    int flags[2][8];                  // each rank: bit 0 a node reached its threshold, bit 1 near the guard
    // every factorisation
    R fB[8];                          // forward aggregate: response to the carry into the rank
    R bB[8];                          // first-node increment: response to the carry from the right
    R bAz[8];                         // first-node increment: response to the forward carry into the rank
    R hh[8];                          // p dt g across the boundary to the next rank
    double best[8];                   // each rank's argmax of sigma - sigma_crit (nucleation)
    int arg[8];
    double tmin[8];                   // each rank's lowest threshold
    double fm[8][4];                  // each rank's product of 2 x 2 chunk matrices (factorisation)
};

// exclusive scan of the chunk maps within the CTA (one barrier), with the
// CTA's carry-in composed in: returns the carry entering this thread's chunk,
// and the CTA's aggregate map -- the inclusive map of the scan's last thread:
// dir 0 (left to right) stored by lane 31 of the last warp in sAg[0..1], to
// be read after the next barrier; dir 1 (right to left) in aggA, aggB of
// lane 0 of warp 0.
template <int DIR, typename R>
__device__ __forceinline__ void cta_scan(R A, R B, R *sA, R *sB, R &exA, R &exB, R &aggA, R &aggB, R *sAg) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // inclusive warp scan
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const R Ao = DIR == 0 ? __shfl_up_sync(full, A, d) : __shfl_down_sync(full, A, d);
        const R Bo = DIR == 0 ? __shfl_up_sync(full, B, d) : __shfl_down_sync(full, B, d);
        if (DIR == 0 ? lane >= d : lane + d < 32) { A = fmx(B, Ao, A); B = B * Bo; }
    }
    const int edge = DIR == 0 ? 31 : 0;
    if (lane == edge) { sA[DIR * 32 + w] = A; sB[DIR * 32 + w] = B; }
    __syncthreads();
    // composite of the earlier warps (fwd: warps < w; bwd: warps > w), as a map
    const int k = DIR == 0 ? lane : nw - 1 - lane;
    const bool take = DIR == 0 ? k < w : k > w;
    R a = take && k >= 0 && k < nw ? sA[DIR * 32 + k] : R(0), b = take && k >= 0 && k < nw ? sB[DIR * 32 + k] : R(1);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const R ao = __shfl_up_sync(full, a, d), bo = __shfl_up_sync(full, b, d);
        if (lane >= d) { a = fmx(b, ao, a); b = b * bo; }
    }
    const R cwA = __shfl_sync(full, a, 31), cwB = __shfl_sync(full, b, 31);
    // this thread's exclusive map within the CTA: (earlier lanes) o (earlier warps)
    const R iA = fmx(B, cwA, A), iB = B * cwB;                 // inclusive
    const R pA = DIR == 0 ? __shfl_up_sync(full, iA, 1) : __shfl_down_sync(full, iA, 1);
    const R pB = DIR == 0 ? __shfl_up_sync(full, iB, 1) : __shfl_down_sync(full, iB, 1);
    const int first = DIR == 0 ? 0 : 31;
    exA = lane == first ? cwA : pA;
    exB = lane == first ? cwB : pB;
    aggA = iA; aggB = iB;
    if (DIR == 0 && w == nw - 1 && lane == 31) { sAg[0] = iA; sAg[1] = iB; }
}

// Cluster version of chain_factor (increment form): every CTA calls it;
// g = team thread, TT = team size.  Two cluster barriers.
template <typename R, int M>
__device__ __noinline__ void chain_factor_cl(const ChainArgs<R> &a, double dt, int n, int TT, int g, int64_t cb,
                                             int64_t cs, int64_t ps, ClSlots<R> *sl, int rank) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double sfm[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    auto node = [&](int i, double &d, double &em, double &ep, bool &is_void) {
        const double gl = i > 0 ? a.g[cs + i] : 0.0, gr = i + 1 < n ? a.g[cs + i + 1] : 0.0;
        is_void = isinf(a.thr[cs + i]);
        d = __fma_rn(dt, __dadd_rn(gl, gr), a.V[cb + i]);
        if (is_void) d = __fma_rn(dt, a.leak[cs + i], d);
        em = -__dmul_rn(dt, gl);
        ep = -__dmul_rn(dt, gr);
    };
    M2 P{1.0, 0.0, 0.0, 1.0};
    for (int k = 0; k < M; ++k) {
        const int i = g * M + k;
        if (i >= n) break;
        double d, em, ep;
        bool v;
        node(i, d, em, ep, v);
        P = m2mul(M2{d, -__dmul_rn(em, em), 1.0, 0.0}, P);
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const M2 o = m2shfl_up(P, d);
        if (lane >= d) P = m2mul(P, o);
    }
    if (lane == 31) { sfm[0][w] = P.a; sfm[1][w] = P.b; sfm[2][w] = P.c; sfm[3][w] = P.d; }
    __syncthreads();
    M2 Cw{1.0, 0.0, 0.0, 1.0};
    for (int k = 0; k < w; ++k) Cw = m2mul(M2{sfm[0][k], sfm[1][k], sfm[2][k], sfm[3][k]}, Cw);
    if (threadIdx.x < 4 * (int)cl.num_blocks()) {         // this CTA's product, pushed to every CTA
        M2 Ag{1.0, 0.0, 0.0, 1.0};
        for (int k = 0; k < nw; ++k) Ag = m2mul(M2{sfm[0][k], sfm[1][k], sfm[2][k], sfm[3][k]}, Ag);
        const int q = threadIdx.x >> 2, e = threadIdx.x & 3;
        cl.map_shared_rank(sl, q)->fm[rank][e] = e == 0 ? Ag.a : e == 1 ? Ag.b : e == 2 ? Ag.c : Ag.d;
    }
    cl.sync();
    // product of the earlier CTAs' aggregates (later on the left)
    M2 Qc{1.0, 0.0, 0.0, 1.0};
    for (int q = 0; q < rank; ++q) Qc = m2mul(M2{sl->fm[q][0], sl->fm[q][1], sl->fm[q][2], sl->fm[q][3]}, Qc);
    const M2 CwT = m2mul(Cw, Qc);
    const M2 incl = m2mul(P, CwT);
    const M2 prev = m2shfl_up(incl, 1);
    const M2 Q = lane == 0 ? CwT : prev;
    double pprev = g == 0 ? 0.0 : __ddiv_rn(Q.c, Q.a);
    for (int k = 0; k < M; ++k) {
        const int i = g * M + k;
        if (i >= n) break;
        double d, em, ep;
        bool is_void;
        node(i, d, em, ep, is_void);
        const double p = __drcp_rn(__fma_rn(-__dmul_rn(em, em), pprev, d));
        const int64_t pk = ps + (int64_t)k * TT + g;
        a.pinv[pk] = p;
        a.alpha[pk] = (R)p;
        a.dtg[pk] = (R)(-em);
        a.dtl[pk] = is_void ? (R)(dt * a.leak[cs + i]) : R(0);
        a.gam[pk] = (R)(p * em);
        a.uu[pk] = (R)(p * ep);
        pprev = p;
    }
    cl.sync();                          // dt g of the next chunk may belong to another CTA
    R acc = R(1);
    for (int k = 0; k < M; ++k) {
        const int64_t pk = ps + (int64_t)k * TT + g;
        const int i = g * M + k;
        a.beta[pk] = i < n ? (R)(dt * a.f[cs + i]) : R(0);
        acc *= a.alpha[pk] * a.dtg[pk];
        a.Pf[pk] = acc;
    }
    acc = R(1);
    for (int k = M - 1; k >= 0; --k) {
        const int64_t pk = ps + (int64_t)k * TT + g;
        const R gn = k + 1 < M ? a.dtg[pk + TT] : (g + 1 < TT ? a.dtg[ps + g + 1] : R(0));
        acc *= a.alpha[pk] * gn;
        a.Pb[pk] = acc;
    }
}

// SMC (FP32): the chunk coefficients (alpha, dt g, dt f, the response w)
// and the thresholds live in dynamic shared memory, [array][k / 4][thread] as
// float4 (20 bytes per node), instead of registers, so that two or more CTAs
// share an SM; the arithmetic and its order are those of the register form.
template <typename R, int M, int CL, int TMAX, bool SMC>
__global__ void __launch_bounds__(TMAX, SMC ? 2 : 1) k_chain_cl(ChainArgs<R> a) {
    static_assert(!SMC || (sizeof(R) == 4 && M % 4 == 0), "shared-memory coefficients: FP32, M a multiple of 4");
    __shared__ R sA[64], sB[64], sL[32], sR[32], sAg[2];
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int s_nv;
    __shared__ int s_node[EMS_MAX_VOIDS];
    __shared__ double s_vol[EMS_MAX_VOIDS], s_coef[EMS_MAX_VOIDS];
    __shared__ double s_dt, s_tbase, s_gthr;
    __shared__ int s_rs, s_sbase, s_refac;
    __shared__ ClSlots<R> sl;
    cg::cluster_group cl = cg::this_cluster();

    const int rank = (int)cl.block_rank();
    const int t = a.trees[blockIdx.x / CL], s = blockIdx.y;
    const int T = blockDim.x, c = threadIdx.x, TT = T * CL, g = rank * T + c;
    const int lane = c & 31, w_ = c >> 5, nw = T >> 5;
    const int64_t cb = a.toff[t];
    const int n = (int)(a.toff[t + 1] - cb);
    const int64_t cs = (int64_t)s * a.N + cb, ps = (int64_t)s * a.P + a.pbase[t];
    const int64_t st = (int64_t)s * a.n_trees + t;
    const int sm = a.sched[st];
    if (a.kr_mode[st] || sm < 0) return;        // uniform over the cluster: every CTA returns
    const int kd = a.kdone[st];
    auto owner = [&](int v) { return (v / M) / T; };   // rank holding node v

    // cluster-wide lowest threshold
    auto thr_min = [&]() -> double {
        double tm = INFINITY;
        for (int i = g; i < n; i += TT) tm = fmin(tm, a.thr[cs + i]);
        tm = block_min(tm, sv);
        if (c < CL) cl.map_shared_rank(&sl, c)->tmin[rank] = tm;
        cl.sync();
        double r = INFINITY;
        for (int q = 0; q < CL; ++q) r = fmin(r, sl.tmin[q]);
        return r;
    };
    double thrmin = thr_min();
    R sg[M], cc[M];                   // state and (FP32) its Kahan compensation
#pragma unroll
    for (int k = 0; k < M; ++k) { sg[k] = a.sig[ps + (int64_t)k * TT + g]; cc[k] = R(0); }

    int rs = sm > 1 ? sm : 1;
    if ((a.n_steps - kd) % rs) rs = 1;
    if (rs > 1) {
        const int nr = __syncthreads_or(near_guard<R, M>(sg, a.guard * thrmin));
        if (c < CL) cl.map_shared_rank(&sl, c)->flags[0][rank] = nr ? 2 : 0;
        cl.sync();
        int any = 0;
        for (int q = 0; q < CL; ++q) any |= sl.flags[0][q];
        cl.sync();
        if (any & 2) {
            rs = 1;
            if (g == 0) a.sched[st] = 0;
        }
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
    }
    cl.sync();                                   // every CTA has read dirty / fdt
    if (g == 0) { a.dirty[st] = 0; a.fdt[st] = s_dt; }
    if (s_refac) {
        chain_factor_cl<R, M>(a, s_dt, n, TT, g, cb, cs, ps, &sl, rank);
    } else {
        const double dt = s_dt;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int i = g * M + k;
            a.beta[ps + (int64_t)k * TT + g] = i < n ? (R)(dt * a.f[cs + i]) : R(0);
        }
    }

    // One cluster barrier per step.  Each CTA solves its part with no carry
    // from the other CTAs: forward values z, backward increments xr.  The
    // true increment is linear in the two carries that cross its ends,
    //   x_k = xr_k + w_k cf + cpb_k cr,
    // cf the forward carry into the thread's chunk, cr the backward one, and
    // cf, cr are affine in the CTA's forward carry-in zin and its right
    // carry-in; the responses (w, exB, bxB, bxAz and each rank's fB, bB, bAz)
    // are constants of the factorisation.  So one exchange per step of each
    // rank's forward aggregate and first-node increment (both without
    // carries) gives every CTA all carries.  The CTA-boundary halos ride
    // along: each CTA sweeps with the halos of the previous step's exchange
    // and corrects with their change d, an increment (exact as the difference
    // of two nearby values): the left neighbour's d adds to zin, the right
    // neighbour's adds to the right carry-in (p dt g d at the last node).
    // Flags raised by step k reach the other CTAs with step k + 1's exchange:
    // that step's work is dropped, the event handled, the step redone.
    // registers: per node p, dt g, dt f and the response w; the thresholds
    // (at a void node: dt leak) in shared memory, this chunk's lowest one
    // in thc for a cheap test; the backward carry products are rebuilt as
    // running products where they are used (the factorisation's order, so
    // the same values)
    R cp[M], cg_[M], cbt[M], w[M], g_next, cpb0, thc;
    R w_first, w_last;                           // (SMC) the response w at the chunk's ends
    R exB = R(1), bxB = R(1), bxAz = R(0);
    __shared__ R s_th_st[SMC ? 1 : M * TMAX];
    extern __shared__ float4 s_c4[];             // (SMC) [4][M / 4][T] coefficients, then [M][T] thresholds
    R *const s_th = SMC ? (R *)(s_c4 + 4 * (M / 4) * T) : s_th_st;
    auto c4 = [&](int arr, int q) -> float4 { return s_c4[(arr * (M / 4) + q) * T + c]; };
    auto put = [&](int arr, int k, R v) { ((float *)s_c4)[((arr * (M / 4) + k / 4) * T + c) * 4 + (k & 3)] = v; };
    unsigned vmask = 0u;
    __shared__ R s_last, s_hh;
    const unsigned full = 0xffffffffu;
    auto load = [&]() {
        cl.sync();                               // coefficients of every CTA written
        vmask = 0u;
        thc = (R)INFINITY;
        for (int q = 0; q < s_nv; ++q)
            if (s_node[q] / M == g) vmask |= 1u << (s_node[q] % M);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int64_t pk = ps + (int64_t)k * TT + g;
            const int i = g * M + k;
            if constexpr (SMC) {
                put(0, k, a.alpha[pk]);
                put(1, k, a.dtg[pk]);
                put(2, k, a.beta[pk]);
            } else {
                cp[k] = a.alpha[pk];
                cg_[k] = a.dtg[pk];
                cbt[k] = a.beta[pk];
                w[k] = a.Pf[pk];
            }
            const R th = ((vmask >> k) & 1u) ? a.dtl[pk]
                                              : (i < n ? (sizeof(R) == 4 ? (R)__double2float_rd(a.thr[cs + i])
                                                                         : (R)a.thr[cs + i])
                                                       : (R)INFINITY);
            s_th[k * T + c] = th;
            if (!((vmask >> k) & 1u)) thc = fmin(thc, th);
        }
        cpb0 = a.Pb[ps + g];
        g_next = g + 1 < TT ? a.dtg[ps + g + 1] : R(0);
        // response of the chunk's backward sweep to a unit forward carry
        if constexpr (SMC) {
            const int64_t pl = ps + (int64_t)(M - 1) * TT + g;
            R wn = a.Pf[pl];
            w_last = wn;
            put(3, M - 1, wn);
#pragma unroll
            for (int k = M - 2; k >= 0; --k) {
                const int64_t pk = ps + (int64_t)k * TT + g;
                wn = fmx(a.alpha[pk] * a.dtg[pk + TT], wn, a.Pf[pk]);
                put(3, k, wn);
            }
            w_first = wn;
            if (c == T - 1) s_hh = a.alpha[pl] * g_next;
        } else {
#pragma unroll
            for (int k = M - 2; k >= 0; --k) w[k] = fmx(cp[k] * cg_[k + 1], w[k + 1], w[k]);
            w_first = w[0];
            w_last = w[M - 1];
            if (c == T - 1) s_hh = cp[M - 1] * g_next;
        }
        R u0, u1, fB, v0, bAz, bB;
        cta_scan<0, R>(R(0), w_last, sA, sB, u0, exB, u1, fB, sAg);
        cta_scan<1, R>(exB * w_first, cpb0, sA, sB, bxAz, bxB, bAz, bB, sAg);
        fB = sAg[1];                             // written before the second scan's barrier
        bAz = __shfl_sync(full, bAz, 0);
        bB = __shfl_sync(full, bB, 0);
        (void)u0; (void)u1; (void)v0;
        if (c < CL) {
            ClSlots<R> *o = cl.map_shared_rank(&sl, c);
            o->fB[rank] = fB; o->bB[rank] = bB; o->bAz[rank] = bAz; o->hh[rank] = s_hh;
        }
        cl.sync();
    };
    load();

    int pending = 0;                             // this CTA's flags from the previous step
    // events of step `ev` (state = after step ev): nucleation, promotion to
    // fine steps; with `refactor` the factors are rebuilt at once, else left
    // to the next launch
    auto handle = [&](int any, int ev, bool refactor) {
        int refac_from = -1;
        if (any & 1) {
            double best = -INFINITY;
            int arg = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int i = g * M + k;
                if (i < n) {
                    const double m = (double)sg[k] - a.thr[cs + i];
                    if (m > best) { best = m; arg = i; }
                }
            }
            block_argmax(best, arg, sv, si);
            if (c < CL) { ClSlots<R> *o = cl.map_shared_rank(&sl, c); o->best[rank] = best; o->arg[rank] = arg; }
#pragma unroll
            for (int k = 0; k < M; ++k) a.sig[ps + (int64_t)k * TT + g] = sg[k];
            cl.sync();
            best = -INFINITY; arg = 0x7fffffff;
            for (int q = 0; q < CL; ++q)
                if (sl.best[q] > best || (sl.best[q] == best && sl.arg[q] < arg)) { best = sl.best[q]; arg = sl.arg[q]; }
            if (best >= 0.0) {
                const int v = arg;
                if (c == 0) {
                    const int nv = s_nv;
                    if (rank == owner(v)) {
                        const double dt = s_dt;
                        auto S_ = [&](int i) { return (double)a.sig[ps + (int64_t)(i % M) * TT + i / M]; };
                        const double gl = v > 0 ? a.g[cs + v] : 0.0, gr = v + 1 < n ? a.g[cs + v + 1] : 0.0;
                        double acc = (a.V[cb + v] + dt * (gl + gr)) * S_(v);
                        if (v > 0) acc -= dt * gl * S_(v - 1);
                        if (v + 1 < n) acc -= dt * gr * S_(v + 1);
                        const double s0 = (acc - dt * a.f[cs + v]) / a.V[cb + v];
                        const double m0 = s0 - a.thr[cs + v];
                        const double frac = m0 < 0.0 ? -m0 / (best - m0) : 0.0;
                        if (nv < a.maxv) {
                            const int64_t e = st * a.maxv + nv;
                            a.v_node[e] = v;
                            a.v_seg[e] = void_segment<R>(a, s, cb + v);
                            a.v_tnuc[e] = s_tbase + ((double)(ev - s_sbase) + frac) * dt;
                            a.v_vol[e] = 0.0;
                            a.v_count[st] = nv + 1;
                            atomicAdd(&a.counters[0], 1);
                        } else {
                            atomicOr(&a.status[kStatusOverflow], 1);
                        }
                        a.thr[cs + v] = INFINITY;
                    }
                    if (nv < a.maxv) {                  // every CTA's copy of the void list
                        s_node[nv] = v; s_vol[nv] = 0.0; s_coef[nv] = s_dt * a.Binv * a.leak[cs + v];
                        s_nv = nv + 1;
                    }
                }
                refac_from = arg;
            }
        }
        bool promoted = false;
        if (any & 2) {
            // coarse steps from ev + 1 on become fine ones
            n_steps = ev + 1 + (n_steps - ev - 1) * s_rs;
            promoted = true;
            __syncthreads();
            if (c == 0) {
                s_tbase += (double)(ev + 1 - s_sbase) * s_dt;
                s_sbase = ev + 1;
                s_dt = a.dt;
                s_rs = 1;
                for (int q = 0; q < s_nv; ++q) s_coef[q] = a.dt * a.Binv * a.leak[cs + s_node[q]];
                if (rank == 0) { a.sched[st] = 0; a.fdt[st] = a.dt; }
            }
            refac_from = 0;
        }
        if (refac_from < 0 || !refactor) return;
        cl.sync();                               // the new threshold is written; every CTA is here
        const double dtf = promoted ? a.dt : s_dt;
        chain_factor_cl<R, M>(a, dtf, n, TT, g, cb, cs, ps, &sl, rank);
        thrmin = thr_min();
        if (c == 0) s_gthr = a.guard * thrmin;
        load();
    };

    // halos: inside the CTA through shared memory, across CTAs through the
    // slots (buffer 1 holds the exchange before step 0)
    if (lane == 31) sL[w_] = sg[M - 1];
    if (lane == 0) sR[w_] = sg[0];
    if (c == T - 1) s_last = sg[M - 1];
    __syncthreads();
    {
        const R fst = __shfl_sync(full, sg[0], 0);
        if (c < CL) { ClSlots<R> *o = cl.map_shared_rank(&sl, c); o->first[1][rank] = fst; o->last[1][rank] = s_last; }
        cl.sync();
    }

    for (int step = 0; step < n_steps;) {
        const int b = step & 1, ob = b ^ 1;
        R left = __shfl_up_sync(full, sg[M - 1], 1);
        R right = __shfl_down_sync(full, sg[0], 1);
        if (lane == 0 && w_ > 0) left = sL[w_ - 1];
        if (lane == 31 && w_ + 1 < nw) right = sR[w_ + 1];
        if (c == 0) left = rank > 0 ? sl.last[ob][rank - 1] : R(0);
        if (c == T - 1) {
            right = rank + 1 < CL ? sl.first[ob][rank + 1] : R(0);
            s_last = sg[M - 1];
        }
        // forward sweep, then the carries within the CTA
        R z = R(0);
        R zr[M];
        if constexpr (SMC) {                     // coefficients by groups of 4 nodes
            // the next group's coefficients are loaded a group ahead
            float4 P = c4(0, 0), G = c4(1, 0), B = c4(2, 0), Pn = P, Bn = B, Gn = G;
            if (M > 4) { Pn = c4(0, 1); Bn = c4(2, 1); Gn = c4(1, 1); }
            R gk = G.x;
            R qprev = gk * (left - sg[0]);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int j = k & 3;
                if (j == 0 && k > 0) {
                    P = Pn; B = Bn; G = Gn;
                    if (k + 4 < M) { Pn = c4(0, (k >> 2) + 1); Bn = c4(2, (k >> 2) + 1); Gn = c4(1, (k >> 2) + 1); }
                }
                const R nxt = k + 1 < M ? sg[k + 1] : right;
                const R gk1 = j < 3 ? f4at(G, j + 1) : (k + 1 < M ? Gn.x : g_next);
                const R qn = gk1 * (sg[k] - nxt);
                R r = qprev - qn + f4at(B, j);
                if ((vmask >> k) & 1u) r -= s_th[k * T + c] * sg[k];
                z = f4at(P, j) * fmx(gk, z, r);
                zr[k] = z;
                qprev = qn;
                gk = gk1;
            }
        } else {
            R gk = cg_[0];
            R qprev = gk * (left - sg[0]);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const R nxt = k + 1 < M ? sg[k + 1] : right;
                const R gk1 = k + 1 < M ? cg_[k + 1] : g_next;
                const R qn = gk1 * (sg[k] - nxt);
                R r = qprev - qn + cbt[k];
                if ((vmask >> k) & 1u) r -= s_th[k * T + c] * sg[k];
                z = cp[k] * fmx(gk, z, r);
                zr[k] = z;
                qprev = qn;
                gk = gk1;
            }
        }
        R exA, u0, agA, u1;
        cta_scan<0, R>(z, w_last, sA, sB, exA, u0, agA, u1, sAg);
        // backward sweep without carries; the first node with this CTA's forward carry
        R x = R(0);
        if constexpr (SMC) {
            // the previous group's coefficients are loaded a group ahead
            float4 P = c4(0, M / 4 - 1), G = c4(1, M / 4 - 1), Gn = G, Pp = P, Gp = G;
            if (M > 4) { Pp = c4(0, M / 4 - 2); Gp = c4(1, M / 4 - 2); }
#pragma unroll
            for (int k = M - 1; k >= 0; --k) {
                const int j = k & 3;
                if (j == 3 && k + 1 < M) {
                    Gn = G; P = Pp; G = Gp;
                    if (k >= 4) { Pp = c4(0, (k >> 2) - 1); Gp = c4(1, (k >> 2) - 1); }
                }
                const R gk1 = j < 3 ? f4at(G, j + 1) : (k + 1 < M ? Gn.x : g_next);
                x = fmx(f4at(P, j) * gk1, x, zr[k]);
                zr[k] = x;
            }
        } else {
#pragma unroll
            for (int k = M - 1; k >= 0; --k) {
                const R gk1 = k + 1 < M ? cg_[k + 1] : g_next;
                x = fmx(cp[k] * gk1, x, zr[k]);
                zr[k] = x;
            }
        }
        R bxA, u2, bgA, u3;
        cta_scan<1, R>(fmx(w_first, exA, zr[0]), cpb0, sA, sB, bxA, u2, bgA, u3, sAg);
        (void)u0; (void)u1; (void)u2; (void)u3;
        agA = sAg[0];                            // written before the second scan's barrier
        bgA = __shfl_sync(full, bgA, 0);
        const R fst = __shfl_sync(full, sg[0], 0);
        if (c < CL) {
            ClSlots<R> *o = cl.map_shared_rank(&sl, c);
            o->fA[b][rank] = agA; o->bA[b][rank] = bgA;
            o->first[b][rank] = fst; o->last[b][rank] = s_last; o->flags[b][rank] = pending;
        }
        cl.sync();
        int any = 0;
#pragma unroll
        for (int q = 0; q < CL; ++q) any |= sl.flags[b][q];
        if (any) {                               // an event of the previous step: handle, redo this step
            pending = 0;
            handle(any, step - 1, true);
            cl.sync();                           // the slots are written again by the redone step
            continue;
        }
        // carries across the ranks, halo changes included:
        //   Y_(q+1) = fB_q Y_q + fA_q + hh_q dfirst_(q+1) + dlast_q   (forward carry into rank q + 1)
        //   C_(q-1) = bA_q + bAz_q Y_q + bB_q (C_q + dfirst_(q+1))    (increment of rank q's first node)
        R Y[CL];
        Y[0] = R(0);
#pragma unroll
        for (int q = 0; q + 1 < CL; ++q)
            Y[q + 1] = fmx(sl.fB[q], Y[q], fmx(sl.hh[q], sl.first[b][q + 1] - sl.first[ob][q + 1], sl.fA[b][q])) +
                       (sl.last[b][q] - sl.last[ob][q]);
        R C = R(0), zin = R(0);
#pragma unroll
        for (int q = CL - 1; q >= 0; --q) {
            if (q == rank) zin = Y[q];
            if (q > rank) {
                const R dn = q + 1 < CL ? sl.first[b][q + 1] - sl.first[ob][q + 1] : R(0);
                C = fmx(sl.bB[q], C + dn, fmx(sl.bAz[q], Y[q], sl.bA[b][q]));
            }
        }
        if (rank + 1 < CL) C += sl.first[b][rank + 1] - sl.first[ob][rank + 1];
        const R cf = fmx(exB, zin, exA);
        const R cr = fmx(bxB, C, fmx(bxAz, zin, bxA));
        R pb = R(1);
        float4 P4, G4, W4, Gn4, Pp4, Gp4, Wp4;
        if constexpr (SMC) {
            P4 = c4(0, M / 4 - 1); G4 = c4(1, M / 4 - 1); W4 = c4(3, M / 4 - 1); Gn4 = G4;
            Pp4 = P4; Gp4 = G4; Wp4 = W4;
            if (M > 4) { Pp4 = c4(0, M / 4 - 2); Gp4 = c4(1, M / 4 - 2); Wp4 = c4(3, M / 4 - 2); }
        }
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            R dk;
            if constexpr (SMC) {
                const int j = k & 3;
                if (j == 3 && k + 1 < M) {
                    Gn4 = G4; P4 = Pp4; G4 = Gp4; W4 = Wp4;
                    if (k >= 4) { Pp4 = c4(0, (k >> 2) - 1); Gp4 = c4(1, (k >> 2) - 1); Wp4 = c4(3, (k >> 2) - 1); }
                }
                pb *= f4at(P4, j) * (j < 3 ? f4at(G4, j + 1) : (k + 1 < M ? Gn4.x : g_next));
                dk = fmx(pb, cr, fmx(f4at(W4, j), cf, zr[k]));
            } else {
                pb *= cp[k] * (k + 1 < M ? cg_[k + 1] : g_next);
                dk = fmx(pb, cr, fmx(w[k], cf, zr[k]));
            }
            if constexpr (sizeof(R) == 4) {               // compensated (Kahan) FP32 update
                const R y = dk - cc[k];
                const R tt = sg[k] + y;
                cc[k] = (tt - sg[k]) - y;
                sg[k] = tt;
            } else {
                sg[k] += dk;
            }
        }
        // void growth by the Robin leak (owner thread only)
        if (vmask) {
            for (int q = 0; q < s_nv; ++q) {
                const int v = s_node[q];
                if (v / M == g) {
                    R val = R(0);
#pragma unroll
                    for (int k = 0; k < M; ++k)
                        if (v % M == k) val = sg[k];
                    s_vol[q] += s_coef[q] * (double)val;
                }
            }
        }
        // nucleation test: the chunk's largest stress against its lowest
        // threshold first, each node against its own only then
        R mx = (R)-INFINITY;
#pragma unroll
        for (int k = 0; k < M; ++k) mx = ((vmask >> k) & 1u) ? mx : fmax(mx, sg[k]);
        bool hit = false;
        if (mx >= thc) {
#pragma unroll
            for (int k = 0; k < M; ++k) hit |= !((vmask >> k) & 1u) && sg[k] >= s_th[k * T + c];
        }
        const bool nr = s_rs > 1 && near_guard<R, M>(sg, s_gthr);
        if (lane == 31) sL[w_] = sg[M - 1];
        if (lane == 0) sR[w_] = sg[0];
        // the flags, and the warp halos for the next step
        pending = __syncthreads_or(hit) ? 1 : 0;
        if (s_rs > 1) pending |= __syncthreads_or(nr) ? 2 : 0;
        ++step;
    }
    // flags of the last step: handled here, the factors rebuilt by the next launch
    {
        const int b = n_steps & 1;
        if (c < CL) cl.map_shared_rank(&sl, c)->flags[b][rank] = pending;
        cl.sync();
        int any = 0;
        for (int q = 0; q < CL; ++q) any |= sl.flags[b][q];
        if (any) {
            handle(any, n_steps - 1, false);
            __syncthreads();
            if (g == 0) a.dirty[st] = 1;
        }
    }
#pragma unroll
    for (int k = 0; k < M; ++k) a.sig[ps + (int64_t)k * TT + g] = sg[k];
    __syncthreads();
    if (c == 0) {
        for (int q = 0; q < s_nv; ++q)
            if (owner(s_node[q]) == rank) a.v_vol[st * a.maxv + q] = s_vol[q];
        if (rank == 0) atomicAdd(a.work, (unsigned long long)n * (unsigned long long)n_steps);
    }
    cl.sync();                                   // no CTA leaves while another may read its slots
}

// raise the dynamic shared-memory limit of a shared-memory variant to what
// TMAX threads need (outside any stream capture)
template <typename R, int M, int CL, int TMAX>
cudaError_t smem_limit() {
    return cudaFuncSetAttribute(k_chain_cl<R, M, CL, TMAX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)cluster_smem_bytes(M, TMAX));
}

// one launch: n_trees chains x S samples, one cluster of CL CTAs per chain
template <typename R, int M, int CL, int TMAX, bool SMC = false>
cudaError_t launch_cl(int T_cta, unsigned n_trees, int S, cudaStream_t st, const ChainArgs<R> &a) {
    if (T_cta > TMAX || T_cta < 32 || T_cta % 32) return cudaErrorInvalidValue;
    // (SMC: the shared-memory limit was raised once by cluster_smem_init)
    const size_t smem = SMC ? cluster_smem_bytes(M, T_cta) : 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(n_trees * CL, S);
    cfg.blockDim = dim3(T_cta);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_chain_cl<R, M, CL, TMAX, SMC>, a);
}

}  // namespace
}  // namespace ems
