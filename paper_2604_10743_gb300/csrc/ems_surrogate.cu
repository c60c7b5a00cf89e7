// ems_surrogate.cu -- features, targets and the step schedule that connect
// the learned surrogate to an engine context.
//
//   k_features   one CTA per (tree, sample): 24 reductions over the tree's
//                nodes and faces (size, length, j, T, grad T, kappa,
//                sigma_crit, the steady state of Sec. III-B, time scales)
//   k_targets    first nucleation time and node from the void table
//   k_schedule   step schedule per (tree, sample) from the network's prediction
// The chain / tree kernels of the stress advance take r-times coarser
// backward-Euler steps for a (tree, sample) the schedule marks r > 1 (and no
// steps for one it marks frozen); everything else runs the plain solver.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ems_internal.cuh"
#include "../../include/ems_surrogate.h"

namespace {

constexpr int NF = EMS_MLP_FEATURES;

struct Acc {                     // per-thread partial reductions
    double s[8];                 // sums
    double mx[7];                // maxima
    double mn[3];                // minima
    double amax;                 // max margin and its node
    int aidx;
    double gmax, gkap;           // max |G| and kappa at that face
    double tl_all;               // min over nodes of the local early-time nucleation estimate
    double tl_mort, tl_ratio;    // same over nodes whose steady state exceeds sigma_crit; thr0 / sigma_ss there
};

__device__ void acc_merge(Acc &a, const Acc &b) {
    for (int k = 0; k < 8; ++k) a.s[k] += b.s[k];
    for (int k = 0; k < 7; ++k) a.mx[k] = fmax(a.mx[k], b.mx[k]);
    for (int k = 0; k < 3; ++k) a.mn[k] = fmin(a.mn[k], b.mn[k]);
    if (b.amax > a.amax || (b.amax == a.amax && b.aidx < a.aidx)) { a.amax = b.amax; a.aidx = b.aidx; }
    if (b.gmax > a.gmax) { a.gmax = b.gmax; a.gkap = b.gkap; }
    a.tl_all = fmin(a.tl_all, b.tl_all);
    if (b.tl_mort < a.tl_mort) { a.tl_mort = b.tl_mort; a.tl_ratio = b.tl_ratio; }
}

__device__ __forceinline__ double lg(double v) { return log10(fmax(v, 1e-300)); }

struct FeatArgs {
    int n_trees, S, n_seg;
    int64_t N;
    double sem, sigma_T;
    const int64_t *toff;
    const int32_t *par, *face_seg, *child_ptr, *child_idx;
    const int8_t *sign;
    const double *dx, *area, *V, *Tn, *Mface, *kap_a, *thr0, *ss, *j, *drop;
    float *x;
};

// sums: 0 L, 1 V, 2 V T, 3 |j| dx, 4 sign j dx, 5 kappa dx, 6 thr0, 7 branch points
// maxima: 0 |j|, 1 T, 2 |Mface|, 3 kappa, 4 sigma_ss, 5 -sigma_ss (min), 6 unused
// minima: 0 T, 1 kappa, 2 thr0
__global__ void __launch_bounds__(256) k_features(FeatArgs a) {
    __shared__ Acc sh[8];
    const int t = blockIdx.x, s = blockIdx.y;
    const int64_t cb = a.toff[t], n = a.toff[t + 1] - cb, cs = (int64_t)s * a.N + cb;
    const double *js = a.j + (int64_t)s * a.n_seg;
    Acc p;
    for (int k = 0; k < 8; ++k) p.s[k] = 0.0;
    for (int k = 0; k < 7; ++k) p.mx[k] = -INFINITY;
    for (int k = 0; k < 3; ++k) p.mn[k] = INFINITY;
    p.amax = -INFINITY; p.aidx = 0x7fffffff; p.gmax = -1.0; p.gkap = 0.0;
    p.tl_all = INFINITY; p.tl_mort = INFINITY; p.tl_ratio = 1.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t gi = cb + i, si = cs + i;
        const double T = a.Tn[gi], v = a.V[gi], th = a.thr0[si], sg = a.ss[si];
        p.s[1] += v; p.s[2] += v * T; p.s[6] += th;
        p.mx[1] = fmax(p.mx[1], T); p.mn[0] = fmin(p.mn[0], T);
        p.mn[2] = fmin(p.mn[2], th);
        p.mx[4] = fmax(p.mx[4], sg); p.mx[5] = fmax(p.mx[5], -sg);
        const double mg = sg - th;
        if (mg > p.amax || (mg == p.amax && (int)i < p.aidx)) { p.amax = mg; p.aidx = (int)i; }
        if (a.child_ptr[gi + 1] - a.child_ptr[gi] >= 2) p.s[7] += 1.0;
        if (a.par[gi] >= 0) {
            const double dx = a.dx[gi], ar = a.area[gi];
            const double jj = a.sign[gi] * js[a.face_seg[gi]];
            const double kap = a.kap_a[si] / ar;
            const double G = a.sem * jj + a.Mface[si];
            p.s[0] += dx; p.s[3] += fabs(jj) * dx; p.s[4] += jj * dx; p.s[5] += kap * dx;
            p.mx[0] = fmax(p.mx[0], fabs(jj)); p.mx[2] = fmax(p.mx[2], fabs(a.Mface[si]));
            p.mx[3] = fmax(p.mx[3], kap); p.mn[1] = fmin(p.mn[1], kap);
            if (fabs(G) > p.gmax) { p.gmax = fabs(G); p.gkap = kap; }
        }
        // Local early-time Korhonen estimate: semi-infinite branches of
        // cross-section a_e and diffusivity kappa_e meet at node i, whose net
        // atom-flux divergence is F_i = (a kappa G)_in - sum (a kappa G)_out.
        // Continuity of sigma and of the flux at the node give
        // sigma_i(t) = 2 F_i sqrt(t) / (sqrt(pi) sum_e a_e sqrt(kappa_e)),
        // so sigma_i reaches thr0_i at t_i = pi (thr0_i S_i / (2 F_i))^2.
        double F = 0.0, Sa = 0.0;
        if (a.par[gi] >= 0) {
            const double ak = a.kap_a[si], ar = a.area[gi];
            F += ak * (a.sem * a.sign[gi] * js[a.face_seg[gi]] + a.Mface[si]);
            Sa += ar * sqrt(ak / ar);
        }
        for (int k = a.child_ptr[gi]; k < a.child_ptr[gi + 1]; ++k) {
            const int32_t ch = a.child_idx[k];
            const double ak = a.kap_a[(int64_t)s * a.N + ch], ar = a.area[ch];
            F -= ak * (a.sem * a.sign[ch] * js[a.face_seg[ch]] + a.Mface[(int64_t)s * a.N + ch]);
            Sa += ar * sqrt(ak / ar);
        }
        if (F > 0.0 && Sa > 0.0) {
            const double q = th * Sa / (2.0 * F);
            const double tl = 3.14159265358979 * q * q;
            p.tl_all = fmin(p.tl_all, tl);
            if (sg > th && tl < p.tl_mort) { p.tl_mort = tl; p.tl_ratio = th / sg; }
        }
    }
    // warp then block merge in fixed order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        Acc q;
        for (int k = 0; k < 8; ++k) q.s[k] = __shfl_down_sync(0xffffffffu, p.s[k], o);
        for (int k = 0; k < 7; ++k) q.mx[k] = __shfl_down_sync(0xffffffffu, p.mx[k], o);
        for (int k = 0; k < 3; ++k) q.mn[k] = __shfl_down_sync(0xffffffffu, p.mn[k], o);
        q.amax = __shfl_down_sync(0xffffffffu, p.amax, o);
        q.aidx = __shfl_down_sync(0xffffffffu, p.aidx, o);
        q.gmax = __shfl_down_sync(0xffffffffu, p.gmax, o);
        q.gkap = __shfl_down_sync(0xffffffffu, p.gkap, o);
        q.tl_all = __shfl_down_sync(0xffffffffu, p.tl_all, o);
        q.tl_mort = __shfl_down_sync(0xffffffffu, p.tl_mort, o);
        q.tl_ratio = __shfl_down_sync(0xffffffffu, p.tl_ratio, o);
        if (lane + o < 32) acc_merge(p, q);
    }
    if (lane == 0) sh[w] = p;
    __syncthreads();
    if (threadIdx.x != 0) return;
    Acc r = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) acc_merge(r, sh[k]);
    const double L = fmax(r.s[0], 1e-12), nn = (double)n;
    const double kbar = r.s[5] / L;
    const double sc = r.mn[2];                                   // weakest critical stress
    const double gk = r.gkap > 0.0 ? r.gkap : kbar;
    // early-time Korhonen estimate at the steepest face: sigma(t) ~ 2 G sqrt(kappa t / pi)
    const double t_early = 3.14159265358979 * sc * sc / (4.0 * fmax(r.gmax * r.gmax, 1e-300) * fmax(gk, 1e-300));
    float *xo = a.x + ((int64_t)s * a.n_trees + t) * NF;
    xo[0] = (float)lg(nn);
    xo[1] = (float)lg(L);
    xo[2] = (float)log10(1.0 + r.s[7]);
    xo[3] = (float)lg(r.mx[0]);
    xo[4] = (float)lg(r.s[3] / L);
    xo[5] = (float)log10(fmin(r.tl_all, 1e13));           // earliest local nucleation estimate
    xo[6] = (float)(r.s[2] / r.s[1]);
    xo[7] = (float)(r.mx[1] - r.mn[0]);
    xo[8] = (float)log10(fmin(r.tl_mort, 1e13));          // same over mortal nodes
    xo[9] = (float)lg(kbar);
    xo[10] = (float)lg(r.mx[3]);
    xo[11] = (float)lg(r.mn[1]);
    xo[12] = (float)(sc * 1e-8);
    xo[13] = (float)(r.s[6] / nn * 1e-8);
    xo[14] = (float)(r.mx[4] * 1e-8);
    xo[15] = (float)(-r.mx[5] * 1e-8);
    xo[16] = (float)(r.amax * 1e-8);
    xo[17] = r.amax > 0.0 ? 1.0f : 0.0f;
    xo[18] = (float)(n > 1 ? (double)r.aidx / (nn - 1.0) : 0.0);
    xo[19] = (float)lg(L * L / fmax(kbar, 1e-300));
    xo[20] = (float)lg(t_early);
    xo[21] = (float)lg(r.gmax);
    xo[22] = (float)r.tl_ratio;                            // thr0 / sigma_ss at that node
    xo[23] = (float)(a.drop[s] * 10.0);
}

__global__ void k_targets(int n_trees, int S, int maxv, const int64_t *toff, const int32_t *v_count,
                          const int32_t *v_node, const double *v_tnuc, const float *feat, double t_cap, float *out,
                          int32_t *sched) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n_trees * S) return;
    const int t = (int)(k % n_trees);
    const int64_t n = toff[t + 1] - toff[t];
    double tn = t_cap, pos = feat[k * NF + 18];
    if (v_count[k] > 0) {
        tn = fmin(v_tnuc[k * maxv], t_cap);
        pos = n > 1 ? (double)v_node[k * maxv] / (double)(n - 1) : 0.0;
        if (sched) sched[k] = -1;                  // first nucleation known: stop stepping
    }
    out[2 * k] = (float)log10(fmax(tn, 1.0));
    out[2 * k + 1] = (float)pos;
}

__global__ void k_schedule(int64_t n, const float *pred, double thr, int coarsen, int32_t *sched) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    sched[k] = (double)pred[2 * k] > thr ? coarsen : 0;
}

}  // namespace

using namespace ems;

namespace ems {
ems_status mlp_predict_async(ems_mlp *m, const float *x, int64_t rows, float *y, int64_t *launches);
ems_status mlp_sync_status(ems_mlp *m);
cudaStream_t mlp_stream(const ems_mlp *m);
}  // namespace ems

namespace {
ems_status features_window(ems_ctx *c) {
    Dev &d = c->d;
    const ems_params &p = c->prm;
    EMS_TRY(window_derive(c));
    EMS_TRY(screen(c));
    FeatArgs a;
    a.n_trees = c->n_trees; a.S = c->S; a.n_seg = c->n_seg; a.N = c->N;
    a.sem = p.e_charge * p.Z_star * p.rho_Cu / p.Omega;
    a.sigma_T = p.sigma_T;
    a.toff = d.toff; a.par = d.par; a.face_seg = d.face_seg; a.child_ptr = d.child_ptr; a.child_idx = d.child_idx;
    a.sign = d.face_sign;
    a.dx = d.face_dx; a.area = d.face_area; a.V = d.V; a.Tn = d.Tn; a.Mface = d.Mface; a.kap_a = d.kap_a;
    a.thr0 = d.thr0; a.ss = d.sig_ss; a.j = d.j; a.drop = d.drop; a.x = d.feat;
    k_features<<<dim3(c->n_trees, c->S), 256, 0, c->stream>>>(a);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

// features of every sample (window by window when the context uses windows)
ems_status features(ems_ctx *c) {
    return each_window(c, [&](int, int) { return features_window(c); });
}
}  // namespace

extern "C" ems_status ems_surrogate_features(ems_ctx *c, float *x) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "features before the first IR solve");
    EMS_TRY(features(c));
    if (x)
        EMS_CUDA(c, cudaMemcpyAsync(x, c->d.feat, sizeof(float) * NF * c->S * c->n_trees, cudaMemcpyDeviceToDevice,
                                    c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_surrogate_targets(ems_ctx *c, double t_cap, int freeze, float *t) {
    if (!c || !t || !(t_cap > 1.0)) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    const int64_t ts = (int64_t)c->S * c->n_trees;
    k_targets<<<(unsigned)((ts + 255) / 256), 256, 0, c->stream>>>(c->n_trees, c->S, c->maxv, c->d.toff,
                                                                  c->d.v_count, c->d.v_node, c->d.v_tnuc, c->d.feat,
                                                                  t_cap, t, freeze ? c->d.sched : nullptr);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    return EMS_OK;
}

extern "C" ems_status ems_surrogate_schedule(ems_ctx *c, ems_mlp *m, double bound, int coarsen, double guard,
                                             int *n_coarse, float *pred) {
    if (!c || !m || !std::isfinite(bound) || coarsen < 2 || !(guard > 0.0 && guard <= 1.0)) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "schedule before the first IR solve");
    const int64_t ts = (int64_t)c->S * c->n_trees;
    EMS_TRY(features(c));
    // the network runs on its own stream: order it after the features
    cudaEvent_t ev;
    EMS_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, c->stream);
    ems_status s = EMS_OK;
    if (cudaStreamWaitEvent(mlp_stream(m), ev, 0) != cudaSuccess) s = EMS_E_CUDA;
    cudaEventDestroy(ev);
    if (s != EMS_OK) return cuda_check(c, cudaErrorInvalidValue, "cudaStreamWaitEvent");
    s = mlp_predict_async(m, c->d.feat, ts, c->d.pred, &c->launches);
    if (s == EMS_OK) s = mlp_sync_status(m);
    if (s != EMS_OK) return fail(c, s, std::string("surrogate network: ") + ems_mlp_last_error(m));
    k_schedule<<<(unsigned)((ts + 255) / 256), 256, 0, c->stream>>>(ts, c->d.pred, bound + log10(c->prm.horizon),
                                                                    coarsen, c->d.sched);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    if (pred) EMS_CUDA(c, cudaMemcpyAsync(pred, c->d.pred, sizeof(float) * 2 * ts, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<int32_t> sk((size_t)ts);
    std::vector<float> pr((size_t)ts * 2);
    EMS_CUDA(c, cudaMemcpyAsync(sk.data(), c->d.sched, 4 * ts, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaMemcpyAsync(pr.data(), c->d.pred, 8 * ts, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<double> first((size_t)c->n_trees, INFINITY);
    for (int q = 0; q < c->S; ++q) {
        int k = 0;
        for (int t = 0; t < c->n_trees; ++t) {
            const size_t st = (size_t)q * c->n_trees + t;
            k += sk[st] > 1;
            first[t] = std::min(first[t], (double)pr[2 * st]);
        }
        if (n_coarse) n_coarse[q] = k;
    }
    c->sched_guard = guard;
    // tree order: earliest predicted nucleation first in every bucket, so
    // the trees that refactor on nucleation start first
    for (auto &b : c->buckets) {
        std::stable_sort(b.trees.begin(), b.trees.end(), [&](int32_t x, int32_t y) { return first[x] < first[y]; });
        EMS_CUDA(c, cudaMemcpyAsync(b.d_trees, b.trees.data(), 4 * b.trees.size(), cudaMemcpyHostToDevice, c->stream));
    }
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMS_OK;
}

extern "C" ems_status ems_surrogate_clear(ems_ctx *c) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    EMS_CUDA(c, cudaMemsetAsync(c->d.sched, 0, sizeof(int32_t) * c->S * c->n_trees, c->stream));
    return EMS_OK;
}

namespace {
// one TTF run's per-sample outputs
struct RunOut {
    std::vector<double> ttf, final_drop;
};

ems_status ttf_run(ems_ctx *c, RunOut &o) {
    o.ttf.assign(c->S_all, 0.0);
    o.final_drop.assign(c->S_all, 0.0);
    ems_ttf_result r{};
    r.ttf = o.ttf.data();
    r.final_drop = o.final_drop.data();
    ems_ttf_opts opts{};
    return ems_ttf(c, &opts, &r);
}

// largest relative difference of TTF (where the reference's is finite) and
// final IR drop; +inf when the sets of finite TTFs differ
double result_error(const RunOut &ref, const RunOut &run) {
    double e = 0.0;
    for (size_t s = 0; s < ref.ttf.size(); ++s) {
        const bool fr = std::isfinite(ref.ttf[s]), fx = std::isfinite(run.ttf[s]);
        if (fr != fx) return INFINITY;
        e = std::max(e, std::fabs(run.final_drop[s] - ref.final_drop[s]) / ref.final_drop[s]);
        if (fr) e = std::max(e, std::fabs(run.ttf[s] - ref.ttf[s]) / std::max(ref.ttf[s], 1e-30));
    }
    return e;
}
}  // namespace

extern "C" ems_status ems_surrogate_validate(ems_ctx *const *ctxs, int n_ctx, ems_mlp *m, const double *cand,
                                             int n_cand, int coarsen, double guard, double tol, double margin,
                                             double *bound, double *log) {
    if (!ctxs || n_ctx < 1 || !m || !cand || n_cand < 1 || coarsen < 2 || !(guard > 0.0 && guard <= 1.0) ||
        !(tol >= 0.0) || !std::isfinite(margin) || !bound)
        return EMS_E_INVAL;
    for (int k = 0; k < n_ctx; ++k) {
        if (!ctxs[k]) return EMS_E_INVAL;
        if (!ctxs[k]->loaded) return fail(ctxs[k], EMS_E_STATE, "no grid loaded");
    }
    *bound = INFINITY;
    // entry states (restored before every run and at the end) and the plain runs
    std::vector<std::vector<char>> state(n_ctx);
    std::vector<RunOut> plain(n_ctx);
    for (int k = 0; k < n_ctx; ++k) {
        ems_ctx *c = ctxs[k];
        size_t nb = 0;
        EMS_TRY(ems_state_export(c, nullptr, &nb));
        state[k].resize(nb);
        EMS_TRY(ems_state_export(c, state[k].data(), &nb));
        EMS_TRY(ems_surrogate_clear(c));
        EMS_TRY(ttf_run(c, plain[k]));
        EMS_TRY(ems_state_import(c, state[k].data(), nb));
    }
    ems_status st = EMS_OK;
    for (int q = 0; q < n_cand && st == EMS_OK; ++q) {
        double worst = 0.0, coarse = 0.0, pairs = 0.0;
        for (int k = 0; k < n_ctx && st == EMS_OK; ++k) {
            ems_ctx *c = ctxs[k];
            std::vector<int> nc(c->S_all, 0);
            RunOut run;
            if ((st = ems_ir_solve(c, nullptr, nullptr)) != EMS_OK) break;
            if ((st = ems_surrogate_schedule(c, m, cand[q], coarsen, guard, nc.data(), nullptr)) != EMS_OK) break;
            if ((st = ttf_run(c, run)) != EMS_OK) break;
            for (int v : nc) coarse += v;
            pairs += (double)c->S_all * c->n_trees;
            worst = std::max(worst, result_error(plain[k], run));
            if ((st = ems_surrogate_clear(c)) != EMS_OK) break;
            st = ems_state_import(c, state[k].data(), state[k].size());
        }
        if (st != EMS_OK) break;
        if (log) {
            log[3 * q] = cand[q];
            log[3 * q + 1] = coarse / std::max(pairs, 1.0);
            log[3 * q + 2] = worst;
        }
        if (worst <= tol) {
            *bound = cand[q] + margin;
            break;
        }
    }
    return st;
}
