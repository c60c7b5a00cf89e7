// ems_krylov.cu -- rational Krylov reduced models of the chain trees
// (Sec. IV-E, Alg. 1, Eq. rak_moment_recurrence .. rak_shift_time).
//
// One CTA per (tree, sample) in the chunk layout of the BE kernels (thread c
// holds nodes c*M .. c*M+M-1, node c*M+k stored at slot k*T + c), one launch
// per aging step.  R is the context's storage precision (basis, stress,
// per-node arithmetic); cross-thread sums, the shifted factors and the small
// dense algebra are FP64.
//
//   build    (cache miss: first use, a new void, a new thermal map, new q or
//            eta) t_s = eta L^2/(pi^2 kappa_bar) and s0 = 1/t_s; the factors of
//            C - t_s A give (s0 C - A)^-1 y = t_s (C - t_s A)^-1 y; starting
//            block [R C s, R f]; block Arnoldi to order q with classical
//            Gram-Schmidt applied twice; base projections A_h = V^T A V and
//            C_h = V^T C V
//   augment  (cache hit, Sec. IV-E.4) the current starting block [R C s, R f]
//            orthogonalised twice against the cached columns into two extra
//            slots, and their rows of A_h and C_h
//   step     M = C_h - dt A_h (Cholesky), propagator F = M^-1 C_h; backward
//            Euler in reduced coordinates in increment form
//            (s_hat(k+1) - s_hat(k) = F (s_hat(k) - s_hat(k-1))) for a chunk of
//            steps kept on chip; a per-node upper bound of the lifted stress
//            over the chunk (per-coordinate extremes) leaves the candidate
//            nodes, which alone are lifted step by step to find the first
//            nucleation; void volumes take per-coordinate step sums; one lift
//            at the end of the chunk that ends the aging step
//   nucleation: lift at that step, record the void, rebuild (A changed) and
//            carry on from there in the same launch
// A build with nothing to reduce or with a rank-deficient block hands the tree
// to full backward Euler for the rest of the aging step (Sec. IV-E.5).
#include "ems_krylov_kernels.cuh"

namespace ems {
namespace {

template <typename R>
ems_status kr_pass(ems_ctx *c, KrArgs<R> &a) {
    for (auto &b : c->buckets) {
        if (!b.chain) continue;
        a.trees = b.d_trees;
        switch (b.M) {
            case 4: EMS_TRY((kr_launch<4, R>(c, b, a))); break;
            case 8: EMS_TRY((kr_launch<8, R>(c, b, a))); break;
            case 16: EMS_TRY((kr_launch<16, R>(c, b, a))); break;
            case 32: EMS_TRY((kr_launch<32, R>(c, b, a))); break;
            case 64: EMS_TRY((kr_launch<64, R>(c, b, a))); break;
            default: return fail(c, EMS_E_STATE, "unsupported chunk length");
        }
    }
    return EMS_OK;
}

ems_status run_pass(ems_ctx *c, double dt, int n_steps, int build_only) {
    if (c->prm.precision == EMS_F32) {
        KrArgs<float> a = kr_args<float>(c, dt, n_steps, build_only);
        return kr_pass<float>(c, a);
    }
    KrArgs<double> a = kr_args<double>(c, dt, n_steps, build_only);
    return kr_pass<double>(c, a);
}

// chunk length of the on-chip trajectory: the propagator and the table in
// about 96 KB of shared memory
int chunk_steps(int rmax, size_t eb) {
    const size_t budget = 96 * 1024, f = eb * (size_t)rmax * rmax;
    long kc = (long)((budget > f ? budget - f : 0) / (eb * (size_t)rmax)) - 1;
    if (kc > 256) kc = 256;
    if (kc < 8) kc = 8;
    return (int)kc;
}

// reduced-model eligibility (Eq. krylov_threshold): chains with n >= max(3q, 30);
// kept on the device and copied into the mode flags before every pass
ems_status ensure_q(ems_ctx *c, int q, double eta) {
    if (c->rmax == 0) return fail(c, EMS_E_STATE, "context created with method EMS_BE: no Krylov storage");
    if (q < 1 || 2 * q + 2 > c->rmax || !(eta > 0.0)) return fail(c, EMS_E_INVAL, "q must be 1..params.krylov_q, eta > 0");
    if (q != c->kr_q || eta != c->kr_eta) {
        c->kr_q = q;
        c->kr_eta = eta;
        c->kr_kc = chunk_steps(c->rmax, c->prm.precision == EMS_F32 ? 4 : 8);
        const int S = c->S, nt = c->n_trees;
        std::vector<int32_t> ok((size_t)S * nt, 0);
        for (int t = 0; t < nt; ++t) {
            const int64_t n = c->trees.off[t + 1] - c->trees.off[t];
            const bool e = c->pack[t].T > 1 && n >= (3 * q > 30 ? 3 * q : 30);
            for (int s = 0; s < S; ++s) ok[(size_t)s * nt + t] = e ? 1 : 0;
        }
        EMS_CUDA(c, cudaMemcpyAsync(c->d.kr_ok, ok.data(), 4 * ok.size(), cudaMemcpyHostToDevice, c->stream));
        EMS_CUDA(c, cudaMemsetAsync(c->d.kr_state, 0, sizeof(int32_t) * S * nt, c->stream));
        EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return EMS_OK;
}

ems_status set_modes(ems_ctx *c) {
    EMS_CUDA(c, cudaMemcpyAsync(c->d.kr_mode, c->d.kr_ok, sizeof(int32_t) * c->S * c->n_trees,
                                cudaMemcpyDeviceToDevice, c->stream));
    return EMS_OK;
}

}  // namespace

ems_status krylov_prepare(ems_ctx *c) {
    return ensure_q(c, c->kr_q > 0 ? c->kr_q : c->prm.krylov_q, c->kr_q > 0 ? c->kr_eta : c->prm.krylov_eta);
}

// one aging step: reduced models for the eligible chains (one launch per
// chunk shape), then backward Euler for the rest and for any tree that fell
// back.  No host synchronisation once krylov_prepare has run, so the TTF
// graph captures it.
ems_status krylov_stress(ems_ctx *c, double dt, int n_steps) {
    cudaStream_t st = c->stream;
    EMS_TRY(set_modes(c));
    EMS_CUDA(c, cudaMemsetAsync(c->d.counters, 0, 3 * sizeof(int32_t), st));
    EMS_CUDA(c, cudaMemsetAsync(c->d.kdone, 0, sizeof(int32_t) * c->S * c->n_trees, st));
    EMS_TRY(run_pass(c, dt, n_steps, 0));
    return launch_be(c, dt, n_steps);
}

ems_status krylov_advance(ems_ctx *c, double dt, int n_steps, int method, int *n_new) {
    (void)method;
    EMS_TRY(krylov_prepare(c));
    EMS_TRY(krylov_stress(c, dt, n_steps));
    c->t += dt * n_steps;
    if (n_new) EMS_CUDA(c, cudaMemcpyAsync(n_new, c->d.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    return EMS_OK;
}

}  // namespace ems

using namespace ems;

extern "C" ems_status ems_krylov_reduce(ems_ctx *c, int q, double eta, int *n_reduced, int *n_fallback) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    if (!c->have_u) return fail(c, EMS_E_STATE, "Krylov reduction before the first IR solve");
    EMS_TRY(ensure_q(c, q, eta));
    EMS_TRY(set_modes(c));
    EMS_TRY(forcing(c));
    EMS_TRY(run_pass(c, 0.0, 0, 1));
    const size_t ts = (size_t)c->S * c->n_trees;
    std::vector<int32_t> state(ts), mode(ts);
    EMS_CUDA(c, cudaMemcpyAsync(state.data(), c->d.kr_state, 4 * ts, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaMemcpyAsync(mode.data(), c->d.kr_ok, 4 * ts, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    int nr = 0, nf = 0;
    for (size_t k = 0; k < ts; ++k) {
        if (!mode[k]) continue;
        if (state[k] == 1) ++nr;
        if (state[k] == 2) ++nf;
    }
    if (n_reduced) *n_reduced = nr;
    if (n_fallback) *n_fallback = nf;
    return check_status(c);
}
