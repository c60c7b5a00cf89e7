// ems_ttf.cu -- coupled aging loop and time to failure (Sec. IV-A, Sec. V).
//
// Per aging step: forcing from the current currents, n_inner backward-Euler
// steps with nucleation, void-growth resistance, IR re-solve, max drop.  The
// only host traffic per aging step is the S drop fractions (and one status
// word); everything else stays on the device.
#include <cmath>
#include <vector>

#include "ems_internal.cuh"

using namespace ems;

extern "C" ems_status ems_ttf(ems_ctx *c, const ems_ttf_opts *opts, ems_ttf_result *out) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    const ems_params &p = c->prm;
    const int n_out = (opts && opts->n_outer > 0) ? opts->n_outer : p.n_outer;
    const double dto = p.horizon / p.n_outer, dti = dto / p.n_inner;
    const double thr = p.ir_fail_frac;
    const int S = c->S;
    cudaStream_t st = c->stream;
    std::vector<double> drop(S), prev(S), ttf(S, INFINITY);
    std::vector<double> all((size_t)S * (n_out + 1));
    std::vector<int32_t> iters(S);
    double it_total = 0.0;
    auto add_iters = [&]() -> ems_status {
        EMS_CUDA(c, cudaMemcpyAsync(iters.data(), c->d.ir_iters, 4 * S, cudaMemcpyDeviceToHost, st));
        EMS_CUDA(c, cudaStreamSynchronize(st));
        for (int s = 0; s < S; ++s) it_total += iters[s];
        return EMS_OK;
    };
    float ms_stress = 0.0f, ms_ir = 0.0f, ms = 0.0f;

    EMS_CUDA(c, cudaEventRecord(c->ev0, st));
    EMS_TRY(ir_assemble_and_solve(c, true));
    EMS_TRY(ir_currents_and_drop(c));
    EMS_CUDA(c, cudaEventRecord(c->ev1, st));
    EMS_CUDA(c, cudaMemcpyAsync(drop.data(), c->d.drop, 8 * S, cudaMemcpyDeviceToHost, st));
    EMS_TRY(check_status(c));
    EMS_TRY(add_iters());
    EMS_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    ms_ir += ms;
    for (int s = 0; s < S; ++s) {
        all[(size_t)s * (n_out + 1)] = drop[s];
        if (drop[s] >= thr) ttf[s] = 0.0;
        if (out && out->drop0) out->drop0[s] = drop[s];
    }
    if (opts && opts->screen) {
        EMS_TRY(screen(c));
        std::vector<uint8_t> mortal((size_t)S * c->n_trees);
        EMS_CUDA(c, cudaMemcpyAsync(mortal.data(), c->d.mortal, mortal.size(), cudaMemcpyDeviceToHost, st));
        EMS_CUDA(c, cudaStreamSynchronize(st));
        if (out && out->n_mortal)
            for (int s = 0; s < S; ++s) {
                int m = 0;
                for (int t = 0; t < c->n_trees; ++t) m += mortal[(size_t)s * c->n_trees + t];
                out->n_mortal[s] = m;
            }
    }
    double node_steps = 0.0;
    for (int k = 0; k < n_out; ++k) {
        const double t_prev = c->t;
        prev = drop;
        EMS_CUDA(c, cudaEventRecord(c->ev0, st));
        EMS_TRY(forcing(c));
        EMS_TRY(advance(c, dti, p.n_inner, nullptr, p.method));
        EMS_CUDA(c, cudaEventRecord(c->ev1, st));
        EMS_TRY(void_update(c, nullptr));
        cudaEvent_t e2, e3;
        EMS_CUDA(c, cudaEventCreate(&e2));
        EMS_CUDA(c, cudaEventCreate(&e3));
        EMS_CUDA(c, cudaEventRecord(e2, st));
        EMS_TRY(ir_assemble_and_solve(c, true));
        EMS_TRY(ir_currents_and_drop(c));
        EMS_CUDA(c, cudaEventRecord(e3, st));
        EMS_CUDA(c, cudaMemcpyAsync(drop.data(), c->d.drop, 8 * S, cudaMemcpyDeviceToHost, st));
        ems_status sx = check_status(c);
        if (sx == EMS_OK) {
            EMS_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
            ms_stress += ms;
            EMS_CUDA(c, cudaEventElapsedTime(&ms, e2, e3));
            ms_ir += ms;
        }
        cudaEventDestroy(e2);
        cudaEventDestroy(e3);
        if (sx != EMS_OK) return sx;
        EMS_TRY(add_iters());
        node_steps += (double)c->N * S * p.n_inner;
        for (int s = 0; s < S; ++s) {
            all[(size_t)s * (n_out + 1) + k + 1] = drop[s];
            if (std::isinf(ttf[s]) && prev[s] < thr && thr <= drop[s])
                ttf[s] = t_prev + (thr - prev[s]) / (drop[s] - prev[s]) * dto;
        }
    }
    if (out) {
        for (int s = 0; s < S; ++s) {
            if (out->ttf) out->ttf[s] = ttf[s];
            if (out->final_drop) out->final_drop[s] = drop[s];
        }
        if (out->drops)
            for (size_t q = 0; q < all.size(); ++q) out->drops[q] = all[q];
        if (out->n_voids) {
            std::vector<int32_t> cnt((size_t)S * c->n_trees);
            EMS_CUDA(c, cudaMemcpyAsync(cnt.data(), c->d.v_count, 4 * cnt.size(), cudaMemcpyDeviceToHost, st));
            EMS_CUDA(c, cudaStreamSynchronize(st));
            for (int s = 0; s < S; ++s) {
                int m = 0;
                for (int t = 0; t < c->n_trees; ++t) m += cnt[(size_t)s * c->n_trees + t];
                out->n_voids[s] = m;
            }
        }
        out->node_steps = node_steps;
        out->stress_ms = ms_stress;
        out->ir_ms = ms_ir;
        out->ir_iterations = it_total;
    }
    return EMS_OK;
}
