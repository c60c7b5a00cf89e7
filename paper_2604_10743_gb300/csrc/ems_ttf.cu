// ems_ttf.cu -- coupled aging loop and time to failure (Sec. IV-A, Sec. V).
//
// Per aging step: forcing from the current currents, n_inner backward-Euler
// steps with nucleation, void-growth resistance, IR re-solve, max drop, TTF
// crossing test.  All aging steps of all samples (BE, or the reduced models
// plus BE for the trees without one) are captured once into a CUDA graph and
// launched as one unit; the crossing test, the time and the PCG iteration
// count live on the device, and the host reads the results once.  The
// host-driven loop remains for runs longer than the configured schedule and
// on request (no_graph).
#include <cmath>
#include <vector>

#include "ems_internal.cuh"

namespace ems {
namespace {

__global__ void k_ttf_init(int S, int stride, double thr, const double *drop, double *ttf, double *drops,
                           double *iters_acc, const int32_t *iters, double t_now, double *gtime, int32_t *gstep) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) {
        drops[(int64_t)s * stride] = drop[s];
        ttf[s] = drop[s] >= thr ? 0.0 : INFINITY;
    }
    if (s == 0) {
        double a = 0.0;
        for (int k = 0; k < S; ++k) a += iters[k];
        *iters_acc = a;
        *gtime = t_now;
        *gstep = 0;
    }
}

// after aging step k: record the drop, detect the first crossing, advance time
__global__ void k_ttf_step(int S, int stride, double thr, double dto, const double *drop, double *ttf,
                           double *drops, double *iters_acc, const int32_t *iters, double *gtime, int32_t *gstep) {
    const int k = *gstep;
    const double t_prev = *gtime;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) {
        const double dp = drops[(int64_t)s * stride + k], dn = drop[s];
        drops[(int64_t)s * stride + k + 1] = dn;
        if (isinf(ttf[s]) && dp < thr && thr <= dn) ttf[s] = t_prev + (thr - dp) / (dn - dp) * dto;
    }
}

__global__ void k_ttf_tick(int S, double dto, const int32_t *iters, double *iters_acc, double *gtime,
                           int32_t *gstep) {
    double a = 0.0;
    for (int k = 0; k < S; ++k) a += iters[k];
    *iters_acc += a;
    *gtime += dto;
    *gstep += 1;
}

void stats(const std::vector<double> &ttf, ems_ttf_result *out) {
    double sum = 0.0, n = 0.0, cens = 0.0;
    for (double v : ttf) {
        if (std::isinf(v)) cens += 1.0;
        else { sum += v; n += 1.0; }
    }
    const double mean = n > 0 ? sum / n : NAN;
    double ss = 0.0;
    for (double v : ttf)
        if (!std::isinf(v)) ss += (v - mean) * (v - mean);
    const double sd = n > 1 ? std::sqrt(ss / (n - 1.0)) : (n == 1 ? 0.0 : NAN);
    out->ttf_mean = mean;
    out->ttf_std = sd;
    out->ttf_cov = sd / mean;
    out->n_censored = cens;
}

}  // namespace
}  // namespace ems

using namespace ems;

namespace {

// mortal-tree counts per sample from the screen's flags (already computed)
ems_status screen_counts(ems_ctx *c, ems_ttf_result *out) {
    const int S = c->S;
    std::vector<uint8_t> mortal((size_t)S * c->n_trees);
    EMS_CUDA(c, cudaMemcpyAsync(mortal.data(), c->d.mortal, mortal.size(), cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (out && out->n_mortal)
        for (int s = 0; s < S; ++s) {
            int m = 0;
            for (int t = 0; t < c->n_trees; ++t) m += mortal[(size_t)s * c->n_trees + t];
            out->n_mortal[s] = m;
        }
    return EMS_OK;
}

ems_status finish(ems_ctx *c, ems_ttf_result *out, const std::vector<double> &ttf, const std::vector<double> &drop,
                  const std::vector<double> &all, double node_steps, float ms_stress, float ms_ir, double it_total) {
    const int S = c->S;
    if (!out) return EMS_OK;
    for (int s = 0; s < S; ++s) {
        if (out->ttf) out->ttf[s] = ttf[s];
        if (out->final_drop) out->final_drop[s] = drop[s];
        if (out->drop0) out->drop0[s] = all[(size_t)s * (all.size() / S)];
    }
    if (out->drops)
        for (size_t q = 0; q < all.size(); ++q) out->drops[q] = all[q];
    if (out->n_voids) {
        std::vector<int32_t> cnt((size_t)S * c->n_trees);
        EMS_CUDA(c, cudaMemcpyAsync(cnt.data(), c->d.v_count, 4 * cnt.size(), cudaMemcpyDeviceToHost, c->stream));
        EMS_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int s = 0; s < S; ++s) {
            int m = 0;
            for (int t = 0; t < c->n_trees; ++t) m += cnt[(size_t)s * c->n_trees + t];
            out->n_voids[s] = m;
        }
    }
    out->node_steps = node_steps;
    unsigned long long work = 0;
    EMS_CUDA(c, cudaMemcpyAsync(&work, c->d.work, sizeof work, cudaMemcpyDeviceToHost, c->stream));
    EMS_CUDA(c, cudaStreamSynchronize(c->stream));
    out->node_steps_executed = (double)work;
    out->stress_ms = ms_stress;
    out->ir_ms = ms_ir;
    out->ir_iterations = it_total;
    stats(ttf, out);
    return EMS_OK;
}

// One aging step of every sample, recorded on c->stream (the capture
// stream): per window of samples, the window's coefficients, forcing, stress
// advance, void update and IR re-solve, then the crossing test; ev holds 4
// events per window (around the stress kernels, around the IR solve).
ems_status record_step(ems_ctx *c, double dto, double dti, bool kr, cudaEvent_t *ev) {
    const ems_params &p = c->prm;
    const int stride = p.n_outer + 1;
    int w = 0;
    EMS_TRY(each_window(c, [&](int, int ns) -> ems_status {
        cudaEvent_t *e = ev + 4 * (size_t)(w++);
        Dev &d = c->d;
        EMS_TRY(window_derive(c));
        EMS_TRY(forcing(c));
        EMS_CUDA(c, cudaEventRecordWithFlags(e[0], c->stream, cudaEventRecordExternal));
        EMS_TRY(kr ? krylov_stress(c, dti, p.n_inner) : launch_be(c, dti, p.n_inner));
        EMS_CUDA(c, cudaEventRecordWithFlags(e[1], c->stream, cudaEventRecordExternal));
        EMS_TRY(void_update(c, nullptr));
        EMS_CUDA(c, cudaEventRecordWithFlags(e[2], c->stream, cudaEventRecordExternal));
        if (windowed(c)) EMS_TRY(gather_x(c));
        EMS_TRY(ir_assemble_and_solve(c, true));
        EMS_TRY(ir_currents_and_drop(c));
        EMS_CUDA(c, cudaEventRecordWithFlags(e[3], c->stream, cudaEventRecordExternal));
        const unsigned gb = (unsigned)((ns + 255) / 256);
        k_ttf_step<<<gb, 256, 0, c->stream>>>(ns, stride, p.ir_fail_frac, dto, d.drop, d.gttf, d.gdrops, d.giters,
                                              d.ir_iters, d.gtime, d.gstep);
        ++c->launches;
        return EMS_OK;
    }));
    k_ttf_tick<<<1, 1, 0, c->stream>>>(c->S_all, dto, c->d.ir_iters, c->d.giters, c->d.gtime, c->d.gstep);
    ++c->launches;
    return EMS_OK;
}

// All aging steps as captured CUDA graphs (BE, or reduced models plus BE).
// Full layout: one graph holds every aging step.  Monte Carlo windows: one
// graph holds one aging step over all windows and is launched n_out times.
ems_status ttf_graph(ems_ctx *c, int n_out, ems_ttf_result *out) {
    const ems_params &p = c->prm;
    const double dto = p.horizon / p.n_outer, dti = dto / p.n_inner;
    const int S = c->S_all, stride = p.n_outer + 1;
    cudaStream_t st = c->stream;
    const unsigned gb = (unsigned)((S + 255) / 256);
    const bool win = windowed(c);
    const int n_win = win ? (S + c->W - 1) / c->W : 1;
    const int steps_per_graph = win ? 1 : n_out;
    EMS_CUDA(c, cudaEventRecord(c->ev0, st));
    EMS_TRY(each_window(c, [&](int, int) -> ems_status {
        if (windowed(c)) EMS_TRY(gather_x(c));
        EMS_TRY(ir_assemble_and_solve(c, true));
        return ir_currents_and_drop(c);
    }));
    Dev &d = c->d;
    k_ttf_init<<<gb, 256, 0, st>>>(S, stride, p.ir_fail_frac, d.drop, d.gttf, d.gdrops, d.giters, d.ir_iters, c->t,
                                   d.gtime, d.gstep);
    ++c->launches;
    EMS_CUDA(c, cudaGetLastError());
    // every tree factors on its first aging step through its dirty flag, so
    // the captured launches never need a global refactor
    EMS_CUDA(c, cudaMemsetAsync(d.kr_mode, 0, sizeof(int32_t) * S * c->n_trees, st));
    EMS_CUDA(c, cudaMemsetAsync(d.kdone, 0, sizeof(int32_t) * S * c->n_trees, st));
    const bool kr = p.method != EMS_BE;
    if (kr) EMS_TRY(krylov_prepare(c));
    if (c->factored_dt != dti) {
        std::vector<int32_t> ones((size_t)S * c->n_trees, 1);
        EMS_CUDA(c, cudaMemcpyAsync(d.dirty, ones.data(), 4 * ones.size(), cudaMemcpyHostToDevice, st));
        EMS_CUDA(c, cudaStreamSynchronize(st));
        c->factored_dt = dti;
    }
    const int graph_key = win ? -1 : n_out;
    if (!c->ttf_graph || c->graph_nout != graph_key || c->graph_dt != dti) {
        if (c->ttf_graph) { cudaGraphExecDestroy(c->ttf_graph); c->ttf_graph = nullptr; }
        cudaGraph_t g = nullptr;
        const int64_t l0 = c->launches;
        for (auto e : c->gev) cudaEventDestroy(e);
        c->gev.assign(4 * (size_t)steps_per_graph * n_win, nullptr);
        for (auto &e : c->gev) EMS_CUDA(c, cudaEventCreate(&e));
        // capture on a library stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph launches on the caller's
        if (!c->cap_stream) EMS_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        const cudaStream_t user = c->stream;
        c->stream = c->cap_stream;
        cudaError_t eb = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (eb != cudaSuccess) { c->stream = user; cudaGetLastError(); return cuda_check(c, eb, "cudaStreamBeginCapture"); }
        c->graph_capturing = true;
        ems_status sx = EMS_OK;
        for (int k = 0; k < steps_per_graph && sx == EMS_OK; ++k)
            sx = record_step(c, dto, dti, kr, &c->gev[4 * (size_t)k * n_win]);
        c->graph_capturing = false;
        map_all(c);
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        c->stream = user;
        if (sx != EMS_OK || e != cudaSuccess) cudaGetLastError();
        if (sx != EMS_OK) { if (g) cudaGraphDestroy(g); return sx; }
        if (e != cudaSuccess) return cuda_check(c, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->ttf_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { c->ttf_graph = nullptr; return cuda_check(c, e, "cudaGraphInstantiate"); }
        c->graph_nout = graph_key;
        c->graph_dt = dti;
        c->graph_launches = c->launches - l0;
        c->launches = l0;                             // counted when launched
    }
    float ms_stress = 0.0f, ms_ir = 0.0f;
    auto add_times = [&]() -> ems_status {
        for (size_t q = 0; q < c->gev.size(); q += 4) {
            float a = 0.0f, b = 0.0f;
            EMS_CUDA(c, cudaEventElapsedTime(&a, c->gev[q], c->gev[q + 1]));
            EMS_CUDA(c, cudaEventElapsedTime(&b, c->gev[q + 2], c->gev[q + 3]));
            ms_stress += a;
            ms_ir += b;
        }
        return EMS_OK;
    };
    for (int k = 0; k < n_out; k += steps_per_graph) {
        EMS_CUDA(c, cudaGraphLaunch(c->ttf_graph, st));
        c->launches += c->graph_launches;
        if (win) {                                    // the step graph's events are re-recorded next launch
            EMS_CUDA(c, cudaStreamSynchronize(st));
            EMS_TRY(add_times());
        }
    }
    EMS_CUDA(c, cudaEventRecord(c->ev1, st));
    std::vector<double> ttf(S), all((size_t)S * stride), drop(S);
    double it_total = 0.0;
    EMS_CUDA(c, cudaMemcpyAsync(ttf.data(), d.gttf, 8 * S, cudaMemcpyDeviceToHost, st));
    EMS_CUDA(c, cudaMemcpyAsync(all.data(), d.gdrops, 8 * all.size(), cudaMemcpyDeviceToHost, st));
    EMS_CUDA(c, cudaMemcpyAsync(&it_total, d.giters, 8, cudaMemcpyDeviceToHost, st));
    EMS_TRY(check_status(c));
    if (!win) EMS_TRY(add_times());
    c->t += dto * n_out;
    std::vector<double> trimmed((size_t)S * (n_out + 1));
    for (int s = 0; s < S; ++s) {
        for (int k = 0; k <= n_out; ++k) trimmed[(size_t)s * (n_out + 1) + k] = all[(size_t)s * stride + k];
        drop[s] = all[(size_t)s * stride + n_out];
    }
    if (out) out->graph_launch = 1.0;
    return finish(c, out, ttf, drop, trimmed, (double)c->N * S * p.n_inner * n_out, ms_stress, ms_ir, it_total);
}

}  // namespace

extern "C" ems_status ems_ttf(ems_ctx *c, const ems_ttf_opts *opts, ems_ttf_result *out) {
    if (!c) return EMS_E_INVAL;
    if (!c->loaded) return fail(c, EMS_E_STATE, "no grid loaded");
    const ems_params &p = c->prm;
    const int n_out = (opts && opts->n_outer > 0) ? opts->n_outer : p.n_outer;
    if (out) out->graph_launch = 0.0;
    EMS_CUDA(c, cudaMemsetAsync(c->d.work, 0, sizeof(unsigned long long), c->stream));
    if (opts && opts->screen) {
        EMS_TRY(each_window(c, [&](int, int) -> ems_status {
            if (windowed(c)) EMS_TRY(gather_x(c));
            EMS_TRY(ir_assemble_and_solve(c, true));
            EMS_TRY(ir_currents_and_drop(c));
            EMS_TRY(window_derive(c));
            return screen(c);
        }));
        EMS_TRY(screen_counts(c, out));
    }
    if (!(opts && opts->no_graph) && n_out <= p.n_outer) return ttf_graph(c, n_out, out);

    const double dto = p.horizon / p.n_outer, dti = dto / p.n_inner;
    const double thr = p.ir_fail_frac;
    const int S = c->S_all;
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
    cudaEvent_t e2, e3;
    EMS_CUDA(c, cudaEventCreate(&e2));
    EMS_CUDA(c, cudaEventCreate(&e3));
    struct Guard {
        cudaEvent_t a, b;
        ~Guard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } guard{e2, e3};

    EMS_CUDA(c, cudaEventRecord(c->ev0, st));
    EMS_TRY(each_window(c, [&](int, int) -> ems_status {
        if (windowed(c)) EMS_TRY(gather_x(c));
        EMS_TRY(ir_assemble_and_solve(c, true));
        return ir_currents_and_drop(c);
    }));
    EMS_CUDA(c, cudaEventRecord(c->ev1, st));
    EMS_CUDA(c, cudaMemcpyAsync(drop.data(), c->d.drop, 8 * S, cudaMemcpyDeviceToHost, st));
    EMS_TRY(check_status(c));
    EMS_TRY(add_iters());
    EMS_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    ms_ir += ms;
    for (int s = 0; s < S; ++s) {
        all[(size_t)s * (n_out + 1)] = drop[s];
        if (drop[s] >= thr) ttf[s] = 0.0;
    }
    double node_steps = 0.0;
    for (int k = 0; k < n_out; ++k) {
        const double t_prev = c->t;
        prev = drop;
        EMS_TRY(each_window(c, [&](int, int) -> ems_status {
            c->t = t_prev;
            EMS_CUDA(c, cudaEventRecord(c->ev0, st));
            EMS_TRY(window_derive(c));
            EMS_TRY(forcing(c));
            EMS_TRY(advance(c, dti, p.n_inner, nullptr, p.method));
            EMS_CUDA(c, cudaEventRecord(c->ev1, st));
            EMS_TRY(void_update(c, nullptr));
            EMS_CUDA(c, cudaEventRecord(e2, st));
            if (windowed(c)) EMS_TRY(gather_x(c));
            EMS_TRY(ir_assemble_and_solve(c, true));
            EMS_TRY(ir_currents_and_drop(c));
            EMS_CUDA(c, cudaEventRecord(e3, st));
            EMS_CUDA(c, cudaStreamSynchronize(st));
            EMS_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
            ms_stress += ms;
            EMS_CUDA(c, cudaEventElapsedTime(&ms, e2, e3));
            ms_ir += ms;
            return EMS_OK;
        }));
        c->t = t_prev + dto;
        EMS_CUDA(c, cudaMemcpyAsync(drop.data(), c->d.drop, 8 * S, cudaMemcpyDeviceToHost, st));
        EMS_TRY(check_status(c));
        EMS_TRY(add_iters());
        node_steps += (double)c->N * S * p.n_inner;
        for (int s = 0; s < S; ++s) {
            all[(size_t)s * (n_out + 1) + k + 1] = drop[s];
            if (std::isinf(ttf[s]) && prev[s] < thr && thr <= drop[s])
                ttf[s] = t_prev + (thr - prev[s]) / (drop[s] - prev[s]) * dto;
        }
    }
    return finish(c, out, ttf, drop, all, node_steps, ms_stress, ms_ir, it_total);
}
