// ems_internal.cuh -- internal definitions of the GB300 EM/TM engine.
//
// Device data layout (all arrays live in one workspace block):
//   canonical per-node arrays   [S][N]  (N = stress nodes, canonical order)
//   packed per-node arrays      [S][P]  (P = padded nodes of the packed layout)
//   per-segment arrays          [S][n_seg]
//   IR arrays                   [S][n_nodes] / CSR [S][nnz]
// A chain tree handled by T threads with chunks of M nodes stores canonical
// node i at packed offset pbase + (i % M) * T + (i / M): at every step of a
// chunk sweep the T threads touch T consecutive elements (coalesced).
// Branched trees use T = 1, M = n (packed == canonical order).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ems.h"

#define EMS_MAX_VOIDS 256     // compile-time cap on void slots per (tree, sample)
#define EMS_MAX_RASTER (1024 * 1024)  // thermal raster values held in the workspace
#define EMS_MAX_PERT 4096             // values of one sample's temperature perturbation raster
// resistance of a via a void has severed (early failure), Ohm
constexpr double kOpenCircuit = 1.0e9;
// polls a grid-barrier wait makes before it gives up (about a second)
constexpr long long kDefaultWaitLimit = 1LL << 24;

namespace ems {

// Multigrid hierarchy of the IR system (ems_mg.cu).  Offsets index the flat
// int / double arrays of the hierarchy (levels >= 1 hold A and its inverse
// diagonal; levels < L-1 hold the prolongation P and restriction R = P^T)
// and the per-sample scratch (e, t on every level, r below the finest).
#define EMS_MG_MAXLV 8
struct MGLevelDesc {
    int n = 0;
    int64_t a_ptr = 0, a_col = 0, a_val = 0, dinv = 0;
    int64_t p_ptr = 0, p_col = 0, p_val = 0, r_ptr = 0, r_col = 0, r_val = 0;
    int64_t e = 0, t = 0, r = 0;
};
struct MGHost {
    int L = 0;                                  // levels (0: no hierarchy)
    MGLevelDesc lv[EMS_MG_MAXLV];
    std::vector<int32_t> ints;
    std::vector<double> dbls;
    int64_t cinv = 0, per_sample = 0, nnz = 0; // coarsest dense inverse offset, scratch per sample
};
struct MGDevice {
    int L = 0;
    int small = 1024;                           // grid mode: block 0 alone runs levels this small
    MGLevelDesc lv[EMS_MG_MAXLV];
    int64_t cinv = 0, per_sample = 0;
    const int32_t *I = nullptr;
    const double *D = nullptr;
    const float *F = nullptr;                   // D rounded to FP32 (the FP32 V-cycle of FP32 contexts)
    double *scratch = nullptr;                  // [S][per_sample]
};

// Largest team (threads per chain) each chunk length supports: the chunk's
// stress lives in registers (M values of R per thread) and the team must fit
// the 64K-register file of one SM.
template <typename R, int M> struct ChainMaxThreads;
template <int M> struct ChainMaxThreads<double, M> {
    static constexpr int value = M <= 4 ? 1024 : M == 8 ? 896 : M == 16 ? 640 : M == 32 ? 384 : 256;
};
// the FP32 kernel solves for the increment; it keeps one chunk in registers
// and stages the forward sweep in shared memory (8 bytes per node, at most
// 160 KB per CTA)
template <int M> struct ChainMaxThreads<float, M> {
    static constexpr int value = M <= 8 ? 1024 : M == 16 ? 640 : M == 32 ? 640 : 320;
};
// minimum resident CTAs the register budget is sized for (launch bounds):
// FP32 chunks of <= 16 nodes get 51 registers so that four 320-thread trees
// share an SM (512 trees of 5,101 nodes then run in one wave on 152 SMs)
template <typename R, int M> struct ChainMinBlocks { static constexpr int value = 1; };
template <> struct ChainMinBlocks<float, 16> { static constexpr int value = 2; };
inline int chain_max_threads(int prec, int M) {
    if (prec == EMS_F32) return M <= 8 ? 1024 : M == 16 ? 640 : M == 32 ? 640 : 320;
    return M <= 4 ? 1024 : M == 8 ? 896 : M == 16 ? 640 : M == 32 ? 384 : 256;
}
// FP32 register-resident kernel: threads a CTA may have per chunk length
// (its state, coefficients and compensation stay in registers)
inline int reg_max_threads(int M) { return M == 4 ? 896 : M == 8 ? 576 : M == 16 ? 320 : 0; }
constexpr size_t kSharedCoefBytes = 200 * 1024; // FP32 streaming kernel: coefficients staged while they fit
// cluster chain kernel: nodes per thread of the built-in choice, and the
// threads a CTA may have for each compiled (precision, M, CL); 0: none.
// FP32 16 per thread: <= 256 threads (255 registers) on 5- and 6-CTA clusters.
inline int cluster_chunk(int prec) { return prec == EMS_F32 ? 16 : 8; }
inline int cluster_max_threads(int prec, int M, int CL) {
    if (prec == EMS_F32) {
        if (M == 16) return (CL == 2 || CL == 4 || CL == 8) ? 320 : (CL == 5 || CL == 6) ? 256 : 0;
        return 0;
    }
    return (M == 8 && (CL == 2 || CL == 4 || CL == 8)) ? 320 : 0;
}
// cluster chain kernel with the coefficients in shared memory (FP32, 16 per
// thread, two or more CTAs per SM): threads a CTA may have per CL, and the
// dynamic shared memory of a CTA (alpha, dt g, dt f, w and the threshold:
// 20 bytes per node)
inline int cluster_smem_max_threads(int M, int CL) {
    return M == 16 ? ((CL == 2 || CL == 4 || CL == 8) ? 320 : (CL == 5 || CL == 6) ? 256 : 0) : 0;
}
inline size_t cluster_smem_bytes(int M, int T_cta) { return (size_t)5 * sizeof(float) * M * T_cta; }
// raises those kernels' shared-memory limit; ems_create calls it, outside any
// stream capture (ems_chain_cl_f32s.cu)
cudaError_t cluster_smem_init();

// host arrays that a pass fills completely: resize leaves trivial elements
// unset instead of zeroing them first (the first touch then happens in the
// filling pass, on its threads)
template <class T>
struct NoInit : std::allocator<T> {
    template <class U> struct rebind { using other = NoInit<U>; };
    NoInit() noexcept = default;
    template <class U> NoInit(const NoInit<U> &) noexcept {}
    template <class U> void construct(U *p) noexcept { ::new (static_cast<void *>(p)) U; }
    template <class U, class... A> void construct(U *p, A &&...a) { ::new (static_cast<void *>(p)) U(static_cast<A &&>(a)...); }
};
template <class T> using hvec = std::vector<T, NoInit<T>>;

// fn(i) for i in [0, n) on the host's cores (an atomic counter hands out the
// items; fn must only write what item i owns)
template <class F>
void parallel_for(int n, F &&fn) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nthr = std::min(std::min(hw, 32), std::max(1, n / 8));
    if (nthr <= 1) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    std::atomic<int> next(0);
    auto work = [&]() {
        for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) fn(i);
    };
    std::vector<std::thread> th;
    th.reserve(nthr - 1);
    for (int k = 1; k < nthr; ++k) th.emplace_back(work);
    work();
    for (auto &x : th) x.join();
}

// ---------------------------------------------------------------------------
// Host-side tree extraction result (canonical order)
// ---------------------------------------------------------------------------
struct HostTrees {
    int n_trees = 0;
    std::vector<int64_t> off;          // [n_trees+1]
    hvec<int32_t> par;                 // tree-local parent, -1 at the root
    hvec<int32_t> face_seg;            // segment of the face to the parent (-1 root)
    hvec<double> face_dx, face_area;
    hvec<int8_t> face_sign;            // +1 if parent->child is the segment's a->b
    hvec<double> x, y;
    hvec<int32_t> owner_seg;           // MC factor segment of the node
    hvec<int32_t> inc_ptr, inc_seg;    // incident tree segments (IR nodes), CSR
    std::vector<int32_t> child_ptr, child_idx;  // tree-local children, CSR over nodes
    std::vector<uint8_t> is_chain;     // per tree
    std::vector<int32_t> tree_of_seg;  // per segment
    hvec<int32_t> ir_id;               // per stress node: its IR node, -1 inside a segment
    hvec<int32_t> ir_par;              // per IR stress node: tree-local index of the parent IR stress node (-1 root)
};

// Packing of one tree
struct TreePack {
    int T, M;          // threads per tree and chunk length (T = 1 for branched)
    int64_t pbase;     // packed base (within one sample)
    int CL = 1;        // CTAs per tree (a thread-block cluster when > 1; T counts all of them)
    int kind = 0;      // EMS_CHAIN_* kernel of a chain
};

struct Bucket {        // trees launched together: same kernel, T, M and CL
    int T, M;
    int CL = 1;        // CTAs per tree: T / CL threads each
    int kind = 0;      // EMS_CHAIN_* (chains)
    bool chain;
    std::vector<int32_t> trees;
    int32_t *d_trees = nullptr;
};

// ---------------------------------------------------------------------------
// Device arrays (pointers into the workspace)
// ---------------------------------------------------------------------------
struct Dev {
    // grid
    int32_t *seg_a, *seg_b;
    double *seg_R0, *seg_W, *seg_H;
    double *R, *j;                     // [S][n_seg]
    // IR (free-node system)
    int32_t *ir_free_of_node;          // node -> free index or -1
    int32_t *ir_node_of_free;          // free index -> node
    int32_t *csr_ptr, *csr_col;        // [nf+1], [nnz]
    int32_t *ent_ptr, *ent_seg;        // per nnz: contributing segments (diag +, off -)
    int8_t *ent_diag;                  // per nnz: 1 if diagonal
    int32_t *rhs_ptr, *rhs_seg;        // per free row: segments to a pad
    double *rhs_padV;                  // matching pad voltage
    double *sink_of_free;              // [nf] current drawn
    double *csr_val;                   // [S][nnz]
    double *ir_b, *ir_dinv;            // [S][nf]
    double *ir_x, *ir_r, *ir_p, *ir_Ap, *ir_z;  // [S][nf]
    float *val32, *dinv32;             // FP32 copies for the inner solve ([S][nnz], [S][nf])
    float *r32, *p32, *Ap32, *z32, *d32;      // [S][nf] inner FP32 CG vectors
    double *u;                         // [S][n_nodes]
    double *pad_V_of_node;             // [n_nodes] NaN if not a pad
    double *drop;                      // [S]
    double *red;                       // reduction scratch
    int32_t *ir_iters;                 // [S]
    unsigned int *gbar;                // grid barrier words
    // trees (canonical)
    int64_t *toff;                     // [n_trees+1]
    int32_t *par, *face_seg, *owner_seg, *inc_ptr, *inc_seg, *child_ptr, *child_idx;
    int8_t *face_sign;
    double *face_dx, *face_area, *nx_, *ny_;
    double *Tn;                        // [N] node temperature
    double *Mface;                     // [S][N] TM term per face (per sample: temperature perturbations)
    double *fb_ka, *fb_g, *fb_M;       // [N] per face without the sample's kappa factor: a kappa, a kappa / dx, M
                                       // (from the node temperatures; rebuilt when they change)
    double *V;                         // [N]
    double *kap_a, *g, *leak, *thr;    // [S][N]
    double *f;                         // [S][N] forcing
    double *sig_ss;                    // [S][N] steady state (screen)
    // packing
    int64_t *pbase;                    // [n_trees]
    int32_t *pT, *pM;                  // [n_trees]
    // packed state and factors: element type is float or double (precision)
    void *sig, *alpha, *beta, *gam, *uu, *Pf, *Pb, *pinv;   // [S][P]
    void *dtg, *dtl;                   // [S][P] FP32 increment form: dt g per face, dt leak per node
    void *kc;                          // [S][P] FP32 streaming chain kernel: compensation of the state sums
    // voids per (sample, tree)
    int32_t *v_count;                  // [S][n_trees]
    int32_t *v_node, *v_seg;           // [S][n_trees][MAXV]
    double *v_vol, *v_tnuc;            // [S][n_trees][MAXV]
    int32_t *dirty;                    // [S][n_trees] refactor needed
    int32_t *status;                   // [8] device error words
    int32_t *counters;                 // [8]
    uint8_t *mortal;                   // [S][n_trees]
    double *ssmax;                     // [S][n_trees]
    double *kfac, *sfac;               // [S][n_seg] MC multipliers (1 when absent)
    double *thr0;                      // [S][N] critical stress without voids
    double *R_prev;                    // [S][n_seg]
    double *raster;                    // thermal raster (up to EMS_MAX_RASTER values)
    double *pert;                      // [S][EMS_MAX_PERT] per-sample temperature perturbation rasters
    // rational Krylov reduced models (allocated when params.method != EMS_BE)
    void *kr_V;                        // [S][RMAX][P] basis columns (context precision); RMAX = 2q + 2
    double *kr_Ah, *kr_Ch;             // [S][nt][RMAX^2] reduced A_h, C_h (cached base block + current block)
    double *kr_Lm, *kr_Xs;             // [S][nt][RMAX^2], [S][nt][RMAX (RMAX+1)] Cholesky / solve scratch
    int32_t *kr_ok;                    // [S][nt] reduced-model eligibility (Eq. krylov_threshold)
    double *kr_sp, *kr_sg, *kr_su, *kr_sPf, *kr_sPb;   // [S][P] factors of C - t_s A
    double *kr_s0;                     // [S][nt] expansion point s0 = 1/t_s
    int32_t *kr_r, *kr_state;          // [S][nt] basis size; 0 none/stale, 1 valid, 2 fall back to BE
    int32_t *kr_mode, *kdone;          // [S][nt] 1 = advanced by the reduced model; steps done
    // device-side TTF bookkeeping (graph-captured runs)
    double *gtime;                     // [1] simulated time at the start of the aging step
    double *gttf, *gdrops, *giters;    // [S], [S][n_outer+1], [1]
    int32_t *gstep;                    // [1] aging steps done
    // learned surrogate: features, predictions and the step schedule
    float *feat, *pred;                // [S][n_trees][24], [S][n_trees][2]
    int32_t *mg_i;                     // multigrid hierarchy (ints, doubles, scratch)
    double *mg_d, *mg_sc;
    float *mg_f;
    int32_t *sched;                    // [S][n_trees] step schedule: <= 1 fine, r > 1 r-times coarser, < 0 frozen
    double *fdt;                       // [S][n_trees] step the packed factors were built for
    unsigned long long *work;          // [1] node-steps the stress kernels executed
    // Joule-heating profile (ems_joule.cu)
    int32_t *ir_id, *ir_par;           // [N] per stress node
    double *node_x, *node_y, *seg_L;   // IR node coordinates [n_nodes], segment lengths [n_seg]
    int8_t *ir_fixed;                  // [n_nodes] 1: temperature given (via between layers, or a pad)
    double *T_ir;                      // [n_nodes] IR node temperatures of the last profile
    int32_t *up_via;                   // [n_nodes] via resistor up to a strictly higher layer, -1 none
};

}  // namespace ems

struct ems_ctx {
    ems_params prm;
    // Monte Carlo layout: S_all samples hold their state; the per-node
    // coefficient arrays and IR work vectors hold W of them (W == S_all: the
    // full layout).  Calls walk the samples in windows of W: S is the number
    // mapped now, starting at win_s0, and d points the per-sample state
    // arrays of d_all at that window.
    int S_all = 1, W = 1, win_s0 = 0;
    ems::Dev d_all{};
    cudaStream_t stream = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    bool loaded = false;
    std::string err;
    // sizes
    int n_nodes = 0, n_seg = 0, n_pads = 0, n_sinks = 0, S = 1;
    int nf = 0;                // free IR nodes
    int64_t nnz = 0;
    int64_t N = 0;             // stress nodes (canonical)
    int64_t P = 0;             // packed stress nodes per sample
    int n_trees = 0;
    int maxv = 16;
    double t = 0.0;            // simulated time
    double factored_dt = -1.0; // dt the packed factors were built for
    bool have_u = false;       // IR solved at least once
    ems::HostTrees trees;
    std::vector<ems::TreePack> pack;
    std::vector<ems::Bucket> buckets;
    std::vector<ems_chain_rule> rules;   // chain shapes for the next load (autotuner's table)
    struct TuneRec { ems_chain_rule shape; double ms; int group; };
    std::vector<TuneRec> tune_log;       // every shape the last autotune timed
    ems::Dev d{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int coop_blocks = 0;       // resident CTAs for the cooperative PCG
    int mg_blocks = 0;         // resident CTAs for the cooperative multigrid PCG
    int mg_cluster = 0;        // CTAs per cluster of the cluster multigrid PCG (0 unknown, -1 none)
    ems::MGDevice mg;          // IR multigrid hierarchy (mg.L = 0: Jacobi only)
    int64_t launches = 0;      // kernels this context has launched
    int cluster_ok = -1;       // cluster PCG residency (-1 unknown, 0 no, 1 yes)
    int64_t ir_iter_total = 0; // PCG iterations accumulated by ems_ttf (inner iterations)
    int rmax = 0;              // Krylov basis capacity (2 q), 0 without Krylov storage
    bool graph_capturing = false;  // kernels read the time from device memory
    cudaGraphExec_t ttf_graph = nullptr;  // captured TTF run and what it was captured for
    cudaStream_t cap_stream = nullptr;    // library stream used only to capture graphs
    int graph_nout = 0;
    int64_t graph_launches = 0;   // kernels inside the captured graph
    std::vector<cudaEvent_t> gev;  // 4 per captured aging step: stress and IR start / end
    double graph_dt = 0.0;
    int kr_q = 0;              // q and eta of the reduced models currently built
    double kr_eta = 1.0;
    int kr_kc = 64;            // steps per on-chip chunk of the reduced trajectory
    double sched_guard = 0.8;  // coarse trees turn fine once sigma >= guard * lowest sigma_crit
    bool joule = false;        // node temperatures hold a Joule-heating profile (not the raster)
    // thermal raster currently set (nx = 0: uniform T0)
    int rnx = 0, rny = 0;
    double rx0 = 0, ry0 = 0, rx1 = 0, ry1 = 0;
    int pnx = 0, pny = 0;      // per-sample perturbation rasters over the map's extent (0: none)
};

namespace ems {

// helpers implemented in ems_host.cu
ems_status fail(ems_ctx *c, ems_status s, const std::string &msg);
ems_status cuda_check(ems_ctx *c, cudaError_t e, const char *what);
size_t elem_bytes(const ems_ctx *c);

// IR (ems_ir.cu, ems_mg.cu)
ems_status ir_assemble_and_solve(ems_ctx *c, bool warm);
ems_status mg_solve(ems_ctx *c);
void mg_build(int nf, const std::vector<int32_t> &ptr, const std::vector<int32_t> &col,
              const std::vector<int32_t> &ent_ptr, const std::vector<int32_t> &ent_seg,
              const std::vector<int8_t> &ent_diag, const double *R0, int min_rows, MGHost &h);
ems_status ir_currents_and_drop(ems_ctx *c);
ems_status currents(ems_ctx *c);
ems_status check_status(ems_ctx *c);

// stress (ems_stress.cu)
ems_status krylov_prepare(ems_ctx *c);
ems_status krylov_stress(ems_ctx *c, double dt, int n_steps);
ems_status node_physics(ems_ctx *c);
ems_status forcing(ems_ctx *c);
ems_status advance(ems_ctx *c, double dt, int n_steps, int *n_new, int method);
ems_status launch_be(ems_ctx *c, double dt, int n_steps);
ems_status void_update(ems_ctx *c, int *n_changed);
ems_status screen(ems_ctx *c);
ems_status pack_sigma(ems_ctx *c, bool to_packed);
ems_status init_sigma(ems_ctx *c);
ems_status sample_physics(ems_ctx *c);     // kappa, conductances, leak, thresholds of the mapped samples
ems_status face_base(ems_ctx *c);          // sample-independent face terms after the node temperatures changed

// Monte Carlo windows (ems_host.cu)
void map_window(ems_ctx *c, int s0, int ns);   // map samples [s0, s0 + ns) (ns <= W)
void map_all(ems_ctx *c);                      // every sample; per-node arrays are window-sized
ems_status gather_x(ems_ctx *c);               // IR initial guess of the mapped samples from u
ems_status window_derive(ems_ctx *c);          // per-node coefficients of the mapped window
// chain shapes: validity of (kind, M, CL) for n nodes (team size in *T), the
// built-in choice, and the rules' choice (backward Euler) over it
bool shape_valid(int64_t n, int prec, int kind, int M, int CL, int *T);
void chain_shape(int64_t n, int prec, int method, const std::vector<ems_chain_rule> *rules, int *T, int *M,
                 int *CL, int *kind);
std::vector<ems_chain_rule> shape_candidates(int64_t n, int prec);

// Krylov (ems_krylov.cu)
ems_status krylov_advance(ems_ctx *c, double dt, int n_steps, int method, int *n_new);

}  // namespace ems

namespace ems {
inline bool windowed(const ems_ctx *c) { return c->W < c->S_all; }

// Run fn(s0, ns) once per window of samples with that window mapped (one
// call over every sample with the full layout), then map every sample again.
template <class F>
ems_status each_window(ems_ctx *c, F &&fn) {
    if (!windowed(c)) return fn(0, c->S_all);
    ems_status st = EMS_OK;
    for (int s0 = 0; s0 < c->S_all && st == EMS_OK; s0 += c->W) {
        map_window(c, s0, c->S_all - s0 < c->W ? c->S_all - s0 : c->W);
        st = fn(s0, c->S);
    }
    map_all(c);
    return st;
}
}  // namespace ems

#define EMS_CUDA(c, call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ems::cuda_check((c), e_, #call); \
    } while (0)
#define EMS_TRY(call)                                       \
    do {                                                    \
        ems_status s_ = (call);                             \
        if (s_ != EMS_OK) return s_;                        \
    } while (0)
