/*
 * ems.h -- C ABI of the GB300 EM/TM stress / void / IR-drop engine.
 *
 * The engine runs the hot path of EMSpice 3 (arXiv 2604.10743) on one GPU:
 * transient electromigration + thermomigration stress on every interconnect
 * tree of a power grid (Korhonen's PDE, Sec. III-D, Eq. tm_aware_korhonen_pde),
 * advanced by backward-Euler steps (Sec. IV-B) or a rational Krylov reduced
 * model (Sec. IV-E), with void nucleation and growth (Sec. III-D.2/3), void
 * resistance write-back (Sec. IV-C) and IR-drop re-solves (Sec. III-C) up to
 * the 10 %-IR-drop time to failure (Sec. V).
 *
 * Conventions
 *   - Every call returns an ems_status; ems_last_error() gives a message.
 *   - All calls on one context are ordered on the context's CUDA stream; a
 *     call that returns host data synchronises that stream.
 *   - Host input arrays are read during the call and not retained.
 *   - Host output arrays are caller-allocated with the sizes stated.
 *   - Units are SI (m, s, Pa, K, A, V, Ohm).
 *   - Monte Carlo: a context holds S >= 1 samples; per-sample outputs are
 *     laid out sample-major ([S][...]).
 *
 * Stress-node order ("canonical order") used by every per-node array:
 *   trees are the connected components of same-layer segments (vias separate
 *   trees), ordered by their smallest segment id.  A tree's nodes are the IR
 *   nodes it touches plus seg_cells-1 interior nodes per segment.  Node 0 is
 *   the root, the lowest-id IR node of degree one in the tree; the rest follow
 *   depth-first, child segments in increasing segment id, each segment's
 *   interior nodes listed from the parent end, then its far IR node.
 *   Trees are concatenated in tree order.
 */
#ifndef EMS_H
#define EMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EMS_OK = 0,
    EMS_E_INVAL = 1,      /* bad argument or input (NaN, negative length, cycle, island) */
    EMS_E_STATE = 2,      /* call out of order (e.g. stress advance before a grid is loaded) */
    EMS_E_NOMEM = 3,      /* workspace too small or device allocation failed */
    EMS_E_CUDA = 4,       /* a CUDA runtime call failed */
    EMS_E_NOCONV = 5,     /* IR PCG did not reach its tolerance within its iteration cap */
    EMS_E_TIMEOUT = 6,    /* a device-side wait ran out its iteration limit */
    EMS_E_BREAKDOWN = 7,  /* Krylov basis broke down (tree falls back to backward Euler) */
    EMS_E_OVERFLOW = 8    /* more voids in one tree than max_voids_per_tree */
} ems_status;

enum { EMS_F64 = 0, EMS_F32 = 1 };                 /* stress-path arithmetic */
enum { EMS_BE = 0, EMS_KRYLOV = 1, EMS_AUTO = 2 }; /* stress method */

/*
 * Material and numerical settings (the paper's YAML parameter file,
 * Sec. IV-A).  Symbols as in Sec. III-D: kappa = D0 exp(-Ea/(k_B T)) B Omega
 * / (k_B T); S = e Z* rho_Cu j / Omega; M = Q* / (Omega T) dT/dx.
 */
typedef struct {
    double e_charge, k_B, Omega, rho_Cu, B_modulus, Z_star, D0, Ea, Q_star;
    double delta;          /* void interface thickness (Robin BC, Eq. incubation_bc) */
    double rho_Ta, h_Ta;   /* barrier resistivity / thickness (void growth dR) */
    double sigma_T;        /* initial residual stress (Eq. tm_aware_korhonen_ic) */
    double sigma_crit;     /* critical stress (nucleation threshold) */
    double T0;             /* uniform temperature when no thermal map is set */
    double horizon;        /* simulated time span (s) */
    int    n_outer, n_inner;      /* aging steps and BE steps per aging step */
    double ir_fail_frac;   /* failure threshold on max IR drop / Vdd */
    double Vdd;            /* supply voltage for the drop fraction */
    int    precision;      /* EMS_F64 or EMS_F32 for the stress path (IR is always FP64) */
    int    method;         /* EMS_BE, EMS_KRYLOV or EMS_AUTO */
    int    krylov_q;       /* Krylov block order q (Alg. 1) */
    double krylov_eta;     /* shift-time factor eta (Eq. rak_shift_time) */
    double ir_rtol;        /* PCG relative residual target (||r|| <= rtol ||b||) */
    int    ir_max_iter;    /* PCG iteration cap (EMS_E_NOCONV beyond it) */
    int    max_voids_per_tree;  /* void slots per (tree, sample), 1..256 */
    int    ir_precond;     /* EMS_PC_AUTO: smoothed-aggregation multigrid V-cycle for systems of
                              >= 1,024 unknowns (hierarchy built once from the initial
                              resistances), Jacobi below; EMS_PC_JACOBI: Jacobi always */
    int    window_samples; /* Monte Carlo memory layout (Sec. IV-F).  0 (or >= n_samples):
                              every per-node coefficient array (kappa a, conductances, leak,
                              thresholds, forcing, factors) and the IR work vectors are held
                              for all samples at once.  W in 1..n_samples-1: only the
                              per-sample state is held for all samples -- packed stress,
                              resistances, node voltages, the kappa / sigma_crit factors per
                              segment, voids -- and the per-node coefficients and IR vectors
                              exist for W samples at a time: every call that steps, solves or
                              reports per-node data walks the samples in windows of W and
                              rebuilds the window's coefficients from the per-segment factors
                              first.  Results are the same as with the full layout; the
                              reduced models (EMS_KRYLOV / EMS_AUTO) need the full layout. */
    double krylov_eps;     /* deflation threshold of the block Arnoldi (Alg. 1): a new column
                              whose norm after orthogonalisation falls below krylov_eps times
                              its block's norm makes the block rank deficient and the tree is
                              sent to backward Euler (Sec. IV-E.5).  0: 1e-10.  Range [0, 1). */
} ems_params;

enum { EMS_PC_AUTO = 0, EMS_PC_JACOBI = 1 };       /* IR preconditioner */

/*
 * Extracted power-grid netlist (Sec. III-C: a resistor network with uniform
 * current density per segment; via resistors optional, Sec. IV-C).  Segment a -> b is the +x direction of its
 * current density.  Pads are Dirichlet voltage sources; sinks draw current.
 * kappa_factor / sigc_factor, when not NULL, are [n_samples][n_seg] Monte
 * Carlo multipliers (Sec. IV-F) on kappa and sigma_crit of every face / node
 * of the segment (a crossing node takes the factor of its lowest-id
 * incident segment within the tree); NULL means one unperturbed sample.
 */
typedef struct {
    int n_nodes;
    const double *node_x, *node_y;
    int n_seg;
    const int32_t *seg_a, *seg_b, *seg_layer, *seg_cells;
    const double *seg_R0, *seg_W, *seg_H, *seg_L;
    int n_pads;
    const int32_t *pad_node;
    const double *pad_V;
    int n_sinks;
    const int32_t *sink_node;
    const double *sink_I;
    int n_samples;
    const double *kappa_factor, *sigc_factor;
    const int8_t *seg_via;   /* optional [n_seg]: 1 marks a via resistor (joins two layers; part of
                                the IR network, of no stress tree); NULL: no explicit vias */
} ems_grid_desc;

typedef struct ems_ctx ems_ctx;

/*
 * SPICE power-grid netlist reader (the paper's PNA-to-SPICE input with every
 * via resistor kept, Sec. IV-A and IV-C).  Elements, one per line:
 *   R<name> <node> <node> <ohm>   a wire when both nodes are on one metal
 *                                 layer, else a via resistor
 *   V<name> <node> 0 <volt>       a supply pad
 *   I<name> <node> 0 <amp>        a sink drawing <amp> from <node>
 * Node names n<layer>_<x>_<y> give the metal layer (1..n_layers) and the
 * position in integer units of coord_unit; "0" / "gnd" is ground.  Lines
 * starting with '*' or '.' are skipped.  A wire's length is the distance of
 * its nodes, its width / thickness those of its layer, its finite-difference
 * cells max(1, floor(L / dx + 1/2)); a via gets via_W x via_W, length via_H, one
 * cell.  Nodes are numbered in order of first appearance, segments and
 * sources in file order.
 */
typedef struct {
    int n_layers;              /* metal layers named in the netlist, 1..n_layers (<= 64) */
    const double *W, *H;       /* [n_layers] wire width and thickness per layer (m) */
    double via_W, via_H;       /* via side and height (m) */
    double coord_unit;         /* metres per unit of the node-name coordinates */
    double dx;                 /* target finite-difference cell length (m) */
} ems_spice_opts;

typedef struct ems_netlist ems_netlist;

/* Parse len bytes of text.  *out receives the netlist (also on EMS_E_INVAL,
 * so that ems_netlist_error() can say which line failed); free it with
 * ems_netlist_free.  EMS_E_INVAL: bad options, a malformed or unsupported
 * line, a resistor to ground, no resistors or no voltage source. */
ems_status ems_spice_parse(const char *text, size_t len, const ems_spice_opts *opts, ems_netlist **out);
/* A grid descriptor whose arrays point into the netlist (valid until freed;
 * n_samples 0, no Monte Carlo factors). */
ems_status ems_netlist_desc(const ems_netlist *nl, ems_grid_desc *desc);
const char *ems_netlist_error(const ems_netlist *nl);
void ems_netlist_free(ems_netlist *nl);

/* Bytes of device workspace a context needs for this grid (with the Monte
 * Carlo layout params->window_samples selects).  Returns 0 if the
 * descriptor is invalid.  Planning the grid (tree extraction, IR structure,
 * multigrid hierarchy) is the work here; the plan stays in host memory for
 * the next ems_load_grid and is used by it when the grid's arrays and the
 * plan-relevant parameters and shape rules hash the same (the next size query
 * or load releases it). */
size_t ems_workspace_bytes(const ems_params *params, const ems_grid_desc *grid);

/*
 * Create a context on the current CUDA device.
 *   stream     cudaStream_t the context orders its work on (NULL = default stream)
 *   workspace  caller-owned device memory of at least ems_workspace_bytes()
 *              for the grid later loaded, 256-byte aligned; NULL lets the
 *              context allocate (and free) its own.  The caller keeps a
 *              caller-owned workspace alive until ems_destroy().
 */
ems_status ems_create(ems_ctx **out, const ems_params *params, void *stream,
                      void *workspace, size_t ws_bytes);
ems_status ems_destroy(ems_ctx *ctx);
const char *ems_last_error(const ems_ctx *ctx);

/*
 * Load the grid (Sec. IV-A: partition into trees): checks the inputs,
 * extracts the trees in canonical order, packs them by size into the
 * chunk-interleaved layout, copies everything to the device, sets every
 * sample's stress to sigma_T, its resistances to R0 and the time to 0.
 * Errors: EMS_E_INVAL for NaN / non-positive geometry, bad indices, a
 * same-layer cycle, or a node not connected to any pad; EMS_E_NOMEM.
 */
ems_status ems_load_grid(ems_ctx *ctx, const ems_grid_desc *grid);

/*
 * Chain solver shapes and the autotuner (batching of Sec. IV-B's per-tree
 * eliminations over every tree and Monte Carlo sample).  A chain of n stress
 * nodes is cut into T team threads of M consecutive nodes (packed node i at
 * (i mod M) T + i / M of its tree's packed block) and advanced by one of:
 *   EMS_CHAIN_GLOBAL    one CTA per (chain, sample), chunks streamed from HBM
 *   EMS_CHAIN_SHARED    (FP32) one CTA, the chunk coefficients staged in shared memory
 *   EMS_CHAIN_REGISTER  (FP32, M <= 16) one CTA, coefficients and state in registers
 *   EMS_CHAIN_CLUSTER   a cluster of CL CTAs (2..8) per (chain, sample), registers,
 *                       M = 16 (FP32) or 8 (FP64); CTAs trade their carries through
 *                       distributed shared memory
 *   EMS_CHAIN_CLUSTER_SHARED  (FP32, M = 16) the cluster kernel with the chunk
 *                       coefficients in shared memory (20 bytes per node), so that
 *                       two CTAs share an SM; CL 2, 4, 8 (<= 320 threads a CTA) or
 *                       5, 6 (<= 256)
 * Every shape solves the same system; results differ by rounding only.
 */
enum { EMS_CHAIN_DEFAULT = 0, EMS_CHAIN_GLOBAL = 1, EMS_CHAIN_SHARED = 2, EMS_CHAIN_REGISTER = 3,
       EMS_CHAIN_CLUSTER = 4, EMS_CHAIN_CLUSTER_SHARED = 5 };
typedef struct {
    int64_t n_lo, n_hi;    /* chains of n_lo..n_hi stress nodes (inclusive) */
    int kind;              /* EMS_CHAIN_*; EMS_CHAIN_DEFAULT leaves the built-in choice */
    int M;                 /* nodes per thread: 4, 8, 16, 32 or 64 */
    int CL;                /* CTAs per chain: 1, or 2..8 with the cluster kinds */
    int T;                 /* out (ems_autotune, ems_chain_candidates): team threads for n_hi */
} ems_chain_rule;

/*
 * Shapes valid for a chain of n nodes at a precision (backward Euler),
 * the built-in choice first.  count: out, number written (at most cap).
 */
ems_status ems_chain_candidates(int64_t n, int precision, ems_chain_rule *out, int cap, int *count);

/*
 * Shape rules for the next ems_load_grid of this context (backward Euler;
 * the reduced models keep the built-in shapes).  The first rule whose range
 * holds a chain's length and whose shape is valid for it applies; chains no
 * rule covers take the built-in choice.  The rules are copied; n_rules = 0
 * clears them.  A caller-provided workspace must be sized for the shapes the
 * rules pick.  Errors: EMS_E_INVAL for an unknown kind, M or CL.
 */
ems_status ems_set_chain_rules(ems_ctx *ctx, const ems_chain_rule *rules, int n_rules);

/* ems_workspace_bytes for a context whose chain shapes follow these rules. */
size_t ems_workspace_bytes_rules(const ems_params *params, const ems_grid_desc *grid,
                                 const ems_chain_rule *rules, int n_rules);

/*
 * Autotuner: for every group of chains the loaded context advances with one
 * launch (one shape), time each valid shape on scratch copies of those
 * chains (their current stress and voids, the first min(max_samples, W)
 * samples): one launch that factorises and runs n_steps backward-Euler steps,
 * then n_steps more timed with CUDA events.  The context's state is left as
 * it was.  rules[k] gets the fastest shape of group k (n_lo / n_hi: the
 * group's chain lengths), ms[k] its time per launch and ms_default[k] the
 * current shape's (optional, may be NULL); n_rules: out, number of groups
 * (at most cap).  Loading the grid again after ems_set_chain_rules(rules)
 * applies the choice.  Needs backward Euler and a solved IR state.
 */
ems_status ems_autotune(ems_ctx *ctx, int n_steps, int max_samples, ems_chain_rule *rules, double *ms,
                        double *ms_default, int cap, int *n_rules);

/*
 * Every shape the last ems_autotune call timed: shapes[k] (n_lo / n_hi: its
 * group's chain lengths), ms[k] its time per launch (-1: the device cannot
 * launch it), group[k] the group's index in the rules.  count: out, number
 * written (at most cap).  Arrays may be NULL with cap = 0 to get the count.
 */
ems_status ems_autotune_log(const ems_ctx *ctx, int cap, ems_chain_rule *shapes, double *ms, int32_t *group,
                            int *count);

/* Number of trees / stress nodes / samples of the loaded grid. */
ems_status ems_dims(const ems_ctx *ctx, int *n_trees, int64_t *n_stress_nodes,
                    int *n_samples);

/*
 * Set the temperature field (Sec. III-A, "via-node temperatures are read
 * from the map"): T at every stress node by bilinear interpolation of the
 * vertex-centred raster T[iy*nx + ix] over [x0,x1] x [y0,y1] (clamped at the
 * border); then kappa per face (Arrhenius at the face's mean temperature)
 * and the thermomigration term M per face.  T == NULL sets uniform params.T0.
 */
ems_status ems_set_thermal_map(ems_ctx *ctx, const double *T, int nx, int ny,
                               double x0, double y0, double x1, double y1);

/*
 * Per-sample temperature-map perturbation (Sec. IV-F: external temperature
 * maps among the inputs a Monte Carlo sample may vary): sample s adds the
 * raster dT[s][iy*nx + ix] (K), vertex-centred over the extent of the map set
 * by ems_set_thermal_map and sampled bilinearly (clamped at the border), to
 * the temperature of every stress node; kappa and the thermomigration term
 * of the sample follow.  dT == NULL removes the perturbations.  The map (or
 * a Joule-heating profile) stays the common base; the surrogate's features
 * keep using the base temperatures.
 *   dT      host [n_samples][ny][nx], nx, ny >= 2, nx * ny <= 4,096
 * EMS_E_STATE without a thermal map; EMS_E_INVAL for a bad size or a
 * non-finite value.
 */
ems_status ems_set_thermal_perturbation(ems_ctx *ctx, const double *dT, int nx, int ny);

/*
 * Joule-heating temperature profile along every branch (Sec. III-A: the
 * stationary thermal equation k T'' + j^2 rho - k (T - T0) / Gamma^2 = 0 with
 * the thermal characteristic length Gamma^2 = t_cu t_ILD k_cu / k_ILD, t_cu
 * the segment's thickness H).  Per segment with end temperatures T1 (end a)
 * and T2 (end b), on x in [-L/2, L/2]:
 *   T(x) = T0 + Tm + (Tbar - T0 - Tm) cosh(x/Gamma) / cosh(L/(2 Gamma))
 *             - Tn sinh(x/Gamma) / sinh(L/(2 Gamma)),
 *   Tm = j^2 rho_Cu Gamma^2 / k_cu, Tbar = (T1 + T2)/2, Tn = (T1 - T2)/2
 * (the printed solution's cos / sin terms solve the equation with the
 * opposite sign of the loss term; this is the form that satisfies it).
 * End temperatures: an IR node that joins segments of different layers (a
 * via) or is a pad takes the thermal map's value (params.T0 without a map);
 * every other IR node is solved from zero net heat flow into its segments
 * (one thread per tree, leaf-to-root elimination).  Uses the current
 * densities of sample 0 (all samples share them until voids form) and the
 * map set by ems_set_thermal_map; the profile replaces the node
 * temperatures, kappa and the thermomigration term follow, and it stays
 * until the next ems_set_thermal_map.
 *   k_cu, k_ild   thermal conductivities of the wire and the dielectric (W/(m K))
 *   t_ild         dielectric thickness (m)
 * EMS_E_STATE before the first IR solve; EMS_E_INVAL for non-positive inputs.
 */
ems_status ems_joule_profile(ems_ctx *ctx, double k_cu, double k_ild, double t_ild);

/* Node temperatures in use (host [n_stress_nodes], canonical order, K). */
ems_status ems_get_node_temperature(ems_ctx *ctx, double *T);

/*
 * IR-drop solve (Sec. III-C, Eq. ir_drop_mna) for every sample with the
 * current resistances: preconditioned CG in FP64 on the conductance matrix of
 * the non-pad nodes (params.ir_precond: a smoothed-aggregation multigrid
 * V-cycle for systems of >= 1,024 unknowns by default, Jacobi below or on
 * request), warm-started from the previous solution; then the segment
 * current densities j = (u_a - u_b) / (R W H).
 *   u_out         optional host [S][n_nodes] node voltages
 *   max_drop_frac optional host [S]: max over nodes of (Vdd - u) / Vdd
 * EMS_E_NOCONV if a sample misses ir_rtol within ir_max_iter iterations.
 */
ems_status ems_ir_solve(ems_ctx *ctx, double *u_out, double *max_drop_frac);

/*
 * Steady-state immortality screen (Sec. III-B) with the current currents
 * and temperatures: per tree, zero flux on every face gives sigma_ss up to
 * a constant fixed by atom conservation; a tree is mortal iff some node's
 * sigma_ss exceeds its critical stress.
 *   mortal        optional host [S][n_trees] (1 = mortal)
 *   sigma_ss_max  optional host [S][n_trees]
 *   sigma_ss      optional host [S][n_stress_nodes] canonical order
 */
ems_status ems_immortality_check(ems_ctx *ctx, uint8_t *mortal, double *sigma_ss_max,
                                 double *sigma_ss);

/*
 * Advance every tree of every sample by n_steps backward-Euler steps of dt
 * (Sec. IV-B; Eq. em_tm_ode: (C - dt A) s^{k+1} = C s^k + dt f) with the
 * current currents, nucleation after every step (the non-void node with the
 * largest sigma - sigma_crit, lowest index on ties, when that is >= 0;
 * Sec. III-D.2), the Robin void stamp from the next step on (Sec. IV-D,
 * Eq. robin_mid_tree) and void-volume growth by the Robin leak
 * (Eq. void_volume_equation).  method EMS_KRYLOV / EMS_AUTO route every
 * chain with n >= max(3q, 30) (Eq. krylov_threshold) through its reduced model
 * (Sec. IV-E): a basis cached per (tree, sample) under the key the paper
 * gives (the descriptor matrices and s0: rebuilt on a new void, a new
 * thermal map or new q / eta), extended on every call by the current
 * starting block [K^-1 C sigma, K^-1 f]; backward Euler in reduced
 * coordinates; the same nucleation rule on the lifted stress.  Other trees,
 * and trees whose basis breaks down, take full backward Euler.
 *   n_new_voids   optional host: voids nucleated during the call (all samples)
 */
ems_status ems_stress_advance(ems_ctx *ctx, double dt, int n_steps, int method,
                              int *n_new_voids);

/*
 * Build the rational Krylov reduced model (Sec. IV-E, Alg. 1) of every tree
 * with n >= max(3q, 30) (Eq. krylov_threshold): shift t_s = eta L_max^2 /
 * (pi^2 kappa_mean) (Eq. rak_shift_time), K = C/t_s - A, starting block
 * [K^-1 C sigma0, K^-1 f], block Arnoldi to order q with classical
 * Gram-Schmidt applied twice (per-thread sums in the context precision, FP64
 * across threads), projections A_h, C_h (Eq. rak_reduced).  Bases already
 * cached are kept.
 *   n_reduced / n_fallback  optional host: trees reduced / sent back to BE
 */
ems_status ems_krylov_reduce(ems_ctx *ctx, int q, double eta, int *n_reduced,
                             int *n_fallback);

/*
 * Void growth resistance write-back (Sec. III-D.3, IV-C).  Late failure:
 * R_s = R0_s + sum over the voids on segment s of
 * max(0, (V_v - W^2 H)/(W H) [rho_Ta/(h_Ta (2H+W)) - rho_Cu/(H W)]).
 * Early failure (grids with explicit via resistors only): a void at an IR
 * node that connects through a via to a strictly higher layer (a node's
 * layer is that of its wire segments) opens the via once its volume exceeds
 * W^2 H of its segment: the via's resistance becomes the open-circuit
 * sentinel 1e9 Ohm.
 *   n_segments_changed  optional host: segments (all samples) whose R changed
 */
ems_status ems_void_update(ems_ctx *ctx, int *n_segments_changed);

typedef struct {
    int screen;        /* 1: run the immortality screen first (reported only) */
    int n_outer;       /* 0: params.n_outer */
    int no_graph;      /* 1: drive the aging steps from the host instead of one CUDA graph */
} ems_ttf_opts;

typedef struct {
    double *ttf;          /* [S] time of the first 10 % crossing (0 if initially above, +inf if never) */
    double *drop0;        /* [S] initial max IR drop fraction */
    double *final_drop;   /* [S] max IR drop fraction at the end */
    int32_t *n_voids;     /* [S] voids at the end */
    int32_t *n_mortal;    /* [S] mortal trees by the screen (if opts.screen) */
    double *drops;        /* optional [S][n_outer+1] drop after every aging step */
    double node_steps;    /* out: sum over trees and samples of nodes x BE steps */
    double stress_ms;     /* out: device time of the stress-advance kernels (ms; graph runs: the
                             chain / tree / reduced-model launches themselves) */
    double ir_ms;         /* out: device time of the IR solves (ms) */
    double ir_iterations; /* out: PCG iterations summed over the IR solves and samples */
    double ttf_mean;      /* out: mean TTF over uncensored samples (NaN if none) */
    double ttf_std;       /* out: sample standard deviation (ddof 1) over uncensored samples */
    double ttf_cov;       /* out: ttf_std / ttf_mean */
    double n_censored;    /* out: samples that never crossed (TTF = +inf) */
    double graph_launch;  /* out: 1 if the aging steps ran as one captured CUDA graph */
    double node_steps_executed; /* out: stress node-steps the kernels ran: less than node_steps
                                   under a surrogate step schedule (coarse steps); the reduced
                                   models count their steps as full-order ones */
} ems_ttf_result;

/*
 * Full coupled aging run (Sec. IV-A, Eq. em_tm_ir_ode; TTF per Sec. V): from
 * the current state, IR solve, then per aging step: stress advance of
 * n_inner steps of horizon/(n_outer n_inner), void update, IR re-solve, max
 * drop; TTF is the linear interpolation of the first crossing of
 * ir_fail_frac.  Host result arrays are caller-allocated (NULL to skip).
 * Unless opts.no_graph (and for n_outer <= params.n_outer) every aging step
 * of every sample, by either method, runs inside one captured CUDA graph: the
 * crossing detection happens on the device and the host reads the results
 * once; Monte Carlo statistics follow Sec. V-D (uncensored samples only).
 */
ems_status ems_ttf(ems_ctx *ctx, const ems_ttf_opts *opts, ems_ttf_result *out);

/* Copies of device state (host buffers, canonical order). */
ems_status ems_get_sigma(ems_ctx *ctx, double *sigma /* [S][n_stress_nodes] */);
ems_status ems_get_currents(ems_ctx *ctx, double *j /* [S][n_seg] */);
ems_status ems_get_resistance(ems_ctx *ctx, double *R /* [S][n_seg] */);
/* Voids of every (tree, sample): up to cap entries, sample-major then tree,
 * then nucleation order.  Returns the count in *n. */
ems_status ems_get_voids(ems_ctx *ctx, int cap, int32_t *sample, int32_t *node,
                         int32_t *seg, double *volume, double *t_nuc, int *n);

/*
 * Iteration limit of the device-side waits of this context (the grid
 * barriers of the cooperative IR solvers): after `polls` polls a wait gives
 * up, every block of the kernel returns, and the call reports
 * EMS_E_TIMEOUT; the context stays usable.  polls >= 1; 0 restores the
 * default, 2^24 polls (about a second).  A guard against a lost participant,
 * not a tuning knob: a limit too small for the work makes solves time out.
 */
ems_status ems_set_wait_limit(ems_ctx *ctx, long long polls);

/* PCG iterations of the last IR solve, per sample (host [S]). */
ems_status ems_ir_iterations(ems_ctx *ctx, int32_t *iters);

/* Number of kernels the context has launched since it was created. */
ems_status ems_launch_count(const ems_ctx *ctx, int64_t *launches);

/*
 * Checkpoint / resume of the aging state (stress, voids, resistances, node
 * voltages, time; Sec. IV-A: the state carried between aging steps).
 * ems_state_export with buf == NULL returns the size in *bytes.
 */
ems_status ems_state_export(ems_ctx *ctx, void *buf, size_t *bytes);
ems_status ems_state_import(ems_ctx *ctx, const void *buf, size_t bytes);

/*
 * Allocation-free PCG solve.  The paper has no counterpart: this is a
 * service of this library for callers that cannot allocate device memory
 * for it -- code that runs under another framework's allocator and may not
 * call cudaMalloc itself, or that cannot accept the device-wide
 * synchronisation a cudaMalloc / cudaFree can cause between its own kernels.
 *
 * Solves A x = b by Jacobi-preconditioned conjugate gradients in FP64 on one
 * CTA, until ||b - A x|| <= rtol ||b|| or max_iter iterations.
 *   n          unknowns, 1..16384
 *   row_ptr    device [n+1], col device [nnz], val device [nnz]: CSR of a
 *              symmetric positive definite A; every row holds its diagonal
 *   b          device [n]
 *   x          device [n]: initial guess in, solution out
 *   iterations optional host: iterations used
 *   stream     cudaStream_t (NULL = default stream); the call synchronises it
 * Returns EMS_OK, EMS_E_INVAL (n beyond 16384, null pointer, rtol <= 0),
 * EMS_E_NOCONV (iteration cap reached) or EMS_E_CUDA.
 *
 * The work vectors live in one file-scope device array (640 KB) that every
 * GPU loading the library holds until the process exits; nothing is
 * allocated or freed.  All calls share that array: calls whose kernels can
 * overlap on one GPU (several streams or threads at once) race and must be
 * serialised by the caller.  The first call on each device looks the
 * array's device address up once, with that device current.
 */
ems_status ems_ir_pcg_noalloc(int n, const int32_t *row_ptr, const int32_t *col, const double *val,
                              const double *b, double *x, double rtol, int max_iter, int *iterations,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif
