/*
 * ems_surrogate.h -- C ABI of the learned surrogate that schedules the
 * stress solve: a multilayer perceptron over per-(tree, sample) features,
 * trained and evaluated on the GPU with BF16 tensor-core kernels (FP32
 * accumulate), and the calls that tie it to an ems_ctx.
 *
 * The surrogate is not part of the paper's method.  The paper simulates
 * every mortal tree up to the horizon (Sec. IV-A) after its steady-state
 * immortality filter (Sec. III-B); the surrogate predicts, per tree and Monte
 * Carlo sample, log10 of the first nucleation time and the critical node, and
 * lets ems_ttf replace the fine steps of a (tree, sample) by coarse ones only
 * where the predicted time, lowered by a bound the caller validated against
 * the plain solver, still lies beyond the horizon.  Every other tree is
 * stepped by the plain solver, unchanged.
 *
 * Network: 24 inputs -> n_hidden layers of 256 ReLU units -> 2 linear outputs
 * (log10 t_nuc in seconds, critical-node position in [0, 1] along the tree's
 * canonical order).  Inputs and targets are standardised inside the library
 * with the statistics set by ems_mlp_set_norm; predictions are returned in
 * the original units.  Loss: half the batch mean of the squared error summed
 * over the two standardised outputs.  Optimiser: Adam with bias correction.
 *
 * Conventions as in ems.h: every call returns an ems_status; all work of one
 * network is ordered on the stream given to ems_mlp_create; calls that
 * return host data synchronise it.  Device arrays are caller-owned unless
 * stated; the network owns the device memory it allocates (weights, Adam
 * moments, training activations) and frees it in ems_mlp_destroy.
 */
#ifndef EMS_SURROGATE_H
#define EMS_SURROGATE_H

#include "ems.h"

#ifdef __cplusplus
extern "C" {
#endif

#define EMS_MLP_FEATURES 24
#define EMS_MLP_OUTPUTS 2
#define EMS_MLP_WIDTH 256

typedef struct ems_mlp ems_mlp;

/*
 * Create a network with n_hidden (1..8) hidden layers of 256 units, weights
 * He-normal from `seed`, biases zero, identity standardisation.  `stream` is
 * a cudaStream_t (NULL = default stream).  Returns EMS_E_INVAL, EMS_E_NOMEM
 * or EMS_E_CUDA on failure (and *out = NULL).
 */
ems_status ems_mlp_create(int n_hidden, uint64_t seed, void *stream, ems_mlp **out);
void ems_mlp_destroy(ems_mlp *mlp);
const char *ems_mlp_last_error(const ems_mlp *mlp);

/* Number of parameters in the flat host layout used below: for each layer in
 * order, W [out x in] row-major, then b [out]. */
int64_t ems_mlp_param_count(const ems_mlp *mlp);
ems_status ems_mlp_set_params(ems_mlp *mlp, const float *host_params);
ems_status ems_mlp_get_params(ems_mlp *mlp, float *host_params);

/* Standardisation: x_s = (x - x_mean) / x_std per feature, t_s = (t - t_mean)
 * / t_std per output.  Host arrays of 24, 24, 2, 2 floats; std must be > 0. */
ems_status ems_mlp_set_norm(ems_mlp *mlp, const float *x_mean, const float *x_std, const float *t_mean,
                            const float *t_std);

/*
 * Standardisation fitted to a record set on the device and installed in the
 * network: per column of x (24 features) and t (2 targets) the mean and the
 * standard deviation (square root of the mean squared deviation, FP64 sums
 * in a fixed order; a column whose deviation is under 1e-6 gets 1).
 *   x, t    device [rows][24], [rows][2] raw features and targets
 *   stats   optional host [52] doubles: x mean[24], x std[24], t mean[2], t std[2]
 * Synchronises the network's stream.  EMS_E_INVAL for rows < 1 or null data.
 */
ems_status ems_mlp_fit_norm(ems_mlp *mlp, const float *x, const float *t, int64_t rows, double *stats);

/*
 * Forward + backward without an update, for gradient checks.
 *   x       device [rows][24] raw features; t device [rows][2] raw targets
 *   grads   host [ems_mlp_param_count]: dL/dparam in the flat layout, with L
 *           the loss on the standardised outputs
 *   loss    optional host: L
 * rows 1..65536.
 */
ems_status ems_mlp_gradients(ems_mlp *mlp, const float *x, const float *t, int rows, float *grads, float *loss);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the batch x, t;
 * *loss (optional, host) receives the loss before the step. */
ems_status ems_mlp_train_step(ems_mlp *mlp, const float *x, const float *t, int rows, float lr, float *loss);

/*
 * Mini-batch training over `rows` records for `epochs` epochs, batches of
 * `batch` rows (a multiple of 64, <= 65536) in an order reshuffled every epoch
 * from `seed`; the last partial batch of an epoch is dropped.
 *   loss_per_epoch  optional host [epochs]: mean batch loss of each epoch
 */
ems_status ems_mlp_train(ems_mlp *mlp, const float *x, const float *t, int64_t rows, int batch, int epochs, float lr,
                         uint64_t seed, float *loss_per_epoch);

/*
 * Inference: y device [rows][2] (log10 t_nuc, critical-node position) from x
 * device [rows][24].  One fused tensor-core kernel runs all layers for 256
 * rows per CTA with the activations kept on chip; any rows >= 0; x must be
 * 16-byte and y 8-byte aligned.
 */
ems_status ems_mlp_predict(ems_mlp *mlp, const float *x, int64_t rows, float *y);

/*
 * Dense-layer primitive of the network, exposed for numerical tests:
 * D[M x N] = scale * A[M x K] B[N x K]^T (+ bias[N]) (ReLU if relu != 0), with A
 * and B row-major BF16 device arrays and FP32 accumulation on the tensor
 * cores.  Outputs (each optional, device): d_f32 [M x N] FP32; d_bf16 [M x N]
 * BF16.  Shapes: M >= 1, N in 16..256 a multiple of 16, K a multiple of 64.
 */
ems_status ems_gemm_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int relu, float scale,
                         float *d_f32, void *d_bf16, void *stream);

/*
 * Features of every (tree, sample) of a loaded context at its current state
 * and currents (requires one IR solve): x device [S * n_trees][24], row
 * s * n_trees + t.  Features are tree size and length, current density,
 * temperature and its gradient, kappa, critical stress, the steady-state
 * stress of the immortality check (Sec. III-B) and two closed-form time
 * scales (diffusion time L^2 / kappa and the early-time Korhonen estimate).
 */
ems_status ems_surrogate_features(ems_ctx *ctx, float *x);

/*
 * Targets of every (tree, sample) from the voids recorded so far: t device
 * [S * n_trees][2] = (log10 of the first nucleation time in seconds, capped at
 * log10(t_cap) and floored at 0; position of that void's node in [0, 1], or
 * of the steady-state critical node when the tree has no void).  Call after
 * ems_surrogate_features on the same context (the fallback position comes
 * from there).  freeze != 0 also stops all further stepping of every (tree,
 * sample) that has a void (until ems_surrogate_clear), so that record
 * generation spends no steps on trees whose first nucleation is known.
 * t_cap > 1.
 */
ems_status ems_surrogate_targets(ems_ctx *ctx, double t_cap, int freeze, float *t);

/*
 * Per-tree step schedule: run the network on the context's features; every
 * (tree, sample) whose predicted log10 t_nuc - bound > log10(horizon) takes
 * `coarsen` (>= 2) times fewer, `coarsen` times longer backward-Euler steps in
 * ems_stress_advance / ems_ttf until ems_surrogate_clear (a call whose fine
 * step count `coarsen` does not divide steps it finely); all others take the
 * plain solver's fine steps.  The plain solver stays the fallback: a coarse
 * (tree, sample) whose stress reaches guard (0 < guard <= 1) times its lowest
 * critical stress switches to fine steps for good, within the step where it
 * does.  Nucleation detection, void growth and resistance write-back run
 * unchanged for both.  The schedule applies to backward-Euler stepping;
 * trees a Krylov reduced model advances are not rescheduled.  The trees of
 * each launch are also reordered by predicted first nucleation (earliest
 * first).  ems_ttf reports the node-steps actually executed in
 * node_steps_executed.
 * n_coarse (optional, host [S]) receives the coarse trees per sample; pred
 * (optional, device [S * n_trees][2]) the raw predictions.
 */
ems_status ems_surrogate_schedule(ems_ctx *ctx, ems_mlp *mlp, double bound, int coarsen, double guard,
                                  int *n_coarse, float *pred);
ems_status ems_surrogate_clear(ems_ctx *ctx);

/*
 * The skip bound, validated end to end against the plain solver, which stays
 * the judge of the schedule's error.  Every context in ctxs (held-out grids,
 * loaded, any Monte Carlo sample count) is run from its current state by
 * ems_ttf twice per candidate comparison: once plain (no schedule; run once
 * per context) and once under ems_surrogate_schedule(ctx, mlp, candidate,
 * coarsen, guard).  A candidate passes when, over every context and sample,
 * the sets of samples with a finite TTF agree and the largest relative
 * difference of TTF (where finite) and of the final IR drop is <= tol.
 * Candidates are tried in the order given (most aggressive first); *bound
 * receives the first passing candidate + margin, or +inf if none passes.
 * Every context is left in the state it had on entry, with no schedule.
 *   log  optional host [n_cand][3]: candidate, fraction of (tree, sample)
 *        pairs scheduled coarse, largest relative error (+inf for a differing
 *        set of failed samples); rows after the passing one are not written
 * EMS_E_INVAL for null or empty inputs, coarsen < 2 or guard outside (0, 1].
 */
ems_status ems_surrogate_validate(ems_ctx *const *ctxs, int n_ctx, ems_mlp *mlp, const double *candidates,
                                  int n_cand, int coarsen, double guard, double tol, double margin,
                                  double *bound, double *log);

#ifdef __cplusplus
}
#endif
#endif
