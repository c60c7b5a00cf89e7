/*
 * ems_oracle.h -- plain FP64 CPU oracle for the per-tree EM/TM stress path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the correctness reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA library.
 *
 * Tree storage (flat over all trees): tree t owns nodes [off[t], off[t+1]).
 * Within a tree, local node 0 is the root and par[i] < i for every other
 * node (par[root] = -1), i.e. the nodes are in a topological order from the
 * root.  The finite-volume face between node i and its parent carries the
 * conductance g[i] = a_e kappa_e / dx_e (g[root] = 0).
 */
#ifndef EMS_ORACLE_H
#define EMS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Backward-Euler advance of every tree (Sec. III-D.4, Eq. em_tm_ode, with the
 * incubation/Robin boundary condition of Eq. incubation_bc / robin_mid_tree):
 *   (C - dt A) sigma^{k+1} = C sigma^k + dt f,
 *   C = diag(V),  A_ij = g_e,  A_ii = -sum g_e - leak_i [i is a void].
 * After every step: void volumes grow by dt/B * leak_v * sigma_v (atom
 * conservation, Eq. void_volume_equation), then the non-void node with the
 * largest sigma_i - sigma_crit_i (lowest index on ties) nucleates a void if
 * that difference is >= 0 (Sec. III-D.2); its Robin leak acts from the next
 * step.  t_nuc is linear interpolation of sigma_v - sigma_crit_v in time.
 *
 *   par, off       tree structure as above (par is tree-local)
 *   V, g, f        node volume, face conductance, forcing (per node)
 *   leak           Robin leak gamma_i = sum_{e at i} a_e kappa_e / delta
 *   sig_crit       per-node critical stress
 *   sigma          in/out state
 *   void_flag      in/out, 1 where a void exists
 *   void_vol       in/out void volume per node
 *   t_nuc          out, set at nodes that nucleate during this call
 *   margin         out per tree (may be NULL): min over steps of
 *                  |max_i (sigma_i - sig_crit_i)| / sig_crit at the argmax
 *   gap            out per tree (may be NULL): min over the nucleations of
 *                  the lead of the chosen node over the runner-up,
 *                  (best - second) / sig_crit at the chosen node (+inf if
 *                  none); small values mark node choices that rounding of
 *                  the stress could change (test bookkeeping only)
 *   n_threads      OpenMP threads over trees (<= 0: library default)
 * Returns the number of voids nucleated.
 */
int orc_advance(int n_trees, const long *off, const int *par,
                const double *V, const double *g, const double *f,
                const double *leak, const double *sig_crit,
                double *sigma, int *void_flag, double *void_vol, double *t_nuc,
                double t0, double dt, int n_steps, double B_modulus,
                double *margin, double *gap, int n_threads);

/*
 * Steady-state stress of each tree with blocking ends and no voids
 * (Sec. III-B): zero flux on every face gives sigma_child - sigma_parent =
 * dxG[child]; the constant is fixed by atom conservation,
 * sum_i V_i (sigma_i - sigma_T) = 0.
 */
void orc_steady(int n_trees, const long *off, const int *par, const double *V,
                const double *dxG, double sigma_T, double *sigma_ss);

#ifdef __cplusplus
}
#endif
#endif
