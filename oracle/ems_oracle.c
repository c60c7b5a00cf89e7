/*
 * ems_oracle.c -- plain FP64 CPU oracle for the per-tree EM/TM stress path.
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
 * Written for clarity, not speed: every backward-Euler step re-assembles the
 * tree matrix and eliminates it leaf-to-root, then substitutes root-to-leaf.
 * Compiled with -ffp-contract=off so results do not depend on whether the
 * host compiler fuses multiply-adds.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "ems_oracle.h"

/*
 * One backward-Euler step on one tree (Sec. III-D.4, Eq. em_tm_ode):
 *   M x = rhs,  M = C - dt A,
 *   M_ii = V_i + dt (sum of g over faces at i) + dt leak_i [void at i],
 *   M_{i,par(i)} = M_{par(i),i} = -dt g_i.
 * Leaf-to-root elimination (children have larger indices than parents),
 * then root-to-leaf substitution.  d and r are scratch of length n.
 */
static void be_step_tree(int n, const int *par, const double *V, const double *g,
                         const double *f, const double *leak, const int *vflag,
                         double dt, double *sigma, double *d, double *r)
{
    int i;
    for (i = 0; i < n; ++i) {
        d[i] = V[i];
        r[i] = V[i] * sigma[i] + dt * f[i];
        if (vflag[i]) d[i] += dt * leak[i];
    }
    for (i = 1; i < n; ++i) {          /* face (i, par(i)) adds to both diagonals */
        d[i] += dt * g[i];
        d[par[i]] += dt * g[i];
    }
    for (i = n - 1; i >= 1; --i) {     /* eliminate node i into its parent */
        double off = -dt * g[i];
        double l = off / d[i];
        d[par[i]] -= l * off;
        r[par[i]] -= l * r[i];
    }
    sigma[0] = r[0] / d[0];
    for (i = 1; i < n; ++i) {
        double off = -dt * g[i];
        sigma[i] = (r[i] - off * sigma[par[i]]) / d[i];
    }
}

int orc_advance(int n_trees, const long *off, const int *par,
                const double *V, const double *g, const double *f,
                const double *leak, const double *sig_crit,
                double *sigma, int *void_flag, double *void_vol, double *t_nuc,
                double t0, double dt, int n_steps, double B_modulus,
                double *margin, double *gap, int n_threads)
{
    int total = 0;
    int t;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (t = 0; t < n_trees; ++t) {
        long b = off[t];
        int n = (int)(off[t + 1] - off[t]);
        const int *P = par + b;
        double *s = sigma + b;
        int *vf = void_flag + b;
        double *vv = void_vol + b;
        double *d = (double *)malloc(sizeof(double) * (size_t)n);
        double *r = (double *)malloc(sizeof(double) * (size_t)n);
        double *prev = (double *)malloc(sizeof(double) * (size_t)n);
        double mmin = INFINITY, gmin = INFINITY;
        int k, i;
        for (k = 0; k < n_steps; ++k) {
            memcpy(prev, s, sizeof(double) * (size_t)n);
            be_step_tree(n, P, V + b, g + b, f + b, leak + b, vf, dt, s, d, r);
            /* void growth by the Robin leak, Eq. void_volume_equation */
            for (i = 0; i < n; ++i)
                if (vf[i]) vv[i] += dt / B_modulus * leak[b + i] * s[i];
            /* nucleation: argmax over non-void nodes, lowest index on ties */
            {
                int arg = -1;
                double best = -INFINITY, second = -INFINITY;
                for (i = 0; i < n; ++i) {
                    double m;
                    if (vf[i]) continue;
                    m = s[i] - sig_crit[b + i];
                    if (m > best) { second = best; best = m; arg = i; }
                    else if (m > second) second = m;
                }
                if (arg >= 0) {
                    double rel = fabs(best) / sig_crit[b + arg];
                    if (rel < mmin) mmin = rel;
                    if (best >= 0.0) {
                        double m0 = prev[arg] - sig_crit[b + arg];
                        double gp = (best - second) / sig_crit[b + arg];
                        if (gp < gmin) gmin = gp;
                        double frac = (m0 < 0.0) ? (-m0) / (best - m0) : 0.0;
                        vf[arg] = 1;
                        vv[arg] = 0.0;
                        t_nuc[b + arg] = t0 + ((double)k + frac) * dt;
                        total += 1;
                    }
                }
            }
        }
        if (margin) margin[t] = mmin;
        if (gap) gap[t] = gmin;
        free(d); free(r); free(prev);
    }
    return total;
}

void orc_steady(int n_trees, const long *off, const int *par, const double *V,
                const double *dxG, double sigma_T, double *sigma_ss)
{
    int t;
    for (t = 0; t < n_trees; ++t) {
        long b = off[t];
        int n = (int)(off[t + 1] - off[t]);
        double sv = 0.0, svp = 0.0, mean;
        int i;
        double *P = sigma_ss + b;
        P[0] = 0.0;
        for (i = 1; i < n; ++i) P[i] = P[par[b + i]] + dxG[b + i];
        for (i = 0; i < n; ++i) { sv += V[b + i]; svp += V[b + i] * P[i]; }
        mean = svp / sv;
        for (i = 0; i < n; ++i) P[i] = sigma_T + P[i] - mean;
    }
}
