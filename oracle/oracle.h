/*
 * SE-RBFNet FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, brute-force restatement of the optimisation hot path of
 * "Approximating Signed Distance Fields With Sparse Ellipsoidal Radial Basis
 * Function Networks" (SE-RBFNet).  It exists to check the CUDA library and is
 * never linked into it: only tests/, the smoke check of __graft_entry__ and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no source,
 * header, table or helper with the GPU path.
 *
 * Conventions (written out again here on purpose, not included from the GPU
 * headers):
 *   - parameters: 10 rows of `cap` doubles, row r at P + r*cap, in the order
 *     cx, cy, cz, d1, d2, d3, theta_x, theta_y, theta_z, w   (Sec. 3.2, Eq. 3-8).
 *     (the float parameters of the GPU path are passed widened to double);
 *   - every quantity is evaluated in double, except the support-membership
 *     predicate and the binning key, which are evaluated in float (parameters
 *     narrowed back to float, exact for widened floats) with the
 *     operation order spelled out in oracle.c (so both sides take the same
 *     integer decision).
 *
 * Parity status per function is stated in oracle.c next to each definition.
 */
#ifndef SERBF_ORACLE_H
#define SERBF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int oracle_version(void);
void oracle_set_threads(int n);

/* Eq. 3-15 / 3-15-1 support radius and membership (float, canonical order) */
float oracle_support_r2(float d1, float d2, float d3, float neg_ln_eps);
int oracle_in_support(float px, float py, float pz, float cx, float cy, float cz, float r2);

/* App. A rotation entries r1..r9, row-major */
void oracle_rotation(double tx, double ty, double tz, double R[9]);

/* Eq. 3-7: one ellipsoidal basis function at point v (no cutoff) */
double oracle_erbf(double vx, double vy, double vz, const double *P, int32_t cap, int32_t j);

/* Eq. 3-10 target normalisation */
void oracle_normalize(const float *S, int64_t n, double *t, double *m_out, double *h_out);

/* Point binning: canonical float cell index, super-major key, stable sort by (key, index) */
void oracle_cell_keys(const float *x, const float *y, const float *z, int64_t n, float ox, float oy,
                      float oz, float h, int32_t nx, int32_t ny, int32_t nz, int32_t sf, uint32_t *key);
void oracle_bin(const float *x, const float *y, const float *z, int64_t n, float ox, float oy, float oz,
                float h, int32_t nx, int32_t ny, int32_t nz, int32_t sf, uint32_t *perm);

/* Eq. 3-15-1 neighbour lists by brute force over all pairs; CSR in both orientations.
 * kcol / pcol may be NULL (count only).  Returns the number of pairs. */
int64_t oracle_neighbors(const float *x, const float *y, const float *z, int64_t n, const double *P,
                         int32_t cap, int32_t m, float neg_ln_eps, int64_t *krow, uint32_t *kcol,
                         int64_t *prow, uint32_t *pcol);

/* Eq. 3-26 forward, Eq. 3-18 filter, Eq. 3-19 loss terms.
 * stats[0]=L2, stats[1]=L1, stats[2]=max|E| over id_all, stats[3]=|id_all|, stats[4]=pairs */
void oracle_forward(const float *x, const float *y, const float *z, const float *t, int64_t n,
                    const double *P, int32_t cap, int32_t m, float neg_ln_eps, double tau1, double tau2,
                    int use_cutoff, double *psi, double *err, uint8_t *mask, double *stats);

/* App. A gradients of L2 = sum_i E_i^2 with E_i := err[i] (points with err[i]==0 skipped).
 * grad: 10 rows of m doubles, same row order as P. */
void oracle_backward(const float *x, const float *y, const float *z, int64_t n, const double *err,
                     const double *P, int32_t cap, int32_t m, float neg_ln_eps, int use_cutoff,
                     double *grad, int64_t *npairs);

/* Eq. 3-21 */
double oracle_alpha(const double *g2w, const double *w, int32_t m);

/* Kingma-Ba Adam, one step on n scalars, step counter t (>=1) */
void oracle_adam(double *p, const double *g, double *mo, double *v, int64_t n, int32_t t, double lr,
                 double b1, double b2, double eps);

/* Algorithm 3 optimiser step and epoch tail (dynamic weighting, Adam, gates) */
typedef struct {
    int32_t epoch;     /* completed epochs */
    int32_t l1_optim;  /* Alg. 3 flag l1_optim */
    int32_t phase2;    /* epoch T^e reached: L2-only, cosine learning rate */
    int32_t adam_t;    /* Adam step counter */
    int32_t do_prune;  /* Eq. 3-27 due at the end of this epoch */
    int32_t do_add;    /* Eq. 3-24 due at the end of this epoch */
    int32_t n_l2;      /* filled entries of l2_hist */
    int32_t n_bf;      /* filled entries of bf_hist */
    int32_t step;      /* steps done in the current epoch (mini-batches) */
    int32_t pad;
    double lr;         /* learning rate of the next epoch */
    double alpha, beta;
    double l2_epoch;   /* sum of the batch L2 values of the current epoch */
    double l2_hist[64];
    int32_t bf_hist[256];
} oracle_state;

typedef struct {
    double lr0, lr_p2, lr_min, beta1, beta2, adam_eps;
    double tau_m, tau_d, tau_l1, tau_l2;
    int32_t k_l1, k_l2, T_e, M_e;
    int32_t epoch_steps; /* optimiser steps per epoch (1: full batch) */
    int32_t pad;
} oracle_cfg;

void oracle_state_init(oracle_state *st, const oracle_cfg *cfg);
/* P: 10 x cap doubles (updated), grad: 10 x m raw L2 gradients, mo/v: 10 x cap Adam moments */
void oracle_step(double *P, int32_t cap, int32_t m, const double *grad, double *mo, double *v,
                 double l2, double max_abs_e, const oracle_cfg *cfg, oracle_state *st);

/* Eq. 3-27 pruning, stable; returns the new kernel count.  mo/v may be NULL. */
int32_t oracle_prune(double *P, double *mo, double *v, int32_t cap, int32_t m, double tau_d);

/* Algorithm 2 (top-k form) and Eq. 3-24 */
int32_t oracle_select_topk(const float *E, const uint8_t *mask, int64_t n, double thresh, int64_t k,
                           int32_t *out);
int32_t oracle_local_max(const float *x, const float *y, const float *z, const float *E,
                         const uint8_t *mask, int64_t n, const int32_t *cand, int32_t nc, float r2,
                         int32_t *out);
void oracle_new_kernel(float px, float py, float pz, float e, double dbar, double eps, double out[10]);

/* Surface extraction (marching tetrahedra), area-weighted sampling and the
 * Sec. 4 metrics HD, CD, CS. */
int64_t oracle_marching_tets(const float *f, int nx, int ny, int nz, const float o[3], float h, float iso, float *tri,
                             int64_t cap);
int oracle_sample_surface(const float *tri, int64_t ntri, const double *u, int64_t ns, float *pts, float *nrm);
void oracle_surface_metrics(const float *A, const float *nA, int64_t na, const float *B, const float *nB, int64_t nb,
                            double out[3]);

/* Algorithm 1 (greedy inscribed spheres) and Eq. 3-12 (isotropic shapes). */
int32_t oracle_inscribed(const float *x, const float *y, const float *z, const float *t, const float *S,
                         int64_t n, int32_t *out, int32_t max_out);
void oracle_init_shape(const double *cx, const double *cy, const double *cz, const double *w, const double *r,
                       int32_t M, double gamma, double *d);

#ifdef __cplusplus
}
#endif
#endif
