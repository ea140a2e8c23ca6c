/*
 * SE-RBFNet FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Every function below follows one passage of the paper and says which.  The
 * arithmetic is double precision, brute force over all (point, kernel) pairs,
 * in the paper's notation.  Only two decisions are taken in float, because the
 * GPU path must take exactly the same integer decision:
 *   - support membership, Eq. 3-15-1:  with d_k the three axis parameters,
 *       lam = min_k fl(d_k*d_k),  r2 = fl(neg_ln_eps / lam),
 *       dx = fl(px-cx) (etc.),  dist2 = fl(fl(fl(dx*dx)+fl(dy*dy))+fl(dz*dz)),
 *       member  <=>  dist2 < r2   (strict, as in Eq. 3-15-1);
 *   - the binning cell index: k = clamp(floor(fl(fl(x-ox)/h)), 0, n-1).
 * The file must be compiled with -ffp-contract=off so that no multiply-add is
 * fused in those two float expressions.
 *
 * Pins (tests/test_oracle_*.py): closed forms, finite differences,
 * invariants, brute force and library special cases; see each function.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { CX = 0, CY, CZ, D1, D2, D3, TX, TY, TZ, W, NPAR };

int oracle_version(void) { return 1; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static double sgn(double v) { return (v > 0) - (v < 0); } /* sign(0)=0, Sec. 3.4.3 */

/* ---------------------------------------------------------------------------
 * Eq. 3-15: lambda_j is the smallest eigenvalue of R^T D^T D R, i.e. the
 * smallest d_jk^2; the support radius is sqrt(-ln(eps)/lambda_j).  We keep the
 * squared radius.  Eq. 3-15-1: F_ij is nonzero only for ||c_j - v_i|| < radius.
 * Pinned by: FP64 margin invariant and brute-force predicate tests.
 */
float oracle_support_r2(float d1, float d2, float d3, float neg_ln_eps) {
    float a = d1 * d1, b = d2 * d2, c = d3 * d3;
    float lam = a;
    if (b < lam) lam = b;
    if (c < lam) lam = c;
    return neg_ln_eps / lam;
}

/* The canonical float squared distance of the membership test: the three
 * differences, then fl(dx dx) and two fused multiply-adds (fmaf rounds once,
 * C99), fmaf(dz, dz, fmaf(dy, dy, dx * dx)).  Reading: the paper states the
 * test in real arithmetic; the float form is fixed so that every
 * implementation takes the same integer decision. */
static float support_d2(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }

int oracle_in_support(float px, float py, float pz, float cx, float cy, float cz, float r2) {
    float dx = px - cx, dy = py - cy, dz = pz - cz;
    return support_d2(dx, dy, dz) < r2;
}

/* ---------------------------------------------------------------------------
 * App. A, rotation matrix entries r1..r9 (row-major).  These equal
 * R_z(theta_x) R_y(theta_y) R_x(theta_z) with the elementary matrices of
 * Eq. 3-6; the App. A entries are taken as the definition of R.
 * Pinned by: product of the Eq. 3-6 elementary matrices built in the test.
 */
void oracle_rotation(double tx, double ty, double tz, double R[9]) {
    double cx = cos(tx), sx = sin(tx), cy = cos(ty), sy = sin(ty), cz = cos(tz), sz = sin(tz);
    R[0] = cx * cy;
    R[1] = -cz * sx - sy * sz * cx;
    R[2] = sx * sz - cx * cz * sy;
    R[3] = cy * sx;
    R[4] = cx * cz - sx * sy * sz;
    R[5] = -sz * cx - cz * sx * sy;
    R[6] = sy;
    R[7] = cy * sz;
    R[8] = cy * cz;
}

/* Eq. 3-7: Phi(x) = exp(-|| D R (x - c) ||^2), D = diag(d1,d2,d3).
 * Pinned by: single-kernel closed forms along rotated principal axes. */
double oracle_erbf(double vx, double vy, double vz, const double *P, int32_t cap, int32_t j) {
    double R[9];
    oracle_rotation(P[TX * cap + j], P[TY * cap + j], P[TZ * cap + j], R);
    double dl[3] = {vx - P[CX * cap + j], vy - P[CY * cap + j], vz - P[CZ * cap + j]};
    double q = 0.0;
    for (int k = 0; k < 3; ++k) {
        double u = R[3 * k + 0] * dl[0] + R[3 * k + 1] * dl[1] + R[3 * k + 2] * dl[2];
        double dk = P[(D1 + k) * cap + j];
        q += (dk * u) * (dk * u);
    }
    return exp(-q);
}

/* ---------------------------------------------------------------------------
 * Eq. 3-10: S_hat = 2 exp(-h (S - m)^2), m = min(S), h = ln 2 / m^2.
 * Pinned by: fixed points S=0 -> 1, S=m -> 2 and S=-m -> 1/8. */
void oracle_normalize(const float *S, int64_t n, double *t, double *m_out, double *h_out) {
    double m = INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if ((double)S[i] < m) m = S[i];
    double h = log(2.0) / (m * m);
    for (int64_t i = 0; i < n; ++i) {
        double s = (double)S[i] - m;
        t[i] = 2.0 * exp(-h * s * s);
    }
    if (m_out) *m_out = m;
    if (h_out) *h_out = h;
}

/* ---------------------------------------------------------------------------
 * Point binning for the neighbour search (Sec. 3.4.4 "nearest-neighbour based"
 * restriction).  The paper does not fix a data structure; the reading used by
 * this project: a uniform cell grid whose cells are grouped into super cells
 * of sf^3 cells, points stably sorted by (super cell, cell in the super cell,
 * index).  Pinned by: numpy lexsort of the same keys. */
static uint32_t cell_axis(float v, float o, float h, int32_t n) {
    float f = (v - o) / h;
    float fl = floorf(f);
    if (!(fl >= 0.0f)) return 0; /* also catches NaN */
    if (fl >= (float)(n - 1)) return (uint32_t)(n - 1);
    return (uint32_t)fl;
}

void oracle_cell_keys(const float *x, const float *y, const float *z, int64_t n, float ox, float oy,
                      float oz, float h, int32_t nx, int32_t ny, int32_t nz, int32_t sf, uint32_t *key) {
    uint32_t nsx = (uint32_t)((nx + sf - 1) / sf), nsy = (uint32_t)((ny + sf - 1) / sf);
    uint32_t s3 = (uint32_t)(sf * sf * sf);
    (void)nz;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t kx = cell_axis(x[i], ox, h, nx), ky = cell_axis(y[i], oy, h, ny),
                 kz = cell_axis(z[i], oz, h, nz);
        uint32_t super = ((kz / sf) * nsy + ky / sf) * nsx + kx / sf;
        uint32_t local = ((kz % sf) * sf + ky % sf) * sf + kx % sf;
        key[i] = super * s3 + local;
    }
}

static const uint32_t *g_sort_keys;
static int cmp_key_index(const void *a, const void *b) {
    uint32_t ia = *(const uint32_t *)a, ib = *(const uint32_t *)b;
    uint32_t ka = g_sort_keys[ia], kb = g_sort_keys[ib];
    if (ka != kb) return ka < kb ? -1 : 1;
    return ia < ib ? -1 : (ia > ib);
}

void oracle_bin(const float *x, const float *y, const float *z, int64_t n, float ox, float oy, float oz,
                float h, int32_t nx, int32_t ny, int32_t nz, int32_t sf, uint32_t *perm) {
    uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    oracle_cell_keys(x, y, z, n, ox, oy, oz, h, nx, ny, nz, sf, key);
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    g_sort_keys = key;
    qsort(perm, (size_t)n, sizeof(uint32_t), cmp_key_index);
    g_sort_keys = NULL;
    free(key);
}

/* ---------------------------------------------------------------------------
 * Eq. 3-15-1 by brute force over every (i, j).  Kernel-major rows list points
 * in ascending index, point-major rows list kernels in ascending index.
 * Pinned by: numpy brute force of the same predicate; FP64 margin test. */
int64_t oracle_neighbors(const float *x, const float *y, const float *z, int64_t n, const double *P,
                         int32_t cap, int32_t m, float neg_ln_eps, int64_t *krow, uint32_t *kcol,
                         int64_t *prow, uint32_t *pcol) {
    float *r2 = (float *)malloc(sizeof(float) * (size_t)(m ? m : 1));
    for (int32_t j = 0; j < m; ++j)
        r2[j] = oracle_support_r2((float)P[D1 * cap + j], (float)P[D2 * cap + j], (float)P[D3 * cap + j], neg_ln_eps);
    /* kernel-major */
    int64_t *kc = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t j = 0; j < m; ++j) {
        int64_t c = 0;
        for (int64_t i = 0; i < n; ++i)
            c += oracle_in_support(x[i], y[i], z[i], (float)P[CX * cap + j], (float)P[CY * cap + j],
                                   (float)P[CZ * cap + j], r2[j]);
        kc[j] = c;
    }
    int64_t tot = 0;
    for (int32_t j = 0; j < m; ++j) {
        int64_t c = kc[j];
        if (krow) krow[j] = tot;
        tot += c;
    }
    if (krow) krow[m] = tot;
    if (kcol) {
#pragma omp parallel for schedule(dynamic, 4)
        for (int32_t j = 0; j < m; ++j) {
            int64_t o = krow[j];
            for (int64_t i = 0; i < n; ++i)
                if (oracle_in_support(x[i], y[i], z[i], (float)P[CX * cap + j], (float)P[CY * cap + j],
                                      (float)P[CZ * cap + j], r2[j]))
                    kcol[o++] = (uint32_t)i;
        }
    }
    /* point-major */
    if (prow) {
        int64_t *pc = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = 0;
            for (int32_t j = 0; j < m; ++j)
                c += oracle_in_support(x[i], y[i], z[i], (float)P[CX * cap + j], (float)P[CY * cap + j],
                                       (float)P[CZ * cap + j], r2[j]);
            pc[i] = c;
        }
        int64_t s = 0;
        for (int64_t i = 0; i < n; ++i) {
            prow[i] = s;
            s += pc[i];
        }
        prow[n] = s;
        free(pc);
        if (pcol) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                int64_t o = prow[i];
                for (int32_t j = 0; j < m; ++j)
                    if (oracle_in_support(x[i], y[i], z[i], (float)P[CX * cap + j], (float)P[CY * cap + j],
                                          (float)P[CZ * cap + j], r2[j]))
                        pcol[o++] = (uint32_t)j;
            }
        }
    }
    free(kc);
    free(r2);
    return tot;
}

/* ---------------------------------------------------------------------------
 * Eq. 3-26: Psi_i = sum_j w_j |w_j| F_ij with F from Eq. 3-15-1 (use_cutoff)
 * or Eq. 3-9 (no cutoff).  Eq. 3-18: id_0 = {tau1 < t < tau2},
 * id_1 = {t <= tau1 and Psi > tau1}, id_2 = {t >= tau2 and Psi < tau2}.
 * Eq. 3-19: L2 = sum over id_all of (Psi - t)^2;  Eq. 3-14_2: L1 = sum |w|.
 * E_i = Psi_i - t_i on id_all and 0 elsewhere (only id_all enters the loss).
 * Pinned by: single-kernel closed forms, superposition, permutation
 * invariance, sphere-SDF mask cases. */
void oracle_forward(const float *x, const float *y, const float *z, const float *t, int64_t n,
                    const double *P, int32_t cap, int32_t m, float neg_ln_eps, double tau1, double tau2,
                    int use_cutoff, double *psi, double *err, uint8_t *mask, double *stats) {
    float *r2 = (float *)malloc(sizeof(float) * (size_t)(m ? m : 1));
    for (int32_t j = 0; j < m; ++j)
        r2[j] = oracle_support_r2((float)P[D1 * cap + j], (float)P[D2 * cap + j], (float)P[D3 * cap + j], neg_ln_eps);
    int64_t *pairs = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        int64_t c = 0;
        for (int32_t j = 0; j < m; ++j) {
            if (use_cutoff && !oracle_in_support(x[i], y[i], z[i], (float)P[CX * cap + j], (float)P[CY * cap + j],
                                                 (float)P[CZ * cap + j], r2[j]))
                continue;
            double w = P[W * cap + j];
            s += w * fabs(w) * oracle_erbf(x[i], y[i], z[i], P, cap, j);
            ++c;
        }
        pairs[i] = c;
        double ti = t[i];
        int in0 = (tau1 < ti) && (ti < tau2);
        int in1 = (ti <= tau1) && (s > tau1);
        int in2 = (ti >= tau2) && (s < tau2);
        uint8_t mk = (uint8_t)(in0 | in1 | in2);
        psi[i] = s;
        mask[i] = mk;
        err[i] = mk ? s - ti : 0.0;
    }
    double l2 = 0.0, l1 = 0.0, mx = 0.0, cnt = 0.0, np = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        np += (double)pairs[i];
        if (!mask[i]) continue;
        l2 += err[i] * err[i];
        if (fabs(err[i]) > mx) mx = fabs(err[i]);
        cnt += 1.0;
    }
    for (int32_t j = 0; j < m; ++j) l1 += fabs((double)P[W * cap + j]);
    stats[0] = l2;
    stats[1] = l1;
    stats[2] = mx;
    stats[3] = cnt;
    stats[4] = np;
    free(pairs);
    free(r2);
}

/* ---------------------------------------------------------------------------
 * App. A, term by term, summed over the points of each kernel's support with
 * E_i = err[i] (points with err == 0 contribute nothing and are skipped).
 *   dL2/dw_j    = sum 4 w sign(w) F E                           (weights)
 *   dL2/dd_jk   = sum -4 sign(w) w^2 d_k F Dt_k^2 E              (axis lengths)
 *   Et          = (d_k^2 w^2 Dt_k F)_k,  Ft = R^T Et
 *   dL2/dc_jk   = sum 4 sign(w) Ft_k E                           (centres)
 *   dL2/dtheta  = sum -4 sign(w) E (Et . (dR/dtheta) Delta)      (angles)
 * with Delta = v - c and Dt = R Delta.  Reading: the theta_x term is
 * Et1*(-Dt2) + Et2*(+Dt1), the derivative of the App. A matrix (the printed
 * second sign is inconsistent with it); the theta_z term's garbled symbols read
 * as Et3 and D^_Y.  Pinned by: central finite differences of the FP64 loss
 * (no cutoff), exact zero theta gradients for isotropic kernels, single-pair
 * closed forms. */
void oracle_backward(const float *x, const float *y, const float *z, int64_t n, const double *err,
                     const double *P, int32_t cap, int32_t m, float neg_ln_eps, int use_cutoff,
                     double *grad, int64_t *npairs) {
    int64_t *pc = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t j = 0; j < m; ++j) {
        double c[3] = {P[CX * cap + j], P[CY * cap + j], P[CZ * cap + j]};
        double d[3] = {P[D1 * cap + j], P[D2 * cap + j], P[D3 * cap + j]};
        double tx = P[TX * cap + j], ty = P[TY * cap + j], tz = P[TZ * cap + j];
        double w = P[W * cap + j];
        double sw = sgn(w);
        double R[9];
        oracle_rotation(tx, ty, tz, R);
        double cxs = cos(tx), sxs = sin(tx), sys = sin(ty), czs = cos(tz), szs = sin(tz);
        float r2 = oracle_support_r2((float)P[D1 * cap + j], (float)P[D2 * cap + j], (float)P[D3 * cap + j], neg_ln_eps);
        double g[NPAR] = {0};
        int64_t cnt = 0;
        for (int64_t i = 0; i < n; ++i) {
            double E = err[i];
            if (E == 0.0) continue;
            if (use_cutoff && !oracle_in_support(x[i], y[i], z[i], (float)P[CX * cap + j], (float)P[CY * cap + j],
                                                 (float)P[CZ * cap + j], r2))
                continue;
            ++cnt;
            double dl[3] = {(double)x[i] - c[0], (double)y[i] - c[1], (double)z[i] - c[2]};
            double Dt[3];
            for (int k = 0; k < 3; ++k) Dt[k] = R[3 * k] * dl[0] + R[3 * k + 1] * dl[1] + R[3 * k + 2] * dl[2];
            double q = 0.0;
            for (int k = 0; k < 3; ++k) q += d[k] * d[k] * Dt[k] * Dt[k];
            double F = exp(-q);
            /* weights */
            g[W] += 4.0 * w * sw * F * E;
            /* axis lengths */
            for (int k = 0; k < 3; ++k) g[D1 + k] += -4.0 * sw * w * w * d[k] * F * Dt[k] * Dt[k] * E;
            /* centres */
            double Et[3];
            for (int k = 0; k < 3; ++k) Et[k] = d[k] * d[k] * w * w * Dt[k] * F;
            double Ft[3];
            for (int k = 0; k < 3; ++k) Ft[k] = R[k] * Et[0] + R[3 + k] * Et[1] + R[6 + k] * Et[2];
            for (int k = 0; k < 3; ++k) g[CX + k] += 4.0 * sw * Ft[k] * E;
            /* theta_x */
            g[TX] += -4.0 * sw * E * (Et[0] * (-Dt[1]) + Et[1] * Dt[0]);
            /* theta_y */
            double DX = -cxs * sys * dl[0] - R[0] * szs * dl[1] - R[0] * czs * dl[2];
            double DY = -sxs * sys * dl[0] - R[3] * szs * dl[1] - R[3] * czs * dl[2];
            double DZ = cos(ty) * dl[0] - sys * szs * dl[1] - sys * czs * dl[2];
            g[TY] += -4.0 * sw * E * (Et[0] * DX + Et[1] * DY + Et[2] * DZ);
            /* theta_z */
            double HX = R[2] * dl[1] - R[1] * dl[2];
            double HY = R[5] * dl[1] - R[4] * dl[2];
            double HZ = R[8] * dl[1] - R[7] * dl[2];
            g[TZ] += -4.0 * sw * E * (Et[0] * HX + Et[1] * HY + Et[2] * HZ);
        }
        for (int r = 0; r < NPAR; ++r) grad[(int64_t)r * m + j] = g[r];
        pc[j] = cnt;
    }
    if (npairs) {
        int64_t s = 0;
        for (int32_t j = 0; j < m; ++j) s += pc[j];
        *npairs = s;
    }
    free(pc);
}

/* ---------------------------------------------------------------------------
 * Eq. 3-21 with g1 = dL1/dW = sign(W), g2 = dL2/dW:
 *   alpha = clip_[0,1]( (g1 - g2)^T g1 / ||g2 - g1||^2 ),  beta = 1 - alpha.
 * Reading: a zero denominator (g1 == g2) leaves every alpha optimal; alpha = 1.
 * Pinned by: brute-force line search of min_a ||a g2 + (1-a) g1||^2. */
double oracle_alpha(const double *g2w, const double *w, int32_t m) {
    double num = 0.0, den = 0.0;
    for (int32_t j = 0; j < m; ++j) {
        double g1 = sgn(w[j]);
        num += (g1 - g2w[j]) * g1;
        den += (g2w[j] - g1) * (g2w[j] - g1);
    }
    if (!(den > 0.0)) return 1.0;
    double a = num / den;
    if (a > 1.0) a = 1.0;
    if (a < 0.0) a = 0.0;
    return a;
}

/* Kingma & Ba, Adam (cited by the paper for every update, Alg. 3).
 * Pinned by: torch.optim.Adam in float64 on the CPU. */
void oracle_adam(double *p, const double *g, double *mo, double *v, int64_t n, int32_t t, double lr,
                 double b1, double b2, double eps) {
    double bc1 = 1.0 - pow(b1, t), bc2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        mo[i] = b1 * mo[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = mo[i] / bc1, vh = v[i] / bc2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ---------------------------------------------------------------------------
 * Algorithm 3, one full-batch epoch after the gradient is known:
 *   - dynamic weighting (Alg. 3 "if l1_optim and Eq. l1_activate2": Eq. 3-21,
 *     else alpha=1, beta=0), combined gradient per Eq. grad of App. A;
 *   - Adam update;
 *   - epoch tail in the order of Algorithm 3: deletion gate (every k^l2
 *     epochs while l1_optim and e_p < T^e), L1 activation (Eq. l1_activate:
 *     population std of the last k^l2 L2 values < tau^l2), addition gate
 *     (Eq. add_activate over the last k^l1 values of b_f), switch to the
 *     L2-only phase at e_p = T^e with a cosine learning rate from lr_p2 to
 *     lr_min at M^e.
 * b_f = #{|w_j| >= tau_d} after the update (Sec. 3.4.3).
 * Parity unpinned beyond its parts (alpha, Adam are pinned); gate timing is
 * checked against hand-built L2 / b_f sequences. */
void oracle_state_init(oracle_state *st, const oracle_cfg *cfg) {
    memset(st, 0, sizeof(*st));
    st->lr = cfg->lr0;
    st->alpha = 1.0;
    st->beta = 0.0;
}

void oracle_step(double *P, int32_t cap, int32_t m, const double *grad, double *mo, double *v,
                 double l2, double max_abs_e, const oracle_cfg *cfg, oracle_state *st) {
    int32_t e = st->epoch + 1;
    double alpha = 1.0;
    if (st->l1_optim && max_abs_e < cfg->tau_m) {
        double *wv = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
        for (int32_t j = 0; j < m; ++j) wv[j] = P[W * cap + j];
        alpha = oracle_alpha(grad + (int64_t)W * m, wv, m);
        free(wv);
    }
    double beta = 1.0 - alpha;
    st->alpha = alpha;
    st->beta = beta;
    st->adam_t += 1;
    double *gk = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
    double *pk = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
    double *mk = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
    double *vk = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
    for (int r = 0; r < NPAR; ++r) {
        for (int32_t j = 0; j < m; ++j) {
            double g = alpha * grad[(int64_t)r * m + j];
            if (r == W) g += beta * sgn(P[W * cap + j]);
            gk[j] = g;
            pk[j] = P[(int64_t)r * cap + j];
            mk[j] = mo[(int64_t)r * cap + j];
            vk[j] = v[(int64_t)r * cap + j];
        }
        oracle_adam(pk, gk, mk, vk, m, st->adam_t, st->lr, cfg->beta1, cfg->beta2, cfg->adam_eps);
        for (int32_t j = 0; j < m; ++j) {
            P[(int64_t)r * cap + j] = pk[j];
            mo[(int64_t)r * cap + j] = mk[j];
            v[(int64_t)r * cap + j] = vk[j];
        }
    }
    free(gk);
    free(pk);
    free(mk);
    free(vk);

    /* Algorithm 3 runs the gates once per epoch, after its last batch: with
     * epoch_steps > 1 mini-batches the L2 of the epoch is the sum of its
     * batch values (reading of the per-epoch L2 for mini-batches) */
    l2 += st->l2_epoch;
    if (st->step + 1 < (cfg->epoch_steps > 1 ? cfg->epoch_steps : 1)) {
        st->step += 1;
        st->l2_epoch = l2;
        return;
    }
    st->step = 0;
    st->l2_epoch = 0.0;

    /* epoch tail */
    st->do_prune = (e % cfg->k_l2 == 0) && st->l1_optim && (e < cfg->T_e);
    int32_t bf = 0;
    for (int32_t j = 0; j < m; ++j) bf += fabs(P[W * cap + j]) >= cfg->tau_d;
    /* histories keep the most recent values in order */
    if (st->n_l2 < cfg->k_l2) {
        st->l2_hist[st->n_l2++] = l2;
    } else {
        memmove(st->l2_hist, st->l2_hist + 1, sizeof(double) * (size_t)(cfg->k_l2 - 1));
        st->l2_hist[cfg->k_l2 - 1] = l2;
    }
    if (st->n_bf < cfg->k_l1) {
        st->bf_hist[st->n_bf++] = bf;
    } else {
        memmove(st->bf_hist, st->bf_hist + 1, sizeof(int32_t) * (size_t)(cfg->k_l1 - 1));
        st->bf_hist[cfg->k_l1 - 1] = bf;
    }
    if (!st->l1_optim && !st->phase2 && e >= cfg->k_l2 && st->n_l2 == cfg->k_l2) {
        double mean = 0.0;
        for (int k = 0; k < cfg->k_l2; ++k) mean += st->l2_hist[k];
        mean /= cfg->k_l2;
        double var = 0.0;
        for (int k = 0; k < cfg->k_l2; ++k) var += (st->l2_hist[k] - mean) * (st->l2_hist[k] - mean);
        var /= cfg->k_l2;
        if (sqrt(var) < cfg->tau_l2) st->l1_optim = 1;
    }
    st->do_add = 0;
    if (st->l1_optim && !st->phase2 && st->n_bf == cfg->k_l1) {
        int32_t lo = st->bf_hist[0], hi = st->bf_hist[0];
        for (int k = 1; k < cfg->k_l1; ++k) {
            if (st->bf_hist[k] < lo) lo = st->bf_hist[k];
            if (st->bf_hist[k] > hi) hi = st->bf_hist[k];
        }
        if ((double)(hi - lo) < cfg->tau_l1) {
            st->do_add = 1;
            st->l1_optim = 0;
        }
    }
    if (e == cfg->T_e) {
        st->phase2 = 1;
        st->l1_optim = 0;
    }
    if (st->phase2) {
        double span = (double)(cfg->M_e - cfg->T_e);
        double p = span > 0 ? (double)(e - cfg->T_e) / span : 1.0;
        if (p > 1.0) p = 1.0;
        st->lr = cfg->lr_min + (cfg->lr_p2 - cfg->lr_min) * 0.5 * (1.0 + cos(M_PI * p));
    } else {
        st->lr = cfg->lr0;
    }
    st->epoch = e;
}

/* Eq. 3-27: delete kernels with |w_j| < tau_d; survivors keep their order.
 * Pinned by: direct property test. */
int32_t oracle_prune(double *P, double *mo, double *v, int32_t cap, int32_t m, double tau_d) {
    int32_t o = 0;
    for (int32_t j = 0; j < m; ++j) {
        if (!(fabs(P[W * cap + j]) >= tau_d)) continue;
        for (int r = 0; r < NPAR; ++r) {
            P[(int64_t)r * cap + o] = P[(int64_t)r * cap + j];
            if (mo) mo[(int64_t)r * cap + o] = mo[(int64_t)r * cap + j];
            if (v) v[(int64_t)r * cap + o] = v[(int64_t)r * cap + j];
        }
        ++o;
    }
    return o;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, candidate set (I_add = {|E_i| > tau_m / 2} over id_all), then the
 * top-k restriction used by this project (k largest |E|, ties by ascending
 * index; output in that order).  thresh = tau_m / 2.
 * Pinned by: Python sorted() on the same keys. */
static const float *g_absE;
static int cmp_topk(const void *a, const void *b) {
    int32_t ia = *(const int32_t *)a, ib = *(const int32_t *)b;
    float ea = fabsf(g_absE[ia]), eb = fabsf(g_absE[ib]);
    if (ea != eb) return ea > eb ? -1 : 1;
    return ia < ib ? -1 : (ia > ib);
}

int32_t oracle_select_topk(const float *E, const uint8_t *mask, int64_t n, double thresh, int64_t k,
                           int32_t *out) {
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t nc = 0;
    for (int64_t i = 0; i < n; ++i)
        if (mask[i] && (double)fabsf(E[i]) > thresh) c[nc++] = (int32_t)i;
    g_absE = E;
    qsort(c, (size_t)nc, sizeof(int32_t), cmp_topk);
    g_absE = NULL;
    int32_t take = (k >= 0 && k < nc) ? (int32_t)k : nc;
    memcpy(out, c, sizeof(int32_t) * (size_t)take);
    free(c);
    return take;
}

/* Algorithm 2, local-maximum test: keep candidate i if |E_i| >= |E_n| for every id_all
 * point n within radius r of v_i (distance test in float, same operation
 * order as the support predicate, <= r2).  Brute force over all points.
 * Pinned by: numpy brute force. */
int32_t oracle_local_max(const float *x, const float *y, const float *z, const float *E,
                         const uint8_t *mask, int64_t n, const int32_t *cand, int32_t nc, float r2,
                         int32_t *out) {
    int32_t o = 0;
    for (int32_t a = 0; a < nc; ++a) {
        int32_t i = cand[a];
        float ei = fabsf(E[i]);
        int ok = 1;
        for (int64_t q = 0; q < n && ok; ++q) {
            if (!mask[q]) continue;
            float dx = x[q] - x[i], dy = y[q] - y[i], dz = z[q] - z[i];
            float d2 = support_d2(dx, dy, dz);
            if (d2 <= r2 && fabsf(E[q]) > ei) ok = 0;
        }
        if (ok) out[o++] = i;
    }
    return o;
}

/* Eq. 3-24: c^a = v_i, W^a = -sign(E) |E| = -E, d^a = sqrt(-ln(eps/|E|) / dbar^2)
 * on all three axes, A^a = 0.  Output in parameter-row order.
 * Pinned by: Phi_new(c + dbar e_k) = eps / |E| (closed form). */
void oracle_new_kernel(float px, float py, float pz, float e, double dbar, double eps, double out[10]) {
    double ae = fabs((double)e);
    double d = sqrt(-log(eps / ae) / (dbar * dbar));
    out[CX] = px;
    out[CY] = py;
    out[CZ] = pz;
    out[D1] = d;
    out[D2] = d;
    out[D3] = d;
    out[TX] = 0.0;
    out[TY] = 0.0;
    out[TZ] = 0.0;
    out[W] = -sgn(e) * ae;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1, greedy largest inscribed spheres over the interior points.
 * Interior: 1 < t < 2 (targets of Eq. 3-10).  d_in = |S|: the exact SDF is
 * the distance to the surface, read as the closest distance to the samples
 * P.  Each round takes the remaining point with the largest d_in (the lowest
 * index among equal values, as an argmax does), appends it (centre, weight
 * t) and keeps only the points whose squared distance to it exceeds r^2,
 * r = its d_in (the printed comparison of a squared distance with r is read
 * as the squared radius).  The distance and r^2 are float with the support
 * predicate's operation order, so another implementation can take the same
 * decisions.  Writes the selected indices in order; returns how many (at
 * most max_out; more are counted but not written).
 * Pinned by: coverage, order and non-overlap properties and a hand example. */
int32_t oracle_inscribed(const float *x, const float *y, const float *z, const float *t, const float *S,
                         int64_t n, int32_t *out, int32_t max_out) {
    uint8_t *alive = (uint8_t *)malloc((size_t)(n ? n : 1));
    int64_t left = 0;
    for (int64_t i = 0; i < n; ++i) {
        alive[i] = (1.0f < t[i]) && (t[i] < 2.0f);
        left += alive[i];
    }
    int32_t cnt = 0;
    while (left > 0) {
        int64_t best = -1;
        float bd = -1.0f;
        for (int64_t i = 0; i < n; ++i)
            if (alive[i] && fabsf(S[i]) > bd) {
                bd = fabsf(S[i]);
                best = i;
            }
        if (cnt < max_out) out[cnt] = (int32_t)best;
        ++cnt;
        const float r2 = bd * bd;
        for (int64_t k = 0; k < n; ++k) {
            if (!alive[k]) continue;
            const float dx = x[k] - x[best], dy = y[k] - y[best], dz = z[k] - z[best];
            const float d2 = support_d2(dx, dy, dz);
            if (!(d2 > r2)) {
                alive[k] = 0;
                --left;
            }
        }
    }
    free(alive);
    return cnt;
}

/* ---------------------------------------------------------------------------
 * Eq. 3-12: isotropic axis parameters from the nearest other centre,
 *     d_j1 = d_j2 = d_j3 = 2 sqrt(-ln(gamma / w_j^2)) / dhat_j,
 * dhat_j = min_i ||c_j - c_i||, i != j (a single centre: dhat = 2 r_j, the
 * diameter of its sphere -- the paper does not cover that case).
 * Pinned by: Eq. 3-11 (w^2 exp(-d^2 (dhat/2)^2) = gamma) and brute force. */
void oracle_init_shape(const double *cx, const double *cy, const double *cz, const double *w, const double *r,
                       int32_t M, double gamma, double *d) {
    for (int32_t j = 0; j < M; ++j) {
        double best = INFINITY;
        for (int32_t i = 0; i < M; ++i) {
            if (i == j) continue;
            const double dx = cx[j] - cx[i], dy = cy[j] - cy[i], dz = cz[j] - cz[i];
            const double dd = sqrt(dx * dx + dy * dy + dz * dz);
            if (dd < best) best = dd;
        }
        if (M == 1) best = 2.0 * r[j];
        d[j] = 2.0 * sqrt(-log(gamma / (w[j] * w[j]))) / best;
    }
}

/* ---------------------------------------------------------------------------
 * Surface extraction and the Sec. 4 surface metrics (the paper extracts the
 * zero level set with marching cubes; this project extracts it with marching
 * tetrahedra, six per grid cube, which needs no case table).
 *
 * Grid: nx*ny*nz values, x fastest; vertex (i, j, k) at o + h (i, j, k).
 * Cube corners are numbered bit0 = x, bit1 = y, bit2 = z; the six
 * tetrahedra of a cube are {0, a, a + b, 7} for the axis orders (a, b) =
 * (1,2) (1,4) (2,1) (2,4) (4,1) (4,2).  Inside means value < iso.  One or
 * three inside vertices give one triangle on the three edges of the lone
 * vertex; two give the quad on the four crossing edges as two triangles.
 * An edge point interpolates linearly from the edge's lower grid index to
 * its higher one, in float with a fixed operation order (so a shared edge
 * gives the same point in every tetrahedron).  Output in cube order, then
 * tetrahedron order. */
static const int MT_TETS[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

static void mt_edge(const float *f, int64_t gu, int64_t gw, int nx, int ny, const float o[3], float h, float iso,
                    float *out) {
    if (gu > gw) {
        int64_t t = gu;
        gu = gw;
        gw = t;
    }
    const float fu = f[gu], fw = f[gw];
    const float t = (iso - fu) / (fw - fu);
    const int64_t iu[3] = {gu % nx, (gu / nx) % ny, gu / ((int64_t)nx * ny)};
    const int64_t iw[3] = {gw % nx, (gw / nx) % ny, gw / ((int64_t)nx * ny)};
    for (int a = 0; a < 3; ++a) {
        const float pu = o[a] + h * (float)iu[a], pw = o[a] + h * (float)iw[a];
        out[a] = pu + t * (pw - pu);
    }
}

/* Writes up to cap triangles (9 floats each); returns the number found. */
int64_t oracle_marching_tets(const float *f, int nx, int ny, int nz, const float o[3], float h, float iso, float *tri,
                             int64_t cap) {
    int64_t cnt = 0;
    for (int k = 0; k + 1 < nz; ++k)
        for (int j = 0; j + 1 < ny; ++j)
            for (int i = 0; i + 1 < nx; ++i) {
                int64_t g[8];
                for (int c = 0; c < 8; ++c)
                    g[c] = ((int64_t)(k + ((c >> 2) & 1)) * ny + (j + ((c >> 1) & 1))) * nx + (i + (c & 1));
                for (int q = 0; q < 6; ++q) {
                    int64_t v[4];
                    int in[4], nin = 0;
                    for (int a = 0; a < 4; ++a) {
                        v[a] = g[MT_TETS[q][a]];
                        in[a] = f[v[a]] < iso;
                        nin += in[a];
                    }
                    if (nin == 0 || nin == 4) continue;
                    float p[4][3];
                    if (nin == 1 || nin == 3) {
                        const int want = nin == 1;
                        int l = 0;
                        while (in[l] != want) ++l;
                        int e = 0;
                        for (int a = 0; a < 4; ++a)
                            if (a != l) mt_edge(f, v[l], v[a], nx, ny, o, h, iso, p[e++]);
                        if (cnt < cap) memcpy(tri + 9 * cnt, p, 9 * sizeof(float));
                        ++cnt;
                    } else {
                        int A = -1, B = -1, Cc = -1, D = -1;
                        for (int a = 0; a < 4; ++a) {
                            if (in[a]) {
                                if (A < 0) A = a; else B = a;
                            } else {
                                if (Cc < 0) Cc = a; else D = a;
                            }
                        }
                        float ac[3], ad[3], bd[3], bc[3];
                        mt_edge(f, v[A], v[Cc], nx, ny, o, h, iso, ac);
                        mt_edge(f, v[A], v[D], nx, ny, o, h, iso, ad);
                        mt_edge(f, v[B], v[D], nx, ny, o, h, iso, bd);
                        mt_edge(f, v[B], v[Cc], nx, ny, o, h, iso, bc);
                        if (cnt < cap) {
                            float *t0 = tri + 9 * cnt;
                            memcpy(t0, ac, 12); memcpy(t0 + 3, ad, 12); memcpy(t0 + 6, bd, 12);
                        }
                        ++cnt;
                        if (cnt < cap) {
                            float *t1 = tri + 9 * cnt;
                            memcpy(t1, ac, 12); memcpy(t1 + 3, bd, 12); memcpy(t1 + 6, bc, 12);
                        }
                        ++cnt;
                    }
                }
            }
    return cnt;
}

/* Triangle area quantised to a 64-bit integer (unit 2^-40): exact prefix
 * sums, so the sampling below picks the same triangle in any order of
 * summation.  Area in float: 0.5 |(b - a) x (c - a)|. */
static uint64_t mt_area_q(const float *t) {
    const float ux = t[3] - t[0], uy = t[4] - t[1], uz = t[5] - t[2];
    const float vx = t[6] - t[0], vy = t[7] - t[1], vz = t[8] - t[2];
    const float cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
    const float a = 0.5f * sqrtf((cx * cx + cy * cy) + cz * cz);
    return (uint64_t)llrint((double)a * 1099511627776.0);
}

/* Area-weighted uniform samples on a triangle soup: sample s picks the
 * triangle whose quantised cumulative area interval holds floor(u[3s] *
 * total), then the point (1 - r) a + r (1 - u[3s+2]) b + r u[3s+2] c with
 * r = sqrt(u[3s+1]), and the unit normal of the triangle.  u: uniform
 * numbers in [0, 1) (drawn by the caller).  Returns 0, or -1 when the soup
 * has no area. */
int oracle_sample_surface(const float *tri, int64_t ntri, const double *u, int64_t ns, float *pts, float *nrm) {
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(ntri + 1));
    cum[0] = 0;
    for (int64_t k = 0; k < ntri; ++k) cum[k + 1] = cum[k] + mt_area_q(tri + 9 * k);
    const uint64_t total = cum[ntri];
    if (total == 0) {
        free(cum);
        return -1;
    }
    for (int64_t s = 0; s < ns; ++s) {
        const uint64_t target = (uint64_t)(u[3 * s] * (double)total);
        int64_t lo = 0, hi = ntri;  /* the k with cum[k] <= target < cum[k+1] */
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            if (cum[mid] <= target) lo = mid; else hi = mid;
        }
        const float *t = tri + 9 * lo;
        const float r = sqrtf((float)u[3 * s + 1]), w = (float)u[3 * s + 2];
        const float ca = 1.0f - r, cb = r * (1.0f - w), cc = r * w;
        for (int a = 0; a < 3; ++a) pts[3 * s + a] = (ca * t[a] + cb * t[3 + a]) + cc * t[6 + a];
        const float ux = t[3] - t[0], uy = t[4] - t[1], uz = t[5] - t[2];
        const float vx = t[6] - t[0], vy = t[7] - t[1], vz = t[8] - t[2];
        const float cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
        const float len = sqrtf((cx * cx + cy * cy) + cz * cz);
        nrm[3 * s] = cx / len;
        nrm[3 * s + 1] = cy / len;
        nrm[3 * s + 2] = cz / len;
    }
    free(cum);
    return 0;
}

/* Sec. 4 metrics between two sampled surfaces A and B (point-to-point):
 * HD = max(max_a d(a, B), max_b d(b, A)); CD = mean_a d(a, B) / 2 +
 * mean_b d(b, A) / 2; CS = the same averages of |n(x) . n(closest(x))|.
 * Nearest point by brute force on float squared distances (ties: lowest
 * index); distances and sums in double.  out = {HD, CD, CS}. */
void oracle_surface_metrics(const float *A, const float *nA, int64_t na, const float *B, const float *nB, int64_t nb,
                            double out[3]) {
    double hd = 0.0, cd = 0.0, cs = 0.0;
    for (int dir = 0; dir < 2; ++dir) {
        const float *P = dir ? B : A, *nP = dir ? nB : nA, *Q = dir ? A : B, *nQ = dir ? nA : nB;
        const int64_t np = dir ? nb : na, nq = dir ? na : nb;
        double dsum = 0.0, csum = 0.0;
        #pragma omp parallel for reduction(+ : dsum, csum) reduction(max : hd)
        for (int64_t i = 0; i < np; ++i) {
            float best = INFINITY;
            int64_t bi = 0;
            for (int64_t j = 0; j < nq; ++j) {
                const float dx = P[3 * i] - Q[3 * j], dy = P[3 * i + 1] - Q[3 * j + 1], dz = P[3 * i + 2] - Q[3 * j + 2];
                const float d2 = (dx * dx + dy * dy) + dz * dz;
                if (d2 < best) {
                    best = d2;
                    bi = j;
                }
            }
            const double d = sqrt((double)best);
            dsum += d;
            if (d > hd) hd = d;
            csum += fabs((double)nP[3 * i] * nQ[3 * bi] + (double)nP[3 * i + 1] * nQ[3 * bi + 1] +
                         (double)nP[3 * i + 2] * nQ[3 * bi + 2]);
        }
        cd += dsum / (2.0 * (double)np);
        cs += csum / (2.0 * (double)np);
    }
    out[0] = hd;
    out[1] = cd;
    out[2] = cs;
}
