/*
 * serbf.h -- C ABI of the GB300 (sm_103a) SE-RBFNet optimisation hot path.
 *
 * The library fits precomputed signed-distance samples with a sparse sum of
 * ellipsoidal radial basis functions, following "Approximating Signed Distance
 * Fields With Sparse Ellipsoidal Radial Basis Function Networks" (SE-RBFNet):
 *
 *   Psi(v_i) = sum_j w_j |w_j| exp(-|| D_j R_j (v_i - c_j) ||^2)      (Eq. 3-26)
 *
 * restricted to the support of each kernel (Eq. 3-15-1), with the loss of
 * Eq. 3-19 over the filtered points of Eq. 3-18, the analytic gradients of
 * App. A, the dynamic weighting of Eq. 3-21 and Adam (Algorithm 3), kernel
 * deletion (Eq. 3-27), adaptive addition (Algorithm 2, Eq. 3-24) and
 * coarse-to-fine refinement (Sec. 3.4.2).
 *
 * Conventions for every entry point
 *   - Pointers named *_dev, and every array argument unless stated otherwise,
 *     are DEVICE pointers owned by the caller.  The library allocates no
 *     memory of its own: scratch lives in a caller-provided device buffer
 *     described by a serbf_workspace (serbf_workspace_bytes/_init).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream unless documented as synchronising.
 *   - Return value: SERBF_OK or a negative SERBF_E* code.  Argument errors are
 *     detected on the host before anything is launched.  Capacity overflows
 *     found on the device set a sticky flag read by serbf_status().
 *   - Parameters: one float array of 10 rows x `cap` columns, row r at p + r*cap,
 *     rows cx, cy, cz, d1, d2, d3, theta_x, theta_y, theta_z, w  (Sec. 3.2;
 *     d_k multiplies the rotated offset, i.e. it is an inverse axis length).
 *     The live count m is a DEVICE int32 so that deletion and addition can run
 *     without a host round trip.
 *   - Points: after serbf_bin_points every per-point array is in BINNED order
 *     (sorted by cell, then original index); perm[k] is the original index of
 *     binned point k.  Neighbour lists index binned points.
 *   - Rotation: R is the matrix whose entries r1..r9 are listed in App. A.
 */
#ifndef SERBF_H
#define SERBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SERBF_OK 0
#define SERBF_EINVAL -1    /* NULL pointer, bad size or bad configuration */
#define SERBF_ENOMEM -2    /* workspace buffer too small */
#define SERBF_ECAPACITY -3 /* a list or array capacity is too small (see serbf_status) */
#define SERBF_ECUDA -4     /* a CUDA launch or copy failed */
#define SERBF_ETIMEOUT -5  /* a bounded device wait gave up */

#define SERBF_NPARAM 10

/* device status flags (bitmask) reported by serbf_status */
#define SERBF_FLAG_SUPER_LIST 1   /* a super-cell candidate list exceeded super_cap */
#define SERBF_FLAG_ADD_CAPACITY 4 /* addition truncated at the parameter capacity */
#define SERBF_FLAG_FIX_RANGE 8    /* serbf_forward_backward: a moment may lie outside the range of its
                                     64-bit fixed-point accumulator (|moment| >= 2^26 bound); the
                                     gradients of that call are not reliable */

/* indices into the double stats[SERBF_NSTATS] device array */
#define SERBF_STAT_L2 0        /* sum over id_all of E_i^2                 (Eq. 3-19) */
#define SERBF_STAT_L1 1        /* sum_j |w_j| before the update            (Eq. 3-14_2) */
#define SERBF_STAT_MAXE 2      /* max over id_all of |E_i|                 (Eq. l1_activate2) */
#define SERBF_STAT_COUNT 3     /* |id_all|                                 (Eq. 3-18) */
#define SERBF_STAT_PAIRS_FWD 4 /* point-kernel pairs evaluated by the forward */
#define SERBF_STAT_PAIRS_BWD 5 /* point-kernel pairs evaluated by the adjoint */
#define SERBF_STAT_ALPHA 6     /* alpha of the last step                   (Eq. 3-21) */
#define SERBF_STAT_BETA 7      /* beta = 1 - alpha */
#define SERBF_STAT_BF 8        /* b_f = #{|w_j| >= tau_d} after the step   (Sec. 3.4.3) */
#define SERBF_STAT_LOSS 9      /* alpha L2 + beta L1 */
#define SERBF_NSTATS 16

/* Hyper-parameters.  serbf_config_default fills the values of the Algorithm 3
 * input line and Sec. 4.1; the Adam moments are the Kingma-Ba defaults. */
typedef struct {
    double eps;        /* epsilon of the support radius, Eq. 3-15 (1e-7) */
    double tau1, tau2; /* point filter, Eq. 3-18 (0.9, 1.1) */
    double tau_m;      /* max-error gate, Eq. l1_activate2 (0.02) */
    double tau_d;      /* deletion threshold, Eq. 3-27 (0.01) */
    double tau_l1;     /* basis-count stability, Eq. add_activate (5) */
    double tau_l2;     /* L2 stability, Eq. l1_activate (0.5) */
    double lr;         /* Adam learning rate of the first phase (0.01) */
    double lr_p2;      /* learning rate at T^e (1e-3), cosine-annealed ... */
    double lr_min;     /* ... to lr_min at M^e (1e-5) */
    double beta1, beta2, adam_eps; /* Adam (0.9, 0.999, 1e-8) */
    double topk_frac;  /* addition keeps the top fraction of id_all by |E| (0.01); <= 0: no limit */
    double add_radius; /* Algorithm 2 local-maximum radius r (world units) */
    double dbar_min;   /* lower clamp of dbar in Eq. 3-24 (world units) */
    int32_t k_l1, k_l2; /* window lengths (50, 10) */
    int32_t T_e, M_e;  /* phase switch and last epoch (1600, 2000) */
    int32_t kahan;     /* 1: compensated per-kernel sums in the adjoint */
    int32_t fwd_warps; /* warps sharing one forward work item: 1, 2, 4 or 8;
                          0 = chosen from the problem size (default) */
    int32_t epoch_steps; /* optimiser steps per epoch: 1 = full batch (default);
                            n > 1: mini-batches, the epoch tail runs every n-th step
                            on the sum of the n batch L2 values */
    int32_t rebuild_levels; /* how serbf_build_neighbors forms the candidate list of each super
                               cell: 1 = tests every kernel; 2 = lists the kernels of each block of
                               2 x 2 x 2 super cells first and filters that list (the same lists,
                               less work when there are many super cells and kernels); 3 = lists
                               blocks of 4 x 4 x 4 super cells first, filters them into the blocks
                               of 2 x 2 x 2 and those into the super cells (the same lists again;
                               the batched epoch takes 2 for 3); 0 = chosen from the problem size
                               (default) */
} serbf_config;

/* Optimiser state of Algorithm 3; lives in DEVICE memory (sizeof bytes). */
typedef struct {
    int32_t epoch;    /* completed epochs e_p */
    int32_t l1_optim; /* Algorithm 3 flag */
    int32_t phase2;   /* e_p reached T^e */
    int32_t adam_t;   /* Adam step counter (reset to 0 when kernels are added) */
    int32_t do_prune; /* Eq. 3-27 due (consumed by serbf_prune) */
    int32_t do_add;   /* Eq. 3-24 due (consumed by serbf_add_kernels) */
    int32_t n_l2, n_bf;
    int32_t m_added, m_pruned;
    int32_t step;     /* steps done in the current epoch (mini-batches) */
    int32_t reserved;
    double lr;        /* learning rate of the next epoch */
    double alpha, beta;
    double l2_epoch;  /* sum of the batch L2 values of the current epoch */
    double l2_hist[64];  /* L2 of epoch e at index (e - 1) mod k_l2 */
    int32_t bf_hist[256]; /* b_f of epoch e at index (e - 1) mod k_l1 */
} serbf_state;

typedef struct {
    const float *x, *y, *z; /* binned coordinates */
    const float *t;         /* normalised targets, Eq. 3-10 (binned) */
    int64_t n;
} serbf_points;

typedef struct {
    float *p;     /* 10 x cap */
    int32_t *m;   /* device: live kernel count */
    int32_t cap;
} serbf_params;

typedef struct {
    int64_t *rowptr; /* rows + 1 entries */
    uint32_t *col;   /* capacity `cap` entries */
    int64_t cap;
} serbf_csr;

typedef struct {
    float origin[3]; /* lower corner of cell (0, 0, 0) */
    float h;         /* cell edge length */
    int32_t n[3];    /* cells per axis */
} serbf_grid;

typedef struct {
    int64_t max_points;   /* training-set capacity */
    int32_t max_kernels;  /* parameter capacity (== serbf_params.cap) */
    int32_t max_cells;    /* >= n[0]*n[1]*n[2] of every grid used */
    int32_t reserved0;    /* must be 0 */
    int32_t super_cap;    /* candidate kernels per super-cell list */
    int32_t super_factor; /* cells per super-cell edge (1..16) */
    int32_t reserved;
} serbf_ws_sizes;

typedef struct serbf_workspace serbf_workspace; /* opaque, host memory of serbf_workspace_struct_size() bytes */

/* ------------------------------------------------------------------ setup */
const char *serbf_version(void);
const char *serbf_status_string(int code);

/* Fills *cfg with the defaults listed above (add_radius and dbar_min 0: the
 * caller sets them from its grid spacing).  Returns SERBF_EINVAL for NULL. */
int serbf_config_default(serbf_config *cfg);

/* Host bytes the caller must provide for one serbf_workspace object. */
size_t serbf_workspace_struct_size(void);

/* Device bytes needed for the given capacities; EINVAL on non-positive sizes. */
int serbf_workspace_bytes(const serbf_ws_sizes *sz, size_t *bytes);

/* Carves the caller's device buffer `dev` (>= serbf_workspace_bytes, 256-byte
 * aligned) into the scratch arrays.  ws points to serbf_workspace_struct_size()
 * bytes of caller-owned host memory.  Synchronous (clears the status word).
 * ENOMEM if `bytes` is too small, EINVAL on bad sizes or alignment. */
int serbf_workspace_init(serbf_workspace *ws, void *dev, size_t bytes, const serbf_ws_sizes *sz);

/* Releases the workspace's host-side CUDA objects (a side stream and two
 * events created by serbf_workspace_init; some calls fork work onto that
 * stream and join it before they return).  The device buffer stays the
 * caller's.  Call it once when the workspace is no longer used, after the
 * work queued with it has been synchronised; the workspace is invalid
 * afterwards (calls return EINVAL).  EINVAL on an uninitialised workspace. */
int serbf_workspace_release(serbf_workspace *ws);

/* Reads and optionally clears the device status flags (synchronises `stream`).
 * needed[0] = largest super-cell list, needed[3] = kernel count an addition
 * asked for, both since the last clear.  Returns SERBF_ECAPACITY when a flag is
 * set, SERBF_OK otherwise. */
int serbf_status(serbf_workspace *ws, int32_t *flags, int64_t needed[4], int clear, void *stream);

/* Writes the initial Algorithm 3 state (epoch 0, l1_optim false, lr = cfg->lr). */
int serbf_state_init(serbf_state *st_dev, const serbf_config *cfg, void *stream);

/* ------------------------------------------------------------------ a1 */
/* Eq. 3-10 (Sec. 3.3): t_i = 2 exp(-h (S_i - m)^2), m = min_i S_i,
 * h = ln 2 / m^2.  Evaluated as 2^(1 - u^2), u = (S_i - m) / m, in float-float
 * arithmetic (no FP64 in the per-sample work): each t_i is the float nearest
 * the exact value, or, where that value lies within about 2^-40 (2^-45 for
 * t_i > 1e-3) of a rounding boundary, its neighbour; targets below the
 * smallest float are 0.  mh_dev[0] = m, mh_dev[1] = h (double).  Requires
 * m != 0 (not detectable on the host; a zero minimum yields NaN at the
 * minimum and 0 elsewhere). */
int serbf_normalize_sdf(const float *S, float *t, int64_t n, double *mh_dev, serbf_workspace *ws,
                        void *stream);

/* Allocation-free form of serbf_normalize_sdf.  The paper has no counterpart.
 * Some callers cannot allocate device memory when they need the target map:
 * an application that hands out device memory only from a pool it set up at
 * start-up, or a loop with a fixed memory budget that must not allocate once
 * it runs.  This entry point takes no workspace: its reduction scratch is a
 * fixed array inside the library (16384 partial minima, 64 KiB on every
 * device that loads the library, held until the process exits), so n is
 * limited to 67,108,864 points; a larger n returns SERBF_ECAPACITY before
 * anything is launched.  mh_dev (2 doubles) is required.  The first call on
 * each device looks up the array's device address and the device's SM count
 * on the host (set-up; make that first call before any stream capture).
 * Targets and m, h are bit-identical to serbf_normalize_sdf.  Every call
 * shares the one array and overwrites it (nothing in it needs clearing), so
 * calls that can overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller. */
int serbf_normalize_sdf_noalloc(const float *S, float *t, int64_t n, double *mh_dev, void *stream);

/* ------------------------------------------------------------------ a2 */
/* Cell binning of the training points (the neighbour structure that serves
 * the support test of Eq. 3-15; the paper leaves its data structure open).
 * Cell index per axis k = clamp(floor(fl(fl(x - origin) / h)), 0, n - 1);
 * cells are grouped into super cells of sf^3 (sf = super_factor) and the key
 * is super-major: ((sk_z * ns_y + sk_y) * ns_x + sk_x) * sf^3 +
 * (l_z * sf + l_y) * sf + l_x with sk = k / sf, l = k % sf, ns = ceil(n / sf).
 * Points are radix-sorted by (key, index).  Writes perm (binned -> original
 * index) and the binned coordinates, and records cell ranges, 32-point tiles
 * (never straddling a super cell) and tile / super-cell bounding boxes in the
 * workspace.  SYNCHRONISES the stream once (reads the tile count).
 * EINVAL: n > max_points, grid cells > max_cells, non-positive h. */
int serbf_bin_points(const float *x, const float *y, const float *z, int64_t n, const serbf_grid *grid,
                     uint32_t *perm, float *xb, float *yb, float *zb, serbf_workspace *ws, void *stream);

/* dst[k] = src[perm[k]] for k < n (puts targets, SDF values, ... into binned order). */
int serbf_gather(const float *src, const uint32_t *perm, float *dst, int64_t n, void *stream);

/* ------------------------------------------------------------------ a3 */
/* Per-step rebuild of the kernel <-> point neighbour structure, Eq. 3-15-1:
 * point v_i is in the support of kernel j iff, in float with no fused
 * multiply-add, fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)) < r2_j where
 * dx = fl(x_i - cx_j), ..., r2_j = fl(fl(-ln eps) / min_k fl(d_jk * d_jk)).
 * Always rebuilds the workspace's cell -> candidate-kernel lists used by
 * serbf_forward / serbf_backward (asynchronous).  If kmajor and/or pmajor is
 * non-NULL it also writes the explicit CSR lists: kernel-major rows (m + 1
 * rowptr entries) list binned point indices in ascending order; point-major
 * rows (n + 1 entries) list kernel indices in ascending order.  Producing CSR
 * lists SYNCHRONISES the stream; when a col capacity is too small the call
 * returns SERBF_ECAPACITY with the pair count in *npairs (rowptr is valid).
 * npairs (host, may be NULL) receives the number of pairs when CSR lists were
 * requested. */
int serbf_build_neighbors(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                          serbf_csr *kmajor, serbf_csr *pmajor, int64_t *npairs, serbf_workspace *ws,
                          void *stream);

/* ------------------------------------------------------------------ initialisation */
/* Algorithm 1 and Eq. 3-12: initial kernels from the interior training points
 * (1 < t < 2).  Greedy largest inscribed spheres: repeatedly the interior point
 * with the largest |S_raw| (the exact SDF value, i.e. the distance to the
 * surface; the first in binned order among equal values) becomes a centre with
 * weight t, and every interior point whose squared distance to it is not above
 * fl(|S|^2) is removed (float distances in the support predicate's operation
 * order).  Then d_1 = d_2 = d_3 = 2 sqrt(-ln(gamma / w^2)) / dhat with dhat the
 * distance to the nearest other centre (one centre alone: twice its |S|),
 * angles 0.  Writes the first min(M, cap) kernels in selection order and sets
 * the device count; *m_out (host, may be NULL) receives M.  Uses the binning
 * of pts (serbf_bin_points) and its scratch.  SYNCHRONISES the stream.
 * ECAPACITY when M > cap (the first cap kernels are written), EINVAL on bad
 * arguments or gamma outside (0, 1). */
int serbf_init_kernels(const serbf_points *pts, const float *S_raw, double gamma, serbf_params *prm, int32_t *m_out,
                       serbf_workspace *ws, void *stream);

/* ------------------------------------------------------------------ evaluation (Sec. 4) */
/* Zero level set of a grid field f (dims[0] x dims[1] x dims[2] values, x
 * fastest; vertex (i, j, k) at origin + h (i, j, k)) as a triangle soup: each
 * grid cube is split into six tetrahedra {0, a, a + b, 7} (corner bits x = 1,
 * y = 2, z = 4; (a, b) = (1,2) (1,4) (2,1) (2,4) (4,1) (4,2)), inside means
 * f < iso, one or three inside vertices give one triangle, two give two; edge
 * points interpolate linearly from the edge's lower grid index in float with
 * a fixed operation order.  Marching tetrahedra stand in for the paper's
 * marching cubes.  tri: cap x 9 floats (device, caller-owned); *ntri (host)
 * receives the count; scratch: (cubes + 1) int64 (device).  Triangles are in
 * cube order.  SYNCHRONISES; ECAPACITY (with *ntri set) when cap is too small. */
int serbf_marching_tets(const float *f, const int32_t dims[3], const float origin[3], float h, float iso, float *tri,
                        int64_t cap, int64_t *ntri, int64_t *scratch, void *stream);

/* Area-weighted samples on a triangle soup (Sec. 4 samples 1e5 points per
 * surface): sample s takes the triangle whose cumulative area interval holds
 * floor(u[3s] * total) (areas quantised to 2^-40 so the sums are exact), then
 * the point (1 - r) a + r (1 - u[3s+2]) b + r u[3s+2] c, r = sqrt(u[3s+1]), and
 * the triangle's unit normal.  u: ns x 3 uniform numbers in [0, 1) (device,
 * drawn by the caller); pts, nrm: ns x 3 floats; scratch: ntri + 1 int64.
 * SYNCHRONISES; EINVAL when the soup has no area. */
int serbf_sample_surface(const float *tri, int64_t ntri, const double *u, int64_t ns, float *pts, float *nrm,
                         int64_t *scratch, void *stream);

/* Sec. 4 metrics between two sampled surfaces (point-to-point, nearest
 * point by brute force, ties to the lowest index): out (host) = {HD, CD, CS}
 * with HD = max(max_a d(a, B), max_b d(b, A)), CD = mean_a d(a, B) / 2 +
 * mean_b d(b, A) / 2, CS = the same means of |n . n_nearest|.  scratch:
 * 2 (na + nb) + 6 doubles (device).  SYNCHRONISES. */
int serbf_surface_metrics(const float *A, const float *nA, int64_t na, const float *B, const float *nB, int64_t nb,
                          double out[3], double *scratch, void *stream);

/* Inverse of Eq. 3-10 on the branch S >= m: S = m + sqrt(-ln(t / 2) / h), with
 * (m, h) as written by serbf_normalize_sdf; t >= 2 gives m, t <= 0 gives +inf. */
int serbf_denormalize_sdf(const float *t, float *S, int64_t n, const double *mh_dev, void *stream);

/* dst[idx[i]] = src[i] (e.g. binned results back to grid order with perm). */
int serbf_scatter(const float *src, const uint32_t *idx, float *dst, int64_t n, void *stream);

/* ------------------------------------------------------------------ a4 */
/* Eq. 3-26 forward over the pairs of Eq. 3-15-1, Eq. 3-18 filter and the
 * Eq. 3-19 loss terms: psi[i], mask[i] (1 = in id_all), err[i] = psi - t on
 * id_all and 0 elsewhere; stats[L2], stats[MAXE], stats[COUNT] and
 * stats[PAIRS_FWD] (device doubles, deterministic).  Pair arithmetic in
 * float; the loss sums are float-float (about 48 bits), reduced in tile
 * order after the pair kernel.  Two launches.  Uses the lists of the last
 * serbf_build_neighbors call for these parameters. */
int serbf_forward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi,
                  float *err, uint8_t *mask, double *stats, serbf_workspace *ws, void *stream);

/* ------------------------------------------------------------------ a5 */
/* App. A gradients of sum_i err_i^2 (i.e. of L2 when err is the forward's E)
 * with respect to all ten parameters of every live kernel, summed over the
 * pairs of Eq. 3-15-1 with err_i != 0; grad is 10 x cap (same rows as p).
 * Basis values are recomputed, never stored.  stats[PAIRS_BWD] receives the
 * number of pairs.  For an arbitrary upstream gradient g of Psi pass
 * err = g / 2.  Uses the lists of the last serbf_build_neighbors call. */
int serbf_backward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                   const float *err, float *grad, double *stats, serbf_workspace *ws, void *stream);

/* Forward and adjoint in one pass (Eq. 3-26, 3-18, 3-19, App. A): the
 * outputs of serbf_forward, and the gradients of L2 = sum_i E_i^2 of
 * serbf_backward with err = the forward's own E (grad is 10 x cap, rows of
 * kernels >= m untouched; stats[PAIRS_BWD] as there).  Each work item's
 * points with E != 0 are taken against its candidate kernels right after
 * its residuals are known; the per-item moments (world frame, float sums;
 * compensated when cfg->kahan is set) are accumulated across items in 64-bit
 * fixed point (unit 2^-36, integer atomics), so the result is deterministic
 * and order-independent, each item's partial rounded to 2^-36; it equals
 * serbf_backward's up to float rounding.  The fixed-point range is
 * |moment| < 2^27: a partial beyond 2^26, or a bound of max|E| x (points
 * within a kernel's support radius) x max(1, min(r^2, far^2)) reaching 2^26
 * (far = distance from the centre to the farthest corner of the points' box), sets
 * SERBF_FLAG_FIX_RANGE (read with serbf_status; the call itself does not
 * wait for the device).  Two launches.  EINVAL as serbf_forward, or when
 * grad is NULL. */
int serbf_forward_backward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi,
                           float *err, uint8_t *mask, float *grad, double *stats, serbf_workspace *ws,
                           void *stream);

/* ------------------------------------------------------------------ a6 */
/* One Algorithm 3 parameter update for the full batch: if l1_optim and
 * stats[MAXE] < tau_m, alpha from Eq. 3-21 on the weight gradients (double),
 * else alpha = 1; beta = 1 - alpha; gradient of Eq. grad (App. A); Adam; then
 * the epoch tail of Algorithm 3 (deletion due, Eq. l1_activate, Eq.
 * add_activate, switch to the L2-only phase with a cosine learning rate at
 * T^e).  grad holds the raw L2 gradients from serbf_backward and is not
 * modified.  adam_m / adam_v are 10 x cap.  Writes stats[L1, ALPHA, BETA, BF,
 * LOSS].  Two launches; ws holds the reduction scratch. */
int serbf_step(serbf_params *prm, const float *grad, float *adam_m, float *adam_v, serbf_state *st_dev,
               double *stats, const serbf_config *cfg, serbf_workspace *ws, void *stream);

/* ------------------------------------------------------------------ a7 */
/* Eq. 3-27: when st->do_prune is set, removes every kernel with |w| < tau_d
 * (stable order), compacting the parameters and the Adam moments and updating
 * the device count; clears do_prune.  A no-op launch otherwise. */
int serbf_prune(serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev,
                const serbf_config *cfg, void *stream);

/* ------------------------------------------------------------------ a8 */
/* Algorithm 2 in its top-k form and Eq. 3-24: when st->do_add is set (or
 * force != 0): candidates are id_all points with |E| > tau_m / 2; the
 * ceil(topk_frac * |id_all|) largest |E| are kept (ties by ascending binned
 * index); a candidate survives if no id_all point within add_radius has a
 * larger |E|; survivors become kernels c = v, w = -E, d = sqrt(ln(|E|/eps)) /
 * dbar on all axes (dbar = max(|S_raw|, dbar_min)), theta = 0, appended in
 * selection order.  Adam moments are reset (reading: new kernels start from
 * zero moments, t = 0).  Sets st->m_added and clears do_add.
 * S_raw: raw signed distances in binned order. */
int serbf_add_kernels(const serbf_points *pts, const float *S_raw, const float *err, const uint8_t *mask,
                      serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev,
                      const double *stats, const serbf_config *cfg, int force, serbf_workspace *ws,
                      void *stream);

/* ------------------------------------------------------------------ a9 */
/* Sec. 3.4.2 coarse-to-fine step: appends the next grid layer (x_new.., t_new,
 * s_new, n_new points) to the original-order training set (x_all.., t_all,
 * s_all holding n_old points and capacity for n_old + n_new; may alias the
 * old arrays), then re-bins the union into perm / xb, yb, zb and gathers t and
 * S into tb / sb.  Parameters are untouched (training continues from them).
 * SYNCHRONISES the stream (through serbf_bin_points). */
int serbf_refine(float *x_all, float *y_all, float *z_all, float *t_all, float *s_all, int64_t n_old,
                 const float *x_new, const float *y_new, const float *z_new, const float *t_new,
                 const float *s_new, int64_t n_new, const serbf_grid *grid, uint32_t *perm, float *xb,
                 float *yb, float *zb, float *tb, float *sb, serbf_workspace *ws, void *stream);

/* ------------------------------------------------------------------ batches of fields */
/* One field of a batch: the arguments of its single-field epoch calls
 * (serbf_build_neighbors, serbf_forward_backward, serbf_step, serbf_prune,
 * serbf_add_kernels), all device buffers owned by the caller, and its binned
 * workspace (serbf_bin_points done).  cfg->fwd_warps is ignored (the batch
 * uses one split for every field); cfg->kahan must be the same for all. */
typedef struct {
    serbf_points pts;
    const float *S_raw;          /* raw signed distances, binned order */
    float *psi, *err;            /* n */
    uint8_t *mask;               /* n */
    serbf_params prm;
    float *grad, *adam_m, *adam_v; /* 10 x cap */
    serbf_state *st;
    double *stats;
    const serbf_config *cfg;
    serbf_workspace *ws;
} serbf_field;

typedef struct serbf_batch serbf_batch; /* opaque, host memory of serbf_batch_struct_size() bytes */

size_t serbf_batch_struct_size(void);

/* Device bytes of the batch tables for nfields (1..1024) fields. */
int serbf_batch_bytes(int32_t nfields, size_t *bytes);

/* Records every field's arguments in the caller's device buffer `dev`
 * (>= serbf_batch_bytes, 256-byte aligned) and sizes the batch's grids.
 * fwd_warps: warps per forward work item for all fields (1, 2, 4, 8; 0 =
 * chosen from the total item count).  Re-initialise after any field is
 * re-binned (refinement).  SYNCHRONISES the stream.  EINVAL on bad fields
 * (not binned, mismatched kahan, NULL buffers), ENOMEM when bytes is too
 * small, ECAPACITY beyond 2^32 work items. */
int serbf_batch_init(serbf_batch *b, const serbf_field *fields, int32_t nfields, int32_t fwd_warps, void *dev,
                     size_t bytes, void *stream);

/* The warps per forward work item the batch uses. */
int serbf_batch_warps(const serbf_batch *b);

/* One Algorithm 3 epoch of every field (full batch): neighbour rebuild
 * (Eq. 3-15-1), fused forward + adjoint (Eq. 3-26, 3-18, 3-19, App. A) as
 * ONE persistent launch over the work items of all fields, the finishing
 * reductions, the Eq. 3-21 / Adam step with the Algorithm 3 gates, Eq. 3-27
 * deletion and Algorithm 2 addition -- twelve launches or fewer whatever
 * the number of fields, asynchronous, capturable into a CUDA graph.  Each
 * field's results are bit-identical to its single-field epoch with the same
 * warps per item (no floating-point atomics; every reduction has a fixed
 * order).  Status flags go to each field's workspace. */
int serbf_epoch_batched(serbf_batch *b, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SERBF_H */
