// Algorithm 3 update for one full-batch epoch: Eq. 3-21 dynamic weighting,
// Adam, and the epoch-tail gates (Eq. 3-27 deletion due, Eq. l1_activate,
// Eq. add_activate, L2-only phase with a cosine learning rate from T^e).  The
// state machine lives on the device so that a step needs no host round trip.
// Two grid-wide launches whose last blocks finish the reductions.  Also the
// Eq. 3-27 compaction.
#include <math.h>
#include <string.h>

#include "common.cuh"

using namespace serbf;

namespace {

constexpr int kStepThreads = 256;

// Block sums of NV float values with float-float trees (FP64 is slow here).
template <int NV>
__device__ void block_sums_ff(const float (&v)[NV], ff (*sh)[NV], ff (&out)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const ff s = warp_sum_ff(ff{v[k], 0.f});
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            ff t = lane < nw ? sh[lane][k] : ff{0.f, 0.f};
            t = warp_sum_ff(t);
            if (lane == 0) sh[32][k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = sh[32][k];
    __syncthreads();
}

// Block sums of three doubles, in a fixed order.
__device__ void block_sums_d3(const double (&v)[3], double (*sh)[3], double (&out)[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double t = lane < nw ? sh[lane][k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) sh[32][k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k] = sh[32][k];
    __syncthreads();
}

__device__ __forceinline__ float sgnf(float v) { return (float)((v > 0.f) - (v < 0.f)); }

struct StepArgs {
    float *__restrict__ p;
    const int32_t *m;
    int cap;
    const float *__restrict__ grad;
    float *__restrict__ am, *__restrict__ av;
    serbf_state *st;
    double *stats;
    serbf_config c;
    float *part;      // per block partial sums
    double *scal;     // alpha, beta, bias corrections for the update kernel
    uint32_t *counter;
};

constexpr int kStateWords = (int)(sizeof(serbf_state) / 4);
static_assert(sizeof(serbf_state) % 8 == 0, "state is copied as 32-bit words");

// ---------------------------------------------------------------- pieces
// The three sums of Eq. 3-21 and Eq. 3-14_2 for kernel j, in double: |w|,
// and with the L1 term on, (g1 - g2) g1 and |g2 - g1|^2 on the weight
// gradients (one term per kernel, so FP64 costs nothing here).
__device__ __forceinline__ void alpha_terms(const StepArgs &a, int j, bool use_l1, double (&part)[3]) {
    const double w = a.p[PW * a.cap + j], g2 = a.grad[PW * a.cap + j];
    part[0] += fabs(w);
    if (use_l1) {
        const double g1 = (double)((w > 0.0) - (w < 0.0));
        part[1] += (g1 - g2) * g1;
        part[2] += (g2 - g1) * (g2 - g1);
    }
}

// alpha of Eq. 3-21 in double (clamped to [0, 1]; 1 when the L1 term is off
// or the two gradients coincide), beta = 1 - alpha, the Adam bias
// corrections; writes the stats.  sc = {alpha, beta, 1 - beta1^t, 1 - beta2^t}.
__device__ __forceinline__ void alpha_finish(const StepArgs &a, bool use_l1, const double (&fin)[3], double (&sc)[4]) {
    const double num = fin[1], den = fin[2];
    double al = 1.0;
    if (use_l1 && den > 0.0) al = fmin(1.0, fmax(0.0, num / den));
    // the Adam bias corrections feed a float update: float powers (a double
    // pow costs microseconds on this part's FP64 unit)
    const float t = (float)(a.st->adam_t + 1);
    sc[0] = al;
    sc[1] = 1.0 - al;
    sc[2] = 1.0f - powf((float)a.c.beta1, t);
    sc[3] = 1.0f - powf((float)a.c.beta2, t);
    a.stats[SERBF_STAT_L1] = fin[0];
    a.stats[SERBF_STAT_ALPHA] = al;
    a.stats[SERBF_STAT_BETA] = 1.0 - al;
}

// tau_d rounded up to float: |w| >= taud decides as in double.
__device__ __forceinline__ float tau_d_float(double tau_d) {
    float t = (float)tau_d;
    if ((double)t < tau_d) t = nextafterf(t, INFINITY);
    return t;
}

// Combined gradient of Eq. grad (App. A) and the Adam update of parameter
// (r, j); returns 1 when it is a weight that stays at or above tau_d (b_f).
__device__ __forceinline__ float adam_param(const StepArgs &a, int r, int j, const float (&sc)[4], float lr,
                                            float taud) {
    const float b1 = (float)a.c.beta1, b2 = (float)a.c.beta2, eps = (float)a.c.adam_eps;
    const int64_t q = (int64_t)r * a.cap + j;
    const float pv = a.p[q];
    float g = sc[0] * a.grad[q];
    if (r == PW) g = fmaf(sc[1], sgnf(pv), g);
    const float mo = fmaf(b1, a.am[q], (1.f - b1) * g);
    const float vo = fmaf(b2, a.av[q], (1.f - b2) * g * g);
    const float pn = pv - lr * (mo / sc[2]) / (sqrtf(vo / sc[3]) + eps);
    a.am[q] = mo;
    a.av[q] = vo;
    a.p[q] = pn;
    return (r == PW && fabsf(pn) >= taud) ? 1.f : 0.f;
}

// The epoch tail of Algorithm 3 on a shared-memory copy of the state, run by
// one warp after the epoch's last step (mini-batches: every epoch_steps-th
// step, on the sum of the batch L2 values): histories, deletion due (every k^l2 epochs while l1_optim and
// e < T^e), Eq. l1_activate (population std of the last k^l2 L2 values <
// tau^l2), Eq. add_activate (range of the last k^l1 values of b_f < tau^l1),
// the L2-only phase with a cosine learning rate from T^e.
__device__ void epoch_tail(const StepArgs &a, serbf_state &st, double bf, double alpha, double beta, int lane) {
    // per step: Adam counter, alpha/beta, the epoch's L2 sum; the gates only
    // after the epoch's last step (every step when epoch_steps <= 1)
    const int steps = a.c.epoch_steps > 1 ? a.c.epoch_steps : 1;
    const double l2_step = a.stats[SERBF_STAT_L2];
    const double l2 = st.l2_epoch + l2_step;
    __syncwarp();
    if (st.step + 1 < steps) {
        if (lane == 0) {
            st.l2_epoch = l2;
            st.step = st.step + 1;
            st.alpha = alpha;
            st.beta = beta;
            st.adam_t = st.adam_t + 1;
            a.stats[SERBF_STAT_BF] = bf;
            a.stats[SERBF_STAT_LOSS] = alpha * l2_step + beta * a.stats[SERBF_STAT_L1];
        }
        return;
    }
    const int e = st.epoch + 1;
    const int kl2 = a.c.k_l2, kl1 = a.c.k_l1;
    int l1n = st.l1_optim;
    const int phase2 = st.phase2;
    if (lane == 0) {
        st.l2_hist[(e - 1) % kl2] = l2;
        st.bf_hist[(e - 1) % kl1] = (int32_t)bf;
        st.n_l2 = min(st.n_l2 + 1, kl2);
        st.n_bf = min(st.n_bf + 1, kl1);
    }
    __syncwarp();
    const int n_l2 = st.n_l2, n_bf = st.n_bf;
    const int do_prune = (e % kl2 == 0) && l1n && (e < a.c.T_e);
    if (!l1n && !phase2 && e >= kl2 && n_l2 == kl2) {
        // population std of the last k_l2 values, in double (the convergence
        // test of Eq. l1_activate; at most 64 values)
        double v = 0.0;
        for (int k = lane; k < kl2; k += 32) v += st.l2_hist[k];
        const double mean = warp_sum(v) / (double)kl2;
        double var = 0.0;
        for (int k = lane; k < kl2; k += 32) {
            const double d = st.l2_hist[k] - mean;
            var += d * d;
        }
        var = warp_sum(var) / (double)kl2;
        if (sqrt(var) < a.c.tau_l2) l1n = 1;
    }
    int do_add = 0;
    if (l1n && !phase2 && n_bf == kl1) {
        int lo = 0x7fffffff, hi = -0x7fffffff;
        for (int k = lane; k < kl1; k += 32) {
            lo = min(lo, st.bf_hist[k]);
            hi = max(hi, st.bf_hist[k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((float)(hi - lo) < (float)a.c.tau_l1) {
            do_add = 1;
            l1n = 0;
        }
    }
    if (lane == 0) {
        int ph = phase2;
        if (e == a.c.T_e) {
            ph = 1;
            l1n = 0;
        }
        float lr_next = (float)a.c.lr;
        if (ph) {
            const float span = (float)(a.c.M_e - a.c.T_e);
            float pr = span > 0.f ? (float)(e - a.c.T_e) / span : 1.f;
            if (pr > 1.f) pr = 1.f;
            lr_next = (float)a.c.lr_min + (float)(a.c.lr_p2 - a.c.lr_min) * 0.5f * (1.f + cospif(pr));
        }
        st.alpha = alpha;
        st.beta = beta;
        st.adam_t = st.adam_t + 1;
        st.step = 0;
        st.l2_epoch = 0.0;
        st.do_prune = do_prune;
        st.do_add = do_add;
        st.l1_optim = l1n;
        st.phase2 = ph;
        st.lr = lr_next;
        st.epoch = e;
        a.stats[SERBF_STAT_BF] = bf;
        a.stats[SERBF_STAT_LOSS] = alpha * l2_step + beta * a.stats[SERBF_STAT_L1];
    }
}

// The epoch tail (warp 0) on a shared-memory copy of the state, written back.
__device__ void finish_step(const StepArgs &a, double bf, double alpha, double beta, uint32_t *s_words) {
    const uint32_t *gw = reinterpret_cast<const uint32_t *>(a.st);
    for (int k = threadIdx.x; k < kStateWords; k += blockDim.x) s_words[k] = gw[k];
    __syncthreads();
    serbf_state &st = *reinterpret_cast<serbf_state *>(s_words);
    if (threadIdx.x < 32) epoch_tail(a, st, bf, alpha, beta, threadIdx.x);
    __syncthreads();
    uint32_t *gwo = reinterpret_cast<uint32_t *>(a.st);
    for (int k = threadIdx.x; k < kStateWords; k += blockDim.x) gwo[k] = s_words[k];
}

// ---------------------------------------------------------------- grid path
// Stage 1 (one thread per kernel, many blocks): the sums of alpha_terms; the
// last block turns them into alpha, beta and the Adam bias corrections.
// Block bx of nbx.
__device__ __forceinline__ void step_alpha_body(const StepArgs &a, int bx, int nbx) {
    __shared__ double sh3[33][3];
    __shared__ bool s_last;
    const int m = *a.m;
    const bool use_l1 = a.st->l1_optim && (a.stats[SERBF_STAT_MAXE] < a.c.tau_m);
    double part[3] = {0.0, 0.0, 0.0};
    const int j = bx * blockDim.x + threadIdx.x;
    if (j < m) alpha_terms(a, j, use_l1, part);
    double tot[3];
    block_sums_d3(part, sh3, tot);
    double *bp = reinterpret_cast<double *>(a.part);  // 3 doubles per block
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) bp[3 * bx + k] = tot[k];
        __threadfence();
        s_last = atomicAdd(a.counter, 1u) == (unsigned)nbx - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc[3] = {0.0, 0.0, 0.0};
    for (unsigned b = threadIdx.x; b < (unsigned)nbx; b += blockDim.x)
        for (int k = 0; k < 3; ++k) acc[k] += __ldcg(bp + 3 * b + k);
    double fin[3];
    block_sums_d3(acc, sh3, fin);
    if (threadIdx.x == 0) {
        double sc[4];
        alpha_finish(a, use_l1, fin, sc);
        for (int k = 0; k < 4; ++k) a.scal[k] = sc[k];
        *a.counter = 0u;
    }
}

__global__ void __launch_bounds__(kStepThreads) k_step_alpha(StepArgs a) {
    pdl_wait();
    pdl_trigger();
    step_alpha_body(a, blockIdx.x, gridDim.x);
}

// Stage 2 (one thread per parameter, many blocks): adam_param; then the last
// block runs the epoch tail.  Block (bx, r) of nbx x 10.
__device__ __forceinline__ void step_adam_body(const StepArgs &a, int bx, int r, int nbx) {
    __shared__ ff sh1[33][1];
    __shared__ bool s_last;
    __shared__ __align__(8) uint32_t s_words[kStateWords];
    const int m = *a.m;
    const int j = bx * blockDim.x + threadIdx.x;
    const float sc[4] = {(float)a.scal[0], (float)a.scal[1], (float)a.scal[2], (float)a.scal[3]};
    const float lr = (float)a.st->lr, taud = tau_d_float(a.c.tau_d);
    float bfc[1] = {0.f};
    if (j < m) bfc[0] = adam_param(a, r, j, sc, lr, taud);
    ff tot[1];
    block_sums_ff<1>(bfc, sh1, tot);
    const unsigned nblocks = (unsigned)nbx * SERBF_NPARAM, bid = (unsigned)r * nbx + bx;
    if (threadIdx.x == 0) {
        a.part[bid] = tot[0].hi;
        __threadfence();
        s_last = atomicAdd(a.counter + 1, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: b_f, then the epoch tail
    float cnt = 0.f;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) cnt += __ldcg(a.part + b);
    float cc[1] = {cnt};
    block_sums_ff<1>(cc, sh1, tot);
    finish_step(a, (double)tot[0].hi + tot[0].lo, a.scal[0], a.scal[1], s_words);
    if (threadIdx.x == 0) a.counter[1] = 0u;
}

__global__ void __launch_bounds__(kStepThreads) k_step_adam(StepArgs a) {
    pdl_wait();
    pdl_trigger();
    step_adam_body(a, blockIdx.x, blockIdx.y, gridDim.x);
}

// Eq. 3-27: stable compaction of the kernels with |w| >= tau_d.
__device__ __forceinline__ void prune_body(float *p, float *am, float *av, int32_t *m_dev, int cap, serbf_state *st,
                                           double tau_d, int force) {
    __shared__ uint32_t tmp[33];
    __shared__ int s_go;
    if (threadIdx.x == 0) s_go = force || st->do_prune;
    __syncthreads();
    if (!s_go) return;
    const int m = *m_dev;
    // |w| >= tau_d in float with tau_d rounded up: the same decision as in double
    float taud = (float)tau_d;
    if ((double)taud < tau_d) taud = nextafterf(taud, INFINITY);
    uint32_t carry = 0;
    for (int j0 = 0; j0 < m; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool live = j < m;
        const uint32_t keep = live && (fabsf(p[PW * cap + j]) >= taud);
        uint32_t tot;
        const uint32_t off = block_exscan(keep, tmp, &tot);
        float v[3][10];
        if (keep) {
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                v[0][r] = p[r * cap + j];
                v[1][r] = am[r * cap + j];
                v[2][r] = av[r * cap + j];
            }
        }
        __syncthreads();
        if (keep) {
            const int o = carry + off;
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                p[r * cap + o] = v[0][r];
                am[r * cap + o] = v[1][r];
                av[r * cap + o] = v[2][r];
            }
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->m_pruned = m - (int)carry;
        st->do_prune = 0;
        *m_dev = (int)carry;
    }
}

__global__ void __launch_bounds__(kStepThreads) k_prune(float *p, float *am, float *av, int32_t *m_dev, int cap,
                                                        serbf_state *st, double tau_d, int force) {
    pdl_wait();
    pdl_trigger();
    prune_body(p, am, av, m_dev, cap, st, tau_d, force);
}

// ---------------------------------------------------------------- batches of fields
// One field's step for the batched epoch: its arguments and its own block
// count (blocks of the batch grid beyond it leave at once, so each field's
// last-block hand-offs count only its own blocks).
struct StepBatch {
    StepArgs a;
    int nb;
};

__global__ void __launch_bounds__(kStepThreads) k_step_alpha_batch(const StepBatch *sb) {
    pdl_wait();
    pdl_trigger();
    const StepBatch &b = sb[blockIdx.y];
    if ((int)blockIdx.x >= b.nb) return;
    step_alpha_body(b.a, blockIdx.x, b.nb);
}

__global__ void __launch_bounds__(kStepThreads) k_step_adam_batch(const StepBatch *sb) {
    pdl_wait();
    pdl_trigger();
    const StepBatch &b = sb[blockIdx.z];
    if ((int)blockIdx.x >= b.nb) return;
    step_adam_body(b.a, blockIdx.x, blockIdx.y, b.nb);
}

// Eq. 3-27 of field blockIdx.x.
__global__ void __launch_bounds__(kStepThreads) k_prune_batch(const StepBatch *sb) {
    pdl_wait();
    pdl_trigger();
    const StepArgs &a = sb[blockIdx.x].a;
    prune_body(a.p, a.am, a.av, const_cast<int32_t *>(a.m), a.cap, a.st, a.c.tau_d, 0);
}

}  // namespace

namespace serbf {

size_t step_args_size() { return sizeof(StepBatch); }

// Host record of one field's step for a batch (out: sizeof(StepBatch) bytes).
int batch_step_args(serbf_params *prm, const float *grad, float *adam_m, float *adam_v, serbf_state *st_dev,
                    double *stats, const serbf_config *cfg, serbf_workspace *ws, void *out, int *nb) {
    if (!prm || !prm->p || !prm->m || prm->cap < 1 || !grad || !adam_m || !adam_v || !st_dev || !stats || !cfg)
        return SERBF_EINVAL;
    if (!ws || ws->magic != kMagic || prm->cap > ws->sz.max_kernels) return SERBF_EINVAL;
    if (cfg->k_l2 < 1 || cfg->k_l2 > 64 || cfg->k_l1 < 1 || cfg->k_l1 > 256) return SERBF_EINVAL;
    if (!(cfg->lr >= 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0))
        return SERBF_EINVAL;
    StepBatch b{StepArgs{prm->p, prm->m, prm->cap, grad, adam_m, adam_v, st_dev, stats, *cfg, ws->step_part,
                         ws->step_scal, ws->counters + 2},
                (prm->cap + kStepThreads - 1) / kStepThreads};
    memcpy(out, &b, sizeof(b));
    *nb = b.nb;
    return SERBF_OK;
}

// The batched step (two launches) and deletion (one).
int batch_step_launch(const void *args, int nfields, int max_nb, cudaStream_t s) {
    const StepBatch *sb = static_cast<const StepBatch *>(args);
    launch_pdl(k_step_alpha_batch, dim3((unsigned)max_nb, (unsigned)nfields), dim3(kStepThreads), 0, s, sb);
    launch_pdl(k_step_adam_batch, dim3((unsigned)max_nb, SERBF_NPARAM, (unsigned)nfields), dim3(kStepThreads), 0, s,
               sb);
    launch_pdl(k_prune_batch, dim3((unsigned)nfields), dim3(kStepThreads), 0, s, sb);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // namespace serbf

extern "C" int serbf_step(serbf_params *prm, const float *grad, float *adam_m, float *adam_v, serbf_state *st_dev,
                          double *stats, const serbf_config *cfg, serbf_workspace *ws, void *stream) {
    SERBF_TRACE();
    if (!prm || !prm->p || !prm->m || prm->cap < 1 || !grad || !adam_m || !adam_v || !st_dev || !stats || !cfg)
        return SERBF_EINVAL;
    if (!ws || ws->magic != kMagic || prm->cap > ws->sz.max_kernels) return SERBF_EINVAL;
    if (cfg->k_l2 < 1 || cfg->k_l2 > 64 || cfg->k_l1 < 1 || cfg->k_l1 > 256) return SERBF_EINVAL;
    if (!(cfg->lr >= 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0))
        return SERBF_EINVAL;
    StepArgs a{prm->p, prm->m, prm->cap, grad, adam_m, adam_v, st_dev, stats, *cfg,
               ws->step_part, ws->step_scal, ws->counters + 2};
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((prm->cap + kStepThreads - 1) / kStepThreads);
    launch_pdl(k_step_alpha, dim3(nb), dim3(kStepThreads), 0, s, a);
    launch_pdl(k_step_adam, dim3(nb, SERBF_NPARAM), dim3(kStepThreads), 0, s, a);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

extern "C" int serbf_prune(serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev,
                           const serbf_config *cfg, void *stream) {
    SERBF_TRACE();
    if (!prm || !prm->p || !prm->m || prm->cap < 1 || !adam_m || !adam_v || !st_dev || !cfg) return SERBF_EINVAL;
    launch_pdl(k_prune, dim3(1), dim3(kStepThreads), 0, (cudaStream_t)stream, prm->p, adam_m, adam_v, prm->m, prm->cap, st_dev,
                                                           cfg->tau_d, 0);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
