// Algorithm 3 update for one full-batch epoch: Eq. 3-21 dynamic weighting
// (double reductions), Adam, and the epoch-tail gates (Eq. 3-27 deletion due,
// Eq. l1_activate, Eq. add_activate, L2-only phase with a cosine learning rate
// from T^e).  A single block: the state machine lives on the device so that a
// step needs no host round trip.  Also the Eq. 3-27 compaction.
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

constexpr int kStepThreads = 1024;

__device__ double block_sum_d(double v, double *sh) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < nw; ++w) r += sh[w];
        sh[32] = r;
    }
    __syncthreads();
    r = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float sgnf(float v) { return (float)((v > 0.f) - (v < 0.f)); }

struct StepArgs {
    float *p;
    const int32_t *m;
    int cap;
    const float *grad;
    float *am, *av;
    serbf_state *st;
    double *stats;
    serbf_config c;
};

__global__ void __launch_bounds__(kStepThreads) k_step(StepArgs a) {
    __shared__ double sh[33];
    __shared__ serbf_state st;
    __shared__ double s_alpha;
    const int m = *a.m, cap = a.cap;
    if (threadIdx.x == 0) st = *a.st;
    __syncthreads();
    const int e = st.epoch + 1;
    const bool use_l1 = st.l1_optim && (a.stats[SERBF_STAT_MAXE] < a.c.tau_m);
    // L1 = sum |w| before the update (Eq. 3-14_2)
    double l1 = 0.0, num = 0.0, den = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double w = a.p[PW * cap + j];
        l1 += fabs(w);
        if (use_l1) {
            const double g1 = (w > 0) - (w < 0), g2 = a.grad[PW * cap + j];
            num += (g1 - g2) * g1;
            den += (g2 - g1) * (g2 - g1);
        }
    }
    l1 = block_sum_d(l1, sh);
    num = block_sum_d(num, sh);
    den = block_sum_d(den, sh);
    if (threadIdx.x == 0) {
        double al = 1.0;
        if (use_l1 && den > 0.0) al = fmin(1.0, fmax(0.0, num / den));
        s_alpha = al;
    }
    __syncthreads();
    const double alpha = s_alpha, beta = 1.0 - alpha;
    const int t = st.adam_t + 1;
    const float lr = (float)st.lr;
    const float b1 = (float)a.c.beta1, b2 = (float)a.c.beta2, eps = (float)a.c.adam_eps;
    const float bc1 = (float)(1.0 - pow(a.c.beta1, t)), bc2 = (float)(1.0 - pow(a.c.beta2, t));
    const float fa = (float)alpha, fb = (float)beta;
    const int64_t total = 10ll * m;
    for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int r = (int)(idx / m), j = (int)(idx - (int64_t)r * m);
        const int64_t q = (int64_t)r * cap + j;
        float g = fa * a.grad[q];
        if (r == PW) g = fmaf(fb, sgnf(a.p[q]), g);
        const float mo = fmaf(b1, a.am[q], (1.f - b1) * g);
        const float vo = fmaf(b2, a.av[q], (1.f - b2) * g * g);
        a.am[q] = mo;
        a.av[q] = vo;
        a.p[q] -= lr * (mo / bc1) / (sqrtf(vo / bc2) + eps);
    }
    __syncthreads();
    double bf = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) bf += fabs((double)a.p[PW * cap + j]) >= a.c.tau_d;
    bf = block_sum_d(bf, sh);
    if (threadIdx.x != 0) return;
    // epoch tail, in the order of Algorithm 3
    st.alpha = alpha;
    st.beta = beta;
    st.adam_t = t;
    st.do_prune = (e % a.c.k_l2 == 0) && st.l1_optim && (e < a.c.T_e);
    const double l2 = a.stats[SERBF_STAT_L2];
    const int kl2 = a.c.k_l2, kl1 = a.c.k_l1;
    if (st.n_l2 < kl2) {
        st.l2_hist[st.n_l2++] = l2;
    } else {
        for (int k = 0; k + 1 < kl2; ++k) st.l2_hist[k] = st.l2_hist[k + 1];
        st.l2_hist[kl2 - 1] = l2;
    }
    if (st.n_bf < kl1) {
        st.bf_hist[st.n_bf++] = (int32_t)bf;
    } else {
        for (int k = 0; k + 1 < kl1; ++k) st.bf_hist[k] = st.bf_hist[k + 1];
        st.bf_hist[kl1 - 1] = (int32_t)bf;
    }
    if (!st.l1_optim && !st.phase2 && e >= kl2 && st.n_l2 == kl2) {
        double mean = 0.0;
        for (int k = 0; k < kl2; ++k) mean += st.l2_hist[k];
        mean /= kl2;
        double var = 0.0;
        for (int k = 0; k < kl2; ++k) var += (st.l2_hist[k] - mean) * (st.l2_hist[k] - mean);
        var /= kl2;
        if (sqrt(var) < a.c.tau_l2) st.l1_optim = 1;
    }
    st.do_add = 0;
    if (st.l1_optim && !st.phase2 && st.n_bf == kl1) {
        int lo = st.bf_hist[0], hi = st.bf_hist[0];
        for (int k = 1; k < kl1; ++k) {
            lo = min(lo, st.bf_hist[k]);
            hi = max(hi, st.bf_hist[k]);
        }
        if ((double)(hi - lo) < a.c.tau_l1) {
            st.do_add = 1;
            st.l1_optim = 0;
        }
    }
    if (e == a.c.T_e) {
        st.phase2 = 1;
        st.l1_optim = 0;
    }
    if (st.phase2) {
        const double span = (double)(a.c.M_e - a.c.T_e);
        double pr = span > 0 ? (double)(e - a.c.T_e) / span : 1.0;
        if (pr > 1.0) pr = 1.0;
        st.lr = a.c.lr_min + (a.c.lr_p2 - a.c.lr_min) * 0.5 * (1.0 + cos(3.14159265358979323846 * pr));
    } else {
        st.lr = a.c.lr;
    }
    st.epoch = e;
    *a.st = st;
    a.stats[SERBF_STAT_L1] = l1;
    a.stats[SERBF_STAT_ALPHA] = alpha;
    a.stats[SERBF_STAT_BETA] = beta;
    a.stats[SERBF_STAT_BF] = bf;
    a.stats[SERBF_STAT_LOSS] = alpha * l2 + beta * l1;
}

// Eq. 3-27: stable compaction of the kernels with |w| >= tau_d.
__global__ void __launch_bounds__(kStepThreads) k_prune(float *p, float *am, float *av, int32_t *m_dev, int cap,
                                                        serbf_state *st, double tau_d, int force) {
    __shared__ uint32_t tmp[33];
    __shared__ int s_go;
    if (threadIdx.x == 0) s_go = force || st->do_prune;
    __syncthreads();
    if (!s_go) return;
    const int m = *m_dev;
    uint32_t carry = 0;
    for (int j0 = 0; j0 < m; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool live = j < m;
        const uint32_t keep = live && (fabs((double)p[PW * cap + j]) >= tau_d);
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

}  // namespace

extern "C" int serbf_step(serbf_params *prm, const float *grad, float *adam_m, float *adam_v, serbf_state *st_dev,
                          double *stats, const serbf_config *cfg, void *stream) {
    if (!prm || !prm->p || !prm->m || prm->cap < 1 || !grad || !adam_m || !adam_v || !st_dev || !stats || !cfg)
        return SERBF_EINVAL;
    if (cfg->k_l2 < 1 || cfg->k_l2 > 64 || cfg->k_l1 < 1 || cfg->k_l1 > 256) return SERBF_EINVAL;
    StepArgs a{prm->p, prm->m, prm->cap, grad, adam_m, adam_v, st_dev, stats, *cfg};
    k_step<<<1, kStepThreads, 0, (cudaStream_t)stream>>>(a);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

extern "C" int serbf_prune(serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev,
                           const serbf_config *cfg, void *stream) {
    if (!prm || !prm->p || !prm->m || prm->cap < 1 || !adam_m || !adam_v || !st_dev || !cfg) return SERBF_EINVAL;
    k_prune<<<1, kStepThreads, 0, (cudaStream_t)stream>>>(prm->p, adam_m, adam_v, prm->m, prm->cap, st_dev,
                                                           cfg->tau_d, 0);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
