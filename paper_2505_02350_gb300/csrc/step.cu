// Algorithm 3 update for one full-batch epoch: Eq. 3-21 dynamic weighting,
// Adam, and the epoch-tail gates (Eq. 3-27 deletion due, Eq. l1_activate,
// Eq. add_activate, L2-only phase with a cosine learning rate from T^e).  Two
// grid-wide launches whose last blocks finish the reductions: the state
// machine lives on the device so that a step needs no host round trip.  Also
// the Eq. 3-27 compaction.
#include <math.h>

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

// Same for three float-float inputs.
__device__ void block_sums_ff3(const ff (&v)[3], ff (*sh)[3], ff (&out)[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const ff s = warp_sum_ff(v[k]);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ff t = lane < nw ? sh[lane][k] : ff{0.f, 0.f};
            t = warp_sum_ff(t);
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
    float *part;      // per block partial sums (float-float pairs)
    double *scal;     // alpha, beta, bias corrections for the update kernel
    uint32_t *counter;
};

constexpr int kStateWords = (int)(sizeof(serbf_state) / 4);
static_assert(sizeof(serbf_state) % 8 == 0, "state is copied as 32-bit words");

// Stage 1 of the update (one thread per kernel, many blocks): L1 = sum |w|
// (Eq. 3-14_2) and the two Eq. 3-21 dot products; the last block turns them
// into alpha and beta and the Adam bias corrections.
__global__ void __launch_bounds__(kStepThreads) k_step_alpha(StepArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ ff sh3[33][3];
    __shared__ bool s_last;
    const int m = *a.m, cap = a.cap;
    const bool use_l1 = a.st->l1_optim && (a.stats[SERBF_STAT_MAXE] < a.c.tau_m);
    float part[3] = {0.f, 0.f, 0.f};
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) {
        const float w = a.p[PW * cap + j], g2 = a.grad[PW * cap + j];
        part[0] = fabsf(w);
        if (use_l1) {
            const float g1 = sgnf(w);
            part[1] = (g1 - g2) * g1;
            part[2] = (g2 - g1) * (g2 - g1);
        }
    }
    ff tot[3];
    block_sums_ff<3>(part, sh3, tot);
    if (threadIdx.x == 0) {
        float *o = a.part + 6 * blockIdx.x;
        for (int k = 0; k < 3; ++k) {
            o[2 * k] = tot[k].hi;
            o[2 * k + 1] = tot[k].lo;
        }
        __threadfence();
        s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ff acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
        for (int k = 0; k < 3; ++k)
            acc[k] = ff_add(acc[k], ff{__ldcg(a.part + 6 * b + 2 * k), __ldcg(a.part + 6 * b + 2 * k + 1)});
    ff fin[3];
    block_sums_ff3(acc, sh3, fin);
    if (threadIdx.x == 0) {
        // float arithmetic from here (FP64 is slow on this part): alpha to ~1e-7
        const float num = fin[1].hi + fin[1].lo, den = fin[2].hi + fin[2].lo;
        float al = 1.f;
        if (use_l1 && den > 0.f) al = fminf(1.f, fmaxf(0.f, num / den));
        const float t = (float)(a.st->adam_t + 1);
        a.scal[0] = al;
        a.scal[1] = 1.f - al;
        a.scal[2] = 1.f - powf((float)a.c.beta1, t);
        a.scal[3] = 1.f - powf((float)a.c.beta2, t);
        a.stats[SERBF_STAT_L1] = (double)fin[0].hi + (double)fin[0].lo;
        a.stats[SERBF_STAT_ALPHA] = al;
        a.stats[SERBF_STAT_BETA] = 1.f - al;
        *a.counter = 0u;
    }
}

// Stage 2 (one thread per parameter, many blocks): the combined gradient of
// Eq. grad (App. A) and the Adam update; then the last block runs the epoch
// tail of Algorithm 3 on a shared-memory copy of the state.
__global__ void __launch_bounds__(kStepThreads) k_step_adam(StepArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ ff sh1[33][1];
    __shared__ bool s_last;
    __shared__ __align__(8) uint32_t s_words[kStateWords];
    const int m = *a.m, cap = a.cap;
    const int r = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    const float alpha = (float)a.scal[0], beta = (float)a.scal[1];
    const float bc1 = (float)a.scal[2], bc2 = (float)a.scal[3];
    const float lr = (float)a.st->lr;
    const float b1 = (float)a.c.beta1, b2 = (float)a.c.beta2, eps = (float)a.c.adam_eps;
    // b_f: |w| >= tau_d decided in float with tau_d rounded up (same decision as in double)
    float taud = (float)a.c.tau_d;
    if ((double)taud < a.c.tau_d) taud = nextafterf(taud, INFINITY);
    float bfc[1] = {0.f};
    if (j < m) {
        const int64_t q = (int64_t)r * cap + j;
        const float pv = a.p[q];
        float g = alpha * a.grad[q];
        if (r == PW) g = fmaf(beta, sgnf(pv), g);
        const float mo = fmaf(b1, a.am[q], (1.f - b1) * g);
        const float vo = fmaf(b2, a.av[q], (1.f - b2) * g * g);
        const float pn = pv - lr * (mo / bc1) / (sqrtf(vo / bc2) + eps);
        a.am[q] = mo;
        a.av[q] = vo;
        a.p[q] = pn;
        if (r == PW) bfc[0] = fabsf(pn) >= taud ? 1.f : 0.f;
    }
    ff tot[1];
    block_sums_ff<1>(bfc, sh1, tot);
    const unsigned nblocks = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        a.part[bid] = tot[0].hi;
        __threadfence();
        s_last = atomicAdd(a.counter + 1, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: b_f, then the epoch tail (warp 0) on a shared copy of the state
    const uint32_t *gw = reinterpret_cast<const uint32_t *>(a.st);
    for (int k = threadIdx.x; k < kStateWords; k += blockDim.x) s_words[k] = gw[k];
    float cnt = 0.f;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) cnt += __ldcg(a.part + b);
    float cc[1] = {cnt};
    block_sums_ff<1>(cc, sh1, tot);
    const double bf = (double)tot[0].hi + tot[0].lo;
    serbf_state &st = *reinterpret_cast<serbf_state *>(s_words);
    const double l2 = a.stats[SERBF_STAT_L2];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
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
            // population std of the last k_l2 values; each double is split into
            // a float-float pair so the mean and deviations keep ~48 bits
            ff v{0.f, 0.f};
            for (int k = lane; k < kl2; k += 32) {
                const double x = st.l2_hist[k];
                const float xh = (float)x;
                v = ff_add(v, ff{xh, (float)(x - (double)xh)});
            }
            v = warp_sum_ff(v);
            const float inv = 1.f / (float)kl2;
            const ff mean{v.hi * inv, v.lo * inv};
            float var = 0.f;
            for (int k = lane; k < kl2; k += 32) {
                const double x = st.l2_hist[k];
                const float xh = (float)x;
                const ff d = ff_add(ff{xh, (float)(x - (double)xh)}, ff{-mean.hi, -mean.lo});
                const float dd = d.hi + d.lo;
                var = fmaf(dd, dd, var);
            }
            var = warp_sum(var) * inv;
            if (sqrtf(var) < (float)a.c.tau_l2) l1n = 1;
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
            st.do_prune = do_prune;
            st.do_add = do_add;
            st.l1_optim = l1n;
            st.phase2 = ph;
            st.lr = lr_next;
            st.epoch = e;
            a.stats[SERBF_STAT_BF] = bf;
            a.stats[SERBF_STAT_LOSS] = (float)alpha * (float)l2 + (float)beta * (float)a.stats[SERBF_STAT_L1];
            a.counter[1] = 0u;
        }
    }
    __syncthreads();
    uint32_t *gwo = reinterpret_cast<uint32_t *>(a.st);
    for (int k = threadIdx.x; k < kStateWords; k += blockDim.x) gwo[k] = s_words[k];
}

// Eq. 3-27: stable compaction of the kernels with |w| >= tau_d.
__global__ void __launch_bounds__(kStepThreads) k_prune(float *p, float *am, float *av, int32_t *m_dev, int cap,
                                                        serbf_state *st, double tau_d, int force) {
    pdl_wait();
    pdl_trigger();
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

}  // namespace

extern "C" int serbf_step(serbf_params *prm, const float *grad, float *adam_m, float *adam_v, serbf_state *st_dev,
                          double *stats, const serbf_config *cfg, serbf_workspace *ws, void *stream) {
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
    if (!prm || !prm->p || !prm->m || prm->cap < 1 || !adam_m || !adam_v || !st_dev || !cfg) return SERBF_EINVAL;
    launch_pdl(k_prune, dim3(1), dim3(kStepThreads), 0, (cudaStream_t)stream, prm->p, adam_m, adam_v, prm->m, prm->cap, st_dev,
                                                           cfg->tau_d, 0);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
