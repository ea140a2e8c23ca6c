// Adaptive basis addition, Algorithm 2 in its top-k form, with the new
// kernel parameters of Eq. 3-24 appended as in Eq. 3-25:
//   1. candidates: id_all points with |E| > tau_m / 2 (Algorithm 2, candidate set);
//   2. keep the k = ceil(topk_frac |id_all|) largest |E| (ties: ascending
//      binned index) with an exact radix select on the float bits of |E|;
//   3. drop a candidate if an id_all point within add_radius has a larger |E|
//      (Algorithm 2, local-maximum test);
//   4. append c = v, w = -E, d = sqrt(-ln(eps / |E|) / dbar^2) on all axes,
//      theta = 0, in selection order; reset the Adam moments.
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

constexpr int kSelMax = 8192;  // largest selection sorted in shared memory
constexpr int kAddThreads = 1024;

__device__ __forceinline__ uint32_t cand_key(const float *E, const uint8_t *mask, int64_t i, double thresh) {
    float a = fabsf(E[i]);
    return (mask[i] && (double)a > thresh) ? __float_as_uint(a) : 0u;
}

__global__ void __launch_bounds__(kAddThreads) k_add_select(const float *E, const uint8_t *mask, int64_t n,
                                                           const double *stats, const serbf_state *st,
                                                           double thresh, double frac, int force,
                                                           unsigned long long *sel, int32_t *info) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ unsigned long long sk[];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t tmp[33];
    __shared__ uint32_t s_prefix, s_remaining, s_all;
    __shared__ int s_go;
    if (threadIdx.x == 0) {
        s_go = force || st->do_add;
        info[0] = s_go;
        info[1] = 0;
    }
    __syncthreads();
    if (!s_go) return;
    int64_t k = kSelMax;
    if (frac > 0.0) k = (int64_t)ceil(frac * stats[SERBF_STAT_COUNT]);
    if (k > kSelMax) k = kSelMax;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_remaining = (uint32_t)k;
        s_all = 0;
    }
    __syncthreads();
    // exact radix select of the k-th largest key, most significant byte first
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d] = 0;
        __syncthreads();
        const uint32_t pre = s_prefix;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            uint32_t key = cand_key(E, mask, i, thresh);
            if (key == 0) continue;
            if (shift < 24 && (key >> (shift + 8)) != (pre >> (shift + 8))) continue;
            atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0 && !s_all) {
            uint32_t above = 0, rem = s_remaining;
            int d = 255;
            for (; d >= 0; --d) {
                if (above + hist[d] >= rem) break;
                above += hist[d];
            }
            if (d < 0) {
                s_all = 1;  // fewer candidates than k under this prefix: take them all
            } else {
                s_prefix = pre | ((uint32_t)d << shift);
                s_remaining = rem - above;
            }
        }
        __syncthreads();
        if (s_all) break;
    }
    // ordered collection: key > T, plus the first `remaining` keys == T
    const uint32_t T = s_all ? 0u : s_prefix;
    const uint32_t need_eq = s_all ? 0u : s_remaining;
    uint32_t carry = 0, carry_eq = 0;
    for (int64_t i0 = 0; i0 < n; i0 += blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const uint32_t key = i < n ? cand_key(E, mask, i, thresh) : 0u;
        const uint32_t eq = (!s_all && key != 0 && key == T) ? 1u : 0u;
        uint32_t teq;
        const uint32_t oeq = block_exscan(eq, tmp, &teq);
        const uint32_t take = (key != 0 && (s_all ? true : key > T)) || (eq && carry_eq + oeq < need_eq);
        uint32_t tt;
        const uint32_t o = block_exscan(take, tmp, &tt);
        if (take && carry + o < (uint32_t)kSelMax)
            sk[carry + o] = ((unsigned long long)(~key) << 32) | (unsigned long long)(uint32_t)i;
        carry += tt;
        carry_eq += teq;
    }
    const uint32_t ns = carry < (uint32_t)kSelMax ? carry : (uint32_t)kSelMax;
    // bitonic sort ascending on (~|E| bits, index): |E| descending, index ascending
    uint32_t P = 1;
    while (P < ns) P <<= 1;
    for (uint32_t q = ns + threadIdx.x; q < P; q += blockDim.x) sk[q] = ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t q = threadIdx.x; q < P / 2; q += blockDim.x) {
                const uint32_t lo = 2 * stride * (q / stride) + (q % stride), hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long a = sk[lo], b = sk[hi];
                if ((a > b) == asc) {
                    sk[lo] = b;
                    sk[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t q = threadIdx.x; q < ns; q += blockDim.x) sel[q] = sk[q];
    if (threadIdx.x == 0) info[1] = (int32_t)ns;
}

// One selected point s (a warp): keep[s] = 0 if an id_all point within the
// radius has a larger |E|.
__device__ __forceinline__ void localmax_one(const float *x, const float *y, const float *z, const float *E,
                                             const uint8_t *mask, const uint32_t *cell_start, serbf_grid g, int sf,
                                             int nsx, int nsy, float r2, int reach, const unsigned long long *sel,
                                             uint32_t *keep, int s, int lane) {
    const uint32_t i = (uint32_t)(sel[s] & 0xffffffffull);
    const float xi = x[i], yi = y[i], zi = z[i], ei = fabsf(E[i]);
    const int kx = cell_axis(xi, g.origin[0], g.h, g.n[0]);
    const int ky = cell_axis(yi, g.origin[1], g.h, g.n[1]);
    const int kz = cell_axis(zi, g.origin[2], g.h, g.n[2]);
    bool bad = false;
    for (int cz = max(0, kz - reach); cz <= min(g.n[2] - 1, kz + reach) && !bad; ++cz)
        for (int cy = max(0, ky - reach); cy <= min(g.n[1] - 1, ky + reach) && !bad; ++cy)
            for (int cx = max(0, kx - reach); cx <= min(g.n[0] - 1, kx + reach) && !bad; ++cx) {
                const uint32_t key = cell_key(cx, cy, cz, sf, nsx, nsy);
                const uint32_t b = cell_start[key], e = cell_start[key + 1];
                for (uint32_t q0 = b; q0 < e && !bad; q0 += 32) {
                    const uint32_t q = q0 + lane;
                    bool v = false;
                    if (q < e && mask[q]) {
                        const float dx = __fsub_rn(x[q], xi), dy = __fsub_rn(y[q], yi), dz = __fsub_rn(z[q], zi);
                        const float d2 =
                            __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                        v = d2 <= r2 && fabsf(E[q]) > ei;
                    }
                    bad = __any_sync(0xffffffffu, v);
                }
            }
    if (lane == 0) keep[s] = !bad;
}

// Warps over the selected points (grid-stride): reject a point if an id_all
// point within the radius has a larger |E| (distance in float, same operation
// order as the support test, <= r2).  One block per SM, so a step without an
// addition retires few blocks.
__global__ void k_add_localmax(const float *x, const float *y, const float *z, const float *E,
                               const uint8_t *mask, const uint32_t *cell_start, serbf_grid g, int sf, int nsx,
                               int nsy, float r2, int reach, const unsigned long long *sel, const int32_t *info,
                               uint32_t *keep) {
    pdl_wait();
    pdl_trigger();
    if (!info[0]) return;
    const int lane = threadIdx.x & 31, nsel = info[1];
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nsel; s += (gridDim.x * blockDim.x) >> 5)
        localmax_one(x, y, z, E, mask, cell_start, g, sf, nsx, nsy, r2, reach, sel, keep, s, lane);
}

__global__ void __launch_bounds__(kAddThreads) k_add_append(const float *x, const float *y, const float *z,
                                                           const float *E, const float *S, double dbar_min,
                                                           double eps, const unsigned long long *sel,
                                                           const uint32_t *keep, int32_t *info, float *p,
                                                           float *am, float *av, int32_t *m_dev, int cap,
                                                           serbf_state *st, int32_t *status, long long *needed) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t tmp[33];
    if (!info[0]) return;
    const int ns = info[1];
    const int m = *m_dev;
    const int room = cap - m;
    uint32_t carry = 0;
    for (int s0 = 0; s0 < ns; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const uint32_t k = s < ns ? keep[s] : 0u;
        uint32_t tot;
        const uint32_t o = block_exscan(k, tmp, &tot);
        if (k && (int)(carry + o) < room) {
            const uint32_t i = (uint32_t)(sel[s] & 0xffffffffull);
            const int j = m + (int)(carry + o);
            const double ae = fabs((double)E[i]);
            const double dbar = fmax(fabs((double)S[i]), dbar_min);
            const double d = sqrt(-log(eps / ae) / (dbar * dbar));
            p[PCX * cap + j] = x[i];
            p[PCY * cap + j] = y[i];
            p[PCZ * cap + j] = z[i];
            p[PD1 * cap + j] = (float)d;
            p[PD2 * cap + j] = (float)d;
            p[PD3 * cap + j] = (float)d;
            p[PTX * cap + j] = 0.f;
            p[PTY * cap + j] = 0.f;
            p[PTZ * cap + j] = 0.f;
            p[PW * cap + j] = -E[i];
        }
        carry += tot;
    }
    const int added = (int)carry < room ? (int)carry : (room > 0 ? room : 0);
    __syncthreads();
    const int mn = m + added;
    for (int64_t q = threadIdx.x; q < 10ll * mn; q += blockDim.x) {
        const int r = (int)(q / mn), j = (int)(q - (int64_t)r * mn);
        am[r * cap + j] = 0.f;
        av[r * cap + j] = 0.f;
    }
    if (threadIdx.x == 0) {
        if ((int)carry > room) {
            atomicOr(status, SERBF_FLAG_ADD_CAPACITY);
            atomicMax(needed + 3, (long long)(m + (int)carry));
        }
        info[2] = (int)carry;
        *m_dev = mn;
        st->m_added = added;
        st->adam_t = 0;
        st->do_add = 0;
        info[0] = 0;
    }
}

}  // namespace

extern "C" int serbf_add_kernels(const serbf_points *pts, const float *S_raw, const float *err, const uint8_t *mask,
                                 serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev,
                                 const double *stats, const serbf_config *cfg, int force, serbf_workspace *ws,
                                 void *stream) {
    SERBF_TRACE();
    if (!pts || !prm || !cfg || !ws || ws->magic != kMagic || !ws->binned) return SERBF_EINVAL;
    if (pts->n != ws->npoints || !prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels)
        return SERBF_EINVAL;
    if (!st_dev || !stats || !adam_m || !adam_v) return SERBF_EINVAL;
    if (pts->n > 0 && (!S_raw || !err || !mask || !pts->x || !pts->y || !pts->z)) return SERBF_EINVAL;
    if (!(cfg->add_radius >= 0.0) || !(cfg->eps > 0.0)) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    static bool attr = false;
    const int smem = kSelMax * (int)sizeof(unsigned long long);
    if (!attr) {
        if (cudaFuncSetAttribute(k_add_select, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return SERBF_ECUDA;
        attr = true;
    }
    launch_pdl(k_add_select, dim3(1), dim3(kAddThreads), smem, s, err, mask, pts->n, stats, st_dev, cfg->tau_m * 0.5, cfg->topk_frac,
                                               force, ws->sel_key, ws->add_info);
    const float r2 = (float)(cfg->add_radius * cfg->add_radius);
    int reach = (int)ceil(cfg->add_radius / ws->grid.h) + 1;
    if (reach > 1 << 20) reach = 1 << 20;
    const unsigned lm_blocks = (unsigned)(ws->sm_count > 0 ? ws->sm_count : 1);
    launch_pdl(k_add_localmax, dim3(lm_blocks), dim3(256), 0, s, pts->x, pts->y, pts->z, err, mask, ws->cell_start, ws->grid, ws->sf,
                                            ws->ns[0], ws->ns[1], r2, reach, ws->sel_key, ws->add_info,
                                            ws->sel_keep);
    launch_pdl(k_add_append, dim3(1), dim3(kAddThreads), 0, s, pts->x, pts->y, pts->z, err, S_raw, cfg->dbar_min, cfg->eps, ws->sel_key,
                                           ws->sel_keep, ws->add_info, prm->p, adam_m, adam_v, prm->m, prm->cap,
                                           st_dev, ws->status, ws->needed);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
