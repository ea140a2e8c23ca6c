// Workspace management, configuration, status, Eq. 3-10 normalisation and
// small utility kernels (scans, gathers).
#include <math.h>
#include <string.h>

#include "common.cuh"

using namespace serbf;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int64_t max_supers_for(int64_t cells, int sf) {
    double e = cbrt((double)cells);
    int64_t per = (int64_t)ceil(e / sf) + 1;
    int64_t s = per * per * per;
    return s < 1 ? 1 : s;
}

// Walks the carve-up; with base == nullptr it only sizes.
struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(int64_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (size_t)(count > 0 ? count : 1);
        return p;
    }
};

bool sizes_ok(const serbf_ws_sizes *s) {
    return s && s->max_points > 0 && s->max_points < (1ll << 31) && s->max_kernels > 0 && s->max_cells > 0 &&
           s->super_cap > 0 && s->super_factor >= 1 && s->super_factor <= 16;
}

void carve(Carver &c, serbf_workspace *w, const serbf_ws_sizes *s) {
    int64_t N = s->max_points, K = s->max_kernels, C = s->max_cells;
    int64_t S = max_supers_for(C, s->super_factor);
    int64_t cps = (int64_t)s->super_factor * s->super_factor * s->super_factor;
    int64_t T = N / kTile + S + 1;
    int64_t SB = (N + kSortTile - 1) / kSortTile;
    if (SB < 1) SB = 1;
    w->max_tiles = T;
    w->max_supers = S;
    w->sort_blocks = SB;
    w->keys0 = c.take<uint32_t>(N);
    w->keys1 = c.take<uint32_t>(N);
    w->vals0 = c.take<uint32_t>(N);
    w->vals1 = c.take<uint32_t>(N);
    w->hist = c.take<uint32_t>(256 * SB + 1);
    w->cell_start = c.take<uint32_t>(S * cps + 1);
    w->super_tile0 = c.take<uint32_t>(S + 1);
    w->tile_super = c.take<uint32_t>(T);
    w->tile_start = c.take<uint32_t>(T);
    const int64_t I = T / 2 + S + 2;
    w->max_items = I;
    w->super_item0 = c.take<uint32_t>(S + 1);
    w->item_rec = c.take<uint4>(I);
    w->item_class = c.take<uint8_t>(I);
    w->class_hist = c.take<uint32_t>((I + kOrderChunk - 1) / kOrderChunk * kCostClasses);
    w->order_rec = c.take<uint4>(I);
    w->sched = c.take<uint32_t>(4);
    w->sched_total = c.take<unsigned long long>(2);
    w->tile_lo = c.take<float4>(T);
    w->tile_hi = c.take<float4>(T);
    w->sup_lo = c.take<float4>(S);
    w->sup_hi = c.take<float4>(S);
    w->kfwd = c.take<float4>(3 * K);
    w->kbwd = c.take<float4>(4 * K);
    w->sup_list = c.take<uint32_t>(S * (int64_t)s->super_cap);
    w->sup_cnt = c.take<uint32_t>(S);
    // balanced grids have about S / 8 blocks of 2 x 2 x 2 super cells; flat
    // ones more, and those rebuild in one level
    w->max_coarse = S / 4 + 16;
    w->crs_list = c.take<uint32_t>(w->max_coarse * (int64_t)s->super_cap);
    w->crs_cnt = c.take<uint32_t>(w->max_coarse);
    w->fwd_part = c.take<FwdPart>(T + 1);
    w->fwd_gpart = c.take<FwdPart>(T / kFwdGroup + 2);
    w->bwd_pairs = c.take<unsigned long long>(K);
    w->adj_fix = c.take<unsigned long long>(K * 10);
    w->adj_pairs = c.take<unsigned long long>(8);
    w->moments = c.take<float>((int64_t)K * kBwdWarpsPerKernel * 22);
    w->nzrec = c.take<float4>(2 * T);
    w->nzc_cnt = c.take<uint32_t>(T);
    w->nz = c.take<float4>(T * kTile);
    w->step_part = c.take<float>(6 * (SERBF_NPARAM * (K / 256 + 1) + 1));
    w->step_scal = c.take<double>(8);
    w->sel_hist = c.take<uint32_t>(kSelBins);
    w->sel_ctl = c.take<uint32_t>(16);
    w->add_info = c.take<int32_t>(16);
    w->status = c.take<int32_t>(16);
    w->needed = c.take<long long>(4);
    w->counters = c.take<uint32_t>(16);
    w->dtmp = c.take<double>(16);
    w->cell_max = c.take<uint32_t>(4);
    w->field_box = c.take<float4>(2);
}

__global__ void k_exscan_u32(uint32_t *a, int64_t n) {
    __shared__ uint32_t tmp[33];
    int64_t per = (n + blockDim.x - 1) / blockDim.x;
    int64_t b = per * threadIdx.x, e = b + per < n ? b + per : n;
    uint32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += a[i];
    uint32_t total;
    uint32_t off = block_exscan(s, tmp, &total);
    for (int64_t i = b; i < e; ++i) {
        uint32_t v = a[i];
        a[i] = off;
        off += v;
    }
    if (threadIdx.x == 0) a[n] = total;
}

__global__ void k_exscan_i64(int64_t *a, int64_t n) {
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long tot;
    int64_t per = (n + blockDim.x - 1) / blockDim.x;
    int64_t b = per * threadIdx.x, e = b + per < n ? b + per : n;
    unsigned long long s = 0;
    for (int64_t i = b; i < e; ++i) s += (unsigned long long)a[i];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = lane < nw ? ws[lane] : 0ull, vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long t = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += t;
        }
        if (lane < nw) ws[lane] = vi - v;
        if (lane == 31) tot = vi;
    }
    __syncthreads();
    unsigned long long off = ws[warp] + inc - s;
    for (int64_t i = b; i < e; ++i) {
        unsigned long long v = (unsigned long long)a[i];
        a[i] = (int64_t)off;
        off += v;
    }
    if (threadIdx.x == 0) a[n] = (int64_t)tot;
}

__global__ void k_gather(const float *src, const uint32_t *perm, float *dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[perm[k]];
}

__device__ __forceinline__ int ordered_key(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ordered_val(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__global__ void k_init_min(int *slot) { *slot = 0x7fffffff; }

__global__ void k_min(const float *S, int64_t n, int *slot) {
    int best = 0x7fffffff;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        best = min(best, ordered_key(S[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMin(slot, best);
}

// Eq. 3-10, double precision per element.
__global__ void k_normalize(const float *S, float *t, int64_t n, const int *slot, double *mh) {
    double m = (double)ordered_val(*slot);
    double h = log(2.0) / (m * m);
    if (blockIdx.x == 0 && threadIdx.x == 0 && mh) {
        mh[0] = m;
        mh[1] = h;
    }
    __shared__ ff c[kEq310Terms];
    if (threadIdx.x == 0) eq310_coefs(c);
    __syncthreads();
    const float mf = ordered_val(*slot);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = eq310_target(S[i], mf, c);
}

__global__ void k_state_init(serbf_state *st, double lr) {
    serbf_state z;
    memset(&z, 0, sizeof(z));
    z.lr = lr;
    z.alpha = 1.0;
    z.beta = 0.0;
    *st = z;
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

namespace serbf {
int launch_exscan_u32(uint32_t *a, int64_t n, cudaStream_t s) {
    k_exscan_u32<<<1, 1024, 0, s>>>(a, n);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
int launch_exscan_i64(int64_t *a, int64_t n, cudaStream_t s) {
    k_exscan_i64<<<1, 1024, 0, s>>>(a, n);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
}  // namespace serbf

extern "C" {

const char *serbf_version(void) { return "serbf 0.3.7 (sm_103a)"; }

const char *serbf_status_string(int code) {
    switch (code) {
        case SERBF_OK: return "ok";
        case SERBF_EINVAL: return "invalid argument";
        case SERBF_ENOMEM: return "workspace too small";
        case SERBF_ECAPACITY: return "capacity exceeded";
        case SERBF_ECUDA: return "CUDA error";
        case SERBF_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

int serbf_config_default(serbf_config *c) {
    if (!c) return SERBF_EINVAL;
    memset(c, 0, sizeof(*c));
    c->eps = 1e-7;
    c->tau1 = 0.9;
    c->tau2 = 1.1;
    c->tau_m = 0.02;
    c->tau_d = 0.01;
    c->tau_l1 = 5.0;
    c->tau_l2 = 0.5;
    c->lr = 0.01;
    c->lr_p2 = 1e-3;
    c->lr_min = 1e-5;
    c->beta1 = 0.9;
    c->beta2 = 0.999;
    c->adam_eps = 1e-8;
    c->topk_frac = 0.01;
    c->add_radius = 0.0;
    c->dbar_min = 0.0;
    c->k_l1 = 50;
    c->k_l2 = 10;
    c->T_e = 1600;
    c->M_e = 2000;
    c->kahan = 0;
    c->epoch_steps = 1;
    return SERBF_OK;
}

size_t serbf_workspace_struct_size(void) { return sizeof(serbf_workspace); }

int serbf_workspace_bytes(const serbf_ws_sizes *sz, size_t *bytes) {
    if (!sizes_ok(sz) || !bytes) return SERBF_EINVAL;
    serbf_workspace tmp;
    memset(&tmp, 0, sizeof(tmp));
    Carver c{nullptr};
    carve(c, &tmp, sz);
    *bytes = align_up(c.off, 256);
    return SERBF_OK;
}

int serbf_workspace_init(serbf_workspace *ws, void *dev, size_t bytes, const serbf_ws_sizes *sz) {
    if (!ws || !dev || !sizes_ok(sz)) return SERBF_EINVAL;
    if (((uintptr_t)dev) % 256) return SERBF_EINVAL;
    size_t need;
    serbf_workspace_bytes(sz, &need);
    if (bytes < need) return SERBF_ENOMEM;
    memset(ws, 0, sizeof(*ws));
    ws->magic = kMagic;
    ws->base = (char *)dev;
    ws->bytes = bytes;
    ws->sz = *sz;
    Carver c{(char *)dev};
    carve(c, ws, sz);
    if (cudaMemset(ws->status, 0, 16 * sizeof(int32_t)) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemset(ws->needed, 0, 4 * sizeof(long long)) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemset(ws->counters, 0, 16 * sizeof(uint32_t)) != cudaSuccess) return SERBF_ECUDA;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return SERBF_ECUDA;
        if (cudaDeviceGetAttribute(&ws->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SERBF_ECUDA;
    }
    if (cudaMemset(ws->add_info, 0, 16 * sizeof(int32_t)) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemset(ws->sel_hist, 0, kSelBins * sizeof(uint32_t)) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemset(ws->cell_max, 0, 4 * sizeof(uint32_t)) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemset(ws->sel_ctl, 0, 16 * sizeof(uint32_t)) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemset(ws->adj_fix, 0, sizeof(unsigned long long) * 10 * (size_t)sz->max_kernels) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaMemset(ws->adj_pairs, 0, sizeof(unsigned long long) * 8) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamCreateWithFlags(&ws->aux, cudaStreamNonBlocking) != cudaSuccess) return SERBF_ECUDA;
    if (cudaEventCreateWithFlags(&ws->ev_fork, cudaEventDisableTiming) != cudaSuccess) return SERBF_ECUDA;
    if (cudaEventCreateWithFlags(&ws->ev_join, cudaEventDisableTiming) != cudaSuccess) return SERBF_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return SERBF_ECUDA;
    return SERBF_OK;
}

int serbf_workspace_release(serbf_workspace *ws) {
    if (!ws || ws->magic != kMagic) return SERBF_EINVAL;
    int rc = SERBF_OK;
    if (ws->aux && cudaStreamSynchronize(ws->aux) != cudaSuccess) rc = SERBF_ECUDA;
    if (ws->aux && cudaStreamDestroy(ws->aux) != cudaSuccess) rc = SERBF_ECUDA;
    if (ws->ev_fork && cudaEventDestroy(ws->ev_fork) != cudaSuccess) rc = SERBF_ECUDA;
    if (ws->ev_join && cudaEventDestroy(ws->ev_join) != cudaSuccess) rc = SERBF_ECUDA;
    ws->aux = nullptr;
    ws->ev_fork = ws->ev_join = nullptr;
    ws->magic = 0;
    return rc;
}

int serbf_status(serbf_workspace *ws, int32_t *flags, int64_t needed[4], int clear, void *stream) {
    if (!ws || ws->magic != kMagic) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t f = 0;
    long long nd[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(&f, ws->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaMemcpyAsync(nd, ws->needed, sizeof(nd), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    if (flags) *flags = f;
    if (needed)
        for (int k = 0; k < 4; ++k) needed[k] = nd[k];
    if (clear) {
        if (cudaMemsetAsync(ws->status, 0, sizeof(int32_t), s) != cudaSuccess) return SERBF_ECUDA;
        if (cudaMemsetAsync(ws->needed, 0, 4 * sizeof(long long), s) != cudaSuccess) return SERBF_ECUDA;
    }
    return f ? SERBF_ECAPACITY : SERBF_OK;
}

int serbf_state_init(serbf_state *st_dev, const serbf_config *cfg, void *stream) {
    if (!st_dev || !cfg) return SERBF_EINVAL;
    k_state_init<<<1, 1, 0, (cudaStream_t)stream>>>(st_dev, cfg->lr);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

int serbf_normalize_sdf(const float *S, float *t, int64_t n, double *mh_dev, serbf_workspace *ws,
                        void *stream) {
    SERBF_TRACE();
    if (!S || !t || n <= 0 || !ws || ws->magic != kMagic) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int *slot = ws->status + 8;
    k_init_min<<<1, 1, 0, s>>>(slot);
    k_min<<<grid_for(n, 256), 256, 0, s>>>(S, n, slot);
    k_normalize<<<grid_for(n, 256), 256, 0, s>>>(S, t, n, slot, mh_dev);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

int serbf_gather(const float *src, const uint32_t *perm, float *dst, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!src || !perm || !dst))) return SERBF_EINVAL;
    if (n == 0) return SERBF_OK;
    k_gather<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(src, perm, dst, n);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // extern "C"
