// Adaptive basis addition, Algorithm 2 in its top-k form, with the new
// kernel parameters of Eq. 3-24 appended as in Eq. 3-25:
//   1. candidates: id_all points with |E| > tau_m / 2 (Algorithm 2, candidate set);
//   2. keep the k = ceil(topk_frac |id_all|) largest |E| (ties: ascending
//      binned index), exactly, for any k;
//   3. drop a candidate if an id_all point within add_radius has a larger |E|
//      (Algorithm 2, local-maximum test);
//   4. append c = v, w = -E, d = sqrt(-ln(eps / |E|) / dbar^2) on all axes,
//      theta = 0, in selection order; reset the Adam moments.
//
// Three launches, each a no-op unless the addition is due:
//   k_add_hist      all blocks: histogram of the candidates by the top 11 bits
//                   of |E| (its float bits; the sign bit is 0); the last block
//                   finds the bin B that holds the k-th largest key;
//   k_add_gather    all blocks: every candidate in a bin >= B (a superset of
//                   the top k) is appended to a list as (~key, index); the
//                   last block sorts that list by (~key, index) ascending --
//                   |E| descending, index ascending -- and keeps the first k;
//   k_add_localmax  warps over the k selected points: the local-maximum test;
//                   the last block appends the survivors in order.
// The selection lists use the binning sort buffers (idle outside binning).
#include <math.h>
#include <string.h>

#include "common.cuh"

using namespace serbf;

namespace {

constexpr int kHistThreads = 512;
constexpr int kGatherThreads = 1024;
constexpr int kBitonicMax = 8192;  // lists up to this size are sorted in shared memory
constexpr int kLmThreads = 256;

// sel_ctl slots
enum { CTL_BIN = 0, CTL_K, CTL_SUPER, CTL_SLOT, CTL_HIST_DONE, CTL_GATHER_DONE, CTL_LM_DONE };

struct AppendArgs {
    const float *x, *y, *z, *E, *S;
    double dbar_min, eps;
    float *p, *am, *av;
    int32_t *m_dev;
    int cap;
    serbf_state *st;
    int32_t *status;
    long long *needed;
};

// Everything the three launches of one addition read.
struct AddArgs {
    const float *E;
    const uint8_t *mask;
    int64_t n;
    const double *stats;
    double thresh, frac;
    int force;
    uint32_t *hist, *ctl;
    int32_t *info;
    uint32_t *hi, *lo, *hi2, *lo2;  // selection lists (binning sort buffers)
    const uint32_t *cell_start;
    serbf_grid g;
    int sf, nsx, nsy;
    float r2;
    int reach;
    AppendArgs ap;
};

__device__ __forceinline__ uint32_t cand_key(const float *E, const uint8_t *mask, int64_t i, double thresh) {
    const float a = fabsf(E[i]);
    return (mask[i] && (double)a > thresh) ? __float_as_uint(a) : 0u;
}

// Last block of a grid to reach this point (after its own writes): true in
// exactly one block.  No block waits for another.
__device__ __forceinline__ bool last_block(uint32_t *counter, bool *s_flag, int nbx) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *s_flag = atomicAdd(counter, 1u) == (unsigned)nbx - 1;
    }
    __syncthreads();
    if (*s_flag) __threadfence();
    return *s_flag;
}

// Block bx of nbx.
__device__ __forceinline__ void add_hist_body(const AddArgs &A, int bx, int nbx) {
    const float *E = A.E;
    const uint8_t *mask = A.mask;
    const int64_t n = A.n;
    const double thresh = A.thresh, frac = A.frac;
    uint32_t *hist = A.hist, *ctl = A.ctl;
    int32_t *info = A.info;
    __shared__ uint32_t sh[kSelBins];
    __shared__ uint32_t tmp[33];
    __shared__ bool s_last;
    const bool go = A.force || A.ap.st->do_add;
    if (!go) {
        if (bx == 0 && threadIdx.x == 0) info[0] = 0;
        return;
    }
    for (int d = threadIdx.x; d < kSelBins; d += blockDim.x) sh[d] = 0u;
    __syncthreads();
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)nbx * blockDim.x) {
        const uint32_t key = cand_key(E, mask, i, thresh);
        if (key) atomicAdd(&sh[key >> 20], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kSelBins; d += blockDim.x)
        if (sh[d]) atomicAdd(&hist[d], sh[d]);
    if (!last_block(&ctl[CTL_HIST_DONE], &s_last, nbx)) return;
    // the last block: bin counts (cleared for the next call), their total C,
    // k and the bin B holding the k-th largest key
    for (int d = threadIdx.x; d < kSelBins; d += blockDim.x) {
        sh[d] = __ldcg(&hist[d]);
        hist[d] = 0u;
    }
    __syncthreads();
    // thread q owns the four bins 2047 - 4q .. 2044 - 4q, largest first
    constexpr int kPer = kSelBins / kHistThreads;
    static_assert(kPer * kHistThreads == kSelBins, "bins per thread");
    uint32_t own = 0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) own += sh[kSelBins - 1 - kPer * threadIdx.x - r];
    uint32_t total;
    const uint32_t above = block_exscan(own, tmp, &total);  // keys in larger bins than this thread's
    int64_t k = total;
    if (frac > 0.0) {
        const double kk = ceil(frac * A.stats[SERBF_STAT_COUNT]);
        if (kk < (double)k) k = (int64_t)kk;
    }
    if (k < 0) k = 0;
    uint32_t run = above;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
        const int d = kSelBins - 1 - kPer * threadIdx.x - r;
        const uint32_t c = sh[d];
        if (k > 0 && run < (uint32_t)k && run + c >= (uint32_t)k) {
            ctl[CTL_BIN] = (uint32_t)d;
            ctl[CTL_SUPER] = run + c;
        }
        run += c;
    }
    if (threadIdx.x == 0) {
        if (k == 0) {
            ctl[CTL_BIN] = kSelBins;  // nothing to select
            ctl[CTL_SUPER] = 0u;
        }
        ctl[CTL_K] = (uint32_t)k;
        ctl[CTL_SLOT] = 0u;
        ctl[CTL_HIST_DONE] = 0u;
        info[0] = 1;
        info[1] = 0;
    }
}

// ---------------------------------------------------------------- block sorts
// Sort the list (hi, lo) of s pairs ascending by (hi, lo), by one block of
// kGatherThreads threads.  Small lists: bitonic network in shared memory.
__device__ void sort_small(uint32_t *hi, uint32_t *lo, uint32_t s, unsigned long long *sk) {
    uint32_t P = 1;
    while (P < s) P <<= 1;
    for (uint32_t q = threadIdx.x; q < P; q += blockDim.x)
        sk[q] = q < s ? (((unsigned long long)hi[q] << 32) | lo[q]) : ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t q = threadIdx.x; q < P / 2; q += blockDim.x) {
                const uint32_t a = 2 * stride * (q / stride) + (q % stride), b = a + stride;
                const bool asc = (a & size) == 0;
                const unsigned long long x = sk[a], y = sk[b];
                if ((x > y) == asc) {
                    sk[a] = y;
                    sk[b] = x;
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t q = threadIdx.x; q < s; q += blockDim.x) {
        hi[q] = (uint32_t)(sk[q] >> 32);
        lo[q] = (uint32_t)sk[q];
    }
    __syncthreads();
}

struct RadixSmem {
    uint32_t base[256];       // running output position of each digit
    uint32_t tile_tot[256];   // digit counts of the current tile
    uint32_t wcnt[32][256];   // per warp and digit: count, then exclusive prefix over warps
    uint32_t tmp[33];
    int skip;
};

__device__ __forceinline__ uint32_t digit_of(const uint32_t *hi, const uint32_t *lo, uint32_t i, int word,
                                              int shift) {
    return ((word ? hi[i] : lo[i]) >> shift) & 255u;
}

// One stable counting pass on an 8-bit digit (word 0: lo, 1: hi) from (shi,
// slo) to (dhi, dlo).  Returns false (and moves nothing) when every element
// has the same digit.  Stability: tiles of blockDim elements in order; within
// a tile, elements of one digit are ranked by warp, then by lane.
__device__ bool radix_pass(const uint32_t *shi, const uint32_t *slo, uint32_t *dhi, uint32_t *dlo, uint32_t s,
                           int word, int shift, RadixSmem &R) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) R.base[d] = 0u;
    if (threadIdx.x == 0) R.skip = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < s; i += blockDim.x) atomicAdd(&R.base[digit_of(shi, slo, i, word, shift)], 1u);
    __syncthreads();
    const uint32_t c = threadIdx.x < 256 ? R.base[threadIdx.x] : 0u;
    if (c == s) R.skip = 1;
    uint32_t tot;
    const uint32_t off = block_exscan(c, R.tmp, &tot);
    const int skip = R.skip;
    __syncthreads();  // every thread has read the flag before the next pass resets it
    if (skip) return false;
    if (threadIdx.x < 256) R.base[threadIdx.x] = off;
    __syncthreads();
    for (uint32_t t0 = 0; t0 < s; t0 += blockDim.x) {
        for (int q = threadIdx.x; q < 32 * 256; q += blockDim.x) (&R.wcnt[0][0])[q] = 0u;
        __syncthreads();
        const uint32_t i = t0 + threadIdx.x;
        const bool valid = i < s;
        const uint32_t d = valid ? digit_of(shi, slo, i, word, shift) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) R.wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < 256) {
            uint32_t run = 0;
            for (int w = 0; w < 32; ++w) {
                const uint32_t v = R.wcnt[w][threadIdx.x];
                R.wcnt[w][threadIdx.x] = run;
                run += v;
            }
            R.tile_tot[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = R.base[d] + R.wcnt[warp][d] + rank;
            dhi[pos] = shi[i];
            dlo[pos] = slo[i];
        }
        __syncthreads();
        if (threadIdx.x < 256) R.base[threadIdx.x] += R.tile_tot[threadIdx.x];
        __syncthreads();
    }
    return true;
}

// Larger lists: LSD radix on the 64-bit (hi, lo) in 8-bit digits, ping-pong
// between (hi, lo) and (hi2, lo2); passes whose digit is the same for every
// element are skipped.  The first `keep` sorted pairs end in (hi, lo).
__device__ void sort_large(uint32_t *hi, uint32_t *lo, uint32_t *hi2, uint32_t *lo2, uint32_t s, uint32_t keep,
                           RadixSmem &R) {
    uint32_t *ah = hi, *al = lo, *bh = hi2, *bl = lo2;
    for (int pass = 0; pass < 8; ++pass) {
        if (radix_pass(ah, al, bh, bl, s, pass >= 4, 8 * (pass & 3), R)) {
            uint32_t *t = ah;
            ah = bh;
            bh = t;
            t = al;
            al = bl;
            bl = t;
        }
    }
    if (ah != hi) {
        for (uint32_t q = threadIdx.x; q < keep; q += blockDim.x) {
            hi[q] = ah[q];
            lo[q] = al[q];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void add_gather_body(const AddArgs &A, int bx, int nbx, unsigned char *smem) {
    const float *E = A.E;
    const uint8_t *mask = A.mask;
    const int64_t n = A.n;
    const double thresh = A.thresh;
    uint32_t *ctl = A.ctl;
    int32_t *info = A.info;
    uint32_t *hi = A.hi, *lo = A.lo, *hi2 = A.hi2, *lo2 = A.lo2;
    __shared__ bool s_last;
    if (!info[0]) return;
    const uint32_t B = ctl[CTL_BIN];
    const int lane = threadIdx.x & 31;
    if (B < (uint32_t)kSelBins) {
        // grid-stride in whole warps, so every lane of a warp takes part in the ballot
        const int64_t stride = (int64_t)nbx * blockDim.x;
        for (int64_t i0 = bx * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
            const int64_t i = i0 + lane;
            const uint32_t key = i < n ? cand_key(E, mask, i, thresh) : 0u;
            const bool take = key != 0u && (key >> 20) >= B;
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (!bal) continue;
            uint32_t base = 0;
            const int leader = __ffs(bal) - 1;
            if (lane == leader) base = atomicAdd(&ctl[CTL_SLOT], (uint32_t)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (take) {
                const uint32_t o = base + __popc(bal & ((1u << lane) - 1u));
                hi[o] = ~key;
                lo[o] = (uint32_t)i;
            }
        }
    }
    if (!last_block(&ctl[CTL_GATHER_DONE], &s_last, nbx)) return;
    const uint32_t s = __ldcg(&ctl[CTL_SLOT]), k = min(ctl[CTL_K], s);
    if (s <= (uint32_t)kBitonicMax)
        sort_small(hi, lo, s, reinterpret_cast<unsigned long long *>(smem));
    else
        sort_large(hi, lo, hi2, lo2, s, k, *reinterpret_cast<RadixSmem *>(smem));
    if (threadIdx.x == 0) {
        info[1] = (int32_t)k;
        ctl[CTL_SLOT] = 0u;
        ctl[CTL_GATHER_DONE] = 0u;
    }
}

// One selected point s (a warp): keep[s] = 0 if an id_all point within the
// radius has a larger |E|.
__device__ __forceinline__ void localmax_one(const float *x, const float *y, const float *z, const float *E,
                                             const uint8_t *mask, const uint32_t *cell_start, serbf_grid g, int sf,
                                             int nsx, int nsy, float r2, int reach, const uint32_t *sel_idx,
                                             uint32_t *keep, int s, int lane) {
    const uint32_t i = sel_idx[s];
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
                        const float d2 = support_d2(dx, dy, dz);
                        v = d2 <= r2 && fabsf(E[q]) > ei;
                    }
                    bad = __any_sync(0xffffffffu, v);
                }
            }
    if (lane == 0) keep[s] = !bad;
}

// Eq. 3-24 / 3-25: the kept points become kernels, appended in selection
// order up to the capacity (a flag and the size needed otherwise); Adam
// restarts from zero moments.  Run by one block.
__device__ void append_kept(const AppendArgs &a, const uint32_t *sel_idx, const uint32_t *keep, int ns, int32_t *info) {
    __shared__ uint32_t tmp[33];
    const int m = *a.m_dev;
    const int room = a.cap - m;
    const int cap = a.cap;
    uint32_t carry = 0;
    for (int s0 = 0; s0 < ns; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const uint32_t k = s < ns ? __ldcg(&keep[s]) : 0u;
        uint32_t tot;
        const uint32_t o = block_exscan(k, tmp, &tot);
        if (k && (int)(carry + o) < room) {
            const uint32_t i = sel_idx[s];
            const int j = m + (int)(carry + o);
            const double ae = fabs((double)a.E[i]);
            const double dbar = fmax(fabs((double)a.S[i]), a.dbar_min);
            const double d = sqrt(-log(a.eps / ae) / (dbar * dbar));
            a.p[PCX * cap + j] = a.x[i];
            a.p[PCY * cap + j] = a.y[i];
            a.p[PCZ * cap + j] = a.z[i];
            a.p[PD1 * cap + j] = (float)d;
            a.p[PD2 * cap + j] = (float)d;
            a.p[PD3 * cap + j] = (float)d;
            a.p[PTX * cap + j] = 0.f;
            a.p[PTY * cap + j] = 0.f;
            a.p[PTZ * cap + j] = 0.f;
            a.p[PW * cap + j] = -a.E[i];
        }
        carry += tot;
    }
    const int added = (int)carry < room ? (int)carry : (room > 0 ? room : 0);
    __syncthreads();
    const int mn = m + added;
    for (int64_t q = threadIdx.x; q < 10ll * mn; q += blockDim.x) {
        const int r = (int)(q / mn), j = (int)(q - (int64_t)r * mn);
        a.am[r * cap + j] = 0.f;
        a.av[r * cap + j] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if ((int)carry > room) {
            atomicOr(a.status, SERBF_FLAG_ADD_CAPACITY);
            atomicMax(a.needed + 3, (long long)(m + (int)carry));
        }
        info[2] = (int)carry;
        *a.m_dev = mn;
        a.st->m_added = added;
        a.st->adam_t = 0;
        a.st->do_add = 0;
        info[0] = 0;
    }
}

// Warps over the selected points (grid-stride): reject a point if an id_all
// point within the radius has a larger |E| (distance in float, same operation
// order as the support test, <= r2).  One block per SM, so a step without an
// addition retires few blocks.  The last block appends the survivors.
__device__ __forceinline__ void add_localmax_body(const AddArgs &A, int bx, int nbx) {
    const AppendArgs &ap = A.ap;
    const uint32_t *sel_idx = A.lo;  // the sorted selection's indices
    uint32_t *keep = A.hi2;          // scratch once the selection is sorted
    __shared__ bool s_last;
    if (!A.info[0]) return;
    const int lane = threadIdx.x & 31, nsel = A.info[1];
    for (int s = (bx * blockDim.x + threadIdx.x) >> 5; s < nsel; s += (nbx * blockDim.x) >> 5)
        localmax_one(ap.x, ap.y, ap.z, ap.E, A.mask, A.cell_start, A.g, A.sf, A.nsx, A.nsy, A.r2, A.reach, sel_idx,
                     keep, s, lane);
    if (!last_block(&A.ctl[CTL_LM_DONE], &s_last, nbx)) return;
    append_kept(ap, sel_idx, keep, nsel, A.info);
    if (threadIdx.x == 0) A.ctl[CTL_LM_DONE] = 0u;
}

__global__ void __launch_bounds__(kHistThreads) k_add_hist(AddArgs A) {
    pdl_wait();
    pdl_trigger();
    add_hist_body(A, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kGatherThreads) k_add_gather(AddArgs A) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    add_gather_body(A, blockIdx.x, gridDim.x, smem);
}

__global__ void __launch_bounds__(kLmThreads) k_add_localmax(AddArgs A) {
    pdl_wait();
    pdl_trigger();
    add_localmax_body(A, blockIdx.x, gridDim.x);
}

// Batches of fields: field blockIdx.y.
__global__ void __launch_bounds__(kHistThreads) k_add_hist_batch(const AddArgs *aa) {
    pdl_wait();
    pdl_trigger();
    add_hist_body(aa[blockIdx.y], blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kGatherThreads) k_add_gather_batch(const AddArgs *aa) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    add_gather_body(aa[blockIdx.y], blockIdx.x, gridDim.x, smem);
}

__global__ void __launch_bounds__(kLmThreads) k_add_localmax_batch(const AddArgs *aa) {
    pdl_wait();
    pdl_trigger();
    add_localmax_body(aa[blockIdx.y], blockIdx.x, gridDim.x);
}

int gather_smem() {
    return (int)(sizeof(RadixSmem) > kBitonicMax * sizeof(unsigned long long) ? sizeof(RadixSmem)
                                                                                : kBitonicMax * sizeof(unsigned long long));
}

// Dynamic shared memory of the gather kernels (once per process).
int gather_attr() {
    static bool done = false;
    if (!done) {
        if (cudaFuncSetAttribute(k_add_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, gather_smem()) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_add_gather_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, gather_smem()) !=
                cudaSuccess)
            return SERBF_ECUDA;
        done = true;
    }
    return SERBF_OK;
}

bool make_add_args(const serbf_points *pts, const float *S_raw, const float *err, const uint8_t *mask,
                   serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev, const double *stats,
                   const serbf_config *cfg, int force, serbf_workspace *ws, AddArgs &A) {
    if (!pts || !prm || !cfg || !ws || ws->magic != kMagic || !ws->binned) return false;
    if (pts->n != ws->npoints || !prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels) return false;
    if (!st_dev || !stats || !adam_m || !adam_v) return false;
    if (pts->n > 0 && (!S_raw || !err || !mask || !pts->x || !pts->y || !pts->z)) return false;
    if (!(cfg->add_radius >= 0.0) || !(cfg->eps > 0.0)) return false;
    A.E = err;
    A.mask = mask;
    A.n = pts->n;
    A.stats = stats;
    A.thresh = cfg->tau_m * 0.5;
    A.frac = cfg->topk_frac;
    A.force = force;
    A.hist = ws->sel_hist;
    A.ctl = ws->sel_ctl;
    A.info = ws->add_info;
    A.hi = ws->keys0;
    A.lo = ws->vals0;
    A.hi2 = ws->keys1;
    A.lo2 = ws->vals1;
    A.cell_start = ws->cell_start;
    A.g = ws->grid;
    A.sf = ws->sf;
    A.nsx = ws->ns[0];
    A.nsy = ws->ns[1];
    A.r2 = (float)(cfg->add_radius * cfg->add_radius);
    int reach = (int)ceil(cfg->add_radius / ws->grid.h) + 1;
    if (reach > 1 << 20) reach = 1 << 20;
    A.reach = reach;
    A.ap = AppendArgs{pts->x, pts->y, pts->z, err, S_raw, cfg->dbar_min, cfg->eps, prm->p, adam_m, adam_v,
                      prm->m, prm->cap, st_dev, ws->status, ws->needed};
    return true;
}

}  // namespace

namespace serbf {

size_t add_args_size() { return sizeof(AddArgs); }

// Host record of one field's addition for a batch (out: sizeof(AddArgs) bytes).
int batch_add_args(const serbf_points *pts, const float *S_raw, const float *err, const uint8_t *mask,
                   serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev, const double *stats,
                   const serbf_config *cfg, serbf_workspace *ws, void *out) {
    AddArgs A;
    if (!make_add_args(pts, S_raw, err, mask, prm, adam_m, adam_v, st_dev, stats, cfg, 0, ws, A)) return SERBF_EINVAL;
    memcpy(out, &A, sizeof(A));
    return SERBF_OK;
}

// The batched addition: three launches, each a no-op for fields whose
// addition is not due.
int batch_add_launch(const void *args, int nfields, int sm_count, cudaStream_t s) {
    if (gather_attr()) return SERBF_ECUDA;
    const AddArgs *aa = static_cast<const AddArgs *>(args);
    const unsigned nsm = (unsigned)(sm_count > 0 ? sm_count : 1);
    launch_pdl(k_add_hist_batch, dim3(2 * nsm, (unsigned)nfields), dim3(kHistThreads), 0, s, aa);
    launch_pdl(k_add_gather_batch, dim3(nsm, (unsigned)nfields), dim3(kGatherThreads), (size_t)gather_smem(), s, aa);
    launch_pdl(k_add_localmax_batch, dim3(nsm, (unsigned)nfields), dim3(kLmThreads), 0, s, aa);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // namespace serbf

extern "C" int serbf_add_kernels(const serbf_points *pts, const float *S_raw, const float *err, const uint8_t *mask,
                                 serbf_params *prm, float *adam_m, float *adam_v, serbf_state *st_dev,
                                 const double *stats, const serbf_config *cfg, int force, serbf_workspace *ws,
                                 void *stream) {
    SERBF_TRACE();
    AddArgs A;
    if (!make_add_args(pts, S_raw, err, mask, prm, adam_m, adam_v, st_dev, stats, cfg, force, ws, A))
        return SERBF_EINVAL;
    if (gather_attr()) return SERBF_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned nsm = (unsigned)(ws->sm_count > 0 ? ws->sm_count : 1);
    launch_pdl(k_add_hist, dim3(2 * nsm), dim3(kHistThreads), 0, s, A);
    launch_pdl(k_add_gather, dim3(nsm), dim3(kGatherThreads), (size_t)gather_smem(), s, A);
    launch_pdl(k_add_localmax, dim3(nsm), dim3(kLmThreads), 0, s, A);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
