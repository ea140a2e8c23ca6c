// Kernel-major adjoint (App. A).  The points with a nonzero residual are first
// compacted within their tile (x, y, z, E as float4 in the tile's 32 slots).
// Then one block per kernel: its warps visit the super cells of the support
// box, keep the tiles whose box the support reaches and that hold nonzero
// residuals, queue those points in a per-warp shared-memory ring, and process
// them 32 at a time: exact support predicate (Eq. 3-15-1), phi recomputed, and
// ten moments of s = phi * E accumulated in the rotated frame u = R (v - c):
//     S0 = sum s,   M1 = sum s u,   M2 = sum s u u^T.
// All ten App. A gradients are linear in these moments (a = w|w|):
//     dL2/dw     =  4 |w| S0
//     dL2/dd_k   = -4 a d_k (M2)_kk
//     dL2/dc     =  4 a R^T (d^2 . M1)
//     dL2/dtheta = -4 a sum_kl d_k^2 K_kl (M2)_kl,   K = (dR/dtheta) R^T
//     (theta_x: K is constant and the sum is (d_2^2 - d_1^2) (M2)_12),
// which is the App. A sum over pairs with Et = w^2 d^2 u F and
// (dR/dtheta) Delta = K u.  The per-kernel reduction is a float-float
// warp-shuffle tree plus fixed-order sums over warps and over the kernel's
// kBwdSplit blocks: no global atomics.
#include <math.h>

#include "common.cuh"

using namespace serbf;

static_assert(kBwdWarpsPerKernel == 32, "the epilogue reduces one partial per lane");

namespace {

// One block per (32-tile chunk, super cell), one warp per tile: compact the
// tile's nonzero-residual points into its 32 slots (x, y, z, E), then warp 0
// packs the chunk's tiles that hold any as two float4 records -- (box lo,
// count) and (box hi, tile id) -- at the chunk's own record slots, so the
// adjoint reads a candidate tile's test data in one round trip.
__global__ void __launch_bounds__(1024) k_nz_compact(const float *x, const float *y, const float *z, const float *err,
                                                     const uint32_t *stile0, const uint32_t *tile_start,
                                                     const uint32_t *cell_start, int cps, const float4 *tlo,
                                                     const float4 *thi, float4 *nz, float4 *rec, uint32_t *ccnt) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t cnt[32];
    const int s = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t t0 = stile0[s], t1 = stile0[s + 1];
    const uint32_t cb = t0 + blockIdx.x * 32u;
    if (cb >= t1) return;
    const uint32_t t = cb + warp;
    uint32_t c = 0;
    if (t < t1) {
        const uint32_t pe = cell_start[(int64_t)(s + 1) * cps];
        const uint32_t i = tile_start[t] + lane;
        const float e = i < pe ? err[i] : 0.f;
        const bool v = e != 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (v) nz[(size_t)t * kTile + __popc(bal & ((1u << lane) - 1u))] = make_float4(x[i], y[i], z[i], e);
        c = __popc(bal);
    }
    if (lane == 0) cnt[warp] = c;
    __syncthreads();
    if (warp != 0) return;
    const uint32_t tt = cb + lane;
    const uint32_t cl = cnt[lane];
    const unsigned bal = __ballot_sync(0xffffffffu, cl != 0);
    if (cl) {
        const uint32_t o = cb + __popc(bal & ((1u << lane) - 1u));
        float4 lo = tlo[tt], hi = thi[tt];
        lo.w = __uint_as_float(cl);
        hi.w = __uint_as_float(tt);
        rec[2 * (size_t)o] = lo;
        rec[2 * (size_t)o + 1] = hi;
    }
    if (lane == 0) ccnt[cb] = __popc(bal);
}

struct BwdArgs {
    const float4 *kbwd;
    const int32_t *m;
    int cap;
    serbf_grid g;
    int sf, nsx, nsy;
    const float4 *slo, *shi;
    const uint32_t *stile0;
    const float4 *tlo, *thi;
    const float4 *nzrec;   // packed records of tiles with nonzero residuals, per 32-tile chunk
    const uint32_t *nzc;   // records per chunk, indexed by the chunk's first tile
    const float4 *nz;
    float *mom;  // per kernel, per warp: 10 float-float moments S0, M1 (3), M2 (6), then the pair count (bits)
};

template <bool KAHAN>
__global__ void __launch_bounds__(kBwdThreads) k_moments(BwdArgs a) {
    pdl_wait();
    pdl_trigger();
    constexpr int NW = kBwdThreads / 32;
    constexpr int RING = 2 * kQueue;  // two points per lane in flight
    __shared__ uint32_t ring[NW][RING];
    const int j = blockIdx.x, split = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = *a.m;
    if (j >= m) return;
    float acc[10], cmp[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = cmp[q] = 0.f;
    uint32_t pairs = 0;
    const float4 k0 = a.kbwd[4 * j], k1 = a.kbwd[4 * j + 1], k2 = a.kbwd[4 * j + 2], k3 = a.kbwd[4 * j + 3];
    const KBox b = kernel_box(k0.x, k0.y, k0.z, k0.w, a.g);
    const int sx0 = b.kx0 / a.sf, sy0 = b.ky0 / a.sf, sz0 = b.kz0 / a.sf;
    const int nbx = b.kx1 / a.sf - sx0 + 1, nby = b.ky1 / a.sf - sy0 + 1, nbz = b.kz1 / a.sf - sz0 + 1;
    const int nsb = nbx * nby * nbz;
    int head = 0, qn = 0;
    uint32_t *q = ring[warp];
    // the kernel's super cells are dealt round-robin to all its warps; a warp
    // tests 32 of its super cells at once (one per lane), then walks the hit
    // ones and their packed nonzero tiles
    const int W = NW * gridDim.y, wid = split * NW + warp;
    for (int base = wid; base < nsb; base += W * 32) {
        const int sb = base + lane * W;
        uint32_t t0 = 0, nt = 0;
        unsigned long long packed = 0;  // chunk counts (6 bits each) of the first 8 chunks
        if (sb < nsb) {
            const int sx = sx0 + sb % nbx, sy = sy0 + (sb / nbx) % nby, sz = sz0 + sb / (nbx * nby);
            const int s = (sz * a.nsy + sy) * a.nsx + sx;
            if (box_d2(k0.x, k0.y, k0.z, a.slo[s], a.shi[s]) < k0.w) {
                t0 = a.stile0[s];
                nt = a.stile0[s + 1] - t0;  // tiles of the super cell
                const uint32_t nch = (nt + 31) / 32;
                for (uint32_t q8 = 0; q8 < 8 && q8 < nch; ++q8)
                    packed |= (unsigned long long)a.nzc[t0 + 32u * q8] << (6 * q8);
                if (!packed && nch <= 8) nt = 0;  // no nonzero tile at all
            }
        }
        unsigned sbal = __ballot_sync(0xffffffffu, nt != 0);
        while (sbal) {
            const int ssrc = __ffs(sbal) - 1;
            sbal &= sbal - 1;
            const uint32_t st0 = __shfl_sync(0xffffffffu, t0, ssrc), snt = __shfl_sync(0xffffffffu, nt, ssrc);
            const unsigned long long spk = __shfl_sync(0xffffffffu, packed, ssrc);
            // the super cell's 32-tile chunks: the first 8 counts came with the
            // super cell's test, later ones are loaded 32 at a time
            const uint32_t nch = (snt + 31) / 32;
            for (uint32_t cg = 0; cg < nch; cg += 32) {
            uint32_t cc_l = 0;
            if (cg + lane < nch)
                cc_l = (cg + lane < 8) ? (uint32_t)((spk >> (6 * (cg + lane))) & 63ull) : a.nzc[st0 + 32u * (cg + lane)];
            unsigned cbal = __ballot_sync(0xffffffffu, cc_l != 0);
            while (cbal) {
                const int csrc = __ffs(cbal) - 1;
                cbal &= cbal - 1;
                const uint32_t cb = st0 + 32u * (cg + csrc), ncr = __shfl_sync(0xffffffffu, cc_l, csrc);
                uint32_t c = 0, t = 0;
                if ((uint32_t)lane < ncr) {
                    const float4 lo = a.nzrec[2 * (size_t)(cb + lane)], hi = a.nzrec[2 * (size_t)(cb + lane) + 1];
                    if (box_d2(k0.x, k0.y, k0.z, lo, hi) < k0.w) {
                        c = __float_as_uint(lo.w);
                        t = __float_as_uint(hi.w);
                    }
                }
                unsigned bal = __ballot_sync(0xffffffffu, c != 0);
                while (bal) {
                    const int src = __ffs(bal) - 1;
                    bal &= bal - 1;
                    const uint32_t cc = __shfl_sync(0xffffffffu, c, src);
                    const uint32_t tt = __shfl_sync(0xffffffffu, t, src);
                    if (lane < (int)cc) q[(head + qn + lane) & (RING - 1)] = tt * kTile + lane;
                    qn += cc;
                    __syncwarp();
                    if (qn >= 64) {
                        const float4 p0 = a.nz[q[(head + lane) & (RING - 1)]];
                        const float4 p1 = a.nz[q[(head + 32 + lane) & (RING - 1)]];
                        accumulate<KAHAN>(p0, k0, k1, k2, k3, acc, cmp, pairs);
                        accumulate<KAHAN>(p1, k0, k1, k2, k3, acc, cmp, pairs);
                        head = (head + 64) & (RING - 1);
                        qn -= 64;
                        __syncwarp();
                    }
                }
            }
            }
        }
    }
    if (lane < qn) accumulate<KAHAN>(a.nz[q[(head + lane) & (RING - 1)]], k0, k1, k2, k3, acc, cmp, pairs);
    if (lane + 32 < qn) accumulate<KAHAN>(a.nz[q[(head + 32 + lane) & (RING - 1)]], k0, k1, k2, k3, acc, cmp, pairs);
    // this warp's share of the kernel's moments, written to the warp's slot
    // (no atomics, no block barrier); the lanes are combined with a plain
    // float shuffle tree, or a float-float one in the compensated mode
    const int slot = split * NW + warp;  // < gridDim.y * NW <= kBwdWarpsPerKernel
    float *o = a.mom + ((int64_t)j * kBwdWarpsPerKernel + slot) * 22;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        ff v;
        if (KAHAN) {
            v = warp_sum_ff(two_sum(acc[r], -cmp[r]));
        } else {
            v = ff{warp_sum(acc[r]), 0.f};
        }
        if (lane == 0) {
            o[2 * r] = v.hi;
            o[2 * r + 1] = v.lo;
        }
    }
    const uint32_t pw = warp_sum(pairs);
    if (lane == 0) o[20] = __uint_as_float(pw);
}

// One warp per kernel: the kBwdWarpsPerKernel partial moments are summed in a
// fixed order (float-float shuffle tree), then lane 0 evaluates the ten App. A
// gradients; the pair count total is a fixed-order sum by the last block.
__global__ void k_grad_epilogue(const float *p, const int32_t *m_dev, int cap, const float *mom, int nparts,
                                float *grad, unsigned long long *pairs, uint32_t *counter, double *stats) {
    pdl_wait();
    pdl_trigger();
    __shared__ bool s_last;
    __shared__ unsigned long long red[32];
    const int m = *m_dev;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j < m) {
        const float *o = mom + ((int64_t)j * kBwdWarpsPerKernel + lane) * 22;
        const bool has = lane < nparts;
        float M[10];
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const ff v = warp_sum_ff(has ? ff{o[2 * r], o[2 * r + 1]} : ff{0.f, 0.f});
            M[r] = v.hi + v.lo;
        }
        const uint32_t np = warp_sum(has ? __float_as_uint(o[20]) : 0u);
        if (lane == 0) {
            pairs[j] = np;
            grad_from_moments(p, cap, j, M, grad);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long t = 0;
    for (int q = threadIdx.x; q < m; q += blockDim.x) t += __ldcg(pairs + q);
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sum = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        stats[SERBF_STAT_PAIRS_BWD] = (double)sum;
        *counter = 0u;
    }
}

}  // namespace

extern "C" int serbf_backward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                              const float *err, float *grad, double *stats, serbf_workspace *ws, void *stream) {
    SERBF_TRACE();
    if (!pts || !prm || !cfg || !ws || ws->magic != kMagic || !ws->binned) return SERBF_EINVAL;
    if (pts->n != ws->npoints || !prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels)
        return SERBF_EINVAL;
    if (!grad || !stats || (pts->n > 0 && (!err || !pts->x || !pts->y || !pts->z))) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nt = ws->ntiles;
    const int cps = ws->sf * ws->sf * ws->sf;
    if (nt > 0)
        launch_pdl(k_nz_compact, dim3((unsigned)ws->max_chunks, (unsigned)ws->nsuper), dim3(1024), 0, s,
            pts->x, pts->y, pts->z, err, ws->super_tile0, ws->tile_start, ws->cell_start, cps, ws->tile_lo,
            ws->tile_hi, ws->nz, ws->nzrec, ws->nzc_cnt);
    BwdArgs a;
    a.kbwd = ws->kbwd;
    a.m = prm->m;
    a.cap = prm->cap;
    a.g = ws->grid;
    a.sf = ws->sf;
    a.nsx = ws->ns[0];
    a.nsy = ws->ns[1];
    a.slo = ws->sup_lo;
    a.shi = ws->sup_hi;
    a.stile0 = ws->super_tile0;
    a.tlo = ws->tile_lo;
    a.thi = ws->tile_hi;
    a.nzrec = ws->nzrec;
    a.nzc = ws->nzc_cnt;
    a.nz = ws->nz;
    a.mom = ws->moments;
    // enough warps in flight: split a kernel's super cells over more blocks when
    // there are few kernels, fewer when there are many (each split adds a
    // per-warp reduction of ten moments)
    int splits = (int)(20480 / ((int64_t)prm->cap * (kBwdThreads / 32)));
    splits = splits < 1 ? 1 : (splits > kBwdSplit ? kBwdSplit : splits);
    const dim3 grid((unsigned)prm->cap, (unsigned)splits);
    if (cfg->kahan)
        launch_pdl(k_moments<true>, dim3(grid), dim3(kBwdThreads), 0, s, a);
    else
        launch_pdl(k_moments<false>, dim3(grid), dim3(kBwdThreads), 0, s, a);
    launch_pdl(k_grad_epilogue, dim3((prm->cap + 7) / 8), dim3(256), 0, s, prm->p, prm->m, prm->cap, ws->moments,
                                                        splits * (kBwdThreads / 32), grad,
                                                           ws->bwd_pairs, ws->counters + 1, stats);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
