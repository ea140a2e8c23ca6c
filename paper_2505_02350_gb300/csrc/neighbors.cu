// Per-step rebuild of the kernel <-> point neighbour structure (Eq. 3-15,
// Eq. 3-15-1): per-kernel records and, per super cell, the list of kernels
// (ascending index) whose support may reach it.  The forward and the adjoint
// refine these lists against tight 32-point tile boxes and apply the exact
// support predicate per pair.  On request the explicit kernel-major and
// point-major CSR lists are produced from the same structure.
#include <math.h>
#include <string.h>

#include "common.cuh"

using namespace serbf;

namespace {

// Per-kernel records.  kfwd: (c, r2), (Q11, Q22, Q33, a), (2Q12, 2Q13, 2Q23, 0)
// with Q = log2(e) R^T D^2 R, so that exp(-||D R (v - c)||^2) = 2^(-dv^T Q dv);
// kbwd: (c, r2) and the rows of R with e_k = log2(e) d_k^2 in .w.
// R is the App. A matrix (entries r1..r9).
__device__ __forceinline__ void prep_kernels(const float *p, int cap, int m, float nle, float4 *kfwd, float4 *kbwd,
                                             int first, int stride) {
    for (int j = first; j < m; j += stride) {
        float cx = p[PCX * cap + j], cy = p[PCY * cap + j], cz = p[PCZ * cap + j];
        float d1 = p[PD1 * cap + j], d2 = p[PD2 * cap + j], d3 = p[PD3 * cap + j];
        float w = p[PW * cap + j];
        float sx, cxs, sy, cys, sz, czs;
        sincosf(p[PTX * cap + j], &sx, &cxs);
        sincosf(p[PTY * cap + j], &sy, &cys);
        sincosf(p[PTZ * cap + j], &sz, &czs);
        float R[9];
        R[0] = cxs * cys;
        R[1] = -czs * sx - sy * sz * cxs;
        R[2] = sx * sz - cxs * czs * sy;
        R[3] = cys * sx;
        R[4] = cxs * czs - sx * sy * sz;
        R[5] = -sz * cxs - czs * sx * sy;
        R[6] = sy;
        R[7] = cys * sz;
        R[8] = cys * czs;
        const float e[3] = {kLog2e * d1 * d1, kLog2e * d2 * d2, kLog2e * d3 * d3};
        float Q[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Q[a][b] = fmaf(e[0] * R[a], R[b], fmaf(e[1] * R[3 + a], R[3 + b], e[2] * R[6 + a] * R[6 + b]));
        float r2 = support_r2(d1, d2, d3, nle);
        float aw = w * fabsf(w);
        kfwd[3 * j + 0] = make_float4(cx, cy, cz, r2);
        kfwd[3 * j + 1] = make_float4(Q[0][0], Q[1][1], Q[2][2], aw);
        kfwd[3 * j + 2] = make_float4(2.f * Q[0][1], 2.f * Q[0][2], 2.f * Q[1][2], 0.f);
        kbwd[4 * j + 0] = make_float4(cx, cy, cz, r2);
        kbwd[4 * j + 1] = make_float4(R[0], R[1], R[2], e[0]);
        kbwd[4 * j + 2] = make_float4(R[3], R[4], R[5], e[1]);
        kbwd[4 * j + 3] = make_float4(R[6], R[7], R[8], e[2]);
    }
}

// The forward's heavy-first order for its next launch: a stable sort of the
// items by the cost class the last forward filed, descending, in two
// launches on the workspace's side stream (next to the neighbour rebuild).
// k_class_count: block b counts the classes of items [b kOrderChunk,
// (b + 1) kOrderChunk).  k_order_items: block b places the same items; a
// class starts after all heavier classes and after this class in earlier
// chunks, and the rank inside the chunk comes from ballots in item order.
__device__ __forceinline__ void class_count_body(const uint8_t *item_class, int64_t nitems, uint32_t *hist, int bx) {
    constexpr int NW = kOrderChunk / 32;
    __shared__ uint32_t s_wcnt[NW][kCostClasses];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)bx * kOrderChunk + threadIdx.x;
    const int cls = i < nitems ? (int)item_class[i] : -1;
#pragma unroll
    for (int c = 0; c < kCostClasses; ++c) {
        const unsigned bal = __ballot_sync(0xffffffffu, cls == c);
        if (lane == 0) s_wcnt[warp][c] = __popc(bal);
    }
    __syncthreads();
    if (threadIdx.x < kCostClasses) {
        uint32_t t = 0;
        for (int w = 0; w < NW; ++w) t += s_wcnt[w][threadIdx.x];
        hist[(size_t)bx * kCostClasses + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kOrderChunk) k_class_count(const uint8_t *item_class, int64_t nitems,
                                                             uint32_t *hist) {
    class_count_body(item_class, nitems, hist, blockIdx.x);
}

__device__ __forceinline__ void order_items_body(const uint8_t *item_class, const uint32_t *hist,
                                                 const uint4 *item_rec, uint4 *order_rec, int64_t nitems, int bx) {
    constexpr int NW = kOrderChunk / 32;
    __shared__ uint32_t s_base[kCostClasses];      // first position of each class for this chunk
    __shared__ uint32_t s_tot[kCostClasses];
    __shared__ uint32_t s_wcnt[NW][kCostClasses];  // per warp: class counts, then offsets
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nchunks = (int)((nitems + kOrderChunk - 1) / kOrderChunk), b = bx;
    // class totals and this class's count in earlier chunks: warp c handles class c
    if (warp < kCostClasses) {
        uint32_t tot = 0, before = 0;
        for (int q = lane; q < nchunks; q += 32) {
            const uint32_t v = hist[(size_t)q * kCostClasses + warp];
            tot += v;
            before += q < b ? v : 0u;
        }
        tot = warp_sum(tot);
        before = warp_sum(before);
        if (lane == 0) {
            s_tot[warp] = tot;
            s_base[warp] = before;
        }
    }
    const int64_t i = (int64_t)b * kOrderChunk + threadIdx.x;
    const int cls = i < nitems ? (int)item_class[i] : -1;
    const uint4 r = i < nitems ? item_rec[i] : make_uint4(0u, 0u, 0u, 0u);
    uint32_t rank = 0;
#pragma unroll
    for (int c = 0; c < kCostClasses; ++c) {
        const unsigned bal = __ballot_sync(0xffffffffu, cls == c);
        if (cls == c) rank = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) s_wcnt[warp][c] = __popc(bal);
    }
    __syncthreads();
    if (threadIdx.x < kCostClasses) {
        const int c = threadIdx.x;
        uint32_t heavier = 0;  // classes are placed in descending order
        for (int q = c + 1; q < kCostClasses; ++q) heavier += s_tot[q];
        uint32_t run = heavier + s_base[c];
        for (int w = 0; w < NW; ++w) {
            const uint32_t v = s_wcnt[w][c];
            s_wcnt[w][c] = run;
            run += v;
        }
    }
    __syncthreads();
    if (cls >= 0) order_rec[s_wcnt[warp][cls] + rank] = r;
}

__global__ void __launch_bounds__(kOrderChunk) k_order_items(const uint8_t *item_class, const uint32_t *hist,
                                                             const uint4 *item_rec, uint4 *order_rec, int64_t nitems) {
    order_items_body(item_class, hist, item_rec, order_rec, nitems, blockIdx.x);
}

// The per-step rebuild in one launch: blocks [0, nsuper) list, per super
// cell, every kernel whose support may reach its box (centre and r2 taken
// from the parameters with the same float operations as the records); the
// remaining blocks write the per-kernel records.
__device__ __forceinline__ void rebuild_body(const float *p, int cap, const int32_t *m_dev, float nle, float4 *kfwd,
                                             float4 *kbwd, const float4 *slo, const float4 *shi, int nsuper,
                                             uint32_t *list, uint32_t *cnt, int scap, int32_t *status,
                                             long long *needed, int bx, int nbx) {
    __shared__ uint32_t tmp[33];
    const int m = *m_dev;
    const int s = bx;
    if (s >= nsuper) {
        prep_kernels(p, cap, m, nle, kfwd, kbwd, (s - nsuper) * blockDim.x + threadIdx.x,
                     (nbx - nsuper) * blockDim.x);
        return;
    }
    const float4 lo = slo[s], hi = shi[s];
    if (!(lo.x <= hi.x)) {
        if (threadIdx.x == 0) cnt[s] = 0;
        return;
    }
    uint32_t count = 0;
    uint32_t *out = list + (size_t)s * scap;
    for (int j0 = 0; j0 < m; j0 += 256) {
        const int j = j0 + threadIdx.x;
        uint32_t hit = 0;
        if (j < m) {
            const float r2 = support_r2(p[PD1 * cap + j], p[PD2 * cap + j], p[PD3 * cap + j], nle);
            hit = box_d2(p[PCX * cap + j], p[PCY * cap + j], p[PCZ * cap + j], lo, hi) < r2;
        }
        uint32_t tot;
        const uint32_t off = block_exscan(hit, tmp, &tot);
        if (hit && count + off < (uint32_t)scap) out[count + off] = (uint32_t)j;
        count += tot;
    }
    if (threadIdx.x == 0) {
        cnt[s] = count;
        if (count > (uint32_t)scap) {
            atomicOr(status, SERBF_FLAG_SUPER_LIST);
            atomicMax(needed + 0, (long long)count);
        }
    }
}

__global__ void __launch_bounds__(256) k_rebuild(const float *p, int cap, const int32_t *m_dev, float nle,
                                                 float4 *kfwd, float4 *kbwd, const float4 *slo, const float4 *shi,
                                                 int nsuper, uint32_t *list, uint32_t *cnt, int scap, int32_t *status,
                                                 long long *needed) {
    pdl_wait();
    pdl_trigger();
    rebuild_body(p, cap, m_dev, nle, kfwd, kbwd, slo, shi, nsuper, list, cnt, scap, status, needed, blockIdx.x,
                 gridDim.x);
}

// Two-level rebuild, for many super cells and kernels.  First launch: blocks
// [0, ncoarse) list, per block of f x f x f super cells (f = 2; 4 for the
// first of three levels), every kernel whose support may reach the union of
// their boxes (as k_rebuild does per super cell); the remaining blocks write
// the per-kernel records.
__device__ __forceinline__ void coarse_lists_body(const float *p, int cap, const int32_t *m_dev, float nle,
                                                  float4 *kfwd, float4 *kbwd, const float4 *slo, const float4 *shi,
                                                  int nsx, int nsy, int nsz, int ncoarse, uint32_t *list,
                                                  uint32_t *cnt, int scap, int bx, int nbx, int f) {
    __shared__ uint32_t tmp[33];
    __shared__ float4 s_lo, s_hi;
    const int m = *m_dev;
    const int c = bx;
    if (c >= ncoarse) {
        prep_kernels(p, cap, m, nle, kfwd, kbwd, (c - ncoarse) * blockDim.x + threadIdx.x,
                     (nbx - ncoarse) * blockDim.x);
        return;
    }
    if (threadIdx.x == 0) {
        const int ncx = (nsx + f - 1) / f, ncy = (nsy + f - 1) / f;
        const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
        float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f), hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        for (int dz = 0; dz < f; ++dz)
            for (int dy = 0; dy < f; ++dy)
                for (int dx = 0; dx < f; ++dx) {
                    const int sx = f * cx + dx, sy = f * cy + dy, sz = f * cz + dz;
                    if (sx >= nsx || sy >= nsy || sz >= nsz) continue;
                    const int sc = (sz * nsy + sy) * nsx + sx;
                    const float4 a = slo[sc], b = shi[sc];
                    lo = make_float4(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, a.z), 0.f);
                    hi = make_float4(fmaxf(hi.x, b.x), fmaxf(hi.y, b.y), fmaxf(hi.z, b.z), 0.f);
                }
        s_lo = lo;
        s_hi = hi;
    }
    __syncthreads();
    const float4 lo = s_lo, hi = s_hi;
    if (!(lo.x <= hi.x)) {
        if (threadIdx.x == 0) cnt[c] = 0;
        return;
    }
    uint32_t count = 0;
    uint32_t *out = list + (size_t)c * scap;
    for (int j0 = 0; j0 < m; j0 += 256) {
        const int j = j0 + threadIdx.x;
        uint32_t hit = 0;
        if (j < m) {
            const float r2 = support_r2(p[PD1 * cap + j], p[PD2 * cap + j], p[PD3 * cap + j], nle);
            hit = box_d2(p[PCX * cap + j], p[PCY * cap + j], p[PCZ * cap + j], lo, hi) < r2;
        }
        uint32_t tot;
        const uint32_t off = block_exscan(hit, tmp, &tot);
        if (hit && count + off < (uint32_t)scap) out[count + off] = (uint32_t)j;
        count += tot;
    }
    if (threadIdx.x == 0) cnt[c] = count;
}

__global__ void __launch_bounds__(256) k_coarse_lists(const float *p, int cap, const int32_t *m_dev, float nle,
                                                      float4 *kfwd, float4 *kbwd, const float4 *slo,
                                                      const float4 *shi, int nsx, int nsy, int nsz, int ncoarse,
                                                      uint32_t *list, uint32_t *cnt, int scap, int f) {
    pdl_wait();
    pdl_trigger();
    coarse_lists_body(p, cap, m_dev, nle, kfwd, kbwd, slo, shi, nsx, nsy, nsz, ncoarse, list, cnt, scap, blockIdx.x,
                      gridDim.x, f);
}

// Middle of three levels: each block of 2 x 2 x 2 super cells keeps the
// kernels of its parent's list (blocks of 4 x 4 x 4 super cells) that reach
// its own box, tested with the records' centre and r2; a parent list that
// overflowed is not used (every kernel is tested).  A kernel that reaches a
// box reaches every box containing it, so the lists equal the one-level ones
// filtered to these blocks.
__device__ __forceinline__ void mid_lists_body(const int32_t *m_dev, const float4 *kfwd, const float4 *slo,
                                               const float4 *shi, int nsx, int nsy, int nsz, int nmid,
                                               const uint32_t *plist, const uint32_t *pcnt, uint32_t *list,
                                               uint32_t *cnt, int scap, int bx) {
    __shared__ uint32_t tmp[33];
    __shared__ float4 s_lo, s_hi;
    const int c = bx;
    if (c >= nmid) return;
    const int ncx = (nsx + 1) >> 1, ncy = (nsy + 1) >> 1;
    const int cx = c % ncx, cy = (c / ncx) % ncy, cz = c / (ncx * ncy);
    if (threadIdx.x == 0) {
        float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f), hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int sx = 2 * cx + dx, sy = 2 * cy + dy, sz = 2 * cz + dz;
                    if (sx >= nsx || sy >= nsy || sz >= nsz) continue;
                    const int sc = (sz * nsy + sy) * nsx + sx;
                    const float4 a = slo[sc], b = shi[sc];
                    lo = make_float4(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, a.z), 0.f);
                    hi = make_float4(fmaxf(hi.x, b.x), fmaxf(hi.y, b.y), fmaxf(hi.z, b.z), 0.f);
                }
        s_lo = lo;
        s_hi = hi;
    }
    __syncthreads();
    const float4 lo = s_lo, hi = s_hi;
    if (!(lo.x <= hi.x)) {
        if (threadIdx.x == 0) cnt[c] = 0;
        return;
    }
    const int npx = (nsx + 3) >> 2, npy = (nsy + 3) >> 2;
    const int pc = ((cz >> 1) * npy + (cy >> 1)) * npx + (cx >> 1);
    const uint32_t pn = pcnt[pc];
    const bool whole = pn > (uint32_t)scap;  // the parent's list overflowed
    const int L = whole ? *m_dev : (int)pn;
    const uint32_t *src = plist + (size_t)pc * scap;
    uint32_t count = 0;
    uint32_t *out = list + (size_t)c * scap;
    for (int q0 = 0; q0 < L; q0 += 256) {
        const int q = q0 + threadIdx.x;
        uint32_t hit = 0, j = 0;
        if (q < L) {
            j = whole ? (uint32_t)q : src[q];
            const float4 k = kfwd[3 * j];
            hit = box_d2(k.x, k.y, k.z, lo, hi) < k.w;
        }
        uint32_t tot;
        const uint32_t off = block_exscan(hit, tmp, &tot);
        if (hit && count + off < (uint32_t)scap) out[count + off] = j;
        count += tot;
    }
    if (threadIdx.x == 0) cnt[c] = count;
}

__global__ void __launch_bounds__(256) k_mid_lists(const int32_t *m_dev, const float4 *kfwd, const float4 *slo,
                                                   const float4 *shi, int nsx, int nsy, int nsz, int nmid,
                                                   const uint32_t *plist, const uint32_t *pcnt, uint32_t *list,
                                                   uint32_t *cnt, int scap) {
    pdl_wait();
    pdl_trigger();
    mid_lists_body(m_dev, kfwd, slo, shi, nsx, nsy, nsz, nmid, plist, pcnt, list, cnt, scap, blockIdx.x);
}

// Second launch: each super cell keeps the kernels of its block's list that
// reach its own box, with the centre and r2 of the records (the values
// k_rebuild computes), so the lists equal the one-level ones: a kernel that
// reaches a super cell's box reaches the block's box, which contains it.  A
// block list that overflowed is not used: its super cells test every kernel.
__device__ __forceinline__ void fine_lists_body(const int32_t *m_dev, const float4 *kfwd, const float4 *slo,
                                                const float4 *shi, int nsx, int nsy, int nsuper, const uint32_t *clist,
                                                const uint32_t *ccnt, uint32_t *list, uint32_t *cnt, int scap,
                                                int32_t *status, long long *needed, int bx) {
    __shared__ uint32_t tmp[33];
    const int s = bx;
    if (s >= nsuper) return;
    const float4 lo = slo[s], hi = shi[s];
    if (!(lo.x <= hi.x)) {
        if (threadIdx.x == 0) cnt[s] = 0;
        return;
    }
    const int sx = s % nsx, sy = (s / nsx) % nsy, sz = s / (nsx * nsy);
    const int ncx = (nsx + 1) >> 1, ncy = (nsy + 1) >> 1;
    const int c = ((sz >> 1) * ncy + (sy >> 1)) * ncx + (sx >> 1);
    const uint32_t cc = ccnt[c];
    const bool whole = cc > (uint32_t)scap;  // the block's list overflowed
    const int L = whole ? *m_dev : (int)cc;
    const uint32_t *src = clist + (size_t)c * scap;
    uint32_t count = 0;
    uint32_t *out = list + (size_t)s * scap;
    for (int q0 = 0; q0 < L; q0 += 256) {
        const int q = q0 + threadIdx.x;
        uint32_t hit = 0, j = 0;
        if (q < L) {
            j = whole ? (uint32_t)q : src[q];
            const float4 k = kfwd[3 * j];
            hit = box_d2(k.x, k.y, k.z, lo, hi) < k.w;
        }
        uint32_t tot;
        const uint32_t off = block_exscan(hit, tmp, &tot);
        if (hit && count + off < (uint32_t)scap) out[count + off] = j;
        count += tot;
    }
    if (threadIdx.x == 0) {
        cnt[s] = count;
        if (count > (uint32_t)scap) {
            atomicOr(status, SERBF_FLAG_SUPER_LIST);
            atomicMax(needed + 0, (long long)count);
        }
    }
}

__global__ void __launch_bounds__(256) k_fine_lists(const int32_t *m_dev, const float4 *kfwd, const float4 *slo,
                                                    const float4 *shi, int nsx, int nsy, int nsuper,
                                                    const uint32_t *clist, const uint32_t *ccnt, uint32_t *list,
                                                    uint32_t *cnt, int scap, int32_t *status, long long *needed) {
    pdl_wait();
    pdl_trigger();
    fine_lists_body(m_dev, kfwd, slo, shi, nsx, nsy, nsuper, clist, ccnt, list, cnt, scap, status, needed,
                    blockIdx.x);
}

// ---------------------------------------------------------------- batches of fields
// One field's neighbour rebuild for the batched epoch: the arguments of the
// single-field launches, and which form (one or two levels) it takes.
struct RebuildArgs {
    const float *p;
    int cap;
    const int32_t *m_dev;
    float nle;
    float4 *kfwd, *kbwd;
    const float4 *slo, *shi;
    int nsx, nsy, nsz, nsuper, ncoarse;
    uint32_t *list, *cnt, *clist, *ccnt;
    int scap;
    int two_level;
    int32_t *status;
    long long *needed;
    int level1_blocks;                 // blocks this field uses in the first launch
    const uint8_t *item_class;         // heavy-first order of the forward's items
    uint32_t *class_hist;
    const uint4 *item_rec;
    uint4 *order_rec;
    int64_t nitems;
};

// Field blockIdx.y: the item order for the next forward (two launches).
__global__ void __launch_bounds__(kOrderChunk) k_class_count_batch(const RebuildArgs *ra) {
    const RebuildArgs &r = ra[blockIdx.y];
    if ((int64_t)blockIdx.x * kOrderChunk >= r.nitems) return;
    class_count_body(r.item_class, r.nitems, r.class_hist, blockIdx.x);
}

__global__ void __launch_bounds__(kOrderChunk) k_order_items_batch(const RebuildArgs *ra) {
    const RebuildArgs &r = ra[blockIdx.y];
    if ((int64_t)blockIdx.x * kOrderChunk >= r.nitems) return;
    order_items_body(r.item_class, r.class_hist, r.item_rec, r.order_rec, r.nitems, blockIdx.x);
}

// First rebuild launch: one-level fields rebuild, two-level fields list the
// kernels of their blocks of 2 x 2 x 2 super cells; both write the records.
__global__ void __launch_bounds__(256) k_rebuild_batch(const RebuildArgs *ra) {
    pdl_wait();
    pdl_trigger();
    const RebuildArgs &r = ra[blockIdx.y];
    if ((int)blockIdx.x >= r.level1_blocks) return;
    if (r.two_level)
        coarse_lists_body(r.p, r.cap, r.m_dev, r.nle, r.kfwd, r.kbwd, r.slo, r.shi, r.nsx, r.nsy, r.nsz, r.ncoarse,
                          r.clist, r.ccnt, r.scap, blockIdx.x, r.level1_blocks, 2);
    else
        rebuild_body(r.p, r.cap, r.m_dev, r.nle, r.kfwd, r.kbwd, r.slo, r.shi, r.nsuper, r.list, r.cnt, r.scap,
                     r.status, r.needed, blockIdx.x, r.level1_blocks);
}

// Second rebuild launch: the super-cell lists of two-level fields.
__global__ void __launch_bounds__(256) k_fine_lists_batch(const RebuildArgs *ra) {
    pdl_wait();
    pdl_trigger();
    const RebuildArgs &r = ra[blockIdx.y];
    if (!r.two_level || (int)blockIdx.x >= r.nsuper) return;
    fine_lists_body(r.m_dev, r.kfwd, r.slo, r.shi, r.nsx, r.nsy, r.nsuper, r.clist, r.ccnt, r.list, r.cnt, r.scap,
                    r.status, r.needed, blockIdx.x);
}

// ---------------------------------------------------------------- point-major CSR
// One warp per tile; lanes are points.  The super cell's list is walked in
// ascending kernel order (entries whose support misses the tile box are
// skipped), so each row comes out sorted.
template <bool FILL>
__global__ void k_pmajor(const float *x, const float *y, const float *z, const uint32_t *tile_super,
                         const uint32_t *tile_start, const float4 *tlo, const float4 *thi, const uint32_t *cell_start,
                         int cps, int64_t ntiles, const uint32_t *slist, const uint32_t *scnt, int scap,
                         const float4 *kfwd, int64_t *rowptr, uint32_t *col) {
    int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    uint32_t s = tile_super[t], p0 = tile_start[t], pe = cell_start[(int64_t)(s + 1) * cps];
    int64_t i = (int64_t)p0 + lane;
    bool valid = i < (int64_t)pe;
    float px = valid ? x[i] : __int_as_float(0x7fc00000);
    float py = valid ? y[i] : 0.f, pz = valid ? z[i] : 0.f;
    float4 lo = tlo[t], hi = thi[t];
    int L = min((int)scnt[s], scap);
    const uint32_t *lst = slist + (size_t)s * scap;
    int64_t o = FILL && valid ? rowptr[i] : 0;
    int64_t n = 0;
    for (int q = 0; q < L; ++q) {
        uint32_t j = lst[q];
        float4 k = kfwd[3 * j];
        if (!(box_d2(k.x, k.y, k.z, lo, hi) < k.w)) continue;
        if (in_support(px, py, pz, k.x, k.y, k.z, k.w)) {
            if (FILL) col[o + n] = j;
            ++n;
        }
    }
    if (!FILL && valid) rowptr[i] = n;
}

// ---------------------------------------------------------------- kernel-major CSR
// One warp per kernel.  Super cells are visited in ascending id, their tiles in
// ascending order and each tile's points in order, which is ascending binned
// index, so each CSR row comes out sorted.
template <bool FILL>
__global__ void k_kmajor(const float *x, const float *y, const float *z, const float4 *kfwd, const int32_t *m_dev,
                         serbf_grid g, int sf, int nsx, int nsy, const float4 *slo, const float4 *shi,
                         const uint32_t *stile0, const uint32_t *tile_start, const float4 *tlo, const float4 *thi,
                         const uint32_t *cell_start, int cps, int64_t *rowptr, uint32_t *col) {
    int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= *m_dev) return;
    float4 k = kfwd[3 * j];
    KBox b = kernel_box(k.x, k.y, k.z, k.w, g);
    int64_t base = FILL ? rowptr[j] : 0;
    uint32_t count = 0;
    for (int sz = b.kz0 / sf; sz <= b.kz1 / sf; ++sz)
        for (int sy = b.ky0 / sf; sy <= b.ky1 / sf; ++sy)
            for (int sx = b.kx0 / sf; sx <= b.kx1 / sf; ++sx) {
                int s = (sz * nsy + sy) * nsx + sx;
                if (!(box_d2(k.x, k.y, k.z, slo[s], shi[s]) < k.w)) continue;
                uint32_t pe_s = cell_start[(int64_t)(s + 1) * cps];
                for (uint32_t t = stile0[s]; t < stile0[s + 1]; ++t) {
                    if (!(box_d2(k.x, k.y, k.z, tlo[t], thi[t]) < k.w)) continue;
                    uint32_t i = tile_start[t] + lane;
                    bool hit = i < pe_s && in_support(x[i], y[i], z[i], k.x, k.y, k.z, k.w);
                    unsigned bal = __ballot_sync(0xffffffffu, hit);
                    if (FILL && hit) col[base + count + __popc(bal & ((1u << lane) - 1u))] = i;
                    count += __popc(bal);
                }
            }
    if (!FILL && lane == 0) rowptr[j] = count;
}

__global__ void k_zero_i64(int64_t *a, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        a[k] = 0;
}

bool ws_ok(const serbf_workspace *ws) { return ws && ws->magic == kMagic && ws->binned; }

// Two levels when asked, or by default once super cells x kernel capacity
// reaches 2^25 box tests: measured, the 256^3 band workload (4913 super
// cells, capacity 32768) rebuilds 4x faster in two levels, while the 128^3
// one (729, 8192) is slower by the extra launch.
bool rebuild_two_level(int levels, int64_t nsuper, int cap) {
    return levels >= 2 || (levels == 0 && nsuper * (int64_t)cap >= (int64_t)1 << 25);
}

// Three levels (blocks of 4 x 4 x 4 super cells against every kernel, then
// blocks of 2 x 2 x 2, then super cells) when asked, or by default once the
// second level alone would make 2^25 box tests: measured, the 256^3 band
// with super cells of 2 x 2 x 2 cells (4913 blocks of 2 x 2 x 2, capacity
// 32768) rebuilds in a fraction of its two-level time.  Single fields only;
// the batched epoch takes two levels.
bool rebuild_three_level(int levels, int64_t ncoarse, int cap) {
    return levels == 3 || (levels == 0 && ncoarse * (int64_t)cap >= (int64_t)1 << 25);
}

}  // namespace

namespace serbf {
}  // namespace serbf

namespace serbf {

size_t rebuild_args_size() { return sizeof(RebuildArgs); }

// Host record of one field's neighbour rebuild for a batch (out:
// sizeof(RebuildArgs) bytes); *level1_blocks, *chunks and *nsuper size the
// batch's grids, *two_level says which form the field takes.
int batch_rebuild_args(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                       serbf_workspace *ws, void *out, int *level1_blocks, int64_t *chunks, int *nsuper,
                       int *two_level) {
    if (!pts || !prm || !cfg || !ws_ok(ws)) return SERBF_EINVAL;
    if (!prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels) return SERBF_EINVAL;
    if (pts->n != ws->npoints) return SERBF_EINVAL;
    if (!(cfg->eps > 0.0 && cfg->eps < 1.0) || cfg->rebuild_levels < 0 || cfg->rebuild_levels > 3) return SERBF_EINVAL;
    RebuildArgs r;
    memset(&r, 0, sizeof(r));
    const int nsx = ws->ns[0], nsy = ws->ns[1], nsz = ws->ns[2];
    const int64_t ncoarse = (int64_t)((nsx + 1) / 2) * ((nsy + 1) / 2) * ((nsz + 1) / 2);
    const int prep_blocks = (prm->cap + 255) / 256;
    r.p = prm->p;
    r.cap = prm->cap;
    r.m_dev = prm->m;
    r.nle = (float)(-log(cfg->eps));
    r.kfwd = ws->kfwd;
    r.kbwd = ws->kbwd;
    r.slo = ws->sup_lo;
    r.shi = ws->sup_hi;
    r.nsx = nsx;
    r.nsy = nsy;
    r.nsz = nsz;
    r.nsuper = ws->nsuper;
    r.ncoarse = (int)ncoarse;
    r.list = ws->sup_list;
    r.cnt = ws->sup_cnt;
    r.clist = ws->crs_list;
    r.ccnt = ws->crs_cnt;
    r.scap = ws->sz.super_cap;
    r.two_level = rebuild_two_level(cfg->rebuild_levels, ws->nsuper, prm->cap) && ncoarse <= ws->max_coarse;
    r.status = ws->status;
    r.needed = ws->needed;
    r.level1_blocks = (r.two_level ? (int)ncoarse : ws->nsuper) + prep_blocks;
    r.item_class = ws->item_class;
    r.class_hist = ws->class_hist;
    r.item_rec = ws->item_rec;
    r.order_rec = ws->order_rec;
    r.nitems = ws->nitems;
    memcpy(out, &r, sizeof(r));
    *level1_blocks = r.level1_blocks;
    *chunks = (ws->nitems + kOrderChunk - 1) / kOrderChunk;
    *nsuper = ws->nsuper;
    *two_level = r.two_level;
    return SERBF_OK;
}

// The batched rebuild: item order (two launches), then the lists and
// records (one launch, two when some field takes two levels).
int batch_rebuild_launch(const void *args, int nfields, int level1_blocks, int64_t chunks, int nsuper, int two_level,
                         cudaStream_t s) {
    const RebuildArgs *ra = static_cast<const RebuildArgs *>(args);
    if (chunks > 0) {
        k_class_count_batch<<<dim3((unsigned)chunks, (unsigned)nfields), kOrderChunk, 0, s>>>(ra);
        k_order_items_batch<<<dim3((unsigned)chunks, (unsigned)nfields), kOrderChunk, 0, s>>>(ra);
    }
    launch_pdl(k_rebuild_batch, dim3((unsigned)level1_blocks, (unsigned)nfields), dim3(256), 0, s, ra);
    if (two_level) launch_pdl(k_fine_lists_batch, dim3((unsigned)nsuper, (unsigned)nfields), dim3(256), 0, s, ra);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // namespace serbf

extern "C" int serbf_build_neighbors(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                                     serbf_csr *kmajor, serbf_csr *pmajor, int64_t *npairs, serbf_workspace *ws,
                                     void *stream) {
    SERBF_TRACE();
    if (!pts || !prm || !cfg || !ws_ok(ws)) return SERBF_EINVAL;
    if (!prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels) return SERBF_EINVAL;
    if (pts->n != ws->npoints || (pts->n > 0 && (!pts->x || !pts->y || !pts->z))) return SERBF_EINVAL;
    if (!(cfg->eps > 0.0 && cfg->eps < 1.0)) return SERBF_EINVAL;
    if (cfg->rebuild_levels < 0 || cfg->rebuild_levels > 3) return SERBF_EINVAL;
    if (kmajor && (!kmajor->rowptr || (kmajor->cap > 0 && !kmajor->col))) return SERBF_EINVAL;
    if (pmajor && (!pmajor->rowptr || (pmajor->cap > 0 && !pmajor->col))) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // fork: the item order for the next forward overlaps the rebuild
    const bool fork = ws->nitems > 0 && ws->aux;
    if (fork) {
        if (cudaEventRecord(ws->ev_fork, s) != cudaSuccess) return SERBF_ECUDA;
        if (cudaStreamWaitEvent(ws->aux, ws->ev_fork, 0) != cudaSuccess) return SERBF_ECUDA;
        const unsigned nchunks = (unsigned)((ws->nitems + kOrderChunk - 1) / kOrderChunk);
        k_class_count<<<nchunks, kOrderChunk, 0, ws->aux>>>(ws->item_class, ws->nitems, ws->class_hist);
        k_order_items<<<nchunks, kOrderChunk, 0, ws->aux>>>(ws->item_class, ws->class_hist, ws->item_rec,
                                                            ws->order_rec, ws->nitems);
        SERBF_CHECK_LAUNCH();
        if (cudaEventRecord(ws->ev_join, ws->aux) != cudaSuccess) return SERBF_ECUDA;
    }
    {
        const float nle = (float)(-log(cfg->eps));
        const int prep_blocks = (prm->cap + 255) / 256;
        const int nsx = ws->ns[0], nsy = ws->ns[1], nsz = ws->ns[2];
        const int64_t ncoarse = (int64_t)((nsx + 1) / 2) * ((nsy + 1) / 2) * ((nsz + 1) / 2);
        const int64_t ntop = (int64_t)((nsx + 3) / 4) * ((nsy + 3) / 4) * ((nsz + 3) / 4);
        if (rebuild_two_level(cfg->rebuild_levels, ws->nsuper, prm->cap) && ncoarse <= ws->max_coarse) {
            if (rebuild_three_level(cfg->rebuild_levels, ncoarse, prm->cap) && ntop <= ws->nsuper) {
                // blocks of 4 x 4 x 4 super cells against every kernel (their
                // lists and counts held in the super cells' storage, which the
                // last level rewrites), then blocks of 2 x 2 x 2
                launch_pdl(k_coarse_lists, dim3((unsigned)(ntop + prep_blocks)), dim3(256), 0, s,
                           (const float *)prm->p, prm->cap, (const int32_t *)prm->m, nle, ws->kfwd, ws->kbwd,
                           (const float4 *)ws->sup_lo, (const float4 *)ws->sup_hi, nsx, nsy, nsz, (int)ntop,
                           ws->sup_list, ws->sup_cnt, ws->sz.super_cap, 4);
                launch_pdl(k_mid_lists, dim3((unsigned)ncoarse), dim3(256), 0, s, (const int32_t *)prm->m,
                           (const float4 *)ws->kfwd, (const float4 *)ws->sup_lo, (const float4 *)ws->sup_hi, nsx, nsy,
                           nsz, (int)ncoarse, (const uint32_t *)ws->sup_list, (const uint32_t *)ws->sup_cnt,
                           ws->crs_list, ws->crs_cnt, ws->sz.super_cap);
            } else {
                launch_pdl(k_coarse_lists, dim3((unsigned)(ncoarse + prep_blocks)), dim3(256), 0, s,
                           (const float *)prm->p, prm->cap, (const int32_t *)prm->m, nle, ws->kfwd, ws->kbwd,
                           (const float4 *)ws->sup_lo, (const float4 *)ws->sup_hi, nsx, nsy, nsz, (int)ncoarse,
                           ws->crs_list, ws->crs_cnt, ws->sz.super_cap, 2);
            }
            launch_pdl(k_fine_lists, dim3(ws->nsuper), dim3(256), 0, s, (const int32_t *)prm->m,
                       (const float4 *)ws->kfwd, (const float4 *)ws->sup_lo, (const float4 *)ws->sup_hi, nsx, nsy,
                       ws->nsuper, (const uint32_t *)ws->crs_list, (const uint32_t *)ws->crs_cnt, ws->sup_list,
                       ws->sup_cnt, ws->sz.super_cap, ws->status, ws->needed);
        } else {
            launch_pdl(k_rebuild, dim3(ws->nsuper + prep_blocks), dim3(256), 0, s, (const float *)prm->p, prm->cap,
                       (const int32_t *)prm->m, nle, ws->kfwd, ws->kbwd, (const float4 *)ws->sup_lo,
                       (const float4 *)ws->sup_hi, ws->nsuper, ws->sup_list, ws->sup_cnt, ws->sz.super_cap,
                       ws->status, ws->needed);
        }
    }
    int rc = SERBF_OK;
    SERBF_CHECK_LAUNCH();
    // join the side stream
    if (fork && cudaStreamWaitEvent(s, ws->ev_join, 0) != cudaSuccess) return SERBF_ECUDA;
    if (!kmajor && !pmajor) return SERBF_OK;

    // Explicit lists: an overflowing candidate list would make them silently
    // incomplete, so the status is checked first.
    int32_t flags;
    rc = serbf_status(ws, &flags, nullptr, 0, stream);
    if (rc) return rc;
    int32_t m = 0;
    if (cudaMemcpyAsync(&m, prm->m, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    const int cps = ws->sf * ws->sf * ws->sf;
    int64_t n = pts->n;
    int64_t total = -1;
    int result = SERBF_OK;
    if (kmajor) {
        unsigned blocks = (unsigned)(((int64_t)m * 32 + 255) / 256);
        k_zero_i64<<<1, 256, 0, s>>>(kmajor->rowptr, (int64_t)m + 1);
        if (m > 0)
            k_kmajor<false><<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->kfwd, prm->m, ws->grid, ws->sf,
                                                   ws->ns[0], ws->ns[1], ws->sup_lo, ws->sup_hi, ws->super_tile0,
                                                   ws->tile_start, ws->tile_lo, ws->tile_hi, ws->cell_start, cps,
                                                   kmajor->rowptr, nullptr);
        rc = launch_exscan_i64(kmajor->rowptr, m, s);
        if (rc) return rc;
        int64_t tot = 0;
        if (cudaMemcpyAsync(&tot, kmajor->rowptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SERBF_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
        total = tot;
        if (tot > kmajor->cap) result = SERBF_ECAPACITY;
        else if (m > 0)
            k_kmajor<true><<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->kfwd, prm->m, ws->grid, ws->sf,
                                                  ws->ns[0], ws->ns[1], ws->sup_lo, ws->sup_hi, ws->super_tile0,
                                                  ws->tile_start, ws->tile_lo, ws->tile_hi, ws->cell_start, cps,
                                                  kmajor->rowptr, kmajor->col);
        SERBF_CHECK_LAUNCH();
    }
    if (pmajor) {
        int64_t nt = ws->ntiles;
        unsigned blocks = (unsigned)((nt * 32 + 255) / 256);
        k_zero_i64<<<64, 256, 0, s>>>(pmajor->rowptr, n + 1);
        if (nt > 0)
            k_pmajor<false><<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->tile_super, ws->tile_start,
                                                   ws->tile_lo, ws->tile_hi, ws->cell_start, cps, nt, ws->sup_list,
                                                   ws->sup_cnt, ws->sz.super_cap, ws->kfwd, pmajor->rowptr, nullptr);
        rc = launch_exscan_i64(pmajor->rowptr, n, s);
        if (rc) return rc;
        int64_t tot = 0;
        if (cudaMemcpyAsync(&tot, pmajor->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SERBF_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
        total = tot;
        if (tot > pmajor->cap) result = SERBF_ECAPACITY;
        else if (nt > 0)
            k_pmajor<true><<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->tile_super, ws->tile_start,
                                                  ws->tile_lo, ws->tile_hi, ws->cell_start, cps, nt, ws->sup_list,
                                                  ws->sup_cnt, ws->sz.super_cap, ws->kfwd, pmajor->rowptr,
                                                  pmajor->col);
        SERBF_CHECK_LAUNCH();
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    if (npairs) *npairs = total;
    return result;
}
