// Point binning (the data structure behind the support test of Eq. 3-15).
//
// Cells of edge h are grouped into super cells of sf^3 cells.  Points are
// radix-sorted by (super cell, cell within the super cell, original index), so
// every super cell -- and every cell -- is a contiguous range of binned
// points.  Each super cell's range is cut into 32-point tiles (one warp each);
// tiles never straddle a super cell, so they are full except the last one of
// each super cell, and a tile's bounding box is tight.  Also the Sec. 3.4.2
// refinement entry point, which re-bins the grown training set.
#include <math.h>

#include <utility>

#include "common.cuh"

using namespace serbf;

namespace {

__global__ void k_keys(const float *x, const float *y, const float *z, int64_t n, serbf_grid g, int sf, int nsx,
                       int nsy, uint32_t *keys, uint32_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int kx = cell_axis(x[i], g.origin[0], g.h, g.n[0]);
        int ky = cell_axis(y[i], g.origin[1], g.h, g.n[1]);
        int kz = cell_axis(z[i], g.origin[2], g.h, g.n[2]);
        keys[i] = cell_key(kx, ky, kz, sf, nsx, nsy);
        vals[i] = (uint32_t)i;
    }
}

__global__ void __launch_bounds__(256) k_radix_hist(const uint32_t *keys, int64_t n, int shift, uint32_t *hist,
                                                    int64_t nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t start = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortTile / 256; ++r) {
        int64_t e = start + r * 256 + threadIdx.x;
        if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: within a block, elements keep their order per digit; blocks
// are placed in order by the digit-major exclusive scan of the histograms.
__global__ void __launch_bounds__(256) k_radix_scatter(const uint32_t *kin, const uint32_t *vin, uint32_t *kout,
                                                       uint32_t *vout, int64_t n, int shift,
                                                       const uint32_t *hist, int64_t nblk) {
    __shared__ uint32_t wcnt[8][257];
    __shared__ uint32_t run[256];
    __shared__ uint32_t base[256];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = hist[(int64_t)tid * nblk + blockIdx.x];
    run[tid] = 0;
    for (int k = tid; k < 8 * 257; k += 256) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    int64_t start = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortTile / 256; ++r) {
        int64_t e = start + r * 256 + tid;
        bool valid = e < n;
        uint32_t key = valid ? kin[e] : 0u, val = valid ? vin[e] : 0u;
        uint32_t d = valid ? (key >> shift) & 255u : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t acc = run[tid];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = acc;
            acc += c;
        }
        run[tid] = acc;
        __syncthreads();
        if (valid) {
            uint32_t pos = base[d] + wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        for (int k = tid; k < 8 * 257; k += 256) (&wcnt[0][0])[k] = 0;
        __syncthreads();
    }
}

__global__ void k_apply_perm(const uint32_t *sorted_vals, const float *x, const float *y, const float *z,
                             int64_t n, uint32_t *perm, float *xb, float *yb, float *zb) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t i = sorted_vals[k];
        perm[k] = i;
        xb[k] = x[i];
        yb[k] = y[i];
        zb[k] = z[i];
    }
}

__global__ void k_zero_u32(uint32_t *a, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        a[k] = 0u;
}

__global__ void k_count_cells(const uint32_t *keys, int64_t n, uint32_t *cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[keys[k]], 1u);
}

// tiles and forward work items per super cell (for the scans that number them)
__global__ void k_super_tiles(const uint32_t *cell_start, int nsuper, int cps, uint32_t *stile, uint32_t *sitem,
                              uint32_t *maxt, uint32_t *maxc) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsuper; s += gridDim.x * blockDim.x) {
        uint32_t b = cell_start[(int64_t)s * cps], e = cell_start[(int64_t)(s + 1) * cps];
        const uint32_t nt = (e - b + kTile - 1) / kTile;
        stile[s] = nt;
        sitem[s] = (nt + 1) / 2;
        atomicMax(maxt, nt);
        // most points in one cell of this super cell (bounds the points in a ball)
        uint32_t mc = 0, prev = b;
        for (int c = 1; c <= cps; ++c) {
            const uint32_t q = cell_start[(int64_t)s * cps + c];
            mc = max(mc, q - prev);
            prev = q;
        }
        atomicMax(maxc, mc);
    }
}

// Tiles of each super cell, and its work items: the tiles at even offsets
// (with the following tile, if any, as the item's second tile).  The first
// forward takes them in this order.
__global__ void k_fill_tiles(const uint32_t *cell_start, const uint32_t *stile0, const uint32_t *sitem0, int nsuper,
                             int cps, uint32_t *tile_super, uint32_t *tile_start, uint4 *item_rec,
                             uint4 *order_rec, uint8_t *item_class) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsuper; s += gridDim.x * blockDim.x) {
        const uint32_t t0 = stile0[s], t1 = stile0[s + 1], i0 = sitem0[s];
        const uint32_t p0 = cell_start[(int64_t)s * cps], pe = cell_start[(int64_t)(s + 1) * cps];
        for (uint32_t t = t0; t < t1; ++t) {
            const uint32_t ps = p0 + (t - t0) * kTile;
            tile_super[t] = (uint32_t)s;
            tile_start[t] = ps;
            if (((t - t0) & 1u) == 0) {
                const uint32_t it = i0 + (t - t0) / 2;
                const uint32_t np = min(pe - ps, 2u * kTile);
                const uint4 r = make_uint4(t, (uint32_t)s, ps, np | (it << 7));
                item_rec[it] = r;
                order_rec[it] = r;
                item_class[it] = 3;  // one class for all until a forward has measured them
            }
        }
    }
}

__device__ __forceinline__ void warp_box(float x, float y, float z, bool v, float4 &lo, float4 &hi) {
    float mnx = v ? x : INFINITY, mny = v ? y : INFINITY, mnz = v ? z : INFINITY;
    float mxx = v ? x : -INFINITY, mxy = v ? y : -INFINITY, mxz = v ? z : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mnz = fminf(mnz, __shfl_xor_sync(0xffffffffu, mnz, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        mxz = fmaxf(mxz, __shfl_xor_sync(0xffffffffu, mxz, o));
    }
    lo = make_float4(mnx, mny, mnz, 0.f);
    hi = make_float4(mxx, mxy, mxz, 0.f);
}

// One warp per tile: the bounding box of its points.
__global__ void k_tile_boxes(const uint32_t *tile_super, const uint32_t *tile_start, const uint32_t *cell_start,
                             int cps, int64_t ntiles, const float *xb, const float *yb, const float *zb, float4 *lo,
                             float4 *hi) {
    int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    uint32_t s = tile_super[t], p0 = tile_start[t], pe = cell_start[(int64_t)(s + 1) * cps];
    uint32_t i = p0 + lane;
    bool v = i < pe;
    float4 a, b;
    warp_box(v ? xb[i] : 0.f, v ? yb[i] : 0.f, v ? zb[i] : 0.f, v, a, b);
    if (lane == 0) {
        lo[t] = a;
        hi[t] = b;
    }
}

// One block: the union of the super-cell boxes (the box of every binned point).
__global__ void k_field_box(const float4 *slo, const float4 *shi, int nsuper, float4 *box) {
    __shared__ float red[6][32];
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int s = threadIdx.x; s < nsuper; s += blockDim.x) {
        const float4 a = slo[s], b = shi[s];
        v[0] = fminf(v[0], a.x);
        v[1] = fminf(v[1], a.y);
        v[2] = fminf(v[2], a.z);
        v[3] = fmaxf(v[3], b.x);
        v[4] = fmaxf(v[4], b.y);
        v[5] = fmaxf(v[5], b.z);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            const float w = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = k < 3 ? fminf(v[k], w) : fmaxf(v[k], w);
        }
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 6; ++k) v[k] = k < 3 ? fminf(v[k], red[k][w]) : fmaxf(v[k], red[k][w]);
        box[0] = make_float4(v[0], v[1], v[2], 0.f);
        box[1] = make_float4(v[3], v[4], v[5], 0.f);
    }
}

// One warp per super cell: union of its tile boxes (empty: +inf / -inf).
__global__ void k_super_boxes(const uint32_t *stile0, int nsuper, const float4 *tlo, const float4 *thi, float4 *slo,
                              float4 *shi) {
    int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (s >= nsuper) return;
    float mnx = INFINITY, mny = INFINITY, mnz = INFINITY, mxx = -INFINITY, mxy = -INFINITY, mxz = -INFINITY;
    for (uint32_t t = stile0[s] + lane; t < stile0[s + 1]; t += 32) {
        float4 a = tlo[t], b = thi[t];
        mnx = fminf(mnx, a.x);
        mny = fminf(mny, a.y);
        mnz = fminf(mnz, a.z);
        mxx = fmaxf(mxx, b.x);
        mxy = fmaxf(mxy, b.y);
        mxz = fmaxf(mxz, b.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mnz = fminf(mnz, __shfl_xor_sync(0xffffffffu, mnz, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        mxz = fmaxf(mxz, __shfl_xor_sync(0xffffffffu, mxz, o));
    }
    if (lane == 0) {
        slo[s] = make_float4(mnx, mny, mnz, 0.f);
        shi[s] = make_float4(mxx, mxy, mxz, 0.f);
    }
}

__global__ void k_concat(float *dst, const float *src, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

int gsz(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

}  // namespace

namespace serbf {

int radix_sort_pairs(uint32_t **k, uint32_t **v, uint32_t **ktmp, uint32_t **vtmp, int64_t n, int bits,
                     uint32_t *hist, cudaStream_t s) {
    const int64_t nblk = (n + kSortTile - 1) / kSortTile;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nblk, 256, 0, s>>>(*k, n, shift, hist, nblk);
        int rc = launch_exscan_u32(hist, 256 * nblk, s);
        if (rc) return rc;
        k_radix_scatter<<<(unsigned)nblk, 256, 0, s>>>(*k, *v, *ktmp, *vtmp, n, shift, hist, nblk);
        std::swap(*k, *ktmp);
        std::swap(*v, *vtmp);
    }
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // namespace serbf

extern "C" int serbf_bin_points(const float *x, const float *y, const float *z, int64_t n, const serbf_grid *grid,
                                uint32_t *perm, float *xb, float *yb, float *zb, serbf_workspace *ws,
                                void *stream) {
    SERBF_TRACE();
    if (!ws || ws->magic != kMagic || !grid || n < 0) return SERBF_EINVAL;
    if (n > 0 && (!x || !y || !z || !perm || !xb || !yb || !zb)) return SERBF_EINVAL;
    if (n > ws->sz.max_points) return SERBF_EINVAL;
    if (!(grid->h > 0.f) || grid->n[0] < 1 || grid->n[1] < 1 || grid->n[2] < 1) return SERBF_EINVAL;
    int64_t cells = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
    if (cells > ws->sz.max_cells) return SERBF_EINVAL;
    const int sf = ws->sz.super_factor, cps = sf * sf * sf;
    const int nsx = (grid->n[0] + sf - 1) / sf, nsy = (grid->n[1] + sf - 1) / sf, nsz = (grid->n[2] + sf - 1) / sf;
    const int64_t nsuper = (int64_t)nsx * nsy * nsz;
    if (nsuper > ws->max_supers) return SERBF_EINVAL;
    const int64_t ncp = nsuper * cps;  // cells including the padding of partial super cells
    cudaStream_t s = (cudaStream_t)stream;
    ws->grid = *grid;
    ws->sf = sf;
    ws->ns[0] = nsx;
    ws->ns[1] = nsy;
    ws->ns[2] = nsz;
    ws->nsuper = (int32_t)nsuper;
    ws->npoints = n;
    ws->binned = 0;

    uint32_t *kin = ws->keys0, *vin = ws->vals0, *kout = ws->keys1, *vout = ws->vals1;
    if (n > 0) {
        k_keys<<<gsz(n, 256), 256, 0, s>>>(x, y, z, n, *grid, sf, nsx, nsy, kin, vin);
        int nbits = 1;
        while (nbits < 32 && (1ll << nbits) < ncp) ++nbits;
        int rc = radix_sort_pairs(&kin, &vin, &kout, &vout, n, nbits, ws->hist, s);
        if (rc) return rc;
        k_apply_perm<<<gsz(n, 256), 256, 0, s>>>(vin, x, y, z, n, perm, xb, yb, zb);
    }
    k_zero_u32<<<gsz(ncp + 1, 256), 256, 0, s>>>(ws->cell_start, ncp + 1);
    if (n > 0) k_count_cells<<<gsz(n, 256), 256, 0, s>>>(kin, n, ws->cell_start);
    int rc = launch_exscan_u32(ws->cell_start, ncp, s);
    if (rc) return rc;
    uint32_t *maxt = ws->counters + 8;
    cudaMemsetAsync(maxt, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(ws->cell_max, 0, sizeof(uint32_t), s);
    k_super_tiles<<<gsz(nsuper, 256), 256, 0, s>>>(ws->cell_start, (int)nsuper, cps, ws->super_tile0,
                                                   ws->super_item0, maxt, ws->cell_max);
    rc = launch_exscan_u32(ws->super_tile0, nsuper, s);
    if (rc) return rc;
    rc = launch_exscan_u32(ws->super_item0, nsuper, s);
    if (rc) return rc;
    k_fill_tiles<<<gsz(nsuper, 256), 256, 0, s>>>(ws->cell_start, ws->super_tile0, ws->super_item0, (int)nsuper, cps,
                                                  ws->tile_super, ws->tile_start, ws->item_rec, ws->order_rec,
                                                  ws->item_class);
    SERBF_CHECK_LAUNCH();
    uint32_t nt = 0, mt = 0, ni = 0;
    if (cudaMemcpyAsync(&nt, ws->super_tile0 + nsuper, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaMemcpyAsync(&ni, ws->super_item0 + nsuper, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaMemcpyAsync(&mt, maxt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    if ((int64_t)nt > ws->max_tiles || ni >= (1u << 25)) return SERBF_ECAPACITY;  // item ids have 25 bits
    ws->nitems = ni;
    // scheduling state: no mean cost yet (the first forward files every item
    // in the same class), no counts
    if (cudaMemsetAsync(ws->sched, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaMemsetAsync(ws->sched_total, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return SERBF_ECUDA;

    ws->ntiles = nt;
    ws->max_chunks = (int32_t)((mt + kTile - 1) / kTile);
    if (nt > 0)
        k_tile_boxes<<<(unsigned)((nt * 32 + 255) / 256), 256, 0, s>>>(ws->tile_super, ws->tile_start, ws->cell_start,
                                                                        cps, nt, xb, yb, zb, ws->tile_lo, ws->tile_hi);
    k_super_boxes<<<(unsigned)((nsuper * 32 + 255) / 256), 256, 0, s>>>(ws->super_tile0, (int)nsuper, ws->tile_lo,
                                                                        ws->tile_hi, ws->sup_lo, ws->sup_hi);
    k_field_box<<<1, 256, 0, s>>>(ws->sup_lo, ws->sup_hi, (int)nsuper, ws->field_box);
    SERBF_CHECK_LAUNCH();
    ws->binned = 1;
    return SERBF_OK;
}

extern "C" int serbf_refine(float *x_all, float *y_all, float *z_all, float *t_all, float *s_all, int64_t n_old,
                            const float *x_new, const float *y_new, const float *z_new, const float *t_new,
                            const float *s_new, int64_t n_new, const serbf_grid *grid, uint32_t *perm, float *xb,
                            float *yb, float *zb, float *tb, float *sb, serbf_workspace *ws, void *stream) {
    SERBF_TRACE();
    if (!ws || ws->magic != kMagic || n_old < 0 || n_new < 0) return SERBF_EINVAL;
    if (!x_all || !y_all || !z_all || !t_all || !s_all || !tb || !sb) return SERBF_EINVAL;
    if (n_new > 0 && (!x_new || !y_new || !z_new || !t_new || !s_new)) return SERBF_EINVAL;
    int64_t n = n_old + n_new;
    if (n > ws->sz.max_points) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_new > 0) {
        k_concat<<<gsz(n_new, 256), 256, 0, s>>>(x_all + n_old, x_new, n_new);
        k_concat<<<gsz(n_new, 256), 256, 0, s>>>(y_all + n_old, y_new, n_new);
        k_concat<<<gsz(n_new, 256), 256, 0, s>>>(z_all + n_old, z_new, n_new);
        k_concat<<<gsz(n_new, 256), 256, 0, s>>>(t_all + n_old, t_new, n_new);
        k_concat<<<gsz(n_new, 256), 256, 0, s>>>(s_all + n_old, s_new, n_new);
        SERBF_CHECK_LAUNCH();
    }
    int rc = serbf_bin_points(x_all, y_all, z_all, n, grid, perm, xb, yb, zb, ws, stream);
    if (rc) return rc;
    rc = serbf_gather(t_all, perm, tb, n, stream);
    if (rc) return rc;
    return serbf_gather(s_all, perm, sb, n, stream);
}
