// Per-step rebuild of the kernel <-> point neighbour structure (Eq. 3-15,
// Eq. 3-15-1): per-kernel records, super-cell and cell candidate lists (every
// list in ascending kernel index), and on request the explicit kernel-major and
// point-major CSR lists.
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

// Per-kernel records.  kfwd: (c, r2), (Q11, Q22, Q33, a), (2Q12, 2Q13, 2Q23, 0)
// with Q = log2(e) R^T D^2 R, so that exp(-||D R (v - c)||^2) = 2^(-dv^T Q dv);
// kbwd: (c, r2) and the rows of R with e_k = log2(e) d_k^2 in .w.
// R is the App. A matrix (entries r1..r9).
__global__ void k_prep(const float *p, int cap, const int32_t *m_dev, float nle, float4 *kfwd, float4 *kbwd) {
    int m = *m_dev;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        float cx = p[PCX * cap + j], cy = p[PCY * cap + j], cz = p[PCZ * cap + j];
        float d1 = p[PD1 * cap + j], d2 = p[PD2 * cap + j], d3 = p[PD3 * cap + j];
        double tx = p[PTX * cap + j], ty = p[PTY * cap + j], tz = p[PTZ * cap + j];
        float w = p[PW * cap + j];
        double sx, cxs, sy, cys, sz, czs;
        sincos(tx, &sx, &cxs);
        sincos(ty, &sy, &cys);
        sincos(tz, &sz, &czs);
        double R[9];
        R[0] = cxs * cys;
        R[1] = -czs * sx - sy * sz * cxs;
        R[2] = sx * sz - cxs * czs * sy;
        R[3] = cys * sx;
        R[4] = cxs * czs - sx * sy * sz;
        R[5] = -sz * cxs - czs * sx * sy;
        R[6] = sy;
        R[7] = cys * sz;
        R[8] = cys * czs;
        double L2E = 1.4426950408889634;
        double e[3] = {L2E * (double)d1 * d1, L2E * (double)d2 * d2, L2E * (double)d3 * d3};
        double Q[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                Q[a][b] = e[0] * R[a] * R[b] + e[1] * R[3 + a] * R[3 + b] + e[2] * R[6 + a] * R[6 + b];
        float r2 = support_r2(d1, d2, d3, nle);
        float aw = w * fabsf(w);
        kfwd[3 * j + 0] = make_float4(cx, cy, cz, r2);
        kfwd[3 * j + 1] = make_float4((float)Q[0][0], (float)Q[1][1], (float)Q[2][2], aw);
        kfwd[3 * j + 2] = make_float4((float)(2.0 * Q[0][1]), (float)(2.0 * Q[0][2]), (float)(2.0 * Q[1][2]), 0.f);
        kbwd[4 * j + 0] = make_float4(cx, cy, cz, r2);
        kbwd[4 * j + 1] = make_float4((float)R[0], (float)R[1], (float)R[2], (float)e[0]);
        kbwd[4 * j + 2] = make_float4((float)R[3], (float)R[4], (float)R[5], (float)e[1]);
        kbwd[4 * j + 3] = make_float4((float)R[6], (float)R[7], (float)R[8], (float)e[2]);
    }
}

// One block per super cell: every kernel whose support may reach the box.
__global__ void __launch_bounds__(256) k_super_lists(const float4 *kfwd, const int32_t *m_dev, const float4 *slo,
                                                     const float4 *shi, uint32_t *list, uint32_t *cnt, int cap,
                                                     int32_t *status, long long *needed) {
    __shared__ uint32_t tmp[33];
    int s = blockIdx.x;
    float4 lo = slo[s], hi = shi[s];
    if (!(lo.x <= hi.x)) {
        if (threadIdx.x == 0) cnt[s] = 0;
        return;
    }
    int m = *m_dev;
    uint32_t count = 0;
    uint32_t *out = list + (size_t)s * cap;
    for (int j0 = 0; j0 < m; j0 += 256) {
        int j = j0 + threadIdx.x;
        uint32_t hit = 0;
        if (j < m) {
            float4 k = kfwd[3 * j];
            hit = box_d2(k.x, k.y, k.z, lo, hi) < k.w;
        }
        uint32_t tot;
        uint32_t off = block_exscan(hit, tmp, &tot);
        if (hit && count + off < (uint32_t)cap) out[count + off] = (uint32_t)j;
        count += tot;
    }
    if (threadIdx.x == 0) {
        cnt[s] = count;
        if (count > (uint32_t)cap) {
            atomicOr(status, SERBF_FLAG_SUPER_LIST);
            atomicMax(needed + 0, (long long)count);
        }
    }
}

// One warp per cell: filter the super-cell list against the cell's box.
__global__ void k_cell_lists(const float4 *kfwd, const float4 *clo, const float4 *chi, int ncells, serbf_grid g,
                             int sf, int nsx, int nsy, const uint32_t *slist, const uint32_t *scnt, int scap,
                             uint32_t *list, uint32_t *cnt, int ccap, int32_t *status, long long *needed) {
    int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (c >= ncells) return;
    float4 lo = clo[c], hi = chi[c];
    if (!(lo.x <= hi.x)) {
        if (lane == 0) cnt[c] = 0;
        return;
    }
    int kx = c % g.n[0], ky = (c / g.n[0]) % g.n[1], kz = c / (g.n[0] * g.n[1]);
    int s = ((kz / sf) * nsy + ky / sf) * nsx + kx / sf;
    int L = min((int)scnt[s], scap);
    const uint32_t *in = slist + (size_t)s * scap;
    uint32_t *out = list + (size_t)c * ccap;
    uint32_t count = 0;
    for (int b = 0; b < L; b += 32) {
        int idx = b + lane;
        bool hit = false;
        uint32_t j = 0;
        if (idx < L) {
            j = in[idx];
            float4 k = kfwd[3 * j];
            hit = box_d2(k.x, k.y, k.z, lo, hi) < k.w;
        }
        unsigned bal = __ballot_sync(0xffffffffu, hit);
        uint32_t rank = __popc(bal & ((1u << lane) - 1u));
        if (hit && count + rank < (uint32_t)ccap) out[count + rank] = j;
        count += __popc(bal);
    }
    if (lane == 0) {
        cnt[c] = count;
        if (count > (uint32_t)ccap) {
            atomicOr(status, SERBF_FLAG_CELL_LIST);
            atomicMax(needed + 1, (long long)count);
        }
    }
}

// ---------------------------------------------------------------- point-major CSR
// One warp per tile; lanes are points, the cell's candidate list is walked in
// ascending kernel order, so each row comes out sorted.
template <bool FILL>
__global__ void k_pmajor(const float *x, const float *y, const float *z, const uint32_t *tile_cell,
                         const uint32_t *tile_start, const uint32_t *cell_start, int64_t ntiles,
                         const uint32_t *clist, const uint32_t *ccnt, int ccap, const float4 *kfwd,
                         int64_t *rowptr, uint32_t *col) {
    int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    uint32_t c = tile_cell[t], p0 = tile_start[t], pe = cell_start[c + 1];
    int64_t i = (int64_t)p0 + lane;
    bool valid = i < (int64_t)pe;
    float px = valid ? x[i] : __int_as_float(0x7fc00000);
    float py = valid ? y[i] : 0.f, pz = valid ? z[i] : 0.f;
    int L = min((int)ccnt[c], ccap);
    const uint32_t *lst = clist + (size_t)c * ccap;
    int64_t o = FILL && valid ? rowptr[i] : 0;
    int64_t n = 0;
    for (int s = 0; s < L; ++s) {
        uint32_t j = lst[s];
        float4 k = kfwd[3 * j];
        if (in_support(px, py, pz, k.x, k.y, k.z, k.w)) {
            if (FILL) col[o + n] = j;
            ++n;
        }
    }
    if (!FILL && valid) rowptr[i] = n;
}

// ---------------------------------------------------------------- kernel-major CSR
// One block per kernel.  Rows of cells are visited in ascending (kz, ky); within
// a row, cells and points are in ascending binned order, so each CSR row comes
// out sorted.  Elements are compacted in order with block scans.
template <bool FILL>
__global__ void __launch_bounds__(256) k_kmajor(const float *x, const float *y, const float *z,
                                                const float4 *kfwd, const int32_t *m_dev, serbf_grid g,
                                                const float4 *clo, const float4 *chi, const uint32_t *cell_start,
                                                int64_t *rowptr, uint32_t *col) {
    __shared__ uint32_t rs[256];
    __shared__ uint32_t ro[257];
    __shared__ uint32_t tmp[33];
    int j = blockIdx.x;
    int m = *m_dev;
    if (j >= m) return;
    float4 k = kfwd[3 * j];
    KBox b = kernel_box(k.x, k.y, k.z, k.w, g);
    int64_t base = FILL ? rowptr[j] : 0;
    uint32_t count = 0;
    for (int r0 = 0; r0 < b.nrows; r0 += 256) {
        int row = r0 + threadIdx.x;
        uint32_t start = 0, len = 0;
        if (row < b.nrows) {
            int c0, c1;
            row_cells(b, row, k.x, k.y, k.z, k.w, clo, chi, g, c0, c1);
            if (c0 >= 0) {
                start = cell_start[c0];
                len = cell_start[c1 + 1] - start;
            }
        }
        uint32_t total;
        uint32_t off = block_exscan(len, tmp, &total);
        rs[threadIdx.x] = start;
        ro[threadIdx.x] = off;
        if (threadIdx.x == 0) ro[256] = total;
        __syncthreads();
        for (uint32_t e0 = 0; e0 < total; e0 += 256) {
            uint32_t e = e0 + threadIdx.x;
            uint32_t hit = 0, idx = 0;
            if (e < total) {
                int lo = 0, hi = 255;
                while (lo < hi) {  // last row with ro[row] <= e
                    int mid = (lo + hi + 1) >> 1;
                    if (ro[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                idx = rs[lo] + (e - ro[lo]);
                hit = in_support(x[idx], y[idx], z[idx], k.x, k.y, k.z, k.w);
            }
            uint32_t tot;
            uint32_t o = block_exscan(hit, tmp, &tot);
            if (FILL && hit) col[base + count + o] = idx;
            count += tot;
        }
        __syncthreads();
    }
    if (!FILL && threadIdx.x == 0) rowptr[j] = count;
}

__global__ void k_zero_i64(int64_t *a, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        a[k] = 0;
}

bool ws_ok(const serbf_workspace *ws) { return ws && ws->magic == kMagic && ws->binned; }

}  // namespace

namespace serbf {
int launch_prep(const serbf_params *prm, const serbf_config *cfg, serbf_workspace *ws, cudaStream_t s) {
    float nle = (float)(-log(cfg->eps));
    int blocks = (prm->cap + 127) / 128;
    k_prep<<<blocks, 128, 0, s>>>(prm->p, prm->cap, prm->m, nle, ws->kfwd, ws->kbwd);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
}  // namespace serbf

extern "C" int serbf_build_neighbors(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                                     serbf_csr *kmajor, serbf_csr *pmajor, int64_t *npairs, serbf_workspace *ws,
                                     void *stream) {
    if (!pts || !prm || !cfg || !ws_ok(ws)) return SERBF_EINVAL;
    if (!prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels) return SERBF_EINVAL;
    if (pts->n != ws->npoints || (pts->n > 0 && (!pts->x || !pts->y || !pts->z))) return SERBF_EINVAL;
    if (!(cfg->eps > 0.0 && cfg->eps < 1.0)) return SERBF_EINVAL;
    if (kmajor && (!kmajor->rowptr || (kmajor->cap > 0 && !kmajor->col))) return SERBF_EINVAL;
    if (pmajor && (!pmajor->rowptr || (pmajor->cap > 0 && !pmajor->col))) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_prep(prm, cfg, ws, s);
    if (rc) return rc;
    k_super_lists<<<ws->nsuper, 256, 0, s>>>(ws->kfwd, prm->m, ws->sup_lo, ws->sup_hi, ws->sup_list, ws->sup_cnt,
                                              ws->sz.super_cap, ws->status, ws->needed);
    k_cell_lists<<<(unsigned)((ws->ncells * 32ll + 255) / 256), 256, 0, s>>>(
        ws->kfwd, ws->cell_lo, ws->cell_hi, ws->ncells, ws->grid, ws->sf, ws->ns[0], ws->ns[1], ws->sup_list,
        ws->sup_cnt, ws->sz.super_cap, ws->cell_list, ws->cell_cnt, ws->sz.cell_cap, ws->status, ws->needed);
    SERBF_CHECK_LAUNCH();
    if (!kmajor && !pmajor) return SERBF_OK;

    // Explicit lists: the capacity overflow of the candidate lists must be
    // excluded first, otherwise the lists would be silently incomplete.
    int32_t flags;
    rc = serbf_status(ws, &flags, nullptr, 0, stream);
    if (rc) return rc;
    int32_t m = 0;
    if (cudaMemcpyAsync(&m, prm->m, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    int64_t n = pts->n;
    int64_t total = -1;
    int result = SERBF_OK;
    if (kmajor) {
        k_zero_i64<<<1, 256, 0, s>>>(kmajor->rowptr, (int64_t)m + 1);
        if (m > 0)
            k_kmajor<false><<<m, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->kfwd, prm->m, ws->grid, ws->cell_lo,
                                              ws->cell_hi, ws->cell_start, kmajor->rowptr, nullptr);
        rc = launch_exscan_i64(kmajor->rowptr, m, s);
        if (rc) return rc;
        int64_t tot = 0;
        if (cudaMemcpyAsync(&tot, kmajor->rowptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SERBF_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
        total = tot;
        if (tot > kmajor->cap) result = SERBF_ECAPACITY;
        else if (m > 0)
            k_kmajor<true><<<m, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->kfwd, prm->m, ws->grid, ws->cell_lo,
                                             ws->cell_hi, ws->cell_start, kmajor->rowptr, kmajor->col);
        SERBF_CHECK_LAUNCH();
    }
    if (pmajor) {
        int64_t nt = ws->ntiles;
        unsigned blocks = (unsigned)((nt * 32 + 255) / 256);
        k_zero_i64<<<64, 256, 0, s>>>(pmajor->rowptr, n + 1);
        if (nt > 0)
            k_pmajor<false><<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->tile_cell, ws->tile_start,
                                                   ws->cell_start, nt, ws->cell_list, ws->cell_cnt,
                                                   ws->sz.cell_cap, ws->kfwd, pmajor->rowptr, nullptr);
        rc = launch_exscan_i64(pmajor->rowptr, n, s);
        if (rc) return rc;
        int64_t tot = 0;
        if (cudaMemcpyAsync(&tot, pmajor->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SERBF_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
        total = tot;
        if (tot > pmajor->cap) result = SERBF_ECAPACITY;
        else if (nt > 0)
            k_pmajor<true><<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, ws->tile_cell, ws->tile_start,
                                                  ws->cell_start, nt, ws->cell_list, ws->cell_cnt, ws->sz.cell_cap,
                                                  ws->kfwd, pmajor->rowptr, pmajor->col);
        SERBF_CHECK_LAUNCH();
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    if (npairs) *npairs = total;
    return result;
}
