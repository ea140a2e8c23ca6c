// Kernel-major adjoint (App. A).  The points with a nonzero residual are first
// compacted per tile (x, y, z, E as float4, binned order).  Then one block per
// kernel walks the cell rows of its support box, gathers the compacted points
// of those rows, applies the exact support predicate (Eq. 3-15-1), recomputes
// phi and accumulates ten moments of s = phi * E in the rotated frame
// u = R (v - c):
//     S0 = sum s,   M1 = sum s u,   M2 = sum s u u^T.
// All ten App. A gradients are linear in these moments (a = w|w|):
//     dL2/dw     =  4 |w| S0
//     dL2/dd_k   = -4 a d_k (M2)_kk
//     dL2/dc     =  4 a R^T (d^2 . M1)
//     dL2/dtheta = -4 a sum_kl d_k^2 K_kl (M2)_kl,   K = (dR/dtheta) R^T,
// which is the App. A sum over pairs with Et = w^2 d^2 u F and
// (dR/dtheta) Delta = K u.  The per-kernel reduction is a warp-shuffle tree
// (double) plus a fixed-order sum over the block's warps: no global atomics.
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

__global__ void k_nz_count(const float *err, const uint32_t *tile_cell, const uint32_t *tile_start,
                           const uint32_t *cell_start, int64_t ntiles, uint32_t *tile_nz) {
    int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    uint32_t c = tile_cell[t], p0 = tile_start[t], pe = cell_start[c + 1];
    uint32_t i = p0 + lane;
    bool nz = i < pe && err[i] != 0.f;
    unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) tile_nz[t] = __popc(bal);
}

__global__ void k_nz_fill(const float *x, const float *y, const float *z, const float *err,
                          const uint32_t *tile_cell, const uint32_t *tile_start, const uint32_t *cell_start,
                          int64_t ntiles, const uint32_t *tile_off, float4 *nz) {
    int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    uint32_t c = tile_cell[t], p0 = tile_start[t], pe = cell_start[c + 1];
    uint32_t i = p0 + lane;
    float e = i < pe ? err[i] : 0.f;
    bool v = e != 0.f;
    unsigned bal = __ballot_sync(0xffffffffu, v);
    if (v) nz[tile_off[t] + __popc(bal & ((1u << lane) - 1u))] = make_float4(x[i], y[i], z[i], e);
}

struct BwdArgs {
    const float4 *kbwd;
    const float *p;
    const int32_t *m;
    int cap;
    serbf_grid g;
    const float4 *clo, *chi;
    const uint32_t *cell_tile0;
    const uint32_t *nz_off;  // per tile exclusive offsets, [ntiles] = total
    const float4 *nz;
    float *grad;
    unsigned long long *pairs;
    uint32_t *counter;
    double *stats;
    int32_t *status;
    long long *needed;
};

__device__ __forceinline__ void kadd(float &s, float &c, float v) {
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

template <bool KAHAN>
__global__ void __launch_bounds__(kBwdThreads) k_moments(BwdArgs a) {
    constexpr int NT = kBwdThreads, NW = kBwdThreads / 32;
    __shared__ uint32_t rs[NT];
    __shared__ uint32_t ro[NT + 1];
    __shared__ uint32_t tmp[33];
    __shared__ double red[NW][11];
    __shared__ bool s_last;
    const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m = *a.m;
    float acc[10], cmp[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = cmp[q] = 0.f;
    uint32_t pairs = 0;
    if (j < m) {
        const float4 k0 = a.kbwd[4 * j], k1 = a.kbwd[4 * j + 1], k2 = a.kbwd[4 * j + 2], k3 = a.kbwd[4 * j + 3];
        const KBox b = kernel_box(k0.x, k0.y, k0.z, k0.w, a.g);
        for (int r0 = 0; r0 < b.nrows; r0 += NT) {
            const int row = r0 + threadIdx.x;
            uint32_t start = 0, len = 0;
            if (row < b.nrows) {
                int c0, c1;
                row_cells(b, row, k0.x, k0.y, k0.z, k0.w, a.clo, a.chi, a.g, c0, c1);
                if (c0 >= 0) {
                    start = a.nz_off[a.cell_tile0[c0]];
                    len = a.nz_off[a.cell_tile0[c1 + 1]] - start;
                }
            }
            uint32_t total;
            const uint32_t off = block_exscan(len, tmp, &total);
            rs[threadIdx.x] = start;
            ro[threadIdx.x] = off;
            __syncthreads();
            for (uint32_t e = threadIdx.x; e < total; e += NT) {
                int lo = 0, hi = NT - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (ro[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                const float4 pt = a.nz[rs[lo] + (e - ro[lo])];
                const float dx = __fsub_rn(pt.x, k0.x), dy = __fsub_rn(pt.y, k0.y), dz = __fsub_rn(pt.z, k0.z);
                const bool in =
                    __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) < k0.w;
                const float u1 = fmaf(k1.z, dz, fmaf(k1.y, dy, k1.x * dx));
                const float u2 = fmaf(k2.z, dz, fmaf(k2.y, dy, k2.x * dx));
                const float u3 = fmaf(k3.z, dz, fmaf(k3.y, dy, k3.x * dx));
                const float q = fmaf(k3.w * u3, u3, fmaf(k2.w * u2, u2, k1.w * u1 * u1));
                const float s = in ? ex2_approx(-q) * pt.w : 0.f;
                pairs += in;
                const float s1 = s * u1, s2 = s * u2, s3 = s * u3;
                if (KAHAN) {
                    kadd(acc[0], cmp[0], s);
                    kadd(acc[1], cmp[1], s1);
                    kadd(acc[2], cmp[2], s2);
                    kadd(acc[3], cmp[3], s3);
                    kadd(acc[4], cmp[4], s1 * u1);
                    kadd(acc[5], cmp[5], s1 * u2);
                    kadd(acc[6], cmp[6], s1 * u3);
                    kadd(acc[7], cmp[7], s2 * u2);
                    kadd(acc[8], cmp[8], s2 * u3);
                    kadd(acc[9], cmp[9], s3 * u3);
                } else {
                    acc[0] += s;
                    acc[1] += s1;
                    acc[2] += s2;
                    acc[3] += s3;
                    acc[4] = fmaf(s1, u1, acc[4]);
                    acc[5] = fmaf(s1, u2, acc[5]);
                    acc[6] = fmaf(s1, u3, acc[6]);
                    acc[7] = fmaf(s2, u2, acc[7]);
                    acc[8] = fmaf(s2, u3, acc[8]);
                    acc[9] = fmaf(s3, u3, acc[9]);
                }
            }
            __syncthreads();
        }
    }
    // segmented reduction for this kernel: warp shuffles in double, then warps in order
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        double v = (double)acc[q] - (KAHAN ? (double)cmp[q] : 0.0);
        v = warp_sum(v);
        if (lane == 0) red[warp][q] = v;
    }
    const double pw = warp_sum((double)pairs);
    if (lane == 0) red[warp][10] = pw;
    __syncthreads();
    if (threadIdx.x == 0) {
        double M[11];
        for (int q = 0; q < 11; ++q) {
            M[q] = 0.0;
            for (int w = 0; w < NW; ++w) M[q] += red[w][q];
        }
        a.pairs[j] = (unsigned long long)M[10];
        if (j < m) {
            const int cap = a.cap;
            const double w = a.p[PW * cap + j];
            const double d[3] = {a.p[PD1 * cap + j], a.p[PD2 * cap + j], a.p[PD3 * cap + j]};
            const double tx = a.p[PTX * cap + j], ty = a.p[PTY * cap + j], tz = a.p[PTZ * cap + j];
            double sx, cx, sy, cy, sz, cz;
            sincos(tx, &sx, &cx);
            sincos(ty, &sy, &cy);
            sincos(tz, &sz, &cz);
            double R[9] = {cx * cy, -cz * sx - sy * sz * cx, sx * sz - cx * cz * sy,
                           cy * sx, cx * cz - sx * sy * sz, -sz * cx - cz * sx * sy,
                           sy,      cy * sz,                cy * cz};
            // derivatives of the App. A entries
            double Ry[9] = {-cx * sy, -cx * cy * sz, -cx * cy * cz, -sx * sy, -sx * cy * sz,
                            -sx * cy * cz, cy, -sy * sz, -sy * cz};
            double Rz[9] = {0.0, R[2], -R[1], 0.0, R[5], -R[4], 0.0, R[8], -R[7]};
            const double aw = w * fabs(w);
            const double S0 = M[0];
            const double M1[3] = {M[1], M[2], M[3]};
            const double M2[3][3] = {{M[4], M[5], M[6]}, {M[5], M[7], M[8]}, {M[6], M[8], M[9]}};
            double g[10];
            g[PW] = 4.0 * fabs(w) * S0;
            for (int k = 0; k < 3; ++k) g[PD1 + k] = -4.0 * aw * d[k] * M2[k][k];
            for (int k = 0; k < 3; ++k) {
                double v = 0.0;
                for (int l = 0; l < 3; ++l) v += R[3 * l + k] * d[l] * d[l] * M1[l];
                g[PCX + k] = 4.0 * aw * v;
            }
            // K = dR R^T; theta_x: K is the constant generator of the leading z-rotation
            double Kx[3][3] = {{0, -1, 0}, {1, 0, 0}, {0, 0, 0}};
            double Ky[3][3], Kz[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    Ky[r][c] = Ry[3 * r] * R[3 * c] + Ry[3 * r + 1] * R[3 * c + 1] + Ry[3 * r + 2] * R[3 * c + 2];
                    Kz[r][c] = Rz[3 * r] * R[3 * c] + Rz[3 * r + 1] * R[3 * c + 1] + Rz[3 * r + 2] * R[3 * c + 2];
                }
            double gx = 0.0, gy = 0.0, gz = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) {
                    const double f = d[r] * d[r] * M2[r][c];
                    gx += f * Kx[r][c];
                    gy += f * Ky[r][c];
                    gz += f * Kz[r][c];
                }
            g[PTX] = -4.0 * aw * gx;
            g[PTY] = -4.0 * aw * gy;
            g[PTZ] = -4.0 * aw * gz;
            for (int r = 0; r < 10; ++r) a.grad[r * cap + j] = (float)g[r];
        }
        __threadfence();
        const uint32_t prev = atomicAdd(a.counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long P = 0;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) P += __ldcg(a.pairs + q);
    P = warp_sum(P);
    if (lane == 0) red[warp][0] = (double)P;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += red[w][0];
        a.stats[SERBF_STAT_PAIRS_BWD] = t;
        *a.counter = 0u;
    }
}

}  // namespace

extern "C" int serbf_backward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                              const float *err, float *grad, double *stats, serbf_workspace *ws, void *stream) {
    if (!pts || !prm || !cfg || !ws || ws->magic != kMagic || !ws->binned) return SERBF_EINVAL;
    if (pts->n != ws->npoints || !prm->p || !prm->m || prm->cap < 1 || prm->cap > ws->sz.max_kernels)
        return SERBF_EINVAL;
    if (!grad || !stats || (pts->n > 0 && (!err || !pts->x || !pts->y || !pts->z))) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t nt = ws->ntiles;
    if (nt > 0) {
        unsigned blocks = (unsigned)((nt * 32 + 255) / 256);
        k_nz_count<<<blocks, 256, 0, s>>>(err, ws->tile_cell, ws->tile_start, ws->cell_start, nt, ws->tile_nz);
        int rc = launch_exscan_u32(ws->tile_nz, nt, s);
        if (rc) return rc;
        k_nz_fill<<<blocks, 256, 0, s>>>(pts->x, pts->y, pts->z, err, ws->tile_cell, ws->tile_start,
                                         ws->cell_start, nt, ws->tile_nz, ws->nz_pts);
    } else {
        cudaMemsetAsync(ws->tile_nz, 0, sizeof(uint32_t), s);
    }
    BwdArgs a;
    a.kbwd = ws->kbwd;
    a.p = prm->p;
    a.m = prm->m;
    a.cap = prm->cap;
    a.g = ws->grid;
    a.clo = ws->cell_lo;
    a.chi = ws->cell_hi;
    a.cell_tile0 = ws->cell_tile0;
    a.nz_off = ws->tile_nz;
    a.nz = ws->nz_pts;
    a.grad = grad;
    a.pairs = ws->bwd_pairs;
    a.counter = ws->counters + 1;
    a.stats = stats;
    a.status = ws->status;
    a.needed = ws->needed;
    if (cfg->kahan)
        k_moments<true><<<prm->cap, kBwdThreads, 0, s>>>(a);
    else
        k_moments<false><<<prm->cap, kBwdThreads, 0, s>>>(a);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
