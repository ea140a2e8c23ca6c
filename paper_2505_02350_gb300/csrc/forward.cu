// Point-major forward (Eq. 3-26) over the support pairs of Eq. 3-15-1, the
// point filter of Eq. 3-18 and the loss terms of Eq. 3-19.
//
// One warp per 32-point tile of a cell; lanes are points.  The warp walks its
// cell's candidate kernels in ascending order: their records are gathered
// from global memory with float4 loads into a per-warp shared-memory batch and
// then read back as warp-wide broadcasts, so every lane evaluates the same
// kernel at once.  Each lane applies the exact support predicate to its own
// point, so the pairs summed are exactly the point-major neighbour rows.
#include "common.cuh"

using namespace serbf;

namespace {

struct FwdArgs {
    const float *x, *y, *z, *t;
    const uint32_t *tile_cell, *tile_start, *cell_start;
    const uint32_t *clist, *ccnt;
    const float4 *kfwd;
    int64_t ntiles;
    int ccap;
    double tau1, tau2;
    float *psi, *err;
    uint8_t *mask;
    FwdPart *part;
    uint32_t *counter;
    double *stats;
};

__global__ void __launch_bounds__(kFwdWarps * 32) k_forward(FwdArgs a) {
    __shared__ float4 sk[kFwdWarps][kFwdBatch][3];
    __shared__ double s_l2[kFwdWarps];
    __shared__ float s_mx[kFwdWarps];
    __shared__ uint32_t s_cnt[kFwdWarps];
    __shared__ unsigned long long s_pairs[kFwdWarps];
    __shared__ bool s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tile = (int64_t)blockIdx.x * kFwdWarps + warp;

    double l2 = 0.0;
    float mx = 0.f;
    uint32_t cnt = 0;
    uint32_t pairs = 0;
    if (tile < a.ntiles) {
        const uint32_t cell = a.tile_cell[tile];
        const uint32_t p0 = a.tile_start[tile], pe = a.cell_start[cell + 1];
        const int64_t i = (int64_t)p0 + lane;
        const bool valid = i < (int64_t)pe;
        // invalid lanes carry NaN so the support test fails for them
        const float px = valid ? a.x[i] : __int_as_float(0x7fc00000);
        const float py = valid ? a.y[i] : 0.f;
        const float pz = valid ? a.z[i] : 0.f;
        const uint32_t *lst = a.clist + (size_t)cell * a.ccap;
        const int L = min((int)a.ccnt[cell], a.ccap);
        float acc = 0.f;
        for (int b0 = 0; b0 < L; b0 += kFwdBatch) {
            const int nb = min(kFwdBatch, L - b0);
            for (int s = lane; s < nb; s += 32) {
                const uint32_t j = lst[b0 + s];
                sk[warp][s][0] = a.kfwd[3 * j + 0];
                sk[warp][s][1] = a.kfwd[3 * j + 1];
                sk[warp][s][2] = a.kfwd[3 * j + 2];
            }
            __syncwarp();
#pragma unroll 4
            for (int s = 0; s < nb; ++s) {
                const float4 k0 = sk[warp][s][0], k1 = sk[warp][s][1], k2 = sk[warp][s][2];
                const float dx = __fsub_rn(px, k0.x), dy = __fsub_rn(py, k0.y), dz = __fsub_rn(pz, k0.z);
                const float xx = __fmul_rn(dx, dx), yy = __fmul_rn(dy, dy), zz = __fmul_rn(dz, dz);
                const bool in = __fadd_rn(__fadd_rn(xx, yy), zz) < k0.w;
                // q = dv^T Q dv (log2 units): dx (Q11 dx + 2Q12 dy + 2Q13 dz) + dy (Q22 dy + 2Q23 dz) + Q33 dz^2
                const float ra = fmaf(k2.y, dz, fmaf(k2.x, dy, k1.x * dx));
                const float rb = fmaf(k2.z, dz, k1.y * dy);
                const float q = fmaf(k1.z, zz, fmaf(dy, rb, dx * ra));
                const float phi = ex2_approx(-q);
                acc = in ? fmaf(k1.w, phi, acc) : acc;
                pairs += in;
            }
            __syncwarp();
        }
        if (valid) {
            const double t = a.t[i];
            const double ps = acc;
            const bool m0 = (a.tau1 < t) && (t < a.tau2);
            const bool m1 = (t <= a.tau1) && (ps > a.tau1);
            const bool m2 = (t >= a.tau2) && (ps < a.tau2);
            const bool mk = m0 || m1 || m2;
            const float e = mk ? __fsub_rn(acc, a.t[i]) : 0.f;
            a.psi[i] = acc;
            a.err[i] = e;
            a.mask[i] = (uint8_t)mk;
            if (mk) {
                l2 = (double)e * (double)e;
                mx = fabsf(e);
                cnt = 1;
            }
        }
    }
    // deterministic reduction: lanes -> warp -> block partial -> last block
    l2 = warp_sum(l2);
    mx = warp_max(mx);
    cnt = warp_sum(cnt);
    unsigned long long pr = warp_sum((unsigned long long)pairs);
    if (lane == 0) {
        s_l2[warp] = l2;
        s_mx[warp] = mx;
        s_cnt[warp] = cnt;
        s_pairs[warp] = pr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        FwdPart p{0.0, 0.f, 0u, 0ull};
        for (int w = 0; w < kFwdWarps; ++w) {
            p.l2 += s_l2[w];
            p.maxe = fmaxf(p.maxe, s_mx[w]);
            p.cnt += s_cnt[w];
            p.pairs += s_pairs[w];
        }
        a.part[blockIdx.x] = p;
        __threadfence();
        const uint32_t prev = atomicAdd(a.counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: fixed-order sum of all block partials
    double L2 = 0.0;
    float MX = 0.f;
    unsigned long long C = 0, P = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const FwdPart *q = a.part + b;
        L2 += __ldcg(&q->l2);
        MX = fmaxf(MX, __ldcg(&q->maxe));
        C += __ldcg(&q->cnt);
        P += __ldcg(&q->pairs);
    }
    L2 = warp_sum(L2);
    MX = warp_max(MX);
    C = warp_sum(C);
    P = warp_sum(P);
    if (lane == 0) {
        s_l2[warp] = L2;
        s_mx[warp] = MX;
        s_cnt[warp] = (uint32_t)C;
        s_pairs[warp] = P;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = 0.0;
        float m = 0.f;
        unsigned long long c = 0, pp = 0;
        for (int w = 0; w < kFwdWarps; ++w) {
            l += s_l2[w];
            m = fmaxf(m, s_mx[w]);
            c += s_cnt[w];
            pp += s_pairs[w];
        }
        a.stats[SERBF_STAT_L2] = l;
        a.stats[SERBF_STAT_MAXE] = m;
        a.stats[SERBF_STAT_COUNT] = (double)c;
        a.stats[SERBF_STAT_PAIRS_FWD] = (double)pp;
        *a.counter = 0u;
    }
}

}  // namespace

extern "C" int serbf_forward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi,
                             float *err, uint8_t *mask, double *stats, serbf_workspace *ws, void *stream) {
    if (!pts || !prm || !cfg || !ws || ws->magic != kMagic || !ws->binned) return SERBF_EINVAL;
    if (pts->n != ws->npoints || !prm->m || !prm->p) return SERBF_EINVAL;
    if (pts->n > 0 && (!pts->x || !pts->y || !pts->z || !pts->t || !psi || !err || !mask)) return SERBF_EINVAL;
    if (!stats) return SERBF_EINVAL;
    FwdArgs a;
    a.x = pts->x;
    a.y = pts->y;
    a.z = pts->z;
    a.t = pts->t;
    a.tile_cell = ws->tile_cell;
    a.tile_start = ws->tile_start;
    a.cell_start = ws->cell_start;
    a.clist = ws->cell_list;
    a.ccnt = ws->cell_cnt;
    a.kfwd = ws->kfwd;
    a.ntiles = ws->ntiles;
    a.ccap = ws->sz.cell_cap;
    a.tau1 = cfg->tau1;
    a.tau2 = cfg->tau2;
    a.psi = psi;
    a.err = err;
    a.mask = mask;
    a.part = ws->fwd_part;
    a.counter = ws->counters + 0;
    a.stats = stats;
    int64_t blocks = (ws->ntiles + kFwdWarps - 1) / kFwdWarps;
    if (blocks < 1) blocks = 1;
    k_forward<<<(unsigned)blocks, kFwdWarps * 32, 0, (cudaStream_t)stream>>>(a);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
