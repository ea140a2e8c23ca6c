// Point-major forward (Eq. 3-26) over the support pairs of Eq. 3-15-1, the
// point filter of Eq. 3-18 and the loss terms of Eq. 3-19.
//
// One warp per 32-point tile; lanes are points.  The warp streams its super
// cell's candidate list (ascending kernel index), keeps the kernels whose
// support reaches the tile's bounding box (one candidate per lane, ballot),
// and gathers their records with float4 loads into a per-warp shared-memory
// ring.  Each full batch of 32 staged kernels is then evaluated with warp-wide
// broadcast reads: every lane applies the exact support predicate to its own
// point, so the pairs summed are exactly the point-major neighbour rows, in
// ascending kernel order.
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

struct FwdArgs {
    const float *x, *y, *z, *t;
    const uint32_t *tile_super, *tile_start, *cell_start;
    const float4 *tile_lo, *tile_hi;
    const uint32_t *slist, *scnt;
    const float4 *kfwd;
    int64_t ntiles;
    int scap, cps;
    float tau1, tau2;  // tau1 rounded down, tau2 rounded up to float: exact double decisions
    float *psi, *err;
    uint8_t *mask;
    FwdPart *part;        // one partial per tile
    FwdPart *gpart;       // one partial per group of kFwdGroup tiles
    uint32_t *group_done; // tiles finished per group
    uint32_t *counter;    // groups finished
    uint32_t *tile_next;  // next tile to take (zeroed before each launch)
    double *stats;
};

// Squared distance from c to the farthest corner of a box, rounded so that
// it is never below the float squared distance of any point inside the box:
// box_far_d2 < r2 means every point of the box is in the support.
__device__ __forceinline__ float box_far_d2(float cx, float cy, float cz, float4 lo, float4 hi) {
    const float ax = fmaxf(__fsub_rn(cx, lo.x), __fsub_rn(hi.x, cx));
    const float ay = fmaxf(__fsub_rn(cy, lo.y), __fsub_rn(hi.y, cy));
    const float az = fmaxf(__fsub_rn(cz, lo.z), __fsub_rn(hi.z, cz));
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
}

// Up to 32 kernels whose support only partly covers the tile: exact predicate per lane.
template <int UNROLL>
__device__ __forceinline__ void eval_partial(const float4 (*ring)[3], int cnt, float px, float py, float pz,
                                            float &acc, uint32_t &n) {
#pragma unroll UNROLL
    for (int q = 0; q < cnt; ++q) {
        {
            const float4 k0 = ring[q][0], k1 = ring[q][1], k2 = ring[q][2];
            const float dx = __fsub_rn(px, k0.x), dy = __fsub_rn(py, k0.y), dz = __fsub_rn(pz, k0.z);
            const float xx = __fmul_rn(dx, dx), yy = __fmul_rn(dy, dy), zz = __fmul_rn(dz, dz);
            const bool in = __fadd_rn(__fadd_rn(xx, yy), zz) < k0.w;
            // q = dv^T Q dv (log2 units): dx (Q11 dx + 2Q12 dy + 2Q13 dz) + dy (Q22 dy + 2Q23 dz) + Q33 dz^2
            const float ra = fmaf(k2.y, dz, fmaf(k2.x, dy, k1.x * dx));
            const float rb = fmaf(k2.z, dz, k1.y * dy);
            const float qv = fmaf(k1.z, zz, fmaf(dy, rb, dx * ra));
            const float phi = ex2_approx(-qv);
            acc = in ? fmaf(k1.w, phi, acc) : acc;
            n += in;
        }
    }
}

// Up to 32 kernels whose support covers the whole tile box: no predicate needed.
template <int UNROLL>
__device__ __forceinline__ void eval_full(const float4 (*ring)[3], int cnt, float px, float py, float pz,
                                         float &acc) {
#pragma unroll UNROLL
    for (int q = 0; q < cnt; ++q) {
        {
            const float4 k0 = ring[q][0], k1 = ring[q][1], k2 = ring[q][2];
            const float dx = px - k0.x, dy = py - k0.y, dz = pz - k0.z;
            const float ra = fmaf(k2.y, dz, fmaf(k2.x, dy, k1.x * dx));
            const float rb = fmaf(k2.z, dz, k1.y * dy);
            const float qv = fmaf(k1.z, dz * dz, fmaf(dy, rb, dx * ra));
            acc = fmaf(k1.w, ex2_approx(-qv), acc);
        }
    }
}

struct TileOut {
    float l2, mx;
    uint32_t cnt, pairs;
};

// One tile (32 binned points) on one warp: stream the super cell's candidate
// list, stage the kernels that reach the tile box, evaluate, write psi, E and
// the mask.  Returns this lane's loss contributions.
__device__ __forceinline__ TileOut forward_tile(const FwdArgs &a, int64_t tile, float4 (*ringP)[3],
                                                float4 (*ringF)[3], int lane) {
    TileOut out{0.f, 0.f, 0u, 0u};
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t sup = a.tile_super[tile];
    const uint32_t p0 = a.tile_start[tile], pe = a.cell_start[(int64_t)(sup + 1) * a.cps];
    const int64_t i = (int64_t)p0 + lane;
    const bool valid = i < (int64_t)pe;
    // invalid lanes carry NaN so the support test fails for them
    const float px = valid ? a.x[i] : __int_as_float(0x7fc00000);
    const float py = valid ? a.y[i] : 0.f;
    const float pz = valid ? a.z[i] : 0.f;
    const float4 lo = a.tile_lo[tile], hi = a.tile_hi[tile];
    const uint32_t *lst = a.slist + (size_t)sup * a.scap;
    const int L = min((int)a.scnt[sup], a.scap);
    int hp = 0, qp = 0, hf = 0, qf = 0;
    uint32_t nfull = 0, np = 0;
    float acc = 0.f;
    uint32_t jn = lane < L ? lst[lane] : 0u;
    for (int b = 0; b < L; b += 32) {
        const uint32_t j = jn;
        const bool live = b + lane < L;
        if (b + 32 + lane < L) jn = lst[b + 32 + lane];  // prefetch the next chunk
        bool part = false, full = false;
        float4 k0;
        if (live) {
            k0 = a.kfwd[3 * j];
            if (box_d2(k0.x, k0.y, k0.z, lo, hi) < k0.w) {
                full = box_far_d2(k0.x, k0.y, k0.z, lo, hi) < k0.w;
                part = !full;
            }
        }
        const unsigned bp = __ballot_sync(0xffffffffu, part), bf = __ballot_sync(0xffffffffu, full);
        if (part || full) {
            float4(*ring)[3] = part ? ringP : ringF;
            const int slot = part ? ((hp + qp + __popc(bp & lt)) & (kQueue - 1))
                                  : ((hf + qf + __popc(bf & lt)) & (kQueue - 1));
            ring[slot][0] = k0;
            ring[slot][1] = a.kfwd[3 * j + 1];
            ring[slot][2] = a.kfwd[3 * j + 2];
        }
        qp += __popc(bp);
        qf += __popc(bf);
        __syncwarp();
        if (qp >= 32) {
            eval_partial<8>(ringP + hp, 32, px, py, pz, acc, np);
            hp ^= 32;
            qp -= 32;
        }
        if (qf >= 32) {
            eval_full<8>(ringF + hf, 32, px, py, pz, acc);
            hf ^= 32;
            qf -= 32;
            nfull += 32;
        }
        __syncwarp();
    }
    // leftovers: head is 0 or 32 and fewer than 32 remain, so they do not wrap
    if (qp > 0) eval_partial<1>(ringP + hp, qp, px, py, pz, acc, np);
    if (qf > 0) {
        eval_full<1>(ringF + hf, qf, px, py, pz, acc);
        nfull += qf;
    }
    __syncwarp();
    if (valid) {
        out.pairs = np + nfull;
        const float t = a.t[i], ps = acc;
        const bool m0 = (a.tau1 < t) && (t < a.tau2);
        const bool m1 = (t <= a.tau1) && (ps > a.tau1);
        const bool m2 = (t >= a.tau2) && (ps < a.tau2);
        const bool mk = m0 || m1 || m2;
        const float e = mk ? __fsub_rn(ps, t) : 0.f;
        a.psi[i] = ps;
        a.err[i] = e;
        a.mask[i] = (uint8_t)mk;
        if (mk) {
            out.l2 = e * e;
            out.mx = fabsf(e);
            out.cnt = 1;
        }
    }
    return out;
}

// Fixed-order warp reduction of tile partials [b, e) into one partial.
__device__ __forceinline__ FwdPart reduce_parts(const FwdPart *p, uint32_t b, uint32_t e, int lane) {
    ff l{0.f, 0.f};
    float mx = 0.f;
    unsigned long long c = 0, pr = 0;
    for (uint32_t q = b + lane; q < e; q += 32) {
        l = ff_add(l, ff{__ldcg(&p[q].l2hi), __ldcg(&p[q].l2lo)});
        mx = fmaxf(mx, __ldcg(&p[q].maxe));
        c += __ldcg(&p[q].cnt);
        pr += __ldcg(&p[q].pairs);
    }
    l = warp_sum_ff(l);
    mx = warp_max(mx);
    c = warp_sum(c);
    pr = warp_sum(pr);
    return FwdPart{l.hi, l.lo, mx, (uint32_t)c, pr};
}

// Persistent warps take tiles from a global counter (heavy and light tiles
// balance out), write one partial per tile, and the partials are reduced in a
// fixed order in two levels (groups of kFwdGroup tiles, then all groups), so
// the loss terms are deterministic whatever warp handled which tile.
__global__ void __launch_bounds__(kFwdWarps * 32) k_forward(FwdArgs a) {
    // two rings per warp (kernels partly / fully covering the tile); a ring
    // holds 64 staged records and is consumed 32 at a time from slot 0 or 32
    __shared__ float4 ringP[kFwdWarps][kQueue][3];
    __shared__ float4 ringF[kFwdWarps][kQueue][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ngroups = (uint32_t)((a.ntiles + kFwdGroup - 1) / kFwdGroup);
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.tile_next, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((int64_t)t >= a.ntiles) break;
        const TileOut o = forward_tile(a, t, ringP[warp], ringF[warp], lane);
        const ff l2 = warp_sum_ff(ff{o.l2, 0.f});
        const float mx = warp_max(o.mx);
        const uint32_t cnt = warp_sum(o.cnt), pr = warp_sum(o.pairs);
        uint32_t done = 0;
        if (lane == 0) {
            a.part[t] = FwdPart{l2.hi, l2.lo, mx, cnt, (unsigned long long)pr};
            __threadfence();
            done = atomicAdd(a.group_done + t / kFwdGroup, 1u);
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        const uint32_t g = t / kFwdGroup;
        const uint32_t gb = g * kFwdGroup;
        const uint32_t ge = (uint32_t)min((int64_t)gb + kFwdGroup, a.ntiles);
        if (done != ge - gb - 1) continue;
        // this warp completed its group: reduce the group's partials
        __threadfence();
        const FwdPart gp = reduce_parts(a.part, gb, ge, lane);
        uint32_t gdone = 0;
        if (lane == 0) {
            a.gpart[g] = gp;
            a.group_done[g] = 0u;
            __threadfence();
            gdone = atomicAdd(a.counter, 1u);
        }
        gdone = __shfl_sync(0xffffffffu, gdone, 0);
        if (gdone != ngroups - 1) continue;
        // the last group: fixed-order sum of all group partials
        __threadfence();
        const FwdPart tot = reduce_parts(a.gpart, 0, ngroups, lane);
        if (lane == 0) {
            a.stats[SERBF_STAT_L2] = (double)tot.l2hi + (double)tot.l2lo;
            a.stats[SERBF_STAT_MAXE] = tot.maxe;
            a.stats[SERBF_STAT_COUNT] = (double)tot.cnt;
            a.stats[SERBF_STAT_PAIRS_FWD] = (double)tot.pairs;
            *a.counter = 0u;
        }
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
    a.tile_super = ws->tile_super;
    a.tile_start = ws->tile_start;
    a.cell_start = ws->cell_start;
    a.tile_lo = ws->tile_lo;
    a.tile_hi = ws->tile_hi;
    a.slist = ws->sup_list;
    a.scnt = ws->sup_cnt;
    a.kfwd = ws->kfwd;
    a.ntiles = ws->ntiles;
    a.scap = ws->sz.super_cap;
    a.cps = ws->sf * ws->sf * ws->sf;
    // float thresholds that give the same decisions as comparing in double:
    // t <= tau1 iff t <= (largest float <= tau1), t >= tau2 iff t >= (smallest float >= tau2)
    a.tau1 = (float)cfg->tau1;
    if ((double)a.tau1 > cfg->tau1) a.tau1 = nextafterf(a.tau1, -INFINITY);
    a.tau2 = (float)cfg->tau2;
    if ((double)a.tau2 < cfg->tau2) a.tau2 = nextafterf(a.tau2, INFINITY);
    a.psi = psi;
    a.err = err;
    a.mask = mask;
    a.part = ws->fwd_part;
    a.gpart = ws->fwd_gpart;
    a.group_done = ws->fwd_group_done;
    a.counter = ws->counters + 0;
    a.tile_next = ws->counters + 4;
    a.stats = stats;
    if (ws->ntiles == 0) {
        // nothing to evaluate: the loss terms are zero
        cudaMemsetAsync(stats + SERBF_STAT_L2, 0, 4 * sizeof(double), (cudaStream_t)stream);
        SERBF_CHECK_LAUNCH();
        return SERBF_OK;
    }
    int64_t blocks = (ws->ntiles + kFwdWarps - 1) / kFwdWarps;
    const int64_t resident = (int64_t)ws->sm_count * kFwdBlocksPerSM;
    if (blocks > resident) blocks = resident;
    // the tile counter is reset before every launch (warps still looking for
    // work may touch it after the last tile is done, so the kernel cannot)
    cudaMemsetAsync(a.tile_next, 0, sizeof(uint32_t), (cudaStream_t)stream);
    k_forward<<<(unsigned)blocks, kFwdWarps * 32, 0, (cudaStream_t)stream>>>(a);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
