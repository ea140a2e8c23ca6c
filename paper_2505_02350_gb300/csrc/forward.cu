// Point-major forward (Eq. 3-26) over the support pairs of Eq. 3-15-1, the
// point filter of Eq. 3-18 and the loss terms of Eq. 3-19.
//
// Work item = up to two consecutive 32-point tiles of one super cell; each
// lane holds one point of each tile.  The warp streams
// its super cell's candidate list (ascending kernel index), keeps the kernels
// whose support reaches the item's bounding box (one candidate per lane,
// ballot), and stages their records in a per-warp shared-memory ring, in
// pairs.  Each batch of 32 staged kernels is then evaluated with broadcast
// 16-byte loads and packed f32x2 arithmetic (two kernels per instruction,
// two points per lane), so every shared-memory load serves four pairs.  A
// kernel whose support covers the whole box skips the predicate; otherwise
// every lane applies the exact support predicate to its own points, so the
// pairs summed are exactly the point-major neighbour rows.
//
// Persistent blocks take items heaviest first (order from the costs measured
// by the previous launch) to keep the tail short; the warps of a block split
// an item's candidate list and combine their sums in a fixed order.
#include <math.h>
#include <string.h>

#include "common.cuh"

using namespace serbf;

namespace {

struct FwdArgs {
    const float *x, *y, *z, *t;
    const uint32_t *tile_super, *tile_start, *cell_start, *stile0;
    const float4 *tile_lo, *tile_hi;
    const uint32_t *slist, *scnt;
    const float4 *kfwd;
    const float4 *kbwd;      // adjoint records (c, r2), rows of R with log2(e) d_k^2
    const uint4 *item_rec;   // item records
    const uint4 *order_rec;  // item records, heaviest class first (stable)
    uint8_t *item_class;     // cost class of each item, for the next order
    uint32_t *sched;         // mean cost of the last launch
    unsigned long long *sched_total;
    int64_t max_items;
    unsigned long long *adj_fix;    // fixed-point moments (fused adjoint)
    unsigned long long *adj_pairs;  // adjoint pair count (fused adjoint)
    int64_t ntiles, nitems;
    int scap, cps;
    float tau1, tau2;  // tau1 rounded down, tau2 rounded up to float: exact double decisions
    float *psi, *err;
    uint8_t *mask;
    FwdPart *part;        // one partial per tile
    uint32_t *item_next;  // next work item to take (zero between launches)
    uint32_t *exit_count; // blocks that have exited (zero between launches)
    int32_t *status;      // device status flags
};

constexpr int kTouch = 256;  // kernels an item's warps remember for its adjoint (more: re-scan the list)
constexpr int kNz = 2 * kTile;

// Two float32 lanes in one 64-bit register: the packed f32x2 arithmetic of
// sm_100+ does two IEEE round-to-nearest operations per instruction, each
// bit-identical to its scalar counterpart.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Staged kernels are stored in pairs, interleaved so that one 16-byte load
// gives the same field of both kernels (a packed f32x2 operand).  Field v of
// the kernel in ring slot s is at float 24 (s / 2) + 2 v + s % 2, with fields
// cx, cy, cz, r2, Q11, Q22, Q33, a = w|w|, 2Q12, 2Q13, 2Q23 (v = 0 .. 10).
constexpr int kPairFloats = 24;

__device__ __forceinline__ void stage(float *ring, int slot, float4 k0, float4 k1, float4 k2) {
    float *b = ring + kPairFloats * (slot >> 1) + (slot & 1);
    b[0] = k0.x;
    b[2] = k0.y;
    b[4] = k0.z;
    b[6] = k0.w;
    b[8] = k1.x;
    b[10] = k1.y;
    b[12] = k1.z;
    b[14] = k1.w;
    b[16] = k2.x;
    b[18] = k2.y;
    b[20] = k2.z;
}

// The empty partner of an odd last kernel: q = 0, a = 0 and r2 < 0, so it
// adds exactly zero and is never counted.
__device__ __forceinline__ void stage_empty(float *ring, int slot) {
    float *b = ring + kPairFloats * (slot >> 1) + (slot & 1);
#pragma unroll
    for (int v = 0; v < 11; ++v) b[2 * v] = 0.f;
    b[6] = -1.f;
}

// Squared distance from c to the farthest corner of a box, rounded so that
// it is never below the support_d2 of any point inside the box:
// box_far_d2 < r2 means every point of the box is in the support.
__device__ __forceinline__ float box_far_d2(float cx, float cy, float cz, float4 lo, float4 hi) {
    const float ax = fmaxf(__fsub_rn(cx, lo.x), __fsub_rn(hi.x, cx));
    const float ay = fmaxf(__fsub_rn(cy, lo.y), __fsub_rn(hi.y, cy));
    const float az = fmaxf(__fsub_rn(cz, lo.z), __fsub_rn(hi.z, cz));
    return support_d2(ax, ay, az);
}

// npairs staged kernel pairs from pair index pb against the lane's two
// points.  PARTIAL: the support only partly covers the item box, so each
// pair takes the exact Eq. 3-15-1 predicate (the operations of support_d2,
// packed: fma(dz, dz, fma(dy, dy, fl(dx dx))) < r2).
template <bool PARTIAL, int UNROLL>
__device__ __forceinline__ void eval_pairs(const float *ring, int pb, int npairs, const f2 (&P)[2][3], f2 (&acc)[2],
                                           uint32_t (&n)[2]) {
#pragma unroll UNROLL
    for (int q = 0; q < npairs; ++q) {
        const ulonglong2 *r = reinterpret_cast<const ulonglong2 *>(ring + kPairFloats * (pb + q));
        const ulonglong2 F0 = r[0], F1 = r[1], F2 = r[2], F3 = r[3], F4 = r[4], F5 = r[5];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const f2 dx = f2_sub(P[p][0], F0.x), dy = f2_sub(P[p][1], F0.y), dz = f2_sub(P[p][2], F1.x);
            const f2 zz = f2_mul(dz, dz);
            // q = dv^T Q dv (log2 units): dx (Q11 dx + 2Q12 dy + 2Q13 dz) + dy (Q22 dy + 2Q23 dz) + Q33 dz^2
            const f2 ra = f2_fma(F4.y, dz, f2_fma(F4.x, dy, f2_mul(F2.x, dx)));
            const f2 rb = f2_fma(F5.x, dz, f2_mul(F2.y, dy));
            const f2 qv = f2_fma(F3.x, zz, f2_fma(dy, rb, f2_mul(dx, ra)));
            float q0, q1;
            f2_unpack(qv, q0, q1);
            float e0 = ex2_approx(-q0), e1 = ex2_approx(-q1);
            if (PARTIAL) {
                const f2 d2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                float d0, d1, r0, r1;
                f2_unpack(d2, d0, d1);
                f2_unpack(F1.y, r0, r1);
                const bool i0 = d0 < r0, i1 = d1 < r1;
                e0 = i0 ? e0 : 0.f;
                e1 = i1 ? e1 : 0.f;
                n[p] += (uint32_t)i0 + (uint32_t)i1;
            }
            acc[p] = f2_fma(F3.y, f2_pack(e0, e1), acc[p]);
        }
    }
}

// Whole-warp reductions in one instruction (redux.sync, sm_100 family): exact
// for integers; min / max of floats select one of the inputs, so the result
// does not depend on the order.
__device__ __forceinline__ uint32_t redux_add(uint32_t v) {
    uint32_t r;
    asm volatile("redux.sync.add.u32 %0, %1, 0xffffffff;" : "=r"(r) : "r"(v));
    return r;
}
__device__ __forceinline__ float redux_min(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float redux_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// Partial of a group of tiles: the loss sum in double (the global loss
// reduction runs in FP64; a tile's own sum of 32 squares is float-float).
struct FwdGPart {
    double l2;
    float maxe;
    uint32_t cnt;
    unsigned long long pairs;
};
static_assert(sizeof(FwdGPart) == sizeof(FwdPart), "group partials reuse the tile-partial storage");

__device__ __forceinline__ double part_l2(const FwdPart *p, uint32_t q) {
    return (double)__ldcg(&p[q].l2hi) + (double)__ldcg(&p[q].l2lo);
}
__device__ __forceinline__ double part_l2(const FwdGPart *p, uint32_t q) { return __ldcg(&p[q].l2); }

// Fixed-order warp reduction of partials [b, e) (of tiles or of groups) into one.
template <typename P>
__device__ __forceinline__ FwdGPart reduce_parts(const P *p, uint32_t b, uint32_t e, int lane) {
    double l = 0.0;
    float mx = 0.f;
    unsigned long long c = 0, pr = 0;
#pragma unroll 4
    for (uint32_t q = b + lane; q < e; q += 32) {
        l += part_l2(p, q);
        mx = fmaxf(mx, __ldcg(&p[q].maxe));
        c += __ldcg(&p[q].cnt);
        pr += __ldcg(&p[q].pairs);
    }
    l = warp_sum(l);
    mx = warp_max(mx);
    c = warp_sum(c);
    pr = warp_sum(pr);
    return FwdGPart{l, mx, (uint32_t)c, pr};
}

// Loss terms of one tile, stored as the tile's partial (lane order within the
// tile).  The partials are reduced in tile order after the launch, so the
// totals do not depend on which warp handled which tile.
__device__ __forceinline__ void finish_tile(const FwdArgs &a, uint32_t t, float l2, float mx_l, uint32_t cnt_l,
                                            uint32_t pairs_l, int lane) {
    const ff l2s = warp_sum_ff(ff{l2, 0.f});
    const float mx = redux_max(mx_l);
    const uint32_t cnt = redux_add(cnt_l), pr = redux_add(pairs_l);
    if (lane == 0) a.part[t] = FwdPart{l2s.hi, l2s.lo, mx, cnt, (unsigned long long)pr};
}

// Eq. 3-18 filter and residual of one point; returns its loss contributions.
__device__ __forceinline__ float point_out(const FwdArgs &a, int64_t i, bool valid, float t, float ps, uint32_t np,
                                           float &l2, float &mx, uint32_t &cnt, uint32_t &pairs) {
    l2 = 0.f;
    mx = 0.f;
    cnt = 0u;
    pairs = 0u;
    if (!valid) return 0.f;
    const bool m0 = (a.tau1 < t) && (t < a.tau2);
    const bool m1 = (t <= a.tau1) && (ps > a.tau1);
    const bool m2 = (t >= a.tau2) && (ps < a.tau2);
    const bool mk = m0 || m1 || m2;
    const float e = mk ? __fsub_rn(ps, t) : 0.f;
    a.psi[i] = ps;
    a.err[i] = e;
    a.mask[i] = (uint8_t)mk;
    pairs = np;
    if (mk) {
        l2 = e * e;
        mx = fabsf(e);
        cnt = 1u;
    }
    return e;
}

// Item geometry shared by the warps of a block.
struct ItemInfo {
    uint32_t t0, sup, item;
    int two;
    int64_t i0, i1;
    int v0, v1;
};

// Decode an item record (first tile, super cell, first point, points | item << 7).
__device__ __forceinline__ ItemInfo item_info(uint4 r, int lane) {
    ItemInfo it;
    const uint32_t np = r.w & 127u;
    it.t0 = r.x;
    it.sup = r.y;
    it.two = np > (uint32_t)kTile;
    it.i0 = (int64_t)r.z + lane;
    it.i1 = it.i0 + kTile;  // the second tile starts kTile points later
    it.v0 = (uint32_t)lane < np;
    it.v1 = (uint32_t)(lane + kTile) < np;
    it.item = r.w >> 7;
    return it;
}

// One warp's share of a work item: candidate chunks w, w + W, w + 2W, ... of
// the super cell's list (32 candidates each) are filtered against the item
// box, staged in pairs and evaluated against the lane's two points.
// Returns the lane's partial sums and pair counts; *cost gets the warp's
// measured work.
template <int G, int ADJ>
__device__ __forceinline__ void forward_share(const FwdArgs &a, const ItemInfo &it, int w, float *ringP, float *ringF,
                                              int lane, f2 (&acc)[2], uint32_t (&n)[2], uint32_t &cost,
                                              uint32_t *touch, int tcap, int &ntouch, float (&tv)[2]) {
    const unsigned lt = (1u << lane) - 1u;
    // invalid lanes carry NaN so the support test fails for them
    const float qnan = __int_as_float(0x7fc00000);
    f2 P[2][3];
    {
        const float x0 = it.v0 ? a.x[it.i0] : qnan, y0 = it.v0 ? a.y[it.i0] : 0.f, z0 = it.v0 ? a.z[it.i0] : 0.f;
        const float x1 = it.v1 ? a.x[it.i1] : qnan, y1 = it.v1 ? a.y[it.i1] : 0.f, z1 = it.v1 ? a.z[it.i1] : 0.f;
        P[0][0] = f2_pack(x0, x0);
        P[0][1] = f2_pack(y0, y0);
        P[0][2] = f2_pack(z0, z0);
        P[1][0] = f2_pack(x1, x1);
        P[1][1] = f2_pack(y1, y1);
        P[1][2] = f2_pack(z1, z1);
        // the targets, for the residuals after the sums (loaded early)
        tv[0] = it.v0 ? a.t[it.i0] : 0.f;
        tv[1] = it.v1 ? a.t[it.i1] : 0.f;
    }
    float4 lo = a.tile_lo[it.t0], hi = a.tile_hi[it.t0];
    if (it.two) {
        const float4 l1 = a.tile_lo[it.t0 + 1], h1 = a.tile_hi[it.t0 + 1];
        lo = make_float4(fminf(lo.x, l1.x), fminf(lo.y, l1.y), fminf(lo.z, l1.z), 0.f);
        hi = make_float4(fmaxf(hi.x, h1.x), fmaxf(hi.y, h1.y), fmaxf(hi.z, h1.z), 0.f);
    }
    const uint32_t *lst = a.slist + (size_t)it.sup * a.scap;
    const int L = min((int)a.scnt[it.sup], a.scap);
    constexpr int kStride = 32 * G;
    int hp = 0, qp = 0, hf = 0, qf = 0;
    uint32_t nfull = 0, npart = 0;
    acc[0] = 0ull;
    acc[1] = 0ull;
    n[0] = 0u;
    n[1] = 0u;
    // software pipeline: records of the next chunk and indices of the one
    // after it are in flight while a chunk is filtered
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int b0 = 32 * w;
    uint32_t jc = b0 + lane < L ? lst[b0 + lane] : 0u;
    float4 c0 = zero4, c1 = zero4, c2 = zero4;
    if (b0 + lane < L) {
        c0 = a.kfwd[3 * jc];
        c1 = a.kfwd[3 * jc + 1];
        c2 = a.kfwd[3 * jc + 2];
    }
    uint32_t jn = b0 + kStride + lane < L ? lst[b0 + kStride + lane] : 0u;
    int nchunks = 0;
    ntouch = 0;
    for (int b = b0; b < L; b += kStride) {
        const float4 k0 = c0, k1 = c1, k2 = c2;
        const uint32_t j = jc;
        const bool live = b + lane < L;
        if (b + kStride + lane < L) {
            c0 = a.kfwd[3 * jn];
            c1 = a.kfwd[3 * jn + 1];
            c2 = a.kfwd[3 * jn + 2];
        }
        jc = jn;
        if (b + 2 * kStride + lane < L) jn = lst[b + 2 * kStride + lane];
        ++nchunks;
        bool part = false, full = false;
        if (live && box_d2(k0.x, k0.y, k0.z, lo, hi) < k0.w) {
            full = box_far_d2(k0.x, k0.y, k0.z, lo, hi) < k0.w;
            part = !full;
        }
        const unsigned bp = __ballot_sync(0xffffffffu, part), bf = __ballot_sync(0xffffffffu, full);
        if (part) stage(ringP, (hp + qp + __popc(bp & lt)) & (kQueue - 1), k0, k1, k2);
        if (full) stage(ringF, (hf + qf + __popc(bf & lt)) & (kQueue - 1), k0, k1, k2);
        if (ADJ) {
            // the kernels that reach the item box, for the adjoint pass
            const unsigned ba = bp | bf;
            const int pos = ntouch + __popc(ba & lt);
            if ((part || full) && pos < tcap) touch[pos] = j;
            ntouch += __popc(ba);
        }
        qp += __popc(bp);
        qf += __popc(bf);
        npart += __popc(bp);
        nfull += __popc(bf);
        __syncwarp();
        if (qp >= 32) {
            eval_pairs<true, 2>(ringP, hp >> 1, 16, P, acc, n);
            hp ^= 32;
            qp -= 32;
        }
        if (qf >= 32) {
            eval_pairs<false, 2>(ringF, hf >> 1, 16, P, acc, n);
            hf ^= 32;
            qf -= 32;
        }
        __syncwarp();
    }
    // leftovers: the head is 0 or 32 and fewer than 32 remain, so they do not
    // wrap; an odd count gets an empty partner
    if (qp & 1) {
        if (lane == 0) stage_empty(ringP, hp + qp);
        __syncwarp();
    }
    if (qf & 1) {
        if (lane == 0) stage_empty(ringF, hf + qf);
        __syncwarp();
    }
    if (qp > 0) eval_pairs<true, 1>(ringP, hp >> 1, (qp + 1) >> 1, P, acc, n);
    if (qf > 0) eval_pairs<false, 1>(ringF, hf >> 1, (qf + 1) >> 1, P, acc, n);
    __syncwarp();
    n[0] += nfull;
    n[1] += nfull;
    // about one unit per filtered candidate, ~6 per fully and ~9 per partly
    // covering kernel
    cost = 32u * (uint32_t)nchunks + 6u * nfull + 9u * npart;
}

// ---------------------------------------------------------------- fused adjoint
// After an item's residuals are known, its points with E != 0 (at most 64,
// in shared memory as x, y, z, E arrays: tile 0 from 0, tile 1 from 32, each
// padded to an even count) are taken against the kernels that reached the
// item box in the forward filter, kept if their support reaches the box of
// those points: lanes are kernels, each lane loops over the points two at a
// time (packed f32x2) and accumulates the ten moments of its kernel in the
// world frame, Delta = v - c:
//     S0 = sum s,  W1 = sum s Delta,  W2 = sum s Delta Delta^T,  s = phi E,
// with phi = 2^(-Delta^T Q Delta) from the forward's own records (so the
// adjoint evaluates the same quadratic form as the forward).  The kernel
// frame moments of App. A are M1 = R W1 and M2 = R W2 R^T, formed once per
// kernel after the launch.  The item's float partial
// moments go to per-kernel 64-bit fixed-point accumulators (unit 2^-36) by
// integer atomics: integer addition is associative, so the totals do not
// depend on the order in which items finish.

// The nz points in pairs: pair k holds points 2k and 2k + 1 as two 16-byte
// words (x0, x1, y0, y1) and (z0, z1, e0, e1), so one pair of points is two
// 16-byte loads that give the packed operands directly.
struct NzPoints {
    float4 v[kNz];  // kNz / 2 pairs, two words each
    __device__ __forceinline__ float &at(int field, int i) {
        // field 0..3 = x, y, z, e of point i
        float4 &w = v[2 * (i >> 1) + (field >> 1)];
        const int k = 2 * (field & 1) + (i & 1);
        return k == 0 ? w.x : (k == 1 ? w.y : (k == 2 ? w.z : w.w));
    }
};

__device__ __forceinline__ f2 f2_dup(float v) { return f2_pack(v, v); }

// v * 2^36 rounded to the nearest integer (ties to even): the scaling by a
// power of two is exact in float, and one hardware conversion rounds (it was
// 9 % faster on the 256^3 field than an integer-only rounding).  |v| >= 2^26
// does not fit the accumulators' range; the caller flags such a partial
// before converting it.
__device__ __forceinline__ long long to_fix36(float v) {
    return __float2ll_rn(__fmul_rn(v, 68719476736.f));
}

// Compensated (Kahan) accumulation of packed pairs: s + v with the lost
// low-order part carried in c.
__device__ __forceinline__ void f2_kadd(f2 &s, f2 &c, f2 v) {
    const f2 y = f2_sub(v, c);
    const f2 t = f2_add(s, y);
    c = f2_sub(f2_sub(t, s), y);
    s = t;
}

// A batch of cnt <= 32 kernels from queue slot head: all nz points of the
// item against each kernel.  A short batch spreads each kernel over
// L = 2, 4 or 8 neighbouring lanes (cnt <= 16, 8, 4) that take every L-th
// point pair; their moments are combined with xor shuffles within the group
// (a fixed order for a given cnt) before the atomics, so short batches do
// not leave most lanes idle.  KAHAN: compensated per-lane sums.
template <bool KAHAN>
__device__ __forceinline__ void adjoint_batch(const FwdArgs &a, const uint32_t *q, int head, int cnt,
                                              const NzPoints &nz, int nc0, int nc1, int lane) {
    const int sh = cnt > 16 ? 0 : (cnt > 8 ? 1 : (cnt > 4 ? 2 : 3));
    const int L = 1 << sh, kl = lane >> sh, sub = lane & (L - 1);
    const bool act = kl < cnt;  // whole groups of L lanes are inactive together
    const uint32_t j = q[(head + (act ? kl : 0)) & (kQueue - 1)];
    const float4 k0 = a.kfwd[3 * j], k1 = a.kfwd[3 * j + 1], k2 = a.kfwd[3 * j + 2];
    const f2 cx = f2_dup(k0.x), cy = f2_dup(k0.y), cz = f2_dup(k0.z);
    const f2 q11 = f2_dup(k1.x), q22 = f2_dup(k1.y), q33 = f2_dup(k1.z);
    const f2 q12 = f2_dup(k2.x), q13 = f2_dup(k2.y), q23 = f2_dup(k2.z);  // 2 Q12, 2 Q13, 2 Q23
    f2 acc[10], cmp[KAHAN ? 10 : 1];
#pragma unroll
    for (int r = 0; r < 10; ++r) acc[r] = 0ull;
#pragma unroll
    for (int r = 0; r < (KAHAN ? 10 : 1); ++r) cmp[r] = 0ull;
#pragma unroll 1
    for (int seg = 0; seg < 2; ++seg) {
        const int base = seg ? kTile : 0, cntp = act ? ((seg ? nc1 : nc0) + 1) >> 1 : 0;
#pragma unroll 4
        for (int pp = sub; pp < cntp; pp += L) {
            const int i = base + 2 * pp;
            const ulonglong2 wa = *reinterpret_cast<const ulonglong2 *>(&nz.v[i]);
            const ulonglong2 wb = *reinterpret_cast<const ulonglong2 *>(&nz.v[i + 1]);
            const f2 px = wa.x, py = wa.y, pz = wb.x, pe = wb.y;
            const f2 dx = f2_sub(px, cx), dy = f2_sub(py, cy), dz = f2_sub(pz, cz);
            const f2 zz = f2_mul(dz, dz);
            // q = Delta^T Q Delta (log2 units), the forward's operation order
            const f2 ra = f2_fma(q13, dz, f2_fma(q12, dy, f2_mul(q11, dx)));
            const f2 rb = f2_fma(q23, dz, f2_mul(q22, dy));
            const f2 qv = f2_fma(q33, zz, f2_fma(dy, rb, f2_mul(dx, ra)));
            float q0, q1;
            f2_unpack(qv, q0, q1);
            float e0 = ex2_approx(-q0), e1 = ex2_approx(-q1);
            // Eq. 3-15-1, the operations of support_d2, packed
            const f2 d2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
            float d0, d1;
            f2_unpack(d2, d0, d1);
            const bool i0 = d0 < k0.w, i1 = d1 < k0.w;
            e0 = i0 ? e0 : 0.f;
            e1 = i1 ? e1 : 0.f;
            const f2 sv = f2_mul(f2_pack(e0, e1), pe);
            const f2 sx = f2_mul(sv, dx), sy = f2_mul(sv, dy), sz = f2_mul(sv, dz);
            if (KAHAN) {
                f2_kadd(acc[0], cmp[0], sv);
                f2_kadd(acc[1], cmp[1], sx);
                f2_kadd(acc[2], cmp[2], sy);
                f2_kadd(acc[3], cmp[3], sz);
                f2_kadd(acc[4], cmp[4], f2_mul(sx, dx));
                f2_kadd(acc[5], cmp[5], f2_mul(sx, dy));
                f2_kadd(acc[6], cmp[6], f2_mul(sx, dz));
                f2_kadd(acc[7], cmp[7], f2_mul(sy, dy));
                f2_kadd(acc[8], cmp[8], f2_mul(sy, dz));
                f2_kadd(acc[9], cmp[9], f2_mul(sz, dz));
            } else {
                acc[0] = f2_add(acc[0], sv);
                acc[1] = f2_add(acc[1], sx);
                acc[2] = f2_add(acc[2], sy);
                acc[3] = f2_add(acc[3], sz);
                acc[4] = f2_fma(sx, dx, acc[4]);
                acc[5] = f2_fma(sx, dy, acc[5]);
                acc[6] = f2_fma(sx, dz, acc[6]);
                acc[7] = f2_fma(sy, dy, acc[7]);
                acc[8] = f2_fma(sy, dz, acc[8]);
                acc[9] = f2_fma(sz, dz, acc[9]);
            }
        }
    }
    float v[10];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        float lo, hi;
        f2_unpack(acc[r], lo, hi);
        if (KAHAN) {
            // the two halves and their compensations, as a float-float sum
            float clo, chi;
            f2_unpack(cmp[r], clo, chi);
            const ff t = ff_add(two_sum(lo, -clo), two_sum(hi, -chi));
            v[r] = t.hi + t.lo;
        } else {
            v[r] = lo + hi;
        }
    }
    for (int o = 1; o < L; o <<= 1) {
#pragma unroll
        for (int r = 0; r < 10; ++r) v[r] += __shfl_xor_sync(0xffffffffu, v[r], o);
    }
    if (act && sub == 0) {
        // a partial at or beyond 2^26 (or not finite) does not fit the
        // fixed-point range: flag it (never taken in a healthy fit)
        bool out = false;
#pragma unroll
        for (int r = 0; r < 10; ++r) out |= !(fabsf(v[r]) < 67108864.f);
        if (out) atomicOr(a.status, SERBF_FLAG_FIX_RANGE);
        unsigned long long *o = a.adj_fix + 10 * (size_t)j;
#pragma unroll
        for (int r = 0; r < 10; ++r)
            if (v[r] != 0.f) atomicAdd(o + r, (unsigned long long)to_fix36(v[r]));
    }
}

// One warp's share of an item's adjoint: the kernels this warp found
// reaching the item box (or, if it found more than tcap, its candidate
// chunks of the super cell's list again), filtered against the nz box.
template <int G, bool KAHAN>
__device__ __forceinline__ void adjoint_share(const FwdArgs &a, const ItemInfo &it, int w, const NzPoints &nz,
                                              int nc0, int nc1, float4 lo, float4 hi, const uint32_t *touch,
                                              int ntouch, int tcap, uint32_t *q, int lane, uint32_t &cost) {
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t *lst = a.slist + (size_t)it.sup * a.scap;
    const bool listed = ntouch <= tcap;
    const int L = listed ? ntouch : min((int)a.scnt[it.sup], a.scap);
    const int b0 = listed ? 0 : 32 * w, stride = listed ? 32 : 32 * G;
    int head = 0, qn = 0, nk = 0;
    for (int b = b0; b < L; b += stride) {
        const bool live = b + lane < L;
        const uint32_t j = live ? (listed ? touch[b + lane] : lst[b + lane]) : 0u;
        bool hit = false;
        if (live) {
            const float4 k0 = a.kfwd[3 * j];
            hit = box_d2(k0.x, k0.y, k0.z, lo, hi) < k0.w;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) q[(head + qn + __popc(bal & lt)) & (kQueue - 1)] = j;
        qn += __popc(bal);
        nk += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
            adjoint_batch<KAHAN>(a, q, head, 32, nz, nc0, nc1, lane);
            head = (head + 32) & (kQueue - 1);
            qn -= 32;
            __syncwarp();
        }
    }
    if (qn > 0) adjoint_batch<KAHAN>(a, q, head, qn, nz, nc0, nc1, lane);
    __syncwarp();
    cost += (uint32_t)(nk * (nc0 + nc1)) / 4u + 32u;
}

// The nz points of one 32-point tile (lanes = points): compacted in lane
// order from `base`, padded to an even count with a copy of the last point
// with E = 0 (it adds zero and is not counted); returns their count and box
// (empty: +inf / -inf).
__device__ __forceinline__ int nz_tile(NzPoints &nzp, int base, bool nz, float x, float y, float z, float e, int lane,
                                       float4 &lo, float4 &hi) {
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    const int cnt = __popc(bal);
    if (nz) {
        const int i = base + __popc(bal & ((1u << lane) - 1u));
        nzp.at(0, i) = x;
        nzp.at(1, i) = y;
        nzp.at(2, i) = z;
        nzp.at(3, i) = e;
    }
    __syncwarp();
    if ((cnt & 1) && lane == 0) {
        // pad: a copy of the last point with E = 0 (finite, adds nothing)
        nzp.at(0, base + cnt) = nzp.at(0, base + cnt - 1);
        nzp.at(1, base + cnt) = nzp.at(1, base + cnt - 1);
        nzp.at(2, base + cnt) = nzp.at(2, base + cnt - 1);
        nzp.at(3, base + cnt) = 0.f;
    }
    float mnx = nz ? x : INFINITY, mny = nz ? y : INFINITY, mnz = nz ? z : INFINITY;
    float mxx = nz ? x : -INFINITY, mxy = nz ? y : -INFINITY, mxz = nz ? z : -INFINITY;
    if (bal) {
        mnx = redux_min(mnx);
        mny = redux_min(mny);
        mnz = redux_min(mnz);
        mxx = redux_max(mxx);
        mxy = redux_max(mxy);
        mxz = redux_max(mxz);
    }
    lo = make_float4(mnx, mny, mnz, 0.f);
    hi = make_float4(mxx, mxy, mxz, 0.f);
    return cnt;
}

__device__ __forceinline__ float4 box_min(float4 a, float4 b) {
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.f);
}
__device__ __forceinline__ float4 box_max(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), 0.f);
}

// ---------------------------------------------------------------- scheduling
// Heavy-first order: blocks claim positions of order_rec, which lists the
// items by the cost class the previous launch measured, heaviest first and
// in natural (spatially coherent) order within a class.  Every launch files
// each item's class for the next order.  Each item is evaluated exactly once
// whatever the order, and the loss partials are reduced by tile index, so
// the order never changes a result.
__device__ __forceinline__ uint4 resolve(const FwdArgs &a, uint32_t k) {
    return (int64_t)k < a.nitems ? a.order_rec[k] : make_uint4(0u, 0u, 0u, 0u);  // w = 0: none left
}

// Class of a measured cost: 0 below mean / 4, then about one class per half
// octave up to 7 at 4 x mean and above (all in class 3 before a mean exists).
__device__ __forceinline__ int cost_class(uint32_t c, uint32_t mean) {
    if (mean == 0) return 3;
    const uint64_t c4 = 4ull * c;
    int k = 0;
    k += c4 >= mean;         // >= mean / 4
    k += c4 >= 2ull * mean;  // >= mean / 2
    k += c4 >= 3ull * mean;  // >= 0.75 mean
    k += c4 >= 4ull * mean;  // >= mean
    k += c4 >= 6ull * mean;  // >= 1.5 mean
    k += c4 >= 8ull * mean;  // >= 2 mean
    k += c4 >= 16ull * mean; // >= 4 mean
    return k;
}

// Files an item's class by its measured cost.
__device__ __forceinline__ void note_cost(const FwdArgs &a, uint32_t mean, uint4 rec, uint32_t c) {
    const uint32_t item = rec.w >> 7;
    const int cls = cost_class(c, mean);
    a.item_class[item] = (uint8_t)cls;
    atomicAdd(a.sched_total, (unsigned long long)c);
}

// Last block out: records the mean cost and resets the claim counters.
__device__ __forceinline__ void sched_finish(const FwdArgs &a) {
    __threadfence();
    if (atomicAdd(a.exit_count, 1u) != gridDim.x - 1) return;
    __threadfence();
    const unsigned long long tot = __ldcg(a.sched_total);
    const unsigned long long mean = a.nitems > 0 ? tot / (unsigned long long)a.nitems : 0ull;
    a.sched[0] = (uint32_t)min(mean, 0xffffffffull);
    *a.sched_total = 0ull;
    *a.item_next = 0u;
    *a.exit_count = 0u;
}

// A batch of fields advanced by one launch: the fields' arguments in device
// memory and their work items concatenated in field order (item_off: prefix
// sums of the item counts).  Blocks claim from one counter over all items.
struct FwdBatch {
    const FwdArgs *args;
    const uint32_t *item_off;  // nfields + 1
    int nfields;
    uint32_t *next, *exit;     // claim and exit counters (zero between launches)
};
constexpr int kMaxBatchFields = 1024;

// Item k of the batch: its field (binary search of the item offsets, read
// through the read-only cache) and record; w = 0 when none is left.
__device__ __forceinline__ uint4 resolve_batch(const FwdBatch &b, uint32_t k, uint32_t &field) {
    const uint32_t *off = b.item_off;
    field = 0;
    if (k >= __ldg(off + b.nfields)) return make_uint4(0u, 0u, 0u, 0u);
    int lo = 0, hi = b.nfields - 1;  // largest f with off[f] <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= k) lo = mid; else hi = mid - 1;
    }
    field = (uint32_t)lo;
    return b.args[lo].order_rec[k - off[lo]];
}

// Last block out of a batch launch: every field's mean cost, and the batch
// counters reset.
__device__ __forceinline__ void sched_finish_batch(const FwdBatch &b) {
    __threadfence();
    if (atomicAdd(b.exit, 1u) != gridDim.x - 1) return;
    __threadfence();
    for (int f = 0; f < b.nfields; ++f) {
        const FwdArgs &a = b.args[f];
        const unsigned long long tot = __ldcg(a.sched_total);
        const unsigned long long mean = a.nitems > 0 ? tot / (unsigned long long)a.nitems : 0ull;
        a.sched[0] = (uint32_t)min(mean, 0xffffffffull);
        *a.sched_total = 0ull;
    }
    *b.next = 0u;
    *b.exit = 0u;
}

// Persistent blocks take work items, heaviest first, from a global counter.
// The G warps of a block share an item (its candidate list split by 32-entry
// chunks); their partial sums are combined in warp order, so Psi does not
// depend on timing.  G = 1 when there are enough items to balance the warps,
// 2 or 4 for small problems.
// ADJ: 0 forward only, 1 with the fused adjoint, 2 with the fused adjoint
// and compensated (Kahan) per-item moment sums.
// BATCH: the items of a batch of fields (b); otherwise of one field (a1).
template <int G, int ADJ, bool BATCH>
__device__ __forceinline__ void forward_loop(const FwdArgs &a1, const FwdBatch &b) {
    // two rings per warp (kernels partly / fully covering the item box); a
    // ring holds 64 staged kernels (32 pairs), consumed 32 at a time from
    // slot 0 or 32
    //
    // Shared memory is kept small: the L1 cache that serves the kernel-record
    // gathers gets what the blocks leave of the SM's unified 256 KB.  The
    // rings are idle during the adjoint, so the nz points live in warp 0's
    // first ring and each warp's adjoint queue in its second.
    constexpr int GR = G > 1 ? G : 1;    // the cross-warp sums exist only for G > 1
    constexpr int RL = G > 1 ? 32 : 1;
    constexpr int kTouchW = G > 1 ? kTouch / 2 : kTouch;  // kernels remembered per warp
    __shared__ __align__(16) float ringP[G][(kQueue / 2) * kPairFloats];
    __shared__ __align__(16) float ringF[G][(kQueue / 2) * kPairFloats];
    __shared__ float2 red_psi[GR][RL];
    __shared__ uint2 red_n[GR][RL];
    __shared__ uint32_t red_cost[G];
    __shared__ uint4 s_rec;
    // fused adjoint: the item's nz points (tile 0 at 0, tile 1 at 32), their
    // counts and boxes, and the kernels each warp found reaching the item
    __shared__ int s_nc[2];
    __shared__ float4 s_box[2][2];
    __shared__ uint32_t touch[ADJ ? G : 1][ADJ ? kTouchW : 1];
    // batch: the arguments of the current item's field
    __shared__ __align__(16) unsigned char s_args[BATCH ? sizeof(FwdArgs) : 16];
    __shared__ uint32_t s_field;
    static_assert(sizeof(NzPoints) <= sizeof(ringP[0]) && kQueue * 4 <= (int)sizeof(ringF[0]), "ring aliases");
    NzPoints &nzs = *reinterpret_cast<NzPoints *>(ringP[0]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *adjq = reinterpret_cast<uint32_t *>(ringF[warp]);
    if (threadIdx.x == 0) {
        if (BATCH) {
            uint32_t f;
            s_rec = resolve_batch(b, atomicAdd(b.next, 1u), f);
            s_field = f;
        } else {
            s_rec = resolve(a1, atomicAdd(a1.item_next, 1u));
        }
    }
    __syncthreads();
    uint4 rec = s_rec;  // the item's record; no points (w = 0) when done
    uint32_t field = BATCH ? s_field : 0u, loaded = ~0u;
    uint32_t mean = BATCH ? 0u : a1.sched[0];
    const FwdArgs &a = BATCH ? *reinterpret_cast<const FwdArgs *>(s_args) : a1;
    while (rec.w != 0u) {
        if (BATCH && field != loaded) {
            // the block's threads copy the field's arguments (block-uniform
            // branch: every thread holds the same record and field)
            if (G == 1) __syncwarp(); else __syncthreads();
            const uint32_t *src = reinterpret_cast<const uint32_t *>(b.args + field);
            uint32_t *dst = reinterpret_cast<uint32_t *>(s_args);
            for (int k = threadIdx.x; k < (int)(sizeof(FwdArgs) / 4); k += blockDim.x) dst[k] = src[k];
            if (G == 1) __syncwarp(); else __syncthreads();
            loaded = field;
            mean = a.sched[0];
        }
        const ItemInfo it = item_info(rec, lane);
        // the next claim is made now, its record is fetched after the sums
        // and used at the end, so neither round trip is on the item's path
        uint32_t knext = 0, fnext = 0;
        if (threadIdx.x == 0) knext = atomicAdd(BATCH ? b.next : a.item_next, 1u);
        f2 acc[2];
        uint32_t n[2], cost;
        int ntouch = 0;
        float tv[2];
        forward_share<G, ADJ>(a, it, warp, ringP[warp], ringF[warp], lane, acc, n, cost, touch[ADJ ? warp : 0],
                              kTouchW, ntouch, tv);
        uint4 rn = make_uint4(0u, 0u, 0u, 0u);
        if (threadIdx.x == 0) rn = BATCH ? resolve_batch(b, knext, fnext) : resolve(a, knext);
        if constexpr (G == 1) {
            // one warp: finish both tiles directly
            float l0, h0, l1, h1;
            f2_unpack(acc[0], l0, h0);
            f2_unpack(acc[1], l1, h1);
            float l2, mx;
            uint32_t cnt, pr;
            const float e0 = point_out(a, it.i0, it.v0, tv[0], l0 + h0, n[0], l2, mx, cnt, pr);
            finish_tile(a, it.t0, l2, mx, cnt, pr, lane);
            float e1 = 0.f;
            if (it.two) {
                e1 = point_out(a, it.i1, it.v1, tv[1], l1 + h1, n[1], l2, mx, cnt, pr);
                finish_tile(a, it.t0 + 1, l2, mx, cnt, pr, lane);
            }
            if (ADJ) {
                // adjoint pairs: every support pair of a point with E != 0
                // (the adjoint takes exactly these)
                const uint32_t pb = redux_add((e0 != 0.f ? n[0] : 0u) + (e1 != 0.f ? n[1] : 0u));
                if (lane == 0 && pb) atomicAdd(a.adj_pairs, (unsigned long long)pb);
                float4 lo0, hi0, lo1, hi1;
                const int nc0 = nz_tile(nzs, 0, e0 != 0.f, a.x[it.v0 ? it.i0 : 0], a.y[it.v0 ? it.i0 : 0],
                                        a.z[it.v0 ? it.i0 : 0], e0, lane, lo0, hi0);
                const int nc1 = nz_tile(nzs, kTile, e1 != 0.f, a.x[it.v1 ? it.i1 : 0], a.y[it.v1 ? it.i1 : 0],
                                        a.z[it.v1 ? it.i1 : 0], e1, lane, lo1, hi1);
                __syncwarp();
                if (nc0 + nc1 > 0)
                    adjoint_share<1, (ADJ > 1)>(a, it, 0, nzs, nc0, nc1, box_min(lo0, lo1), box_max(hi0, hi1), touch[0],
                                                ntouch, kTouchW, adjq, lane, cost);
                __syncwarp();
            }
            if (lane == 0) note_cost(a, mean, rec, cost);
            rec.x = __shfl_sync(0xffffffffu, rn.x, 0);
            rec.y = __shfl_sync(0xffffffffu, rn.y, 0);
            rec.z = __shfl_sync(0xffffffffu, rn.z, 0);
            rec.w = __shfl_sync(0xffffffffu, rn.w, 0);
            if (BATCH) field = __shfl_sync(0xffffffffu, fnext, 0);
            continue;
        } else {
        {
            float l0, h0, l1, h1;
            f2_unpack(acc[0], l0, h0);
            f2_unpack(acc[1], l1, h1);
            red_psi[warp][lane] = make_float2(l0 + h0, l1 + h1);
            red_n[warp][lane] = make_uint2(n[0], n[1]);
            if (lane == 0) red_cost[warp] = cost;
        }
        __syncthreads();
        // warp 0 finishes the first tile, warp 1 the second (if any)
        if (warp < 2 && (warp == 0 || it.two)) {
            float ps = 0.f;
            uint32_t np = 0;
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const float2 v = red_psi[q][lane];
                const uint2 c = red_n[q][lane];
                ps += warp ? v.y : v.x;
                np += warp ? c.y : c.x;
            }
            float l2, mx;
            uint32_t cnt, pr;
            const int64_t i = warp ? it.i1 : it.i0;
            const bool v = warp ? it.v1 : it.v0;
            const float e = point_out(a, i, v, warp ? tv[1] : tv[0], ps, np, l2, mx, cnt, pr);
            finish_tile(a, it.t0 + warp, l2, mx, cnt, pr, lane);
            if (ADJ) {
                // adjoint pairs: every support pair of a point with E != 0
                const uint32_t pb = redux_add(e != 0.f ? np : 0u);
                if (lane == 0 && pb) atomicAdd(a.adj_pairs, (unsigned long long)pb);
                float4 lo, hi;
                const int nc = nz_tile(nzs, kTile * warp, e != 0.f, a.x[v ? i : 0], a.y[v ? i : 0],
                                       a.z[v ? i : 0], e, lane, lo, hi);
                if (lane == 0) {
                    s_nc[warp] = nc;
                    s_box[warp][0] = lo;
                    s_box[warp][1] = hi;
                    if (warp == 0 && !it.two) s_nc[1] = 0;
                }
            }
            if (warp == 0 && lane == 0) {
                if (!ADJ) {
                    uint32_t c = 0;
#pragma unroll
                    for (int q = 0; q < G; ++q) c += red_cost[q];
                    note_cost(a, mean, rec, c);
                }
                s_rec = rn;
                if (BATCH) s_field = fnext;
            }
        }
        if (ADJ) {
            __syncthreads();
            const int nc0 = s_nc[0], nc1 = s_nc[1];
            if (nc0 + nc1 > 0) {
                const float4 lo = nc1 ? (nc0 ? box_min(s_box[0][0], s_box[1][0]) : s_box[1][0]) : s_box[0][0];
                const float4 hi = nc1 ? (nc0 ? box_max(s_box[0][1], s_box[1][1]) : s_box[1][1]) : s_box[0][1];
                uint32_t c = 0;
                adjoint_share<G, (ADJ > 1)>(a, it, warp, nzs, nc0, nc1, lo, hi, touch[warp], ntouch, kTouchW, adjq,
                                            lane, c);
                if (lane == 0) red_cost[warp] += c;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t c = 0;
#pragma unroll
                for (int q = 0; q < G; ++q) c += red_cost[q];
                note_cost(a, mean, rec, c);
            }
        }
        __syncthreads();
        rec = s_rec;
        if (BATCH) field = s_field;
        }
    }
    // the last block out prepares the next launch: every block has made its
    // last claim and recorded its costs before it counts itself out
    if (threadIdx.x == 0) {
        if (BATCH)
            sched_finish_batch(b);
        else
            sched_finish(a1);
    }
}

// Resident warps per SM (the register budget): 20 for the fused variants
// with 1 or 2 warps per item and 16 with 4, 24 for eight warps and for the
// forward alone (20 with one warp); measured on the 128^3 and 256^3 fields,
// other bounds were slower.
#define SERBF_FWD_BOUNDS(G, ADJ) __launch_bounds__(G * 32, (G == 8 ? 24 : (ADJ ? (G == 4 ? 16 : 20) : (G == 1 ? 20 : 24))) / G)

template <int G, int ADJ>
__global__ void SERBF_FWD_BOUNDS(G, ADJ) k_forward(FwdArgs a) {
    pdl_wait();
    pdl_trigger();
    forward_loop<G, ADJ, false>(a, FwdBatch{});
}

// One launch over the work items of every field of a batch.
template <int G, int ADJ>
__global__ void SERBF_FWD_BOUNDS(G, ADJ) k_forward_batch(FwdBatch b) {
    pdl_wait();
    pdl_trigger();
    forward_loop<G, ADJ, true>(FwdArgs{}, b);
}

template <int G, int ADJ>
int launch_forward(const FwdArgs &a, int64_t nitems, int sm_count, cudaStream_t s) {
    static int per_sm = 0;  // resident blocks per SM (same for every device of one kind)
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forward<G, ADJ>, G * 32, 0) != cudaSuccess ||
            nb < 1)
            return SERBF_ECUDA;
        per_sm = nb;
    }
    int64_t blocks = nitems;
    const int64_t resident = (int64_t)sm_count * per_sm;
    if (blocks > resident) blocks = resident;
    launch_pdl(k_forward<G, ADJ>, dim3((unsigned)blocks), dim3(G * 32), 0, s, a);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

template <int G>
int64_t forward_groups(int sm_count) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forward<G, 0>, G * 32, 0) != cudaSuccess ||
            nb < 1)
            nb = 1;
        per_sm = nb;
    }
    return (int64_t)sm_count * per_sm;
}

// After the forward: the Eq. 3-19 loss terms from the tile partials in tile
// order (a warp per group of kFwdGroup tiles, then the last block over the
// group partials), and with the fused adjoint the ten App. A gradients of each
// kernel from its fixed-point moments (a thread per kernel, accumulators
// cleared for the next launch).  The last block writes the totals.
constexpr float kFixUnitF = 1.4551915228366852e-11f;  // 2^-36
constexpr int kFinishThreads = 256;

struct FinishArgs {
    const FwdPart *part;
    FwdGPart *gpart;
    int64_t ntiles;
    const float *p;
    const int32_t *m_dev;
    int cap;
    unsigned long long *fix, *pairs;
    float *grad;
    uint32_t *counter;
    double *stats;
    const float4 *kbwd;      // (c, r2) of each kernel
    float cell_h;            // binning cell edge
    uint32_t *cell_max;      // [0] most points in one cell, [1] running range bound (float bits)
    const float4 *field_box; // box of all binned points
    float npoints;
    int32_t *status;
};

// Upper bound of |moment| / max|E| for kernel j (centre c, support radius
// r): a pair has phi <= 1 and every component of v - c is at most the
// distance from c to the farthest corner of the points' box, and below r,
// so every moment of the kernel is at most (points within r of c) * max|E| *
// max(1, min(r^2, far^2)); the points within r are at most the points of
// the field and at most (cells a ball of radius r can touch) * (most points
// in one cell).
__device__ __forceinline__ float moment_bound(float4 k0, float h, uint32_t cell_max, const float4 *box, float npts) {
    const float nc = ceilf(2.f * sqrtf(k0.w) / h) + 2.f;
    const float far2 = box_far_d2(k0.x, k0.y, k0.z, box[0], box[1]);
    return fmaxf(1.f, fminf(k0.w, far2)) * fminf(npts, nc * nc * nc * (float)cell_max);
}

// Block bx of nbx.
template <bool ADJ>
__device__ __forceinline__ void fwd_finish_body(const FinishArgs &f, int bx, int nbx) {
    __shared__ bool s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ngroups = (f.ntiles + kFwdGroup - 1) / kFwdGroup;
    const int64_t g = (int64_t)bx * (kFinishThreads / 32) + warp;
    if (g < ngroups) {
        const uint32_t gb = (uint32_t)(g * kFwdGroup);
        const uint32_t ge = (uint32_t)min((int64_t)gb + kFwdGroup, f.ntiles);
        const FwdGPart gp = reduce_parts(f.part, gb, ge, lane);
        if (lane == 0) f.gpart[g] = gp;
    }
    if (ADJ) {
        const int m = *f.m_dev;
        const int j = bx * blockDim.x + threadIdx.x;
        if (j < m) {
            unsigned long long *o = f.fix + 10 * (size_t)j;
            float M[10];
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                // int64 -> float from its two 32-bit halves and one FMA;
                // relative error ~1e-7
                const long long v = (long long)o[r];
                const float hi = (float)(int)(v >> 32), lo = (float)(uint32_t)(v & 0xffffffffll);
                M[r] = fmaf(hi, 4294967296.f, lo) * kFixUnitF;
                o[r] = 0ull;
            }
            grad_from_moments<true>(f.p, f.cap, j, M, f.grad);
            // positive floats order like their bits (NaN orders above +inf)
            atomicMax(&f.cell_max[1], __float_as_uint(moment_bound(f.kbwd[4 * j], f.cell_h, f.cell_max[0],
                                                                   f.field_box, f.npoints)));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(f.counter, 1u) == (unsigned)nbx - 1;
    }
    __syncthreads();
    if (!s_last || warp != 0) return;
    __threadfence();
    const FwdGPart tot = reduce_parts(f.gpart, 0, (uint32_t)ngroups, lane);
    if (lane == 0) {
        f.stats[SERBF_STAT_L2] = tot.l2;
        f.stats[SERBF_STAT_MAXE] = tot.maxe;
        f.stats[SERBF_STAT_COUNT] = (double)tot.cnt;
        f.stats[SERBF_STAT_PAIRS_FWD] = (double)tot.pairs;
        if (ADJ) {
            f.stats[SERBF_STAT_PAIRS_BWD] = (double)__ldcg(f.pairs);
            *f.pairs = 0ull;
            // the int64 sums hold |moment| < 2^27 (unit 2^-36); flag when the
            // bound reaches 2^26, or is not finite
            const float bound = __uint_as_float(__ldcg(&f.cell_max[1])) * tot.maxe;
            if (!(bound < 67108864.f)) atomicOr(f.status, SERBF_FLAG_FIX_RANGE);
            f.cell_max[1] = 0u;
        }
        *f.counter = 0u;
    }
}

template <bool ADJ>
__global__ void __launch_bounds__(kFinishThreads) k_fwd_finish(FinishArgs f) {
    pdl_wait();
    pdl_trigger();
    fwd_finish_body<ADJ>(f, blockIdx.x, gridDim.x);
}

// Batch: field blockIdx.y.
template <bool ADJ>
__global__ void __launch_bounds__(kFinishThreads) k_fwd_finish_batch(const FinishArgs *fa) {
    pdl_wait();
    pdl_trigger();
    const FinishArgs f = fa[blockIdx.y];
    fwd_finish_body<ADJ>(f, blockIdx.x, gridDim.x);
}

// The arguments of one forward (+ adjoint) call; false on bad arguments.
bool make_args(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi, float *err,
               uint8_t *mask, float *grad, double *stats, serbf_workspace *ws, FwdArgs &a, FinishArgs &f,
               int64_t &finish_blocks) {
    if (!pts || !prm || !cfg || !ws || ws->magic != kMagic || !ws->binned) return false;
    if (pts->n != ws->npoints || !prm->m || !prm->p) return false;
    if (pts->n > 0 && (!pts->x || !pts->y || !pts->z || !pts->t || !psi || !err || !mask)) return false;
    if (!stats) return false;
    const bool adj = grad != nullptr;
    if (cfg->fwd_warps != 0 && cfg->fwd_warps != 1 && cfg->fwd_warps != 2 && cfg->fwd_warps != 4 && cfg->fwd_warps != 8)
        return false;
    if (adj && (prm->cap < 1 || prm->cap > ws->sz.max_kernels)) return false;
    a.x = pts->x;
    a.y = pts->y;
    a.z = pts->z;
    a.t = pts->t;
    a.tile_super = ws->tile_super;
    a.stile0 = ws->super_tile0;
    a.item_rec = ws->item_rec;
    a.order_rec = ws->order_rec;
    a.item_class = ws->item_class;
    a.sched = ws->sched;
    a.sched_total = ws->sched_total;
    a.max_items = ws->max_items;
    a.nitems = ws->nitems;
    a.tile_start = ws->tile_start;
    a.cell_start = ws->cell_start;
    a.tile_lo = ws->tile_lo;
    a.tile_hi = ws->tile_hi;
    a.slist = ws->sup_list;
    a.scnt = ws->sup_cnt;
    a.kfwd = ws->kfwd;
    a.kbwd = ws->kbwd;
    a.adj_fix = ws->adj_fix;
    a.adj_pairs = ws->adj_pairs;
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
    a.item_next = ws->counters + 4;
    a.exit_count = ws->counters + 6;
    a.status = ws->status;
    f.part = ws->fwd_part;
    f.gpart = reinterpret_cast<FwdGPart *>(ws->fwd_gpart);
    f.ntiles = ws->ntiles;
    f.p = prm->p;
    f.m_dev = prm->m;
    f.cap = prm->cap;
    f.fix = ws->adj_fix;
    f.pairs = ws->adj_pairs;
    f.grad = grad;
    f.counter = ws->counters + 5;
    f.stats = stats;
    f.kbwd = ws->kbwd;
    f.cell_h = ws->grid.h;
    f.cell_max = ws->cell_max;
    f.field_box = ws->field_box;
    f.npoints = (float)ws->npoints;
    f.status = ws->status;
    const int64_t ngroups = (ws->ntiles + kFwdGroup - 1) / kFwdGroup;
    int64_t nb = (ngroups + kFinishThreads / 32 - 1) / (kFinishThreads / 32);
    if (adj) nb = max(nb, (int64_t)((prm->cap + kFinishThreads - 1) / kFinishThreads));
    finish_blocks = nb < 1 ? 1 : nb;
    return true;
}

// Warps per item: the fewest that still leave about four items per group of
// warps for the heavy-first balancing, unless the configuration fixes it.
int pick_warps(int64_t nitems, int sm_count, int fixed) {
    if (fixed == 1 || fixed == 2 || fixed == 4 || fixed == 8) return fixed;
    return nitems >= 4 * forward_groups<1>(sm_count) ? 1 : (nitems >= 4 * forward_groups<2>(sm_count) ? 2 : 4);
}

int forward_impl(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi, float *err,
                 uint8_t *mask, float *grad, double *stats, serbf_workspace *ws, void *stream) {
    FwdArgs a;
    FinishArgs f;
    int64_t nb = 1;
    if (!make_args(pts, prm, cfg, psi, err, mask, grad, stats, ws, a, f, nb)) return SERBF_EINVAL;
    const bool adj = grad != nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = SERBF_OK;
    if (ws->ntiles > 0) {
        const int64_t ni = ws->nitems;
        const int G = pick_warps(ni, ws->sm_count, cfg->fwd_warps);
        const int mode = adj ? (cfg->kahan ? 2 : 1) : 0;
        switch (G * 4 + mode) {
            case 4: rc = launch_forward<1, 0>(a, ni, ws->sm_count, s); break;
            case 5: rc = launch_forward<1, 1>(a, ni, ws->sm_count, s); break;
            case 6: rc = launch_forward<1, 2>(a, ni, ws->sm_count, s); break;
            case 8: rc = launch_forward<2, 0>(a, ni, ws->sm_count, s); break;
            case 9: rc = launch_forward<2, 1>(a, ni, ws->sm_count, s); break;
            case 10: rc = launch_forward<2, 2>(a, ni, ws->sm_count, s); break;
            case 16: rc = launch_forward<4, 0>(a, ni, ws->sm_count, s); break;
            case 17: rc = launch_forward<4, 1>(a, ni, ws->sm_count, s); break;
            case 18: rc = launch_forward<4, 2>(a, ni, ws->sm_count, s); break;
            case 32: rc = launch_forward<8, 0>(a, ni, ws->sm_count, s); break;
            case 33: rc = launch_forward<8, 1>(a, ni, ws->sm_count, s); break;
            default: rc = launch_forward<8, 2>(a, ni, ws->sm_count, s); break;
        }
    }
    if (rc) return rc;
    if (adj)
        launch_pdl(k_fwd_finish<true>, dim3((unsigned)nb), dim3(kFinishThreads), 0, s, f);
    else
        launch_pdl(k_fwd_finish<false>, dim3((unsigned)nb), dim3(kFinishThreads), 0, s, f);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

template <int G, int ADJ>
int launch_forward_batch(const FwdBatch &b, int64_t nitems, int sm_count, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forward_batch<G, ADJ>, G * 32, 0) != cudaSuccess ||
            nb < 1)
            return SERBF_ECUDA;
        per_sm = nb;
    }
    int64_t blocks = nitems;
    const int64_t resident = (int64_t)sm_count * per_sm;
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    launch_pdl(k_forward_batch<G, ADJ>, dim3((unsigned)blocks), dim3(G * 32), 0, s, b);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // namespace

namespace serbf {

size_t fwd_args_size() { return sizeof(FwdArgs); }
size_t finish_args_size() { return sizeof(FinishArgs); }

// Host records of one field's fused forward + adjoint (out: sizeof(FwdArgs)
// and sizeof(FinishArgs) bytes) and the finishing kernel's block count.
int batch_forward_args(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi,
                       float *err, uint8_t *mask, float *grad, double *stats, serbf_workspace *ws, void *fwd_out,
                       void *fin_out, int64_t *finish_blocks) {
    FwdArgs a;
    FinishArgs f;
    if (!make_args(pts, prm, cfg, psi, err, mask, grad, stats, ws, a, f, *finish_blocks)) return SERBF_EINVAL;
    memcpy(fwd_out, &a, sizeof(a));
    memcpy(fin_out, &f, sizeof(f));
    return SERBF_OK;
}

int batch_pick_warps(int64_t nitems, int sm_count, int fixed) { return pick_warps(nitems, sm_count, fixed); }

// One persistent launch over the items of every field, then the finishing
// kernel of every field (grid.y = field).  args / fin / item_off / counters
// are device arrays written by the batch set-up.
int batch_forward_launch(const void *args, const void *fin, const uint32_t *item_off, int nfields, uint32_t *counters,
                         int64_t total_items, int64_t finish_blocks, int G, int kahan, int sm_count, cudaStream_t s) {
    if (nfields < 1 || nfields > kMaxBatchFields) return SERBF_EINVAL;
    FwdBatch b{static_cast<const FwdArgs *>(args), item_off, nfields, counters, counters + 1};
    int rc = SERBF_OK;
    if (total_items > 0) {
        switch (G * 2 + (kahan ? 1 : 0)) {
            case 2: rc = launch_forward_batch<1, 1>(b, total_items, sm_count, s); break;
            case 3: rc = launch_forward_batch<1, 2>(b, total_items, sm_count, s); break;
            case 4: rc = launch_forward_batch<2, 1>(b, total_items, sm_count, s); break;
            case 5: rc = launch_forward_batch<2, 2>(b, total_items, sm_count, s); break;
            case 8: rc = launch_forward_batch<4, 1>(b, total_items, sm_count, s); break;
            case 9: rc = launch_forward_batch<4, 2>(b, total_items, sm_count, s); break;
            case 16: rc = launch_forward_batch<8, 1>(b, total_items, sm_count, s); break;
            case 17: rc = launch_forward_batch<8, 2>(b, total_items, sm_count, s); break;
            default: return SERBF_EINVAL;
        }
    }
    if (rc) return rc;
    launch_pdl(k_fwd_finish_batch<true>, dim3((unsigned)finish_blocks, (unsigned)nfields), dim3(kFinishThreads), 0, s,
               static_cast<const FinishArgs *>(fin));
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

}  // namespace serbf

extern "C" int serbf_forward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg, float *psi,
                             float *err, uint8_t *mask, double *stats, serbf_workspace *ws, void *stream) {
    SERBF_TRACE();
    return forward_impl(pts, prm, cfg, psi, err, mask, nullptr, stats, ws, stream);
}

extern "C" int serbf_forward_backward(const serbf_points *pts, const serbf_params *prm, const serbf_config *cfg,
                                      float *psi, float *err, uint8_t *mask, float *grad, double *stats,
                                      serbf_workspace *ws, void *stream) {
    SERBF_TRACE();
    if (!grad) return SERBF_EINVAL;
    return forward_impl(pts, prm, cfg, psi, err, mask, grad, stats, ws, stream);
}
