// Internal definitions shared by the CUDA translation units of libserbf.
// Nothing here is part of the public ABI (include/serbf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "serbf.h"
#include <nvtx3/nvToolsExt.h>

namespace serbf {

// An NVTX range named after a host entry point, for timelines and ncu --nvtx
// filters; without an attached tool the calls return at once.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
};
#define SERBF_TRACE() serbf::TraceRange serbf_trace_range_(__func__)


constexpr uint64_t kMagic = 0x53455242465753ull;  // "SERBFWS"
constexpr int kTile = 32;                         // points per forward/backward tile (one warp)
constexpr int kSortTile = 4096;                   // elements per radix-sort block
constexpr int kQueue = 64;                        // per-warp ring of staged candidates
constexpr int kFwdGroup = 64;                     // tiles per first-level forward reduction group
constexpr double kFixUnit = 1.0 / 68719476736.0;  // 2^-36: fixed-point unit of the fused adjoint's moments
constexpr int kCostClasses = 8;                   // cost classes of the forward's heavy-first schedule
constexpr int kOrderChunk = 1024;                 // items per block of the class sort
constexpr int kBwdThreads = 64;                   // threads per adjoint block
constexpr int kBwdSplit = 16;                     // most blocks per kernel in the adjoint
constexpr int kBwdWarpsPerKernel = kBwdSplit * kBwdThreads / 32;  // == 32, one epilogue lane each
constexpr int kMaxRowsPerKernel = 1 << 16;        // cell rows a kernel support may span
constexpr float kLog2e = 1.4426950408889634f;
constexpr int kSelBins = 2048;                    // addition: histogram bins over bits 30..20 of |E|

// Parameter rows (Sec. 3.2): centre, axis parameters d, angles, weight.
enum { PCX = 0, PCY, PCZ, PD1, PD2, PD3, PTX, PTY, PTZ, PW };

// Per-block partials of the forward reduction (L2 as a float-float pair).
struct FwdPart {
    float l2hi, l2lo;
    float maxe;
    uint32_t cnt;
    unsigned long long pairs;
};

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys (8 bits per pass, kSortTile elements per block; hist holds
// 256 x blocks + 1 words).  On return *k and *v point to whichever of the two
// buffer pairs holds the result.  Defined in bin.cu.
int radix_sort_pairs(uint32_t **k, uint32_t **v, uint32_t **ktmp, uint32_t **vtmp, int64_t n, int bits,
                     uint32_t *hist, cudaStream_t s);

}  // namespace serbf

// Host-side description of the caller's scratch buffer.
struct serbf_workspace {
    uint64_t magic;
    char *base;
    size_t bytes;
    serbf_ws_sizes sz;
    int64_t max_tiles;
    int64_t max_supers;
    int64_t max_items;
    int64_t sort_blocks;
    // grid recorded by serbf_bin_points
    serbf_grid grid;
    int32_t sf;       // cells per super-cell edge
    int32_t ns[3];    // super cells per axis
    int32_t nsuper;
    int32_t binned;
    int64_t npoints;
    int64_t ntiles;
    int64_t nitems;      // forward work items (one or two tiles of one super cell)
    int32_t sm_count;
    int32_t max_chunks;  // most 32-tile chunks in one super cell
    // side stream for work that overlaps the main stream inside one call
    // (fork and join through the two events; capturable into a CUDA graph)
    cudaStream_t aux;
    cudaEvent_t ev_fork, ev_join;
    // binning
    uint32_t *keys0, *keys1, *vals0, *vals1, *hist;
    uint32_t *cell_start;   // nsuper * sf^3 + 1 (super-major cell order)
    uint32_t *super_tile0;  // nsuper + 1: first tile of each super cell
    uint32_t *tile_super, *tile_start;
    float4 *tile_lo, *tile_hi;
    // forward work items: tiles at even offsets within their super cell,
    // taken together with the next tile of the same super cell if any.
    // Item record: (first tile, super cell, first point, points | item << 7).
    uint32_t *super_item0;  // nsuper + 1: first item of each super cell
    uint4 *item_rec;        // record of each item, in item order
    // heavy-first order of the forward: each launch files every item into a
    // cost class (item_class); a stable sort by class, descending (class
    // counts per chunk of kOrderChunk items in class_hist), gives the next
    // launch's order (order_rec).
    uint8_t *item_class;    // max_items
    uint32_t *class_hist;   // chunks x kCostClasses
    uint4 *order_rec;       // max_items
    uint32_t *sched;        // [0] mean cost of the last launch
    unsigned long long *sched_total;  // cost sum of the running launch
    float4 *sup_lo, *sup_hi;
    // per-kernel records
    float4 *kfwd;  // 3 per kernel
    float4 *kbwd;  // 4 per kernel
    // candidate lists (ascending kernel index) per super cell
    uint32_t *sup_list, *sup_cnt;
    uint32_t *crs_list, *crs_cnt;  // lists of blocks of 2 x 2 x 2 super cells (two-level rebuild)
    int64_t max_coarse;            // blocks the coarse lists have room for
    // reductions
    serbf::FwdPart *fwd_part;     // max_tiles
    serbf::FwdPart *fwd_gpart;    // max_tiles / kFwdGroup + 1
    unsigned long long *bwd_pairs;
    unsigned long long *adj_fix;    // max_kernels x 10: fixed-point moments of the fused adjoint
    unsigned long long *adj_pairs;  // [8]: [0] adjoint pairs of the fused adjoint
    float *moments;     // max_kernels x kBwdWarpsPerKernel x 22 (float-float partial moments, pairs)
    float4 *nzrec;      // per 32-tile chunk of a super cell: packed (box, count, id) of its tiles
                        // with nonzero residuals, at the chunk's own slots (2 float4 per tile)
    uint32_t *nzc_cnt;  // indexed by the chunk's first tile: number of such tiles in the chunk
    float4 *nz;         // 32 slots per tile: (x, y, z, E) of its nonzero-residual points
    // optimiser step scratch
    float *step_part;   // per-block partial sums
    double *step_scal;  // alpha, beta, Adam bias corrections
    // addition scratch (the selection itself lives in the binning sort
    // buffers keys0/vals0 and keys1/vals1, idle outside binning)
    uint32_t *sel_hist;           // kSelBins: candidate counts by the top bits of |E| (zero between calls)
    uint32_t *sel_ctl;            // [16]: threshold bin, k, slot and block counters
    int32_t *add_info;            // [0] active, [1] selected, [2] kept
    // status and counters
    int32_t *status;              // [0] flags
    long long *needed;            // [4]
    uint32_t *counters;           // [8] last-block counters
    double *dtmp;                 // [16]
    uint32_t *cell_max;           // [4]: [0] most points in one binning cell, [1] fixed-point range bound (float bits)
    float4 *field_box;            // [2]: lower and upper corner of all binned points
};

#define SERBF_CHECK_LAUNCH()                                   \
    do {                                                       \
        if (cudaGetLastError() != cudaSuccess) return SERBF_ECUDA; \
    } while (0)

namespace serbf {

// ---------------------------------------------------------------- dependent launches
// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while its predecessor on the stream is still running (inside a
// CUDA graph as well); it calls pdl_wait() before it touches anything, which
// returns once the predecessor has finished and its writes are visible, and
// pdl_trigger() to let its own successor be scheduled.  This hides the launch
// gap between the short kernels of one epoch.  In a kernel launched without
// the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Params>(args)...);
}

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Squared distance of the support test (Eq. 3-15-1) in its canonical float
// form: dx = fl(px - cx) and likewise for y, z, then
// d2 = fma(dz, dz, fma(dy, dy, fl(dx * dx))), each fma rounded once.  Every
// implementation (the scalar and packed kernels, the oracle) spells out the
// same three operations, so no compiler contraction can change the value.
__device__ __forceinline__ float support_d2(float dx, float dy, float dz) {
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Eq. 3-15-1 membership, float, fixed operation order.
__device__ __forceinline__ bool in_support(float px, float py, float pz, float cx, float cy, float cz,
                                           float r2) {
    const float dx = __fsub_rn(px, cx), dy = __fsub_rn(py, cy), dz = __fsub_rn(pz, cz);
    return support_d2(dx, dy, dz) < r2;
}

// Squared distance from c to a box, rounded so that it never exceeds the
// support_d2 of any point inside the box (every step is a monotone rounding
// of a smaller exact value, and fma with non-negative terms is monotone in
// each argument), hence box_d2 < r2 is a superset of the membership test for
// points in the box.
__device__ __forceinline__ float box_d2(float cx, float cy, float cz, float4 lo, float4 hi) {
    float ax = cx < lo.x ? __fsub_rn(lo.x, cx) : (cx > hi.x ? __fsub_rn(cx, hi.x) : 0.f);
    float ay = cy < lo.y ? __fsub_rn(lo.y, cy) : (cy > hi.y ? __fsub_rn(cy, hi.y) : 0.f);
    float az = cz < lo.z ? __fsub_rn(lo.z, cz) : (cz > hi.z ? __fsub_rn(cz, hi.z) : 0.f);
    return support_d2(ax, ay, az);
}

__device__ __forceinline__ float support_r2(float d1, float d2, float d3, float nle) {
    float a = __fmul_rn(d1, d1), b = __fmul_rn(d2, d2), c = __fmul_rn(d3, d3);
    float lam = a;
    if (b < lam) lam = b;
    if (c < lam) lam = c;
    return __fdiv_rn(nle, lam);
}

__device__ __forceinline__ int cell_axis(float v, float o, float h, int n) {
    float f = floorf(__fdiv_rn(__fsub_rn(v, o), h));
    if (!(f >= 0.f)) return 0;
    if (f >= (float)(n - 1)) return n - 1;
    return (int)f;
}

// Super-major cell key: super cell id * sf^3 + cell id inside the super cell.
__device__ __forceinline__ uint32_t cell_key(int kx, int ky, int kz, int sf, int nsx, int nsy) {
    const int sx = kx / sf, sy = ky / sf, sz = kz / sf;
    const int lx = kx - sx * sf, ly = ky - sy * sf, lz = kz - sz * sf;
    const uint32_t sup = ((uint32_t)sz * (uint32_t)nsy + (uint32_t)sy) * (uint32_t)nsx + (uint32_t)sx;
    return sup * (uint32_t)(sf * sf * sf) + (uint32_t)((lz * sf + ly) * sf + lx);
}

// Float-float ("double-float") accumulator: hi + lo carries about 48 bits.
// FP64 throughput on this part is a small fraction of FP32, so per-point and
// per-pair sums use this instead of double.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s.hi, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}

__device__ __forceinline__ ff ff_add(ff a, float b) { return ff_add(a, ff{b, 0.f}); }

// a * b exactly, as a float-float pair (the fused multiply-add gives the
// rounding error of the product).
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const ff p = two_prod(a.hi, b.hi);
    const float lo = __fadd_rn(p.lo, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
    const float hi = __fadd_rn(p.hi, lo);
    return {hi, __fsub_rn(lo, __fsub_rn(hi, p.hi))};
}

// a / b for a float-float a: the float quotient, then one correction from
// the exact remainder.
__device__ __forceinline__ ff ff_div(ff a, float b) {
    const float q1 = __fdiv_rn(a.hi, b);
    const ff p = two_prod(q1, b);
    const ff r = ff_add(a, ff{-p.hi, -p.lo});
    const float q2 = __fdiv_rn(r.hi, b);
    const float hi = __fadd_rn(q1, q2);
    return {hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}

// Eq. 3-10 without FP64 (this part's FP64 rate is a small fraction of its
// FP32 rate).  t = 2 exp(-h (S - m)^2) with h = ln 2 / m^2 is 2^(1 - u^2),
// u = (S - m) / m.  The exponent z = 1 - u^2 is formed in float-float (exact
// difference, then a quotient and a square to about 2^-46), split as
// z = n + f with n an integer and |f| <= 1/2, and 2^f = exp(f ln 2) is summed
// as its Taylor series to degree 11 in float-float (the first omitted term is
// below 1e-14).  The result is the float nearest the exact value except where
// that value lies within about 2^-40 of a rounding boundary (then one of the
// two neighbours).  c[k] = (ln 2)^k / k! as float-float, from eq310_coefs.
constexpr int kEq310Terms = 12;
__device__ __forceinline__ void eq310_coefs(ff *c) {
    double t = 1.0;
    for (int k = 0; k < kEq310Terms; ++k) {
        const float hi = (float)t;
        c[k] = ff{hi, (float)(t - (double)hi)};
        t = t * 0.6931471805599453094172321 / (double)(k + 1);
    }
}
__device__ __forceinline__ float eq310_target(float S, float m, const ff *c) {
    const ff s = two_sum(S, -m);  // S - m, exactly
    const ff u = ff_div(s, m);
    const ff u2 = ff_mul(u, u);
    const ff z = ff_add(ff{1.f, 0.f}, ff{-u2.hi, -u2.lo});
    if (z.hi != z.hi) return z.hi;  // NaN in, NaN out (m = 0 and S = 0)
    if (z.hi < -160.f) return 0.f;  // below the smallest float
    const float n = rintf(z.hi);
    const ff f = ff_add(z, -n);
    ff p = c[kEq310Terms - 1];
#pragma unroll
    for (int k = kEq310Terms - 2; k >= 0; --k) p = ff_add(ff_mul(p, f), c[k]);
    if (n > -126.f) return ldexpf(__fadd_rn(p.hi, p.lo), (int)n);  // normal: one rounding, exact scaling
    // below 2^-125 the floats are the multiples of 2^-149: round p 2^n onto
    // that grid directly (rounding p first and scaling after would round twice)
    const float sc = ldexpf(1.f, (int)n + 149);  // 2^-11 .. 2^23, exact
    const float q = __fmul_rn(p.hi, sc), r = __fmul_rn(p.lo, sc);
    float k = rintf(q);
    const float d = __fsub_rn(q, k);  // exact; |r| is below half a unit of q
    if (d == 0.5f && r > 0.f) k = __fadd_rn(k, 1.f);
    if (d == -0.5f && r < 0.f) k = __fsub_rn(k, 1.f);
    return __fmul_rn(k, 1.40129846432481707e-45f);  // k 2^-149, exact
}

__device__ __forceinline__ ff warp_sum_ff(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Inclusive warp scan.
__device__ __forceinline__ uint32_t warp_iscan(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive block scan (blockDim.x multiple of 32, <= 1024); every thread
// must call it.  `tmp` needs 33 entries of shared memory.
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t *tmp, uint32_t *total) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_iscan(v);
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? tmp[lane] : 0u;
        uint32_t si = warp_iscan(s);
        if (lane < nw) tmp[lane] = si - s;
        if (lane == 31) tmp[32] = si;
    }
    __syncthreads();
    uint32_t r = tmp[warp] + inc - v;
    if (total) *total = tmp[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- adjoint helpers
// One adjoint pair: point (x, y, z, E) against a kernel record k0 = (c, r2),
// k1..k3 = rows of R with e_k = log2(e) d_k^2 in .w.  Adds s = phi E and its
// moments in the rotated frame u = R (v - c): S0, M1 (3), M2 (6, upper).
__device__ __forceinline__ void kadd(float &s, float &c, float v) {
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

template <bool KAHAN>
__device__ __forceinline__ void accumulate(const float4 &pt, const float4 &k0, const float4 &k1, const float4 &k2,
                                           const float4 &k3, float (&acc)[10], float (&cmp)[10], uint32_t &pairs) {
    const float dx = __fsub_rn(pt.x, k0.x), dy = __fsub_rn(pt.y, k0.y), dz = __fsub_rn(pt.z, k0.z);
    const bool in = support_d2(dx, dy, dz) < k0.w;
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

// The ten App. A gradients of kernel j from its moments (a = w|w|):
//     dL2/dw     =  4 |w| S0
//     dL2/dd_k   = -4 a d_k (M2)_kk
//     dL2/dc     =  4 a R^T (d^2 . M1)
//     dL2/dtheta = -4 a sum_kl d_k^2 K_kl (M2)_kl,   K = (dR/dtheta) R^T
// (theta_x: K is constant and the sum is (d_2^2 - d_1^2) (M2)_12).
// WORLD: the moments come in the world frame (W1 = sum s Delta, W2 = sum s
// Delta Delta^T with Delta = v - c) and are rotated first: M1 = R W1,
// M2 = R W2 R^T.
template <bool WORLD = false>
__device__ __forceinline__ void grad_from_moments(const float *p, int cap, int j, const float (&Min)[10], float *grad) {
    const float w = p[PW * cap + j];
    const float d[3] = {p[PD1 * cap + j], p[PD2 * cap + j], p[PD3 * cap + j]};
    float sx, cx, sy, cy, sz, cz;
    sincosf(p[PTX * cap + j], &sx, &cx);
    sincosf(p[PTY * cap + j], &sy, &cy);
    sincosf(p[PTZ * cap + j], &sz, &cz);
    const float R[9] = {cx * cy, -cz * sx - sy * sz * cx, sx * sz - cx * cz * sy,
                        cy * sx, cx * cz - sx * sy * sz, -sz * cx - cz * sx * sy,
                        sy,      cy * sz,                cy * cz};
    // derivatives of the App. A entries with respect to theta_y and theta_z
    const float Ry[9] = {-cx * sy, -cx * cy * sz, -cx * cy * cz, -sx * sy, -sx * cy * sz,
                         -sx * cy * cz, cy, -sy * sz, -sy * cz};
    const float Rz[9] = {0.f, R[2], -R[1], 0.f, R[5], -R[4], 0.f, R[8], -R[7]};
    float M[10];
#pragma unroll
    for (int r = 0; r < 10; ++r) M[r] = Min[r];
    if (WORLD) {
        const float W2[3][3] = {{Min[4], Min[5], Min[6]}, {Min[5], Min[7], Min[8]}, {Min[6], Min[8], Min[9]}};
        float T[3][3];  // R W2
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M[1 + k] = R[3 * k] * Min[1] + R[3 * k + 1] * Min[2] + R[3 * k + 2] * Min[3];
#pragma unroll
            for (int b = 0; b < 3; ++b) T[k][b] = R[3 * k] * W2[0][b] + R[3 * k + 1] * W2[1][b] + R[3 * k + 2] * W2[2][b];
        }
        const int idx[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int k = idx[q][0], l = idx[q][1];
            M[4 + q] = T[k][0] * R[3 * l] + T[k][1] * R[3 * l + 1] + T[k][2] * R[3 * l + 2];
        }
    }
    const float aw = w * fabsf(w);
    const float M2[3][3] = {{M[4], M[5], M[6]}, {M[5], M[7], M[8]}, {M[6], M[8], M[9]}};
    grad[PW * cap + j] = 4.f * fabsf(w) * M[0];
    for (int k = 0; k < 3; ++k) grad[(PD1 + k) * cap + j] = -4.f * aw * d[k] * M2[k][k];
    for (int k = 0; k < 3; ++k) {
        float v = 0.f;
        for (int l = 0; l < 3; ++l) v = fmaf(R[3 * l + k] * d[l] * d[l], M[1 + l], v);
        grad[(PCX + k) * cap + j] = 4.f * aw * v;
    }
    // for theta_x, K is the constant generator [[0,-1,0],[1,0,0],[0,0,0]]
    float gy = 0.f, gz = 0.f;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            const float Ky = Ry[3 * r] * R[3 * c] + Ry[3 * r + 1] * R[3 * c + 1] + Ry[3 * r + 2] * R[3 * c + 2];
            const float Kz = Rz[3 * r] * R[3 * c] + Rz[3 * r + 1] * R[3 * c + 1] + Rz[3 * r + 2] * R[3 * c + 2];
            const float f = d[r] * d[r] * M2[r][c];
            gy = fmaf(f, Ky, gy);
            gz = fmaf(f, Kz, gz);
        }
    const float gx = (d[1] * d[1] - d[0] * d[0]) * M2[0][1];
    grad[PTX * cap + j] = -4.f * aw * gx;
    grad[PTY * cap + j] = -4.f * aw * gy;
    grad[PTZ * cap + j] = -4.f * aw * gz;
}

// Cell-index bounding box of a kernel's support sphere (with one cell of
// margin for rounding) and its cell rows (fixed kz, ky; x varies).
struct KBox {
    int kx0, kx1, ky0, ky1, kz0, kz1, nyr, nrows;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ KBox kernel_box(float cx, float cy, float cz, float r2, const serbf_grid &g) {
    KBox b;
    float r = sqrtf(r2);
    if (!(r < 1e30f) || !(cx == cx) || !(cy == cy) || !(cz == cz)) {
        b.kx0 = 0;
        b.kx1 = g.n[0] - 1;
        b.ky0 = 0;
        b.ky1 = g.n[1] - 1;
        b.kz0 = 0;
        b.kz1 = g.n[2] - 1;
    } else {
        float ih = 1.0f / g.h;
        // clamp in float before converting so huge radii cannot overflow int
        auto cidx = [&](float v, int n) { return (int)fminf(fmaxf(floorf(v * ih), -4.f), (float)n + 4.f); };
        b.kx0 = clampi(cidx(cx - r - g.origin[0], g.n[0]) - 1, 0, g.n[0] - 1);
        b.kx1 = clampi(cidx(cx + r - g.origin[0], g.n[0]) + 1, 0, g.n[0] - 1);
        b.ky0 = clampi(cidx(cy - r - g.origin[1], g.n[1]) - 1, 0, g.n[1] - 1);
        b.ky1 = clampi(cidx(cy + r - g.origin[1], g.n[1]) + 1, 0, g.n[1] - 1);
        b.kz0 = clampi(cidx(cz - r - g.origin[2], g.n[2]) - 1, 0, g.n[2] - 1);
        b.kz1 = clampi(cidx(cz + r - g.origin[2], g.n[2]) + 1, 0, g.n[2] - 1);
    }
    b.nyr = b.ky1 - b.ky0 + 1;
    b.nrows = b.nyr * (b.kz1 - b.kz0 + 1);
    return b;
}

}  // namespace serbf

// ---------------------------------------------------------------- cross-unit launchers
namespace serbf {
int launch_exscan_u32(uint32_t *a, int64_t n, cudaStream_t s);  // in place, a[n] = total
int launch_exscan_i64(int64_t *a, int64_t n, cudaStream_t s);   // in place, a[n] = total
}  // namespace serbf
