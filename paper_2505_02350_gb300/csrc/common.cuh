// Internal definitions shared by the CUDA translation units of libserbf.
// Nothing here is part of the public ABI (include/serbf.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "serbf.h"

namespace serbf {

constexpr uint64_t kMagic = 0x53455242465753ull;  // "SERBFWS"
constexpr int kTile = 32;                         // points per forward/backward tile (one warp)
constexpr int kSortTile = 4096;                   // elements per radix-sort block
constexpr int kFwdWarps = 2;                      // warps (tiles) per forward block
constexpr int kQueue = 64;                        // per-warp ring of staged candidates
constexpr int kFwdGroup = 64;                     // tiles per first-level forward reduction group
constexpr int kFwdBlocksPerSM = 16;               // resident forward blocks per SM (register bound)
constexpr int kBwdThreads = 64;                   // threads per adjoint block
constexpr int kBwdSplit = 16;                     // most blocks per kernel in the adjoint
constexpr int kBwdWarpsPerKernel = kBwdSplit * kBwdThreads / 32;  // == 32, one epilogue lane each
constexpr int kMaxRowsPerKernel = 1 << 16;        // cell rows a kernel support may span
constexpr float kLog2e = 1.4426950408889634f;

// Parameter rows (Sec. 3.2): centre, axis parameters d, angles, weight.
enum { PCX = 0, PCY, PCZ, PD1, PD2, PD3, PTX, PTY, PTZ, PW };

// Per-block partials of the forward reduction (L2 as a float-float pair).
struct FwdPart {
    float l2hi, l2lo;
    float maxe;
    uint32_t cnt;
    unsigned long long pairs;
};

}  // namespace serbf

// Host-side description of the caller's scratch buffer.
struct serbf_workspace {
    uint64_t magic;
    char *base;
    size_t bytes;
    serbf_ws_sizes sz;
    int64_t max_tiles;
    int64_t max_supers;
    int64_t sort_blocks;
    // grid recorded by serbf_bin_points
    serbf_grid grid;
    int32_t sf;       // cells per super-cell edge
    int32_t ns[3];    // super cells per axis
    int32_t nsuper;
    int32_t binned;
    int64_t npoints;
    int64_t ntiles;
    int32_t sm_count;
    int32_t max_chunks;  // most 32-tile chunks in one super cell
    // binning
    uint32_t *keys0, *keys1, *vals0, *vals1, *hist;
    uint32_t *cell_start;   // nsuper * sf^3 + 1 (super-major cell order)
    uint32_t *super_tile0;  // nsuper + 1: first tile of each super cell
    uint32_t *tile_super, *tile_start;
    float4 *tile_lo, *tile_hi;
    float4 *sup_lo, *sup_hi;
    // per-kernel records
    float4 *kfwd;  // 3 per kernel
    float4 *kbwd;  // 4 per kernel
    // candidate lists (ascending kernel index) per super cell
    uint32_t *sup_list, *sup_cnt;
    // reductions
    serbf::FwdPart *fwd_part;     // max_tiles
    serbf::FwdPart *fwd_gpart;    // max_tiles / kFwdGroup + 1
    uint32_t *fwd_group_done;     // max_tiles / kFwdGroup + 1 (kept zero between launches)
    unsigned long long *bwd_pairs;
    float *moments;     // max_kernels x kBwdWarpsPerKernel x 22 (float-float partial moments, pairs)
    float4 *nzrec;      // per 32-tile chunk of a super cell: packed (box, count, id) of its tiles
                        // with nonzero residuals, at the chunk's own slots (2 float4 per tile)
    uint32_t *nzc_cnt;  // indexed by the chunk's first tile: number of such tiles in the chunk
    float4 *nz;         // 32 slots per tile: (x, y, z, E) of its nonzero-residual points
    // optimiser step scratch
    float *step_part;   // per-block partial sums
    double *step_scal;  // alpha, beta, Adam bias corrections
    // addition scratch
    unsigned long long *sel_key;  // max(max_kernels, 8192)
    uint32_t *sel_keep;           // max(max_kernels, 8192)
    int32_t *add_info;            // [0] active, [1] selected, [2] kept
    // status and counters
    int32_t *status;              // [0] flags
    long long *needed;            // [4]
    uint32_t *counters;           // [8] last-block counters
    double *dtmp;                 // [16]
};

#define SERBF_CHECK_LAUNCH()                                   \
    do {                                                       \
        if (cudaGetLastError() != cudaSuccess) return SERBF_ECUDA; \
    } while (0)

namespace serbf {

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Eq. 3-15-1 membership, float, fixed operation order, never contracted.
__device__ __forceinline__ bool in_support(float px, float py, float pz, float cx, float cy, float cz,
                                           float r2) {
    float dx = __fsub_rn(px, cx), dy = __fsub_rn(py, cy), dz = __fsub_rn(pz, cz);
    float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return d2 < r2;
}

// Squared distance from c to a box, rounded so that it never exceeds the
// float squared distance of any point inside the box (every step is a
// monotone rounding of a smaller exact value), hence box_d2 < r2 is a superset
// of the membership test for points in the box.
__device__ __forceinline__ float box_d2(float cx, float cy, float cz, float4 lo, float4 hi) {
    float ax = cx < lo.x ? __fsub_rn(lo.x, cx) : (cx > hi.x ? __fsub_rn(cx, hi.x) : 0.f);
    float ay = cy < lo.y ? __fsub_rn(lo.y, cy) : (cy > hi.y ? __fsub_rn(cy, hi.y) : 0.f);
    float az = cz < lo.z ? __fsub_rn(lo.z, cz) : (cz > hi.z ? __fsub_rn(cz, hi.z) : 0.f);
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
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
int launch_prep(const serbf_params *prm, const serbf_config *cfg, serbf_workspace *ws, cudaStream_t s);
}  // namespace serbf
