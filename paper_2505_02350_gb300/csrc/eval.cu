// Evaluation of a fit (Sec. 4): the zero level set of a grid field as
// triangles, area-weighted samples on it, and the point-to-point surface
// metrics HD, CD and CS between two sampled surfaces; plus the inverse of
// Eq. 3-10 and an index scatter to bring binned results back to grid order.
//
// The paper extracts the surface with marching cubes; here every grid cube
// is split into six tetrahedra {0, a, a + b, 7} (corner bits x = 1, y = 2,
// z = 4; axis orders (a, b) = (1,2) (1,4) (2,1) (2,4) (4,1) (4,2)), which needs
// no case table.  Inside means value < iso.  A tetrahedron with one or three
// inside vertices gives one triangle on the lone vertex's three edges, with
// two it gives the quad on the four crossing edges as two triangles.  Edge
// points interpolate from the edge's lower grid index to the higher one in
// float with a fixed operation order, so results are reproducible bit for
// bit and a shared edge gives the same point everywhere.  Output is in cube
// order (counts, exclusive scan, write).
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

__constant__ int c_tets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};

struct Grid3 {
    int nx, ny, nz;
    float o[3];
    float h;
};

__device__ __forceinline__ int64_t corner(const Grid3 &g, int64_t cube, int c) {
    const int64_t cx = g.nx - 1, cy = g.ny - 1;
    const int64_t i = cube % cx, j = (cube / cx) % cy, k = cube / (cx * cy);
    return ((k + ((c >> 2) & 1)) * g.ny + (j + ((c >> 1) & 1))) * g.nx + (i + (c & 1));
}

__device__ __forceinline__ int tet_mask(const float *f, const Grid3 &g, int64_t cube, int q, float iso, int64_t (&v)[4]) {
    int m = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = corner(g, cube, c_tets[q][a]);
        m |= (f[v[a]] < iso) << a;
    }
    return m;
}

__device__ __forceinline__ int tris_of(int m) {
    const int n = __popc(m);
    return (n == 0 || n == 4) ? 0 : (n == 2 ? 2 : 1);
}

__device__ __forceinline__ void edge_point(const float *f, const Grid3 &g, int64_t gu, int64_t gw, float iso,
                                           float *out) {
    if (gu > gw) {
        const int64_t t = gu;
        gu = gw;
        gw = t;
    }
    const float fu = f[gu], fw = f[gw];
    const float t = __fdiv_rn(__fsub_rn(iso, fu), __fsub_rn(fw, fu));
    const int64_t iu[3] = {gu % g.nx, (gu / g.nx) % g.ny, gu / ((int64_t)g.nx * g.ny)};
    const int64_t iw[3] = {gw % g.nx, (gw / g.nx) % g.ny, gw / ((int64_t)g.nx * g.ny)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float pu = __fadd_rn(g.o[a], __fmul_rn(g.h, (float)iu[a]));
        const float pw = __fadd_rn(g.o[a], __fmul_rn(g.h, (float)iw[a]));
        out[a] = __fadd_rn(pu, __fmul_rn(t, __fsub_rn(pw, pu)));
    }
}

__global__ void k_mt_count(const float *f, Grid3 g, float iso, int64_t ncubes, int64_t *cnt) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncubes; c += (int64_t)gridDim.x * blockDim.x) {
        int n = 0;
        for (int q = 0; q < 6; ++q) {
            int64_t v[4];
            n += tris_of(tet_mask(f, g, c, q, iso, v));
        }
        cnt[c] = n;
    }
}

__global__ void k_mt_write(const float *f, Grid3 g, float iso, int64_t ncubes, const int64_t *off, float *tri) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncubes; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = off[c];
        for (int q = 0; q < 6; ++q) {
            int64_t v[4];
            const int m = tet_mask(f, g, c, q, iso, v);
            const int nin = __popc(m);
            if (nin == 0 || nin == 4) continue;
            if (nin != 2) {
                const int want = nin == 1;
                int l = 0;
                while (((m >> l) & 1) != want) ++l;
                float *t = tri + 9 * o;
                int e = 0;
                for (int a = 0; a < 4; ++a)
                    if (a != l) edge_point(f, g, v[l], v[a], iso, t + 3 * e++);
                ++o;
            } else {
                int A = -1, B = -1, C = -1, D = -1;
                for (int a = 0; a < 4; ++a) {
                    if ((m >> a) & 1) {
                        if (A < 0) A = a; else B = a;
                    } else {
                        if (C < 0) C = a; else D = a;
                    }
                }
                float ac[3], ad[3], bd[3], bc[3];
                edge_point(f, g, v[A], v[C], iso, ac);
                edge_point(f, g, v[A], v[D], iso, ad);
                edge_point(f, g, v[B], v[D], iso, bd);
                edge_point(f, g, v[B], v[C], iso, bc);
                float *t0 = tri + 9 * o, *t1 = t0 + 9;
                for (int a = 0; a < 3; ++a) {
                    t0[a] = ac[a];
                    t0[3 + a] = ad[a];
                    t0[6 + a] = bd[a];
                    t1[a] = ac[a];
                    t1[3 + a] = bd[a];
                    t1[6 + a] = bc[a];
                }
                o += 2;
            }
        }
    }
}

// Cross product of the triangle's edges, float, fixed operation order.
__device__ __forceinline__ void tri_cross(const float *t, float &cx, float &cy, float &cz) {
    const float ux = __fsub_rn(t[3], t[0]), uy = __fsub_rn(t[4], t[1]), uz = __fsub_rn(t[5], t[2]);
    const float vx = __fsub_rn(t[6], t[0]), vy = __fsub_rn(t[7], t[1]), vz = __fsub_rn(t[8], t[2]);
    cx = __fsub_rn(__fmul_rn(uy, vz), __fmul_rn(uz, vy));
    cy = __fsub_rn(__fmul_rn(uz, vx), __fmul_rn(ux, vz));
    cz = __fsub_rn(__fmul_rn(ux, vy), __fmul_rn(uy, vx));
}

__device__ __forceinline__ float norm3(float cx, float cy, float cz) {
    return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz)));
}

// Triangle areas quantised to 64-bit integers (unit 2^-40): exact prefix sums.
__global__ void k_area_q(const float *tri, int64_t ntri, int64_t *q) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ntri; k += (int64_t)gridDim.x * blockDim.x) {
        float cx, cy, cz;
        tri_cross(tri + 9 * k, cx, cy, cz);
        const float a = __fmul_rn(0.5f, norm3(cx, cy, cz));
        q[k] = __double2ll_rn(__dmul_rn((double)a, 1099511627776.0));
    }
}

__global__ void k_sample(const float *tri, int64_t ntri, const int64_t *cum, const double *u, int64_t ns, float *pts,
                         float *nrm) {
    const uint64_t total = (uint64_t)cum[ntri];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t target = (uint64_t)__dmul_rn(u[3 * s], (double)total);
        int64_t lo = 0, hi = ntri;  // the k with cum[k] <= target < cum[k + 1]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            if ((uint64_t)cum[mid] <= target) lo = mid; else hi = mid;
        }
        const float *t = tri + 9 * lo;
        const float r = __fsqrt_rn(__double2float_rn(u[3 * s + 1])), w = __double2float_rn(u[3 * s + 2]);
        const float ca = __fsub_rn(1.0f, r), cb = __fmul_rn(r, __fsub_rn(1.0f, w)), cc = __fmul_rn(r, w);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            pts[3 * s + a] = __fadd_rn(__fadd_rn(__fmul_rn(ca, t[a]), __fmul_rn(cb, t[3 + a])), __fmul_rn(cc, t[6 + a]));
        float cx, cy, cz;
        tri_cross(t, cx, cy, cz);
        const float len = norm3(cx, cy, cz);
        nrm[3 * s] = __fdiv_rn(cx, len);
        nrm[3 * s + 1] = __fdiv_rn(cy, len);
        nrm[3 * s + 2] = __fdiv_rn(cz, len);
    }
}

// Nearest point of Q for every point of P (brute force, Q streamed through
// shared memory in tiles; ties: the lowest index): its distance and
// |n_P . n_Q| in double.
constexpr int kNnThreads = 256;
__global__ void __launch_bounds__(kNnThreads) k_nearest(const float *P, const float *nP, int64_t np, const float *Q,
                                                        const float *nQ, int64_t nq, double *dist, double *cosv) {
    __shared__ float sq[kNnThreads * 3];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool live = i < np;
    const float px = live ? P[3 * i] : 0.f, py = live ? P[3 * i + 1] : 0.f, pz = live ? P[3 * i + 2] : 0.f;
    float best = INFINITY;
    int64_t bi = 0;
    for (int64_t j0 = 0; j0 < nq; j0 += kNnThreads) {
        __syncthreads();
        const int64_t jl = j0 + threadIdx.x;
        if (jl < nq) {
            sq[3 * threadIdx.x] = Q[3 * jl];
            sq[3 * threadIdx.x + 1] = Q[3 * jl + 1];
            sq[3 * threadIdx.x + 2] = Q[3 * jl + 2];
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kNnThreads, nq - j0);
        for (int k = 0; k < cnt; ++k) {
            const float dx = __fsub_rn(px, sq[3 * k]), dy = __fsub_rn(py, sq[3 * k + 1]), dz = __fsub_rn(pz, sq[3 * k + 2]);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            if (d2 < best) {
                best = d2;
                bi = j0 + k;
            }
        }
    }
    if (!live) return;
    dist[i] = __dsqrt_rn((double)best);
    const double c = __dadd_rn(__dadd_rn(__dmul_rn((double)nP[3 * i], (double)nQ[3 * bi]),
                                         __dmul_rn((double)nP[3 * i + 1], (double)nQ[3 * bi + 1])),
                               __dmul_rn((double)nP[3 * i + 2], (double)nQ[3 * bi + 2]));
    cosv[i] = fabs(c);
}

// One block: max and sums of the two per-point arrays (fixed order).
__global__ void k_metric_sums(const double *d, const double *c, int64_t n, double *out) {
    __shared__ double sd[32], sc[32], sm[32];
    double s = 0.0, cs = 0.0, mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        s += d[i];
        cs += c[i];
        mx = fmax(mx, d[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sd[warp] = s;
        sc[warp] = cs;
        sm[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sd[w];
            b += sc[w];
            m = fmax(m, sm[w]);
        }
        out[0] = m;
        out[1] = a;
        out[2] = b;
    }
}

// Inverse of Eq. 3-10 on the branch S >= m: S = m + sqrt(-ln(t / 2) / h)
// (t >= 2 maps to m, t <= 0 to +inf).
__global__ void k_denormalize(const float *t, float *S, int64_t n, const double *mh) {
    const double m = mh[0], h = mh[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)t[i];
        double s;
        if (v >= 2.0) s = m;
        else if (v <= 0.0) s = INFINITY;
        else s = m + sqrt(-log(v * 0.5) / h);
        S[i] = (float)s;
    }
}

__global__ void k_scatter(const float *src, const uint32_t *idx, float *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i]] = src[i];
}

int blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

extern "C" int serbf_marching_tets(const float *f, const int32_t dims[3], const float origin[3], float h, float iso,
                                   float *tri, int64_t cap, int64_t *ntri, int64_t *scratch, void *stream) {
    SERBF_TRACE();
    if (!f || !dims || !origin || !ntri || !scratch || !(h > 0.f)) return SERBF_EINVAL;
    if (dims[0] < 2 || dims[1] < 2 || dims[2] < 2 || (cap > 0 && !tri)) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Grid3 g{dims[0], dims[1], dims[2], {origin[0], origin[1], origin[2]}, h};
    const int64_t ncubes = (int64_t)(dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1);
    k_mt_count<<<blocks_for(ncubes), 256, 0, s>>>(f, g, iso, ncubes, scratch);
    int rc = launch_exscan_i64(scratch, ncubes, s);
    if (rc) return rc;
    int64_t n = 0;
    if (cudaMemcpyAsync(&n, scratch + ncubes, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    *ntri = n;
    if (n > cap) return SERBF_ECAPACITY;
    k_mt_write<<<blocks_for(ncubes), 256, 0, s>>>(f, g, iso, ncubes, scratch, tri);
    SERBF_CHECK_LAUNCH();
    return cudaStreamSynchronize(s) == cudaSuccess ? SERBF_OK : SERBF_ECUDA;
}

extern "C" int serbf_sample_surface(const float *tri, int64_t ntri, const double *u, int64_t ns, float *pts, float *nrm,
                                    int64_t *scratch, void *stream) {
    SERBF_TRACE();
    if (!tri || ntri < 1 || !u || ns < 0 || (ns > 0 && (!pts || !nrm)) || !scratch) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    k_area_q<<<blocks_for(ntri), 256, 0, s>>>(tri, ntri, scratch);
    int rc = launch_exscan_i64(scratch, ntri, s);
    if (rc) return rc;
    int64_t total = 0;
    if (cudaMemcpyAsync(&total, scratch + ntri, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    if (total <= 0) return SERBF_EINVAL;
    if (ns > 0) k_sample<<<blocks_for(ns), 256, 0, s>>>(tri, ntri, scratch, u, ns, pts, nrm);
    SERBF_CHECK_LAUNCH();
    return cudaStreamSynchronize(s) == cudaSuccess ? SERBF_OK : SERBF_ECUDA;
}

extern "C" int serbf_surface_metrics(const float *A, const float *nA, int64_t na, const float *B, const float *nB,
                                     int64_t nb, double out[3], double *scratch, void *stream) {
    SERBF_TRACE();
    if (!A || !nA || !B || !nB || na < 1 || nb < 1 || !out || !scratch) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *dA = scratch, *cA = dA + na, *dB = cA + na, *cB = dB + nb, *red = cB + nb;
    k_nearest<<<(unsigned)((na + kNnThreads - 1) / kNnThreads), kNnThreads, 0, s>>>(A, nA, na, B, nB, nb, dA, cA);
    k_nearest<<<(unsigned)((nb + kNnThreads - 1) / kNnThreads), kNnThreads, 0, s>>>(B, nB, nb, A, nA, na, dB, cB);
    k_metric_sums<<<1, 1024, 0, s>>>(dA, cA, na, red);
    k_metric_sums<<<1, 1024, 0, s>>>(dB, cB, nb, red + 3);
    SERBF_CHECK_LAUNCH();
    double r[6];
    if (cudaMemcpyAsync(r, red, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    out[0] = fmax(r[0], r[3]);
    out[1] = r[1] / (2.0 * (double)na) + r[4] / (2.0 * (double)nb);
    out[2] = r[2] / (2.0 * (double)na) + r[5] / (2.0 * (double)nb);
    return SERBF_OK;
}

extern "C" int serbf_denormalize_sdf(const float *t, float *S, int64_t n, const double *mh_dev, void *stream) {
    if (n < 0 || (n > 0 && (!t || !S || !mh_dev))) return SERBF_EINVAL;
    if (n > 0) k_denormalize<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(t, S, n, mh_dev);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}

extern "C" int serbf_scatter(const float *src, const uint32_t *idx, float *dst, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!src || !idx || !dst))) return SERBF_EINVAL;
    if (n > 0) k_scatter<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(src, idx, dst, n);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
