// Initial kernels: Algorithm 1 (greedy largest inscribed spheres over the
// interior training points) and Eq. 3-12 (isotropic axis parameters from the
// nearest other centre), once before the fit.
//
// The interior points (1 < t < 2, Eq. 3-10) are sorted by d_in = |S|
// descending (stable, so equal values keep the binned order: the first
// maximum is taken, as an argmax does).  One block then walks that order:
// the first point not yet removed is the next centre; every interior point
// within its sphere -- found through the binning cells of the sphere's box --
// is removed.  The removal test is the float squared distance in the support
// predicate's operation order against fl(r r), so the decisions are exact
// and reproducible.
#include <math.h>

#include "common.cuh"

using namespace serbf;

namespace {

constexpr int kInitThreads = 1024;

// Sort keys: interior points by |S| descending (inverted float bits of a
// positive value), everything else last.
__global__ void k_init_keys(const float *t, const float *S, int64_t n, uint32_t *keys, uint32_t *vals,
                            uint32_t *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool in = (1.0f < t[i]) && (t[i] < 2.0f);
        keys[i] = in ? ~__float_as_uint(fabsf(S[i])) : 0xffffffffu;
        vals[i] = (uint32_t)i;
        const unsigned b = __ballot_sync(__activemask(), in);
        if ((threadIdx.x & 31) == __ffs(__activemask()) - 1 && b) atomicAdd(count, (uint32_t)__popc(b));
    }
}

// rank[binned index] = position in the sorted interior order, or ~0u.
__global__ void k_init_rank(const uint32_t *sorted_vals, int64_t n, const uint32_t *count, uint32_t *rank) {
    const int64_t nin = *count;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        rank[sorted_vals[k]] = k < nin ? (uint32_t)k : 0xffffffffu;
}

struct InitArgs {
    const float *x, *y, *z, *S;
    const uint32_t *order;  // binned indices of the interior points, |S| descending
    const uint32_t *count;  // number of interior points
    const uint32_t *rank;
    uint8_t *removed;       // per sorted position
    const uint32_t *cell_start;
    serbf_grid g;
    int sf, nsx, nsy;
    uint32_t *centres;      // binned indices of the centres, in selection order
    int32_t cap;
    uint32_t *ncentres;
};

// Algorithm 1, one block.  Terminates: every round removes at least its own
// centre and the scan pointer only moves forward.
__global__ void __launch_bounds__(kInitThreads) k_inscribed(InitArgs a) {
    __shared__ int64_t s_first;
    __shared__ int s_found;
    const int64_t nin = *a.count;
    for (int64_t q = threadIdx.x; q < nin; q += blockDim.x) a.removed[q] = 0;
    __syncthreads();
    int64_t ptr = 0;
    uint32_t cnt = 0;
    for (;;) {
        // the first position >= ptr not yet removed
        if (threadIdx.x == 0) {
            s_first = -1;
            s_found = 0;
        }
        __syncthreads();
        while (ptr < nin) {
            const int64_t q = ptr + threadIdx.x;
            const bool ok = q < nin && !a.removed[q];
            if (ok) atomicOr(&s_found, 1);
            __syncthreads();
            if (s_found) {
                // lowest candidate: warp minima, then a shared minimum
                if (ok) atomicMin(reinterpret_cast<unsigned long long *>(&s_first), (unsigned long long)q);
                break;
            }
            ptr += blockDim.x;
            __syncthreads();
        }
        __syncthreads();
        if (!s_found) break;
        const int64_t p = s_first;
        const uint32_t i = a.order[p];
        const float cx = a.x[i], cy = a.y[i], cz = a.z[i];
        const float r = fabsf(a.S[i]);
        const float r2 = __fmul_rn(r, r);
        if (threadIdx.x == 0) {
            if ((int32_t)cnt < a.cap) a.centres[cnt] = i;
            a.removed[p] = 1;
        }
        ++cnt;
        // remove the interior points within the sphere (cells of its box)
        const KBox b = kernel_box(cx, cy, cz, r2, a.g);
        const int nx = b.kx1 - b.kx0 + 1;
        const int64_t ncells = (int64_t)nx * b.nrows;
        for (int64_t c = threadIdx.x; c < ncells; c += blockDim.x) {
            const int kx = b.kx0 + (int)(c % nx);
            const int row = (int)(c / nx);
            const int ky = b.ky0 + row % b.nyr, kz = b.kz0 + row / b.nyr;
            const uint32_t key = cell_key(kx, ky, kz, a.sf, a.nsx, a.nsy);
            for (uint32_t k = a.cell_start[key]; k < a.cell_start[key + 1]; ++k) {
                const uint32_t rk = a.rank[k];
                if (rk == 0xffffffffu || a.removed[rk]) continue;
                const float dx = __fsub_rn(a.x[k], cx), dy = __fsub_rn(a.y[k], cy), dz = __fsub_rn(a.z[k], cz);
                const float d2 = support_d2(dx, dy, dz);
                if (!(d2 > r2)) a.removed[rk] = 1;
            }
        }
        ptr = p + 1;
        __syncthreads();
    }
    if (threadIdx.x == 0) *a.ncentres = cnt;
}

// Eq. 3-12 for the selected centres (thread per centre): dhat = distance to
// the nearest other centre (a single centre: twice its radius), then
// d = 2 sqrt(-ln(gamma / w^2)) / dhat on all axes, angles 0, w = t.
__global__ void k_init_params(const float *x, const float *y, const float *z, const float *t, const float *S,
                              const uint32_t *centres, const uint32_t *ncentres, int32_t cap, float gamma, float *p,
                              int32_t *m_dev) {
    const int M = (int)min(*ncentres, (uint32_t)cap);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) *m_dev = M;
    if (j >= M) return;
    const uint32_t cj = centres[j];
    const float px = x[cj], py = y[cj], pz = z[cj];
    float best = INFINITY;
    for (int i = 0; i < M; ++i) {
        if (i == j) continue;
        const uint32_t ci = centres[i];
        const float dx = x[ci] - px, dy = y[ci] - py, dz = z[ci] - pz;
        best = fminf(best, dx * dx + dy * dy + dz * dz);
    }
    const float dhat = M > 1 ? sqrtf(best) : 2.f * fabsf(S[cj]);
    const float w = t[cj];
    const float d = 2.f * sqrtf(-logf(gamma / (w * w))) / dhat;
    p[PCX * cap + j] = px;
    p[PCY * cap + j] = py;
    p[PCZ * cap + j] = pz;
    p[PD1 * cap + j] = d;
    p[PD2 * cap + j] = d;
    p[PD3 * cap + j] = d;
    p[PTX * cap + j] = 0.f;
    p[PTY * cap + j] = 0.f;
    p[PTZ * cap + j] = 0.f;
    p[PW * cap + j] = w;
}

}  // namespace

extern "C" int serbf_init_kernels(const serbf_points *pts, const float *S_raw, double gamma, serbf_params *prm,
                                  int32_t *m_out, serbf_workspace *ws, void *stream) {
    SERBF_TRACE();
    if (!pts || !prm || !prm->p || !prm->m || prm->cap < 1 || !ws || ws->magic != kMagic || !ws->binned)
        return SERBF_EINVAL;
    if (pts->n != ws->npoints || prm->cap > ws->sz.max_kernels || !(gamma > 0.0 && gamma < 1.0)) return SERBF_EINVAL;
    const int64_t n = pts->n;
    if (n > 0 && (!pts->x || !pts->y || !pts->z || !pts->t || !S_raw)) return SERBF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *count = ws->counters + 10, *ncent = ws->counters + 11;
    if (cudaMemsetAsync(count, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return SERBF_ECUDA;
    uint32_t *k = ws->keys0, *v = ws->vals0, *kt = ws->keys1, *vt = ws->vals1;
    const int grid = (int)((n + 255) / 256 < 152 * 64 ? (n + 255) / 256 : 152 * 64);
    if (n > 0) {
        k_init_keys<<<grid > 0 ? grid : 1, 256, 0, s>>>(pts->t, S_raw, n, k, v, count);
        int rc = radix_sort_pairs(&k, &v, &kt, &vt, n, 32, ws->hist, s);
        if (rc) return rc;
        // kt now holds scratch: the rank of each binned point
        k_init_rank<<<grid > 0 ? grid : 1, 256, 0, s>>>(v, n, count, kt);
        InitArgs a;
        a.x = pts->x;
        a.y = pts->y;
        a.z = pts->z;
        a.S = S_raw;
        a.order = v;
        a.count = count;
        a.rank = kt;
        a.removed = reinterpret_cast<uint8_t *>(ws->nz);  // >= 16 bytes per point, free between epochs
        a.cell_start = ws->cell_start;
        a.g = ws->grid;
        a.sf = ws->sf;
        a.nsx = ws->ns[0];
        a.nsy = ws->ns[1];
        a.centres = vt;  // the sort's other value buffer is free now
        a.cap = prm->cap;
        a.ncentres = ncent;
        k_inscribed<<<1, kInitThreads, 0, s>>>(a);
        k_init_params<<<(prm->cap + 255) / 256, 256, 0, s>>>(pts->x, pts->y, pts->z, pts->t, S_raw, vt, ncent,
                                                             prm->cap, (float)gamma, prm->p, prm->m);
    } else {
        if (cudaMemsetAsync(prm->m, 0, sizeof(int32_t), s) != cudaSuccess) return SERBF_ECUDA;
    }
    SERBF_CHECK_LAUNCH();
    uint32_t found = 0;
    if (cudaMemcpyAsync(&found, ncent, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SERBF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SERBF_ECUDA;
    if (m_out) *m_out = (int32_t)found;
    return (int64_t)found > prm->cap ? SERBF_ECAPACITY : SERBF_OK;
}
