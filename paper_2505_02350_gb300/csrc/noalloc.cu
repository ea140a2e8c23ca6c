// Allocation-free variant of the Eq. 3-10 target normalisation.
//
// serbf_normalize_sdf keeps its reduction scratch in the caller's workspace,
// which the caller has to allocate on the device first.  This variant keeps the
// scratch in a fixed array of this library instead, for callers that cannot
// allocate device memory at the point where they need the normalisation: an
// application that only hands out buffers from its own pool, or a loop that
// must not allocate once it runs.
#include <math.h>

#include <mutex>

#include "common.cuh"

using namespace serbf;

namespace {

constexpr int kNaItemsPerBlock = 4096;  // points reduced by one block
constexpr int kNaMaxBlocks = 16384;     // partial minima the scratch array holds
constexpr int64_t kNaMaxPoints = (int64_t)kNaItemsPerBlock * kNaMaxBlocks;  // 67,108,864
constexpr int kNaMaxDevices = 64;

// One partial minimum per block (order-preserving int encoding of the float).
// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) int g_na_scratch[kNaMaxBlocks];

std::mutex g_na_mutex;
int *g_na_ptr[kNaMaxDevices] = {nullptr};
int g_na_sms[kNaMaxDevices] = {0};

// Device address of the scratch array on the current device and the device's
// SM count, looked up once per device (the symbol's host-side name is not a
// device address).
int na_setup(int **out, int *sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SERBF_ECUDA;
    if (dev < 0 || dev >= kNaMaxDevices) return SERBF_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return SERBF_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return SERBF_ECUDA;
        g_na_sms[dev] = n;
        g_na_ptr[dev] = static_cast<int *>(p);
    }
    *out = g_na_ptr[dev];
    *sms = g_na_sms[dev];
    return SERBF_OK;
}

__device__ __forceinline__ int na_key(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float na_val(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// Every block writes the minimum of its chunk: no slot needs clearing first.
__global__ void __launch_bounds__(256) k_na_min(const float *S, int64_t n, int *partial) {
    __shared__ int red[8];
    const int64_t b0 = (int64_t)blockIdx.x * kNaItemsPerBlock;
    int best = 0x7fffffff;
    for (int k = threadIdx.x; k < kNaItemsPerBlock; k += blockDim.x) {
        const int64_t i = b0 + k;
        if (i < n) best = min(best, na_key(S[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) best = min(best, red[w]);
        partial[blockIdx.x] = best;
    }
}

// m = min S, h = ln 2 / m^2 (Eq. 3-10), written to the caller's mh[2].
__global__ void __launch_bounds__(256) k_na_finish(const int *partial, int nblocks, double *mh) {
    __shared__ int red[8];
    int best = 0x7fffffff;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) best = min(best, partial[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) best = min(best, red[w]);
        const double m = (double)na_val(best);
        mh[0] = m;
        mh[1] = log(2.0) / (m * m);
    }
}

// Eq. 3-10 per element with the workspace version's arithmetic
// (eq310_target), so both give identical targets.
__global__ void k_na_apply(const float *S, float *t, int64_t n, const double *mh) {
    __shared__ ff c[kEq310Terms];
    if (threadIdx.x == 0) eq310_coefs(c);
    __syncthreads();
    const float m = (float)mh[0];  // the minimum sample, exactly
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = eq310_target(S[i], m, c);
}

}  // namespace

extern "C" int serbf_normalize_sdf_noalloc(const float *S, float *t, int64_t n, double *mh_dev, void *stream) {
    if (!S || !t || !mh_dev || n <= 0) return SERBF_EINVAL;
    if (n > kNaMaxPoints) return SERBF_ECAPACITY;
    int *scratch = nullptr;
    int sms = 0;
    int rc = na_setup(&scratch, &sms);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)((n + kNaItemsPerBlock - 1) / kNaItemsPerBlock);
    k_na_min<<<nblocks, 256, 0, s>>>(S, n, scratch);
    k_na_finish<<<1, 256, 0, s>>>(scratch, nblocks, mh_dev);
    int64_t ab = (n + 255) / 256;
    if (ab > (int64_t)sms * 8) ab = (int64_t)sms * 8;  // grid-stride: 8 blocks of 256 per SM
    k_na_apply<<<(unsigned)ab, 256, 0, s>>>(S, t, n, mh_dev);
    SERBF_CHECK_LAUNCH();
    return SERBF_OK;
}
