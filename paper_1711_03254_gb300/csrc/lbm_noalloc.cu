// Allocation-free variant of the FP64 field reductions (lbm_field_sums_static).
//
// Some callers cannot allocate device memory at the point where they need a
// check of mass and momentum: code running inside a pre-sized memory pool
// (an allocator that must not grow), real-time loops that forbid cudaMalloc
// because it synchronises the device, and embedding hosts that own all GPU
// memory themselves.  This entry point therefore keeps its per-block partial
// sums in a fixed, file-scope device array instead of allocating them.
//
// The array lives in every GPU that loads the library until the process
// exits (kStaticBlocks * kStaticMaxBatch * 8 doubles = 1 MiB).  Host code sees
// `g_sum_scratch` only as a host-side stand-in, so the device address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.  All calls share the array: two calls that overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <mutex>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kStaticThreads = 256;
constexpr int kStaticBlocks = 256;    // partial sums per instance
constexpr int kStaticMaxBatch = 64;   // instances per call
constexpr int kStaticVals = 8;        // M1 M2 Px Py Pz max|u| non-finite count, pad

static __device__ __align__(256) double g_sum_scratch[kStaticMaxBatch * kStaticBlocks * kStaticVals];

__device__ __forceinline__ double ws_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double ws_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// acc[5] is a maximum, the others sums; the block result goes to out[0..7].
__device__ void static_block_reduce(double (&acc)[kStaticVals], double *out) {
    __shared__ double sh[kStaticThreads / 32][kStaticVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < kStaticVals; ++c) acc[c] = c == 5 ? ws_max(acc[c]) : ws_sum(acc[c]);
    if (lane == 0)
        for (int c = 0; c < kStaticVals; ++c) sh[warp][c] = acc[c];
    __syncthreads();
    if (warp == 0) {
        for (int c = 0; c < kStaticVals; ++c) {
            double v = lane < kStaticThreads / 32 ? sh[lane][c] : 0.0;
            v = c == 5 ? ws_max(v) : ws_sum(v);
            if (lane == 0) out[c] = v;
        }
    }
}

__global__ void __launch_bounds__(kStaticThreads)
k_static_partial(const double *__restrict__ r1, const double *__restrict__ r2, const double *__restrict__ u,
                 const uint8_t *__restrict__ type, long long n, double *__restrict__ scratch) {
    const int b = blockIdx.y;
    double acc[kStaticVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long stride = (long long)kStaticBlocks * kStaticThreads;
    for (long long k = (long long)blockIdx.x * kStaticThreads + threadIdx.x; k < n; k += stride) {
        const long long gk = (long long)b * n + k;
        if (type[gk] == kSolid) continue;
        const double a = r1[gk], c = r2[gk];
        const double ux = u[3 * gk], uy = u[3 * gk + 1], uz = u[3 * gk + 2];
        const double rho = a + c, uu = ux * ux + uy * uy + uz * uz;
        acc[0] += a;
        acc[1] += c;
        acc[2] += rho * ux;
        acc[3] += rho * uy;
        acc[4] += rho * uz;
        const bool finite = isfinite(rho) && isfinite(uu);
        acc[5] = fmax(acc[5], finite ? sqrt(uu) : 0.0);
        acc[6] += finite ? 0.0 : 1.0;
    }
    static_block_reduce(acc, scratch + ((long long)b * kStaticBlocks + blockIdx.x) * kStaticVals);
}

__global__ void __launch_bounds__(kStaticThreads)
k_static_final(const double *__restrict__ scratch, double *__restrict__ out) {
    const int b = blockIdx.x;
    double acc[kStaticVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < kStaticBlocks; k += kStaticThreads) {
        const double *p = scratch + ((long long)b * kStaticBlocks + k) * kStaticVals;
        for (int c = 0; c < kStaticVals; ++c) acc[c] = c == 5 ? fmax(acc[c], p[c]) : acc[c] + p[c];
    }
    __shared__ double res[kStaticVals];
    static_block_reduce(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        double *o = out + (long long)b * 6;
        for (int c = 0; c < 5; ++c) o[c] = res[c];
        o[5] = res[6] > 0 ? nan("") : res[5];
    }
}

namespace {
std::mutex g_sym_mu;
double *g_sym_ptr[64] = {nullptr};  // device address of g_sum_scratch, per device
}  // namespace

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_field_sums_static(const double *rho1, const double *rho2, const double *u,
                                            const uint8_t *cell_type, long long ncells, int batch, double *out,
                                            void *stream) {
    if (!rho1 || !rho2 || !u || !cell_type || !out || ncells < 1 || batch < 1) return LBM_ERR_ARG;
    if (batch > kStaticMaxBatch) return LBM_ERR_ARG;  // the fixed scratch holds 64 instances
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LBM_ERR_CUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_sym_mu);
        if (!g_sym_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sum_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
            g_sym_ptr[dev] = (double *)p;
        }
        scratch = g_sym_ptr[dev];
    }
    // cudaLaunchKernel returns the error of this launch itself, so an error
    // left pending by some other launch on this thread is neither reported
    // here nor cleared
    cudaStream_t s = (cudaStream_t)stream;
    long long n = ncells;
    void *pargs[] = {(void *)&rho1, (void *)&rho2, (void *)&u, (void *)&cell_type, (void *)&n, (void *)&scratch};
    if (cudaLaunchKernel((const void *)k_static_partial, dim3(kStaticBlocks, (unsigned)batch, 1),
                         dim3(kStaticThreads, 1, 1), pargs, 0, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    const double *sc = scratch;
    void *fargs[] = {(void *)&sc, (void *)&out};
    if (cudaLaunchKernel((const void *)k_static_final, dim3((unsigned)batch, 1, 1), dim3(kStaticThreads, 1, 1), fargs,
                         0, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}
