// S8: FP64 reductions of the macroscopic fields, per instance: component
// masses, momentum sum rho u_F, |u - u_snap|^2, |u|^2, max |u_F| and a count of
// non-finite values.  Warp shuffles, then shared memory, then a second kernel
// that adds the per-block partials in a fixed order, so the result does not
// depend on scheduling.  The velocity snapshot for the residual is refreshed
// in the same pass.
#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kRedThreads = 256;
constexpr int kRedVals = 9;  // m1 m2 px py pz d2 u2 umax bad
constexpr int kRedGroup = 8; // cells per FP32 partial sum (FP32 fields)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction of kRedVals values (the 8th is a max), written by thread 0.
__device__ void block_reduce(double (&acc)[kRedVals], double *out) {
    __shared__ double sh[kRedThreads / 32][kRedVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < kRedVals; ++c) acc[c] = c == 7 ? warp_max(acc[c]) : warp_sum(acc[c]);
    if (lane == 0)
        for (int c = 0; c < kRedVals; ++c) sh[warp][c] = acc[c];
    __syncthreads();
    if (warp == 0) {
        for (int c = 0; c < kRedVals; ++c) {
            double v = lane < kRedThreads / 32 ? sh[lane][c] : (c == 7 ? 0.0 : 0.0);
            v = c == 7 ? warp_max(v) : warp_sum(v);
            if (lane == 0) out[c] = v;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_reduce_partial(const T *__restrict__ macro, T *__restrict__ usnap,
                                                                const uint32_t *__restrict__ link, Grid g,
                                                                double *__restrict__ partial, int nblk) {
    const int b = blockIdx.y;
    const T *mac = macro + (long long)b * 5 * g.n;
    T *us = usnap + (long long)b * 3 * g.n;
    const uint32_t *lk = link + (long long)b * g.n;
    double acc[kRedVals] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const long long stride = (long long)nblk * kRedThreads;
    if constexpr (std::is_same<T, float>::value) {
        // FP32 fields: the per-cell terms in FP32 (exact products of FP32
        // values but for one rounding each), summed in FP32 over groups of
        // kRedGroup cells of the thread's sequence and the group sums in FP64.
        // GB300's FP64 pipe (2 lanes per clock per SM) made the all-FP64 pass
        // ten times slower than its memory traffic.
        float part[7] = {0, 0, 0, 0, 0, 0, 0}, umax = 0.f;
        int n_in = 0;
        for (long long k = (long long)blockIdx.x * kRedThreads + threadIdx.x; k < g.n; k += stride) {
            if (cell_type(lk[k]) != kSolid) {
                const float r1 = mac[k], r2 = mac[g.n + k];
                const float ux = mac[2 * g.n + k], uy = mac[3 * g.n + k], uz = mac[4 * g.n + k];
                const float dx = ux - us[k], dy = uy - us[g.n + k], dz = uz - us[2 * g.n + k];
                const float rho = r1 + r2;
                part[0] += r1;
                part[1] += r2;
                part[2] += rho * ux;
                part[3] += rho * uy;
                part[4] += rho * uz;
                part[5] += dx * dx + dy * dy + dz * dz;
                const float uu = ux * ux + uy * uy + uz * uz;
                part[6] += uu;
                const bool finite = isfinite(r1) && isfinite(r2) && isfinite(uu);
                umax = fmaxf(umax, finite ? uu : 0.f);
                if (!finite) acc[8] += 1.0;
                us[k] = ux;
                us[g.n + k] = uy;
                us[2 * g.n + k] = uz;
            }
            if (++n_in == kRedGroup) {
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    acc[c] += (double)part[c];
                    part[c] = 0.f;
                }
                n_in = 0;
            }
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[c] += (double)part[c];
        acc[7] = (double)umax;
    } else {
        for (long long k = (long long)blockIdx.x * kRedThreads + threadIdx.x; k < g.n; k += stride) {
            if (cell_type(lk[k]) == kSolid) continue;
            const double r1 = (double)mac[k], r2 = (double)mac[g.n + k];
            const double ux = (double)mac[2 * g.n + k], uy = (double)mac[3 * g.n + k], uz = (double)mac[4 * g.n + k];
            const double sx = (double)us[k], sy = (double)us[g.n + k], sz = (double)us[2 * g.n + k];
            const double rho = r1 + r2;
            acc[0] += r1;
            acc[1] += r2;
            acc[2] += rho * ux;
            acc[3] += rho * uy;
            acc[4] += rho * uz;
            acc[5] += (ux - sx) * (ux - sx) + (uy - sy) * (uy - sy) + (uz - sz) * (uz - sz);
            const double uu = ux * ux + uy * uy + uz * uz;
            acc[6] += uu;
            const bool finite = isfinite(r1) && isfinite(r2) && isfinite(uu);
            // max |u|^2 here, its root once in k_reduce_final (sqrt is monotonic and
            // correctly rounded, so the result is the same); GB300's FP64 pipe is
            // what bounds this pass
            acc[7] = fmax(acc[7], finite ? uu : 0.0);
            if (!finite) acc[8] += 1.0;
            us[k] = mac[2 * g.n + k];
            us[g.n + k] = mac[3 * g.n + k];
            us[2 * g.n + k] = mac[4 * g.n + k];
        }
    }
    block_reduce(acc, partial + ((long long)b * nblk + blockIdx.x) * kRedVals);
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double *__restrict__ partial, int nblk,
                                                              double *__restrict__ out) {
    const int b = blockIdx.x;
    double acc[kRedVals] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < nblk; k += kRedThreads) {
        const double *p = partial + ((long long)b * nblk + k) * kRedVals;
        for (int c = 0; c < kRedVals; ++c) acc[c] = c == 7 ? fmax(acc[c], p[c]) : acc[c] + p[c];
    }
    block_reduce(acc, out + (long long)b * kRedVals);
    if (threadIdx.x == 0) out[(long long)b * kRedVals + 7] = sqrt(out[(long long)b * kRedVals + 7]);
}

// up to 8 blocks per SM of the 152 (a full SM of 256-thread blocks)
int reduce_blocks(long long n) {
    long long b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < 1216 ? b : 1216);
}

cudaError_t launch_reduce(const ReduceArgs &a, int *launches) {
    const dim3 grid((unsigned)a.nblk, (unsigned)a.batch, 1);
    if (a.fp64)
        k_reduce_partial<double><<<grid, kRedThreads, 0, a.stream>>>((const double *)a.macro, (double *)a.usnap,
                                                                     a.link, a.g, a.partial, a.nblk);
    else
        k_reduce_partial<float><<<grid, kRedThreads, 0, a.stream>>>((const float *)a.macro, (float *)a.usnap, a.link,
                                                                    a.g, a.partial, a.nblk);
    k_reduce_final<<<a.batch, kRedThreads, 0, a.stream>>>(a.partial, a.nblk, a.out);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace lbm
