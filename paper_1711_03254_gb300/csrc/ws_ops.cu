// Elementwise pieces of the warm-start surrogate: pooling, upsampling and
// their adjoints, ReLU adjoint, masked MSE loss, Adam, FP32 -> BF16 copies.
// One thread per output element; channels-last tensors with row strides.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ws.h"

namespace ws {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void decode(long long i, int C, int W, int H, int D, int &c, int &x, int &y, int &z,
                                       int &n) {
    c = (int)(i % C);
    long long q = i / C;
    x = (int)(q % W);
    q /= W;
    y = (int)(q % H);
    q /= H;
    z = (int)(q % D);
    n = (int)(q / D);
}

__device__ __forceinline__ long long at(int n, int z, int y, int x, int D, int H, int W, int ld) {
    return ((((long long)n * D + z) * H + y) * W + x) * ld;
}

// y (D/2 x H/2 x W/2) = mean of 2x2x2 children of x (D x H x W)
__global__ void k_pool(const bf16 *__restrict__ x, int ldx, bf16 *__restrict__ y, int ldy, int N, int D, int H, int W,
                       int C) {
    const int Do = D / 2, Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Do * Ho * Wo * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int c, xo, yo, zo, n;
    decode(i, C, Wo, Ho, Do, c, xo, yo, zo, n);
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) s += __bfloat162float(x[at(n, 2 * zo + a, 2 * yo + b, 2 * xo + d, D, H, W, ldx) + c]);
    y[at(n, zo, yo, xo, Do, Ho, Wo, ldy) + c] = __float2bfloat16_rn(s * 0.125f);
}

// dx (D x H x W) = dy(parent) / 8
__global__ void k_pool_bwd(const bf16 *__restrict__ dy, int ldy, bf16 *__restrict__ dx, int ldx, int N, int D, int H,
                           int W, int C, int accumulate) {
    const long long total = (long long)N * D * H * W * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int c, x, y, z, n;
    decode(i, C, W, H, D, c, x, y, z, n);
    float g = __bfloat162float(dy[at(n, z / 2, y / 2, x / 2, D / 2, H / 2, W / 2, ldy) + c]) * 0.125f;
    bf16 *o = dx + at(n, z, y, x, D, H, W, ldx) + c;
    if (accumulate) g += __bfloat162float(*o);
    *o = __float2bfloat16_rn(g);
}

// y (2D x 2H x 2W) = x(parent)
__global__ void k_up(const bf16 *__restrict__ x, int ldx, bf16 *__restrict__ y, int ldy, int N, int D, int H, int W,
                     int C) {
    const int Do = 2 * D, Ho = 2 * H, Wo = 2 * W;
    const long long total = (long long)N * Do * Ho * Wo * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int c, xo, yo, zo, n;
    decode(i, C, Wo, Ho, Do, c, xo, yo, zo, n);
    y[at(n, zo, yo, xo, Do, Ho, Wo, ldy) + c] = x[at(n, zo / 2, yo / 2, xo / 2, D, H, W, ldx) + c];
}

// dx (D x H x W) (+)= sum of the 8 children of dy (2D x 2H x 2W)
__global__ void k_up_bwd(const bf16 *__restrict__ dy, int ldy, bf16 *__restrict__ dx, int ldx, int N, int D, int H,
                         int W, int C, int accumulate) {
    const long long total = (long long)N * D * H * W * C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int c, x, y, z, n;
    decode(i, C, W, H, D, c, x, y, z, n);
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d)
                s += __bfloat162float(dy[at(n, 2 * z + a, 2 * y + b, 2 * x + d, 2 * D, 2 * H, 2 * W, ldy) + c]);
    bf16 *o = dx + at(n, z, y, x, D, H, W, ldx) + c;
    if (accumulate) s += __bfloat162float(*o);
    *o = __float2bfloat16_rn(s);
}

__global__ void k_relu_bwd(const bf16 *__restrict__ y, int ldy, bf16 *__restrict__ dy, int lddy, long long P, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    const long long p = i / C;
    const int c = (int)(i % C);
    if (!(__bfloat162float(y[p * ldy + c]) > 0.f)) dy[p * lddy + c] = __float2bfloat16_rn(0.f);
}

__global__ void k_mse(const float *__restrict__ pred, int ldp, const float *__restrict__ target,
                      const uint8_t *__restrict__ mask, const float *__restrict__ wch, bf16 *__restrict__ dpred,
                      int lddp, float *__restrict__ loss, long long P, int C, float inv_count) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (p < P) {
        const bool m = mask[p] != 0;
        for (int c = 0; c < lddp; ++c) {
            float g = 0.f;
            if (m && c < C) {
                const float d = pred[p * ldp + c] - target[p * C + c];
                l += wch[c] * d * d * inv_count;
                g = 2.f * wch[c] * d * inv_count;
            }
            dpred[p * lddp + c] = __float2bfloat16_rn(g);
        }
    }
    // block reduction of the loss
    __shared__ float sh[256];
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0]);
}

__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v, float *__restrict__ g,
                       bf16 *__restrict__ wb, long long n, float lr_t, float b1, float b2, float eps, float wd) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i] + wd * w[i];
    g[i] = 0.f;  // the gradient buffer is ready for the next accumulation
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr_t * mi / (sqrtf(vi) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float *__restrict__ x, int ldx, bf16 *__restrict__ y, int ldy, long long P, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * C) return;
    const long long p = i / C;
    const int c = (int)(i % C);
    y[p * ldy + c] = __float2bfloat16_rn(x[p * ldx + c]);
}

static unsigned blocks_for(long long total) { return (unsigned)((total + 255) / 256); }
static bool dims_ok(int N, int D, int H, int W, int C) { return N > 0 && D > 0 && H > 0 && W > 0 && C > 0; }

}  // namespace ws

using namespace ws;

extern "C" {

int ws_avgpool2(const void *x, int ldx, void *y, int ldy, int N, int D, int H, int W, int C, void *stream) {
    if (!x || !y || !dims_ok(N, D, H, W, C) || (D | H | W) & 1 || ldx < C || ldy < C) return 1;
    const long long total = (long long)N * (D / 2) * (H / 2) * (W / 2) * C;
    k_pool<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, ldx, (bf16 *)y, ldy, N, D, H, W, C);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_avgpool2_bwd(const void *dy, int ldy, void *dx, int ldx, int N, int D, int H, int W, int C, int accumulate,
                    void *stream) {
    if (!dy || !dx || !dims_ok(N, D, H, W, C) || (D | H | W) & 1 || ldx < C || ldy < C) return 1;
    const long long total = (long long)N * D * H * W * C;
    k_pool_bwd<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, ldy, (bf16 *)dx, ldx, N, D, H,
                                                                    W, C, accumulate);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_upsample2(const void *x, int ldx, void *y, int ldy, int N, int D, int H, int W, int C, void *stream) {
    if (!x || !y || !dims_ok(N, D, H, W, C) || ldx < C || ldy < C) return 1;
    const long long total = (long long)N * 8 * D * H * W * C;
    k_up<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, ldx, (bf16 *)y, ldy, N, D, H, W, C);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_upsample2_bwd(const void *dy, int ldy, void *dx, int ldx, int N, int D, int H, int W, int C, int accumulate,
                     void *stream) {
    if (!dy || !dx || !dims_ok(N, D, H, W, C) || ldx < C || ldy < C) return 1;
    const long long total = (long long)N * D * H * W * C;
    k_up_bwd<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, ldy, (bf16 *)dx, ldx, N, D, H, W,
                                                                  C, accumulate);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_relu_bwd(const void *y, int ldy, void *dy, int lddy, long long P, int C, void *stream) {
    if (!y || !dy || P < 1 || C < 1 || ldy < C || lddy < C) return 1;
    k_relu_bwd<<<blocks_for(P * C), 256, 0, (cudaStream_t)stream>>>((const bf16 *)y, ldy, (bf16 *)dy, lddy, P, C);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_mse_loss(const float *pred, int ldp, const float *target, const uint8_t *mask, const float *wch, void *dpred,
                int lddp, float *loss, long long P, int C, void *stream) {
    if (!pred || !target || !mask || !wch || !dpred || !loss || P < 1 || C < 1 || ldp < C || lddp < C) return 1;
    k_mse<<<blocks_for(P), 256, 0, (cudaStream_t)stream>>>(pred, ldp, target, mask, wch, (bf16 *)dpred, lddp, loss,
                                                           P, C, 1.0f / (float)(P * C));
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_adam(float *w, float *m, float *v, float *g, void *wb, long long n, float lr_t, float beta1, float beta2,
            float eps, float weight_decay, void *stream) {
    if (!w || !m || !v || !g || n < 1) return 1;
    k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(w, m, v, g, (bf16 *)wb, n, lr_t, beta1, beta2, eps,
                                                            weight_decay);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_to_bf16(const float *x, int ldx, void *y, int ldy, long long P, int C, void *stream) {
    if (!x || !y || P < 1 || C < 1 || ldx < C || ldy < C) return 1;
    k_to_bf16<<<blocks_for(P * C), 256, 0, (cudaStream_t)stream>>>(x, ldx, (bf16 *)y, ldy, P, C);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
