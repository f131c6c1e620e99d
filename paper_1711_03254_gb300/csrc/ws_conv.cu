// Tensor-core kernels of the warm-start surrogate (3-D convolutional U-Net):
// BF16 operands, FP32 accumulation.
//
//   ws_conv3d_fwd        implicit GEMM  Y[p, co] = b[co] + sum_{t, ci} W[co, t, ci] X[p + t - r, ci]
//                        (M = positions, N = output channels, K = taps x input channels),
//                        optional ReLU, BF16 or FP32 output.
//   ws_conv3d_bwd_data   the same kernel on dY with the weights flipped and transposed
//                        (ws_conv3d_flip_weights).
//   ws_conv3d_bwd_weight dW[co, t, ci] += sum_p dY[p, co] X[p + t - r, ci]: one GEMM per tap
//                        (M = Co, N = Ci, K = positions), split over position chunks.
//
// The products use warp-level mma.sync m16n8k16 BF16 instructions fed by
// ldmatrix from cp.async double-buffered shared-memory tiles.
//
// Activations are channels-last with a row stride (ld) and a channel offset,
// so concatenations are views of one buffer.  Channel counts are multiples of
// 16 (the host checks).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ws.h"

namespace ws {

using bf16 = __nv_bfloat16;

struct Act {
    int N, D, H, W;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;  // zero-fill when the source is outside the volume
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void *p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void ldmatrix_x4_trans(unsigned (&r)[4], const void *p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------------ forward

constexpr int FBM = 128, FBN = 64, FBK = 16, FPAD = 8;
constexpr int FTHREADS = 256;

// X: [P][ldx] (channel offset already applied), Wt: [Co][KV][Ci], Y: [P][ldy]
template <bool OUT_F32>
__global__ void __launch_bounds__(FTHREADS) k_conv_fwd(const bf16 *__restrict__ X, int ldx, const bf16 *__restrict__ Wt,
                                                       const float *__restrict__ bias, void *__restrict__ Y, int ldy,
                                                       Act a, int Ci, int Co, int k, int relu) {
    __shared__ __align__(16) bf16 sA[2][FBM][FBK + FPAD];
    __shared__ __align__(16) bf16 sB[2][FBN][FBK + FPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;  // 4 x 2 warps, 32 x 32 each
    const long long P = (long long)a.N * a.D * a.H * a.W;
    const long long m0 = (long long)blockIdx.x * FBM;
    const int n0 = blockIdx.y * FBN;
    const int r = k / 2, KV = k * k * k;

    // the A row and half-row this thread loads
    const int arow = tid >> 1, ahalf = (tid & 1) * 8;
    const long long p = m0 + arow;
    int pn = 0, pz = 0, py = 0, px = 0;
    const bool prow = p < P;
    if (prow) {
        long long q = p;
        px = (int)(q % a.W); q /= a.W;
        py = (int)(q % a.H); q /= a.H;
        pz = (int)(q % a.D); q /= a.D;
        pn = (int)q;
    }
    const int brow = tid >> 1, bhalf = (tid & 1) * 8;  // threads 0..127 load B
    const int nchunk = Ci / FBK;
    const int iters = KV * nchunk;

    auto load_stage = [&](int it, int st) {
        const int t = it / nchunk, c0 = (it - t * nchunk) * FBK;
        const int tz = t / (k * k), ty = (t / k) % k, tx = t % k;
        const int zz = pz + tz - r, yy = py + ty - r, xx = px + tx - r;
        const bool ok = prow && zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        const long long src = ok ? ((((long long)pn * a.D + zz) * a.H + yy) * a.W + xx) * ldx + c0 + ahalf : 0;
        cp_async16(&sA[st][arow][ahalf], X + src, ok);
        if (tid < FBN * 2) {
            const int co = n0 + brow;
            const bool okb = co < Co;
            const long long bsrc = okb ? ((long long)co * KV + t) * Ci + c0 + bhalf : 0;
            cp_async16(&sB[st][brow][bhalf], Wt + bsrc, okb);
        }
        cp_async_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;

    load_stage(0, 0);
    for (int it = 0; it < iters; ++it) {
        const int st = it & 1;
        cp_async_wait0();
        __syncthreads();
        if (it + 1 < iters) load_stage(it + 1, st ^ 1);
        unsigned af[2][4], bfr[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            const int row = wm * 32 + mi * 16 + ((lane >> 3) & 1) * 8 + (lane & 7);
            const int col = (lane >> 4) * 8;
            ldmatrix_x4(af[mi], &sA[st][row][col]);
        }
#pragma unroll
        for (int nj = 0; nj < 2; ++nj) {
            const int mtx = lane >> 3;
            const int row = wn * 32 + nj * 16 + (mtx >> 1) * 8 + (lane & 7);
            const int col = (mtx & 1) * 8;
            ldmatrix_x4(bfr[nj], &sB[st][row][col]);
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni)
                mma_bf16(acc[mi][ni], af[mi], bfr[ni >> 1][(ni & 1) * 2], bfr[ni >> 1][(ni & 1) * 2 + 1]);
        __syncthreads();
    }

    // epilogue: bias, ReLU, store
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long row = m0 + wm * 32 + mi * 16 + (lane >> 2) + h * 8;
                const int col = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
                if (row >= P || col >= Co) continue;
                float v0 = acc[mi][ni][h * 2], v1 = acc[mi][ni][h * 2 + 1];
                if (bias) {
                    v0 += bias[col];
                    v1 += bias[col + 1];
                }
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (OUT_F32) {
                    float2 *dst = reinterpret_cast<float2 *>((float *)Y + row * ldy + col);
                    *dst = make_float2(v0, v1);
                } else {
                    __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>((bf16 *)Y + row * ldy + col);
                    *dst = __floats2bfloat162_rn(v0, v1);
                }
            }
}

// W' [Ci][KV][Co] = W [Co][KV-1-t][Ci]: backward-data weights
__global__ void k_flip_weights(const bf16 *__restrict__ W, bf16 *__restrict__ Wf, int Co, int KV, int Ci) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)Co * KV * Ci;
    if (i >= total) return;
    const int ci = (int)(i % Ci);
    const int t = (int)((i / Ci) % KV);
    const int co = (int)(i / ((long long)Ci * KV));
    Wf[((long long)ci * KV + (KV - 1 - t)) * Co + co] = W[i];
}

// ------------------------------------------------------------------ backward weight

constexpr int WBM = 64, WBN = 64, WBK = 32, WPAD = 8;
constexpr int WTHREADS = 256;

// dW[co][t][ci] += sum_{p in chunk} dY[p][co] X[p + t - r][ci]
__global__ void __launch_bounds__(WTHREADS) k_conv_wgrad(const bf16 *__restrict__ X, int ldx,
                                                         const bf16 *__restrict__ dY, int ldy,
                                                         float *__restrict__ dW, Act a, int Ci, int Co, int k,
                                                         long long chunk) {
    __shared__ __align__(16) bf16 sY[2][WBK][WBM + WPAD];  // [p][co]
    __shared__ __align__(16) bf16 sX[2][WBK][WBN + WPAD];  // [p][ci]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps: 32 (co) x 16 (ci) each
    const int KV = k * k * k, r = k / 2;
    const int t = blockIdx.z % KV;
    const long long kc = blockIdx.z / KV;  // position chunk
    const int co0 = blockIdx.y * WBM;
    const int ci0 = blockIdx.x * WBN;
    const long long P = (long long)a.N * a.D * a.H * a.W;
    const long long pbeg = kc * chunk, pend = pbeg + chunk < P ? pbeg + chunk : P;
    const int tz = t / (k * k), ty = (t / k) % k, tx = t % k;

    // load mapping: 32 rows (positions) x 64 channels = 32 x 8 vectors of 16 B: 256 threads, one each
    const int lrow = tid >> 3, lcol = (tid & 7) * 8;
    auto load_stage = [&](long long pb, int st) {
        const long long p = pb + lrow;
        bool okp = p < pend;
        long long srcx = 0, srcy = 0;
        bool okx = false;
        if (okp) {
            long long q = p;
            const int px = (int)(q % a.W); q /= a.W;
            const int py = (int)(q % a.H); q /= a.H;
            const int pz = (int)(q % a.D); q /= a.D;
            const int pn = (int)q;
            const int zz = pz + tz - r, yy = py + ty - r, xx = px + tx - r;
            okx = zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            if (okx) srcx = ((((long long)pn * a.D + zz) * a.H + yy) * a.W + xx) * ldx + ci0 + lcol;
            srcy = p * ldy + co0 + lcol;
        }
        const bool oky = okp && co0 + lcol < Co;
        okx = okx && ci0 + lcol < Ci;
        cp_async16(&sY[st][lrow][lcol], dY + (oky ? srcy : 0), oky);
        cp_async16(&sX[st][lrow][lcol], X + (okx ? srcx : 0), okx);
        cp_async_commit();
    };

    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;

    const int iters = (int)((pend - pbeg + WBK - 1) / WBK);
    if (iters > 0) load_stage(pbeg, 0);
    for (int it = 0; it < iters; ++it) {
        const int st = it & 1;
        cp_async_wait0();
        __syncthreads();
        if (it + 1 < iters) load_stage(pbeg + (long long)(it + 1) * WBK, st ^ 1);
#pragma unroll
        for (int ks = 0; ks < WBK / 16; ++ks) {
            // A = dY^T (m = co, k = p): smem [p][co] holds A transposed -> ldmatrix.trans
            unsigned af[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int mtx = lane >> 3;
                const int prow = ks * 16 + (mtx >> 1) * 8 + (lane & 7);
                const int ccol = wm * 32 + mi * 16 + (mtx & 1) * 8;
                ldmatrix_x4_trans(af[mi], &sY[st][prow][ccol]);
            }
            // B (k = p, n = ci): smem [p][ci] is k-major -> ldmatrix.trans gives the col-major fragment
            unsigned bfr[4];
            {
                const int mtx = lane >> 3;
                const int prow = ks * 16 + (mtx & 1) * 8 + (lane & 7);
                const int ccol = wn * 16 + (mtx >> 1) * 8;
                ldmatrix_x4_trans(bfr, &sX[st][prow][ccol]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 2; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni * 2], bfr[ni * 2 + 1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = co0 + wm * 32 + mi * 16 + (lane >> 2) + h * 8;
                const int ci = ci0 + wn * 16 + ni * 8 + (lane & 3) * 2;
                if (co >= Co || ci >= Ci) continue;
                float *dst = dW + ((long long)co * KV + t) * Ci + ci;
                atomicAdd(dst, acc[mi][ni][h * 2]);
                atomicAdd(dst + 1, acc[mi][ni][h * 2 + 1]);
            }
}

// db[co] += sum_p dY[p][co]
__global__ void k_bias_grad(const bf16 *__restrict__ dY, int ldy, float *__restrict__ db, long long P, int Co) {
    const int co = blockIdx.y * 32 + (threadIdx.x & 31);
    const int lanes = blockDim.x / 32;
    float s = 0.f;
    if (co < Co)
        for (long long p = (long long)blockIdx.x * lanes + (threadIdx.x >> 5); p < P; p += (long long)gridDim.x * lanes)
            s += __bfloat162float(dY[p * ldy + co]);
    __shared__ float sh[32][33];
    sh[threadIdx.x >> 5][threadIdx.x & 31] = s;
    __syncthreads();
    if (threadIdx.x < 32 && co < Co) {
        float t = 0.f;
        for (int w = 0; w < lanes; ++w) t += sh[w][threadIdx.x];
        atomicAdd(db + co, t);
    }
}

}  // namespace ws

using namespace ws;

static bool bad_channels(int c) { return c < 16 || (c % 16) != 0; }

extern "C" {

int ws_conv3d_fwd(const void *x, int ldx, const void *w, const float *bias, void *y, int ldy, int y_f32, int N, int D,
                  int H, int W, int Ci, int Co, int k, int relu, void *stream) {
    if (!x || !w || !y || N < 1 || D < 1 || H < 1 || W < 1 || (k != 1 && k != 3)) return 1;
    if (bad_channels(Ci) || bad_channels(Co) || ldx < Ci || ldy < Co || (ldx % 8) || (ldy % 2)) return 1;
    if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(w) & 15)) return 1;
    Act a{N, D, H, W};
    const long long P = (long long)N * D * H * W;
    const dim3 grid((unsigned)((P + FBM - 1) / FBM), (unsigned)((Co + FBN - 1) / FBN), 1);
    cudaStream_t s = (cudaStream_t)stream;
    if (y_f32)
        k_conv_fwd<true><<<grid, FTHREADS, 0, s>>>((const bf16 *)x, ldx, (const bf16 *)w, bias, y, ldy, a, Ci, Co, k,
                                                   relu);
    else
        k_conv_fwd<false><<<grid, FTHREADS, 0, s>>>((const bf16 *)x, ldx, (const bf16 *)w, bias, y, ldy, a, Ci, Co, k,
                                                    relu);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_conv3d_flip_weights(const void *w, void *wf, int Co, int Ci, int k, void *stream) {
    if (!w || !wf || Co < 1 || Ci < 1 || (k != 1 && k != 3)) return 1;
    const int KV = k * k * k;
    const long long total = (long long)Co * KV * Ci;
    k_flip_weights<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const bf16 *)w, (bf16 *)wf, Co,
                                                                                      KV, Ci);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_conv3d_bwd_weight(const void *x, int ldx, const void *dy, int ldy, float *dw, float *db, int N, int D, int H,
                         int W, int Ci, int Co, int k, void *stream) {
    if (!x || !dy || !dw || N < 1 || D < 1 || H < 1 || W < 1 || (k != 1 && k != 3)) return 1;
    if (bad_channels(Ci) || bad_channels(Co) || ldx < Ci || ldy < Co || (ldx % 8) || (ldy % 8)) return 1;
    Act a{N, D, H, W};
    const long long P = (long long)N * D * H * W;
    const int KV = k * k * k;
    long long chunk = 4096;
    long long nk = (P + chunk - 1) / chunk;
    if (nk * KV > 60000) {  // grid.z limit
        nk = 60000 / KV;
        chunk = (P + nk - 1) / nk;
        chunk = (chunk + WBK - 1) / WBK * WBK;
        nk = (P + chunk - 1) / chunk;
    }
    const dim3 grid((unsigned)((Ci + WBN - 1) / WBN), (unsigned)((Co + WBM - 1) / WBM), (unsigned)(nk * KV));
    cudaStream_t s = (cudaStream_t)stream;
    k_conv_wgrad<<<grid, WTHREADS, 0, s>>>((const bf16 *)x, ldx, (const bf16 *)dy, ldy, dw, a, Ci, Co, k, chunk);
    if (db) {
        const long long blocks = (P + 8 * 64 - 1) / (8 * 64);
        const dim3 g2((unsigned)(blocks < 1024 ? blocks : 1024), (unsigned)((Co + 31) / 32), 1);
        k_bias_grad<<<g2, 256, 0, s>>>((const bf16 *)dy, ldy, db, P, Co);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
