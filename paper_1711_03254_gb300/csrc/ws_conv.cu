// Tensor-core kernels of the warm-start surrogate (3-D convolutional U-Net):
// BF16 operands, FP32 accumulation.
//
//   ws_conv3d_fwd        implicit GEMM  Y[p, co] = b[co] + sum_{t, ci} W[co, t, ci] X[p + t - r, ci]
//                        (M = positions, N = output channels, K = taps x input channels),
//                        optional ReLU, BF16 or FP32 output.
//   ws_conv3d_bwd_data   the same kernel on dY with the weights flipped and transposed
//                        (ws_conv3d_flip_weights).
//   ws_conv3d_bwd_weight dW[co, t, ci] += sum_p dY[p, co] X[p + t - r, ci]: rows (t, ci) x Co
//                        (M = taps x Ci, N = Co, K = positions), split over position chunks.
//
// All three products run on the tcgen05 tensor cores with the accumulator in
// tensor memory.  Kernels:
//   k_conv3_fwd_res, k_conv3_fwd_pers   forward (and data gradient) for 3x3x3, the
//                                       input tile resident in shared memory (TMA),
//                                       the taps as shifted descriptors; one block
//                                       per tile or one persistent block per SM
//   k_conv3_wgrad_res, k_conv3_wgrad_dz weight gradient for 3x3x3 from TMA line boxes,
//                                       tap pairs or dz slots as M rows
//   k_conv_fwd_tc, k_conv_wgrad_tc      the gathered kernels (cp.async, two stages):
//                                       1x1x1 and the shapes no resident plan fits
// The host picks among them (ws_conv3d_fwd_algo, ws_conv3d_bwd_weight_algo).
//
// Activations are channels-last with a row stride (ld) and a channel offset,
// so concatenations are views of one buffer.  Channel counts are multiples of
// 16 (the host checks).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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


// ------------------------------------------------------------------ forward, tcgen05
// The same implicit GEMM on the 5th-generation tensor cores: D[p, co] (FP32,
// in tensor memory) += A[p, k] B[co, k] with A the gathered input rows and B
// the weights, both K-major BF16 in shared memory, issued by one thread as
// tcgen05.mma (M = 128 positions, N = Co <= 256, K = 16 per instruction).
// Operand tiles use the no-swizzle canonical layout: 8-row x 16-byte core
// matrices, the two core matrices of a 16-wide K chunk 128 B apart (leading
// byte offset) and consecutive 8-row groups 256 B apart (stride byte offset).
// Two shared-memory stages of 4 K chunks each: cp.async fills one stage while
// the tensor cores work on the other; an mbarrier per stage, signalled by
// tcgen05.commit, says when a stage's MMAs are done.  Every wait is bounded:
// on expiry the kernel records the fault in g_tc_timeout and stops issuing.
constexpr int TBM = 128, TKC = 4, TTHREADS = 128;

__device__ int g_tc_timeout;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major canonical layout
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long it = 0; it < (1L << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    atomicExch(&g_tc_timeout, 1);
    return false;
}

template <bool OUT_F32>
__global__ void __launch_bounds__(TTHREADS) k_conv_fwd_tc(const bf16 *__restrict__ X, int ldx,
                                                         const bf16 *__restrict__ Wt, const float *__restrict__ bias,
                                                         void *__restrict__ Y, int ldy, Act a, int Ci, int Co, int k,
                                                         int relu, int tmem_cols) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int BN = Co;
    const uint32_t a_chunk = TBM * 32, b_chunk = (uint32_t)BN * 32;
    const uint32_t stage_bytes = TKC * (a_chunk + b_chunk);
    unsigned char *stage0 = sm;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 2 * stage_bytes);  // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const long long P = (long long)a.N * a.D * a.H * a.W;
    const long long m0 = (long long)blockIdx.x * TBM;
    const int r = k / 2, KV = k * k * k, cchunks = Ci / 16;
    const int nkc = KV * cchunks, nkb = (nkc + TKC - 1) / TKC;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tslot;

    // the two A rows this thread gathers (rows tid >> 1 and 64 + (tid >> 1)), half kh = tid & 1
    const int kh = tid & 1;
    int pn[2], pz[2], py[2], px[2];
    bool prow[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const long long p = m0 + j * 64 + (tid >> 1);
        prow[j] = p < P;
        long long q = prow[j] ? p : 0;
        px[j] = (int)(q % a.W); q /= a.W;
        py[j] = (int)(q % a.H); q /= a.H;
        pz[j] = (int)(q % a.D); q /= a.D;
        pn[j] = (int)q;
    }
    auto load_block = [&](int kb, int st) {
        unsigned char *sa = stage0 + st * stage_bytes;
        unsigned char *sb = sa + TKC * a_chunk;
        for (int c = 0; c < TKC; ++c) {
            const int kc = kb * TKC + c;
            if (kc >= nkc) break;
            const int t = kc / cchunks, c0 = (kc - t * cchunks) * 16;
            const int tz = t / (k * k), ty = (t / k) % k, tx = t % k;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int row = j * 64 + (tid >> 1);
                const int zz = pz[j] + tz - r, yy = py[j] + ty - r, xx = px[j] + tx - r;
                const bool ok = prow[j] && zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                const long long src =
                    ok ? ((((long long)pn[j] * a.D + zz) * a.H + yy) * a.W + xx) * ldx + c0 + kh * 8 : 0;
                cp_async16(sa + c * a_chunk + ((row >> 3) * 2 + kh) * 128 + (row & 7) * 16, X + src, ok);
            }
            for (int q = tid; q < BN * 2; q += TTHREADS) {
                const int n = q >> 1, h = q & 1;
                const long long src = ((long long)n * KV + t) * Ci + c0 + h * 8;
                cp_async16(sb + c * b_chunk + ((n >> 3) * 2 + h) * 128 + (n & 7) * 16, Wt + src, true);
            }
        }
        cp_async_commit();
    };

    const uint32_t idesc = umma_idesc_bf16(TBM, BN);
    bool ok_run = true;
    load_block(0, 0);
    for (int kb = 0; kb < nkb && ok_run; ++kb) {
        const int st = kb & 1;
        if (kb + 1 < nkb) {
            const int s1 = (kb + 1) & 1;
            if (kb + 1 >= 2) {
                // the stage is free once the MMAs of block kb - 1 are done (uniform decision)
                const bool okw = mbar_wait(smem_u32(&mbar[s1]), (uint32_t)(((kb - 1) >> 1) & 1));
                if (!__syncthreads_and(okw)) {
                    ok_run = false;
                    break;
                }
            }
            load_block(kb + 1, s1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::);
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t sa = smem_u32(stage0 + st * stage_bytes), sb = sa + TKC * a_chunk;
            for (int c = 0; c < TKC; ++c) {
                const int kc = kb * TKC + c;
                if (kc >= nkc) break;
                const uint64_t ad = umma_desc(sa + c * a_chunk, 128, 256);
                const uint64_t bd = umma_desc(sb + c * b_chunk, 128, 256);
                const uint32_t acc = kc > 0 ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mbar[st])));
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
    if (ok_run) {
        const bool okw = mbar_wait(smem_u32(&mbar[(nkb - 1) & 1]), (uint32_t)(((nkb - 1) >> 1) & 1));
        ok_run = __syncthreads_and(okw);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    if (ok_run) {
        // epilogue: warp w owns accumulator rows (TMEM lanes) 32 w .. 32 w + 31
        const long long row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
            if (row < P) {
                float o[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    float x = __uint_as_float(v[e]);
                    if (bias) x += bias[c0 + e];
                    if (relu) x = fmaxf(x, 0.f);
                    o[e] = x;
                }
                if (OUT_F32) {
                    float4 *dst = reinterpret_cast<float4 *>((float *)Y + row * ldy + c0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) dst[e] = make_float4(o[4 * e], o[4 * e + 1], o[4 * e + 2], o[4 * e + 3]);
                } else {
                    __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>((bf16 *)Y + row * ldy + c0);
#pragma unroll
                    for (int e = 0; e < 8; ++e) dst[e] = __floats2bfloat162_rn(o[2 * e], o[2 * e + 1]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
    }
}

// ------------------------------------------------------------------ forward, resident tiles (3x3x3)
// k_conv3_fwd_res: the same convolution for k = 3 with the input tile held in
// shared memory instead of gathered per tap.  A block owns the outputs of
// `by` consecutive lines of one plane.  Its input is loaded plane by plane by
// TMA: for the K-step (16-channel chunk c, plane offset dz) one box of
// (by + 2) lines x (W + 2) columns x 8 channels per K half, halo included
// (outside the volume the tensor map fills zeros), lands as rows of 16 bytes
// in the order (line, column).  In that layout an output row q = l (W + 2) + x
// and its input at tap (dy, dx) are a fixed distance apart, dy (W + 2) + dx
// rows, so the A operand of a tap is the same shared-memory tile seen through
// a descriptor that starts 16 (dy (W + 2) + dx) bytes further: the 9 taps of a
// plane cost one load.  The rows between two lines (the x halo) are computed
// and discarded.  The no-swizzle K-major layout has rows 16 bytes apart
// within a core matrix and, with a stride byte offset of 128, across core
// matrices, so any 16-byte start is a valid tile; the two K halves of a chunk
// are separate boxes one leading byte offset apart.  The weights of the 9 taps
// of (c, dz) arrive by TMA as [tap][K half][Co rows] tiles.
//
// Roles: thread 0 issues the TMA loads into a ring of stages, thread 32
// issues the MMAs (M = 128 rows per tile, N = Co, K = 16) into one
// accumulator per 128-row tile in tensor memory and releases each stage with
// tcgen05.commit; all four warps run the epilogue.  Every wait is bounded; a
// thread that gives up records it in g_tc_timeout, the MMA thread still
// commits what it issued and the TMA thread waits for its loads in flight,
// and the block writes nothing.
constexpr int RTHREADS = 128;

struct ResPlan {
    int by, nyt, pitch, ntiles, stages, cols, per_sm;
    uint32_t a_half, stage_bytes, tx_bytes;
};

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
        : "memory");
}

template <bool OUT_F32>
__global__ void __launch_bounds__(RTHREADS) k_conv3_fwd_res(const __grid_constant__ CUtensorMap xmap,
                                                           const __grid_constant__ CUtensorMap wmap,
                                                           const float *__restrict__ bias, void *__restrict__ Y,
                                                           int ldy, Act a, int Ci, int Co, int relu, ResPlan pl) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = pl.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + (size_t)NS * pl.stage_bytes);
    uint64_t *empty = full + NS;
    uint64_t *done = empty + NS;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    // the tile: lines y0 .. y0 + lt - 1 of plane z of sample n
    const int yt = blockIdx.x % pl.nyt, zn = blockIdx.x / pl.nyt;
    const int z = zn % a.D, n = zn / a.D;
    const int y0 = yt * pl.by, lt = min(pl.by, a.H - y0);
    const int nt = ((lt - 1) * pl.pitch + a.W + 127) / 128;
    // K-steps (chunk, dz) over the planes inside the volume
    const int dz_lo = z == 0 ? 1 : 0, dz_hi = z == a.D - 1 ? 1 : 2, ndz = dz_hi - dz_lo + 1;
    const int nsteps = (Ci / 16) * ndz;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(pl.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int s = 0; s < 2 * NS + 1; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tslot;
    const uint32_t base = smem_u32(sm);

    if (tid == 0) {
        // TMA producer
        int issued = 0;
        for (int s = 0; s < nsteps; ++s) {
            const int st = s % NS;
            if (s >= NS && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((s / NS) - 1) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            const int c = s / ndz, dz = dz_lo + s % ndz;
            const uint32_t fb = smem_u32(&full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(pl.tx_bytes)
                         : "memory");
            const uint32_t sa = base + (uint32_t)st * pl.stage_bytes, sb = sa + 2 * pl.a_half;
            tma_load_5d(sa, &xmap, c * 16, -1, y0 - 1, z + dz - 1, n, fb);
            tma_load_5d(sa + pl.a_half, &xmap, c * 16 + 8, -1, y0 - 1, z + dz - 1, n, fb);
            for (int t9 = 0; t9 < 9; ++t9)
                for (int h = 0; h < 2; ++h)
                    tma_load_3d(sb + (uint32_t)(t9 * 2 + h) * (uint32_t)Co * 16u, &wmap, c * 16 + 8 * h, dz * 9 + t9,
                                0, fb);
            issued = s + 1;
        }
        // wait for the loads still in flight (the last phase issued on each stage)
        for (int st = 0; st < NS && st < issued; ++st) {
            const int last = st + ((issued - 1 - st) / NS) * NS;
            mbar_wait(smem_u32(&full[st]), (uint32_t)((last / NS) & 1));
        }
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = umma_idesc_bf16(128, Co);
        for (int s = 0; s < nsteps; ++s) {
            const int st = s % NS;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((s / NS) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t sa = base + (uint32_t)st * pl.stage_bytes, sb = sa + 2 * pl.a_half;
            // descriptors of the taps: a base descriptor's start-address field (16-byte
            // units) plus the tap's offset (all addresses stay below 256 KB)
            const uint64_t ad0 = umma_desc(sa, pl.a_half, 128), bd0 = umma_desc(sb, (uint32_t)Co * 16u, 128);
            const uint32_t pitch = (uint32_t)pl.pitch, bstep = 2u * (uint32_t)Co;
            for (int j = 0; j < nt; ++j) {
                const uint64_t aj = ad0 + (uint64_t)(128 * j);
                const uint32_t dj = tmem + (uint32_t)(j * Co);
#pragma unroll
                for (int t9 = 0; t9 < 9; ++t9) {
                    const uint32_t dy = (uint32_t)(t9 / 3), dx = (uint32_t)(t9 % 3);
                    const uint64_t ad = aj + (uint64_t)(dy * pitch + dx);
                    const uint64_t bd = bd0 + (uint64_t)((uint32_t)t9 * bstep);
                    const uint32_t acc = (s > 0 || t9 > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dj),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&empty[st])));
        }
        // arrives once every MMA issued above has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(done)));
    }
    __syncwarp();
    const bool okw = mbar_wait(smem_u32(done), 0u);
    const bool ok_run = __syncthreads_and(okw) && *(volatile int *)abort_flag == 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    if (ok_run) {
        // epilogue: warp w owns accumulator rows (TMEM lanes) 32 w .. 32 w + 31 of every tile
        for (int j = 0; j < nt; ++j) {
            const int q = 128 * j + 32 * warp + lane;
            const int line = q / pl.pitch, x = q - line * pl.pitch;
            const bool valid = x < a.W && line < lt;
            const long long row = (((long long)n * a.D + z) * a.H + y0 + line) * a.W + x;
            for (int c0 = 0; c0 < Co; c0 += 16) {
                uint32_t v[16];
                const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * Co + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
                if (valid) {
                    float o[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        float xv = __uint_as_float(v[e]);
                        if (bias) xv += bias[c0 + e];
                        if (relu) xv = fmaxf(xv, 0.f);
                        o[e] = xv;
                    }
                    if (OUT_F32) {
                        float4 *dst = reinterpret_cast<float4 *>((float *)Y + row * ldy + c0);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            dst[e] = make_float4(o[4 * e], o[4 * e + 1], o[4 * e + 2], o[4 * e + 3]);
                    } else {
                        uint4 *dst = reinterpret_cast<uint4 *>((bf16 *)Y + row * ldy + c0);
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            uint4 u;
                            __nv_bfloat162 h0 = __floats2bfloat162_rn(o[8 * e], o[8 * e + 1]);
                            __nv_bfloat162 h1 = __floats2bfloat162_rn(o[8 * e + 2], o[8 * e + 3]);
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(o[8 * e + 4], o[8 * e + 5]);
                            __nv_bfloat162 h3 = __floats2bfloat162_rn(o[8 * e + 6], o[8 * e + 7]);
                            u.x = *reinterpret_cast<uint32_t *>(&h0);
                            u.y = *reinterpret_cast<uint32_t *>(&h1);
                            u.z = *reinterpret_cast<uint32_t *>(&h2);
                            u.w = *reinterpret_cast<uint32_t *>(&h3);
                            dst[e] = u;
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(pl.cols));
    }
}

// ------------------------------------------------------------------ forward, persistent resident tiles
// k_conv3_fwd_pers: the tiles of k_conv3_fwd_res (same loads, descriptors and
// accumulation order, so the same bits) computed by one persistent block per
// SM that strides over the tiles, with two accumulator buffers in tensor
// memory so that the epilogue of one tile overlaps the MMAs of the next.
// Warp 0 (one thread) issues TMA into the ring of stages across tiles, warp 1
// (one thread) issues the MMAs, warps 2-5 run the epilogue (warp w reads the
// TMEM lanes 32 (w mod 4) ..).  Barriers: full / empty per stage, tfull per
// buffer (tcgen05.commit after a tile's last K-step), tempty per buffer (one
// arrival per epilogue warp once it has read the tile).  Every wait is bounded;
// a role that gives up sets a shared flag, the others stop at their next wait,
// the MMA thread waits for its MMAs and the TMA thread for its loads before
// the block releases its tensor memory.
constexpr int PTHREADS = 192;

struct ResTile {
    int n, z, y0, lt, nt, dz_lo, ndz, nsteps;
};

__device__ __forceinline__ ResTile res_tile(int t, const Act &a, const ResPlan &pl, int Ci) {
    ResTile r;
    const int yt = t % pl.nyt, zn = t / pl.nyt;
    r.z = zn % a.D;
    r.n = zn / a.D;
    r.y0 = yt * pl.by;
    r.lt = min(pl.by, a.H - r.y0);
    r.nt = ((r.lt - 1) * pl.pitch + a.W + 127) / 128;
    r.dz_lo = r.z == 0 ? 1 : 0;
    r.ndz = (r.z == a.D - 1 ? 1 : 2) - r.dz_lo + 1;
    r.nsteps = (Ci / 16) * r.ndz;
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

template <bool OUT_F32>
__global__ void __launch_bounds__(PTHREADS, 1) k_conv3_fwd_pers(const __grid_constant__ CUtensorMap xmap,
                                                               const __grid_constant__ CUtensorMap wmap,
                                                               const float *__restrict__ bias, void *__restrict__ Y,
                                                               int ldy, Act a, int Ci, int Co, int relu, ResPlan pl,
                                                               int ntile_total, uint32_t buf_cols) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = pl.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + (size_t)NS * pl.stage_bytes);
    uint64_t *empty = full + NS;
    uint64_t *tfull = empty + NS;  // [2]
    uint64_t *tempty = tfull + 2;  // [2]
    uint64_t *done = tempty + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(pl.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int s = 0; s < 2 * NS + 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
        for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(&tempty[b])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(done)));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tslot;
    const uint32_t base = smem_u32(sm);

    if (tid == 0) {
        // TMA producer: K-steps of this block's tiles in turn, through the ring
        int g = 0, issued = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntile_total && ok; t += gridDim.x) {
            const ResTile r = res_tile(t, a, pl, Ci);
            for (int s = 0; s < r.nsteps; ++s, ++g) {
                const int st = g % NS;
                if ((g >= NS && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((g / NS) - 1) & 1))) || *abort_flag) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                const int c = s / r.ndz, dz = r.dz_lo + s % r.ndz;
                const uint32_t fb = smem_u32(&full[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(pl.tx_bytes)
                             : "memory");
                const uint32_t sa = base + (uint32_t)st * pl.stage_bytes, sb = sa + 2 * pl.a_half;
                tma_load_5d(sa, &xmap, c * 16, -1, r.y0 - 1, r.z + dz - 1, r.n, fb);
                tma_load_5d(sa + pl.a_half, &xmap, c * 16 + 8, -1, r.y0 - 1, r.z + dz - 1, r.n, fb);
                for (int t9 = 0; t9 < 9; ++t9)
                    for (int h = 0; h < 2; ++h)
                        tma_load_3d(sb + (uint32_t)(t9 * 2 + h) * (uint32_t)Co * 16u, &wmap, c * 16 + 8 * h,
                                    dz * 9 + t9, 0, fb);
                issued = g + 1;
            }
        }
        // wait for the loads still in flight (the last phase issued on each stage)
        for (int st = 0; st < NS && st < issued; ++st) {
            const int last = st + ((issued - 1 - st) / NS) * NS;
            mbar_wait(smem_u32(&full[st]), (uint32_t)((last / NS) & 1));
        }
    } else if (tid == 32) {
        // MMA issuer: tile i accumulates into buffer i & 1
        const uint32_t idesc = umma_idesc_bf16(128, Co);
        int g = 0, i = 0;
        for (int t = blockIdx.x; t < ntile_total; t += gridDim.x, ++i) {
            const ResTile r = res_tile(t, a, pl, Ci);
            const int buf = i & 1;
            if ((i >= 2 && !mbar_wait(smem_u32(&tempty[buf]), (uint32_t)(((i / 2) - 1) & 1))) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t dbase = tmem + (uint32_t)buf * buf_cols;
            bool ok = true;
            for (int s = 0; s < r.nsteps; ++s, ++g) {
                const int st = g % NS;
                if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((g / NS) & 1)) || *abort_flag) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
                const uint32_t sa = base + (uint32_t)st * pl.stage_bytes, sb = sa + 2 * pl.a_half;
                // descriptors of the taps: the start-address field (16-byte units) of a base
                // descriptor plus the tap's offset (all addresses stay below 256 KB)
                const uint64_t ad0 = umma_desc(sa, pl.a_half, 128), bd0 = umma_desc(sb, (uint32_t)Co * 16u, 128);
                const uint32_t pitch = (uint32_t)pl.pitch, bstep = 2u * (uint32_t)Co;
                for (int j = 0; j < r.nt; ++j) {
                    const uint64_t aj = ad0 + (uint64_t)(128 * j);
                    const uint32_t dj = dbase + (uint32_t)(j * Co);
#pragma unroll
                    for (int t9 = 0; t9 < 9; ++t9) {
                        const uint32_t dy = (uint32_t)(t9 / 3), dx = (uint32_t)(t9 % 3);
                        const uint64_t ad = aj + (uint64_t)(dy * pitch + dx);
                        const uint64_t bd = bd0 + (uint64_t)((uint32_t)t9 * bstep);
                        const uint32_t acc = (s > 0 || t9 > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dj),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&empty[st])));
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&tfull[buf])));
        }
        // arrives once every MMA issued above has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(done)));
        mbar_wait(smem_u32(done), 0u);
    } else if (warp >= 2) {
        // epilogue: warp w reads the accumulator rows (TMEM lanes) 32 (w mod 4) .. of every tile
        const int q4 = warp & 3;
        int i = 0;
        for (int t = blockIdx.x; t < ntile_total; t += gridDim.x, ++i) {
            const int buf = i & 1;
            const bool okw = mbar_wait(smem_u32(&tfull[buf]), (uint32_t)((i / 2) & 1));
            if (!__all_sync(0xFFFFFFFFu, okw) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const ResTile r = res_tile(t, a, pl, Ci);
            for (int j = 0; j < r.nt; ++j) {
                const int q = 128 * j + 32 * q4 + lane;
                const int line = q / pl.pitch, x = q - line * pl.pitch;
                const bool valid = x < a.W && line < r.lt;
                const long long row = (((long long)r.n * a.D + r.z) * a.H + r.y0 + line) * a.W + x;
                for (int c0 = 0; c0 < Co; c0 += 16) {
                    uint32_t v[16];
                    const uint32_t addr =
                        tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)buf * buf_cols + (uint32_t)(j * Co + c0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];\n"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(addr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
                    if (valid) {
                        float o[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            float xv = __uint_as_float(v[e]);
                            if (bias) xv += bias[c0 + e];
                            if (relu) xv = fmaxf(xv, 0.f);
                            o[e] = xv;
                        }
                        if (OUT_F32) {
                            float4 *dst = reinterpret_cast<float4 *>((float *)Y + row * ldy + c0);
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                dst[e] = make_float4(o[4 * e], o[4 * e + 1], o[4 * e + 2], o[4 * e + 3]);
                        } else {
                            uint4 *dst = reinterpret_cast<uint4 *>((bf16 *)Y + row * ldy + c0);
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                __nv_bfloat162 h[4];
#pragma unroll
                                for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(o[8 * e + 2 * k], o[8 * e + 2 * k + 1]);
                                uint4 u;
                                u.x = *reinterpret_cast<uint32_t *>(&h[0]);
                                u.y = *reinterpret_cast<uint32_t *>(&h[1]);
                                u.z = *reinterpret_cast<uint32_t *>(&h[2]);
                                u.w = *reinterpret_cast<uint32_t *>(&h[3]);
                                dst[e] = u;
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(pl.cols));
    }
    if (tid == 0 && *abort_flag) atomicExch(&g_tc_timeout, 1);
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

// ------------------------------------------------------------------ backward weight, tcgen05
// dW[co][t][ci] += sum_p X[p + t - r][ci] dY[p][co] as D[m][co] with rows
// m = t * Ci + ci (M = 128 rows of (tap, channel) per block, so the 32-channel
// layers fill the MMA), N = Co <= 256, K = positions of one chunk.  Both
// operands are MN-major in shared memory (for one position, 8 consecutive
// channels form a 16-byte row of a core matrix): the two core matrices of a
// 16-position K chunk sit 128 B apart, 8-row groups 256 B apart.  Blocks of
// 64 positions, two stages, bounded mbarrier waits as in k_conv_fwd_tc.  One
// block per (row tile, chunk) writes its partial tile part[chunk][row][co];
// k_wgrad_sum adds the chunks into dW in chunk order, so the result does not
// depend on scheduling.
constexpr int WTK = 64, WTTHREADS = 128;

__global__ void __launch_bounds__(WTTHREADS) k_conv_wgrad_tc(const bf16 *__restrict__ X, int ldx,
                                                            const bf16 *__restrict__ dY, int ldy,
                                                            float *__restrict__ part, Act a, int Ci, int Co, int k,
                                                            long long chunk, int tmem_cols, uint32_t lbo,
                                                            uint32_t sbo) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t a_chunk = 128 * 32, b_chunk = (uint32_t)Co * 32;  // one 16-position K chunk
    const uint32_t stage_bytes = 4 * (a_chunk + b_chunk);
    unsigned char *stage0 = sm;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 2 * stage_bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int KV = k * k * k, r = k / 2, rows = KV * Ci;
    const int m0 = blockIdx.x * 128;
    const long long P = (long long)a.N * a.D * a.H * a.W;
    const long long pbeg = (long long)blockIdx.y * chunk, pend = pbeg + chunk < P ? pbeg + chunk : P;
    const int nkb = (int)((pend - pbeg + WTK - 1) / WTK);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tslot;

    // this thread copies position j = tid & 63 of each block, for row groups
    // g = (tid >> 6) + 2 q of A and channel groups of B
    const int j = tid & 63, g0 = tid >> 6;
    auto load_block = [&](int kb, int st) {
        unsigned char *sa = stage0 + st * stage_bytes;
        unsigned char *sb = sa + 4 * a_chunk;
        const long long p = pbeg + (long long)kb * WTK + j;
        const bool pin = p < pend;
        int pn = 0, pz = 0, py = 0, px = 0;
        if (pin) {
            long long q = p;
            px = (int)(q % a.W); q /= a.W;
            py = (int)(q % a.H); q /= a.H;
            pz = (int)(q % a.D); q /= a.D;
            pn = (int)q;
        }
        const uint32_t off = (uint32_t)((j >> 3) & 1) * 128 + (uint32_t)(j & 7) * 16;  // K group, row
        const int c = j >> 4;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int g = g0 + 2 * q;
            const int row0 = m0 + 8 * g;
            bool ok = pin && row0 < rows;
            long long src = 0;
            if (ok) {
                const int t = row0 / Ci, ci0 = row0 - t * Ci;
                const int tz = t / (k * k), ty = (t / k) % k, tx = t % k;
                const int zz = pz + tz - r, yy = py + ty - r, xx = px + tx - r;
                ok = zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                if (ok) src = ((((long long)pn * a.D + zz) * a.H + yy) * a.W + xx) * ldx + ci0;
            }
            cp_async16(sa + c * a_chunk + g * 256 + off, X + src, ok);
        }
        for (int ng = g0; ng < Co / 8; ng += 2) {
            const long long src = pin ? p * ldy + 8 * ng : 0;
            cp_async16(sb + c * b_chunk + ng * 256 + off, dY + src, pin);
        }
        cp_async_commit();
    };

    // MN-major A and B (bits 15, 16), FP32 accumulator, BF16 operands
    const uint32_t idesc = umma_idesc_bf16(128, Co) | (1u << 15) | (1u << 16);
    bool ok_run = nkb > 0;
    if (ok_run) load_block(0, 0);
    for (int kb = 0; kb < nkb && ok_run; ++kb) {
        const int st = kb & 1;
        if (kb + 1 < nkb) {
            const int s1 = (kb + 1) & 1;
            if (kb + 1 >= 2) {
                const bool okw = mbar_wait(smem_u32(&mbar[s1]), (uint32_t)(((kb - 1) >> 1) & 1));
                if (!__syncthreads_and(okw)) {
                    ok_run = false;
                    break;
                }
            }
            load_block(kb + 1, s1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::);
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t sa = smem_u32(stage0 + st * stage_bytes), sb = sa + 4 * a_chunk;
            for (int c = 0; c < 4; ++c) {
                const uint64_t ad = umma_desc(sa + c * a_chunk, lbo, sbo);
                const uint64_t bd = umma_desc(sb + c * b_chunk, lbo, sbo);
                const uint32_t acc = (kb > 0 || c > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mbar[st])));
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
    if (ok_run) {
        const bool okw = mbar_wait(smem_u32(&mbar[(nkb - 1) & 1]), (uint32_t)(((nkb - 1) >> 1) & 1));
        ok_run = __syncthreads_and(okw);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    // this block's partial rows: part[chunk][m0 + 0..127][0..Co)
    float *prow = part + ((size_t)blockIdx.y * gridDim.x * 128 + (size_t)(m0 + warp * 32 + lane)) * Co;
    if (!ok_run)
        for (int c = 0; c < Co; ++c) prow[c] = 0.f;  // the status flag reports the failure
    if (ok_run) {
        for (int c0 = 0; c0 < Co; c0 += 16) {
            uint32_t v[16];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
            for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4 *>(prow + c0 + e) = make_float4(
                    __uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
    }
}

// ------------------------------------------------------------------ backward weight, resident tiles (3x3x3)
// k_conv3_wgrad_res: dW[co][t][ci] = sum_p dY[p][co] X[p + t - 1][ci] with the
// positions of a run of `by` lines as K, M = 128 rows of (tap pair (dz, dy),
// ci) and N = Co.  Per K-block (by lines y0.. of plane z of sample n) TMA
// loads, for each (dz, dy) of the block's tile and each 8-channel group, the
// box of X at lines y0 + dy - 1 .., plane z + dz - 1, columns -1 .. W (one
// region of 16-byte rows in the order (line, column)), and the box of dY at
// lines y0 .., columns 0 .. W + 1 (zeros beyond W, so the two columns that
// pad each line add nothing).  In that order the input of tap dx for the
// position in row q sits in row q + dx of the X region: the three dx taps are
// the same regions seen through descriptors 16 dx bytes apart.  Both operands
// are MN-major (8 channels of one position form a 16-byte row; K pairs 128 B
// apart, 8-channel groups one region apart).  M holds 128 / ci_blk tap pairs
// of ci_blk channels; a block owns one such tile of one channel block and a
// range of K-blocks, accumulates [dx][M][Co] in tensor memory and writes its
// partial rows part[pb][t * Ci + ci][co]; k_wgrad_sum adds the partials in
// order.  With bpart given, one unused tap-pair slot of the last tile holds
// ones instead of X, which makes its rows the bias-gradient partial
// sum_p dY[p][co] (bpart[pb][co]).  Rows that TMA never writes (each region's tail, the regions of tap
// pairs past the ninth) are zeroed once, so they add exact zeros.  Roles,
// barriers and bounded waits as in k_conv3_fwd_res.
struct WgPlan {
    int by, nyb, pitch, ksteps, J, ci_blk, ntile, npb, kpb, stages, cols;
    uint32_t region, stage_bytes;
};

__global__ void __launch_bounds__(RTHREADS) k_conv3_wgrad_res(const __grid_constant__ CUtensorMap xmap,
                                                             const __grid_constant__ CUtensorMap dymap,
                                                             float *__restrict__ part, float *__restrict__ bpart,
                                                             Act a, int Ci, int Co, WgPlan pl) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = pl.stages, G = pl.ci_blk / 8, NB = Co / 8;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + (size_t)NS * pl.stage_bytes);
    uint64_t *empty = full + NS;
    uint64_t *done = empty + NS;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const int pb = blockIdx.x, cb = blockIdx.y / pl.ntile, ti = blockIdx.y % pl.ntile;
    const int nkb = a.N * a.D * pl.nyb;
    const int kb0 = pb * pl.kpb, kb1 = min(kb0 + pl.kpb, nkb);
    const int nsteps = kb1 > kb0 ? kb1 - kb0 : 0;
    const int nreal = min(pl.J, 9 - ti * pl.J);  // tap pairs of this tile (>= 1)
    const uint32_t tx = (uint32_t)(nreal * G + NB) * (uint32_t)(pl.by * pl.pitch) * 16u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(pl.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int s = 0; s < 2 * NS + 1; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    // the bias gradient rides in the first unused tap-pair slot of the last
    // tile of channel block 0: a region of ones gives rows sum_p dY[p][co]
    const int jb = (bpart && cb == 0 && ti == pl.ntile - 1 && nreal < pl.J) ? nreal : -1;
    {
        uint4 *z4 = reinterpret_cast<uint4 *>(sm);
        const uint32_t n16 = (uint32_t)NS * pl.stage_bytes / 16u, per_region = pl.region / 16u;
        const uint32_t per_stage = pl.stage_bytes / 16u, ones = 0x3F803F80u;  // BF16 1.0 twice
        for (uint32_t i = tid; i < n16; i += RTHREADS) {
            const bool one = jb >= 0 && (i % per_stage) / per_region == (uint32_t)(jb * G);
            z4[i] = one ? make_uint4(ones, ones, ones, ones) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    // the zeros are read by the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tslot;
    const uint32_t base = smem_u32(sm);

    if (tid == 0) {
        int issued = 0;
        for (int s = 0; s < nsteps; ++s) {
            const int st = s % NS;
            if (s >= NS && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((s / NS) - 1) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            const int kb = kb0 + s;
            const int yb = kb % pl.nyb, z = (kb / pl.nyb) % a.D, n = kb / (pl.nyb * a.D);
            const int y0 = yb * pl.by;
            const uint32_t fb = smem_u32(&full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(tx) : "memory");
            const uint32_t sa = base + (uint32_t)st * pl.stage_bytes;
            for (int j = 0; j < nreal; ++j) {
                const int m = ti * pl.J + j, dz = m / 3, dy = m - 3 * dz;
                for (int g = 0; g < G; ++g)
                    tma_load_5d(sa + (uint32_t)(j * G + g) * pl.region, &xmap, cb * pl.ci_blk + 8 * g, -1,
                                y0 + dy - 1, z + dz - 1, n, fb);
            }
            for (int g = 0; g < NB; ++g)
                tma_load_5d(sa + (uint32_t)(16 + g) * pl.region, &dymap, 8 * g, 0, y0, z, n, fb);
            issued = s + 1;
        }
        for (int st = 0; st < NS && st < issued; ++st) {
            const int last = st + ((issued - 1 - st) / NS) * NS;
            mbar_wait(smem_u32(&full[st]), (uint32_t)((last / NS) & 1));
        }
    } else if (tid == 32) {
        // MN-major A and B (bits 15, 16), FP32 accumulator, BF16 operands
        const uint32_t idesc = umma_idesc_bf16(128, Co) | (1u << 15) | (1u << 16);
        for (int s = 0; s < nsteps; ++s) {
            const int st = s % NS;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((s / NS) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t sa = base + (uint32_t)st * pl.stage_bytes, sb = sa + 16u * pl.region;
            for (int ks = 0; ks < pl.ksteps; ++ks) {
                const uint64_t bd = umma_desc(sb + (uint32_t)ks * 256u, 128, pl.region);
                for (int dx = 0; dx < 3; ++dx) {
                    const uint64_t ad = umma_desc(sa + (uint32_t)(ks * 16 + dx) * 16u, 128, pl.region);
                    const uint32_t acc = (s > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(dx * Co)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&empty[st])));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(done)));
    }
    __syncwarp();
    const bool okw = mbar_wait(smem_u32(done), 0u);
    const bool ok_run = __syncthreads_and(okw) && *(volatile int *)abort_flag == 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    // this thread's accumulator row: tap pair m = ti J + j, channel cb ci_blk + cl
    // (the bias row is the first row of slot jb)
    const int r = 32 * warp + lane, j = r / pl.ci_blk, cl = r - j * pl.ci_blk, m = ti * pl.J + j;
    const bool real = m < 9, brow = jb >= 0 && j == jb && cl == 0;
    for (int dx = 0; dx < 3; ++dx) {
        const int t = (real ? m : 0) * 3 + dx;
        float *prow = part + ((size_t)pb * 27 * Ci + (size_t)t * Ci + (size_t)(cb * pl.ci_blk + cl)) * Co;
        for (int c0 = 0; c0 < Co; c0 += 16) {
            if (ok_run && nsteps > 0) {
                uint32_t v[16];
                const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dx * Co + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
                if (real)
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4 *>(prow + c0 + e) =
                            make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                                        __uint_as_float(v[e + 3]));
                if (brow && dx == 0)
#pragma unroll
                    for (int e = 0; e < 16; ++e) bpart[(size_t)pb * Co + c0 + e] = __uint_as_float(v[e]);
            } else {
                // no K-block here, or a wait gave up (the status flag reports it): zero partials
                if (real)
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4 *>(prow + c0 + e) = make_float4(0.f, 0.f, 0.f, 0.f);
                if (brow && dx == 0)
                    for (int e = 0; e < 16; ++e) bpart[(size_t)pb * Co + c0 + e] = 0.f;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(pl.cols));
    }
}

// k_conv3_wgrad_dz: the weight gradient for Co <= 48 with all nine in-plane
// taps as descriptor shifts.  M = 128 rows = 4 slots of 32 channels: slot dz
// (0, 1, 2) holds, per 8-channel group, the box of X at plane z + dz - 1, lines
// y0 - 1 .. y0 + by, columns -1 .. W, so that the input of tap (dy, dx) for the
// position in row q of the dY box sits in row q + dy (W + 2) + dx; slot 3 holds
// ones in its first group (the bias gradient, channel block 0 only) and reads
// whatever follows in its other groups (rows that are dropped).  Per K-step
// nine MMAs, one per (dy, dx), into accumulators [dy][dx][M][Co] (9 Co tensor
// memory columns).  Each X line is loaded three times (once per dz) instead of
// nine.  Region order per stage: 12 X regions (slot, group), the ones region,
// then the dY regions, padded with zero regions up to 16; all regions have
// the same size, so the 16 M groups are one stride byte offset apart.
// Partials, bounded waits and roles as in k_conv3_wgrad_res.
__global__ void __launch_bounds__(RTHREADS) k_conv3_wgrad_dz(const __grid_constant__ CUtensorMap xmap,
                                                            const __grid_constant__ CUtensorMap dymap,
                                                            float *__restrict__ part, float *__restrict__ bpart,
                                                            Act a, int Ci, int Co, WgPlan pl) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = pl.stages, NB = Co / 8;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + (size_t)NS * pl.stage_bytes);
    uint64_t *empty = full + NS;
    uint64_t *done = empty + NS;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const int pb = blockIdx.x, cb = blockIdx.y;
    const int nkb = a.N * a.D * pl.nyb;
    const int kb0 = pb * pl.kpb, kb1 = min(kb0 + pl.kpb, nkb);
    const int nsteps = kb1 > kb0 ? kb1 - kb0 : 0;
    const uint32_t rows_x = (uint32_t)((pl.by + 2) * pl.pitch), rows_y = (uint32_t)(pl.by * pl.pitch);
    const uint32_t tx = (12u * rows_x + (uint32_t)NB * rows_y) * 16u;
    const bool fold = bpart && cb == 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(pl.cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int s = 0; s < 2 * NS + 1; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    {
        // zeros everywhere (region tails, padding regions), ones in region 12 when folding the bias
        uint4 *z4 = reinterpret_cast<uint4 *>(sm);
        const uint32_t n16 = (uint32_t)NS * pl.stage_bytes / 16u, per_region = pl.region / 16u;
        const uint32_t per_stage = pl.stage_bytes / 16u, ones = 0x3F803F80u;  // BF16 1.0 twice
        for (uint32_t i = tid; i < n16; i += RTHREADS) {
            const bool one = fold && (i % per_stage) / per_region == 12u;
            z4[i] = one ? make_uint4(ones, ones, ones, ones) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tslot;
    const uint32_t base = smem_u32(sm);

    if (tid == 0) {
        int issued = 0;
        for (int s = 0; s < nsteps; ++s) {
            const int st = s % NS;
            if (s >= NS && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((s / NS) - 1) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            const int kb = kb0 + s;
            const int yb = kb % pl.nyb, z = (kb / pl.nyb) % a.D, n = kb / (pl.nyb * a.D);
            const int y0 = yb * pl.by;
            const uint32_t fb = smem_u32(&full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(tx) : "memory");
            const uint32_t sa = base + (uint32_t)st * pl.stage_bytes;
            for (int dz = 0; dz < 3; ++dz)
                for (int g = 0; g < 4; ++g)
                    tma_load_5d(sa + (uint32_t)(dz * 4 + g) * pl.region, &xmap, cb * 32 + 8 * g, -1, y0 - 1,
                                z + dz - 1, n, fb);
            for (int g = 0; g < NB; ++g)
                tma_load_5d(sa + (uint32_t)(13 + g) * pl.region, &dymap, 8 * g, 0, y0, z, n, fb);
            issued = s + 1;
        }
        for (int st = 0; st < NS && st < issued; ++st) {
            const int last = st + ((issued - 1 - st) / NS) * NS;
            mbar_wait(smem_u32(&full[st]), (uint32_t)((last / NS) & 1));
        }
    } else if (tid == 32) {
        // MN-major A and B (bits 15, 16), FP32 accumulator, BF16 operands
        const uint32_t idesc = umma_idesc_bf16(128, Co) | (1u << 15) | (1u << 16);
        for (int s = 0; s < nsteps; ++s) {
            const int st = s % NS;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((s / NS) & 1))) {
                atomicExch(abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t sa = base + (uint32_t)st * pl.stage_bytes, sb = sa + 13u * pl.region;
            for (int ks = 0; ks < pl.ksteps; ++ks) {
                const uint64_t bd = umma_desc(sb + (uint32_t)ks * 256u, 128, pl.region);
                for (int t9 = 0; t9 < 9; ++t9) {
                    const int dy = t9 / 3, dx = t9 - 3 * dy;
                    const uint64_t ad =
                        umma_desc(sa + (uint32_t)(ks * 16 + dy * pl.pitch + dx) * 16u, 128, pl.region);
                    const uint32_t acc = (s > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(t9 * Co)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&empty[st])));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(done)));
    }
    __syncwarp();
    const bool okw = mbar_wait(smem_u32(done), 0u);
    const bool ok_run = __syncthreads_and(okw) && *(volatile int *)abort_flag == 0;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    // this thread's accumulator row: slot dz = r / 32, channel cb 32 + r % 32 (the bias row is row 96)
    const int r = 32 * warp + lane, slot = r >> 5, cl = r & 31;
    const bool real = slot < 3, brow = fold && r == 96;
    for (int t9 = 0; t9 < 9; ++t9) {
        const int t = (real ? slot : 0) * 9 + t9;
        float *prow = part + ((size_t)pb * 27 * Ci + (size_t)t * Ci + (size_t)(cb * 32 + cl)) * Co;
        for (int c0 = 0; c0 < Co; c0 += 16) {
            if (ok_run && nsteps > 0) {
                uint32_t v[16];
                const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t9 * Co + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
                if (real)
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4 *>(prow + c0 + e) =
                            make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]), __uint_as_float(v[e + 2]),
                                        __uint_as_float(v[e + 3]));
                if (brow && t9 == 0)
#pragma unroll
                    for (int e = 0; e < 16; ++e) bpart[(size_t)pb * Co + c0 + e] = __uint_as_float(v[e]);
            } else {
                if (real)
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4 *>(prow + c0 + e) = make_float4(0.f, 0.f, 0.f, 0.f);
                if (brow && t9 == 0)
                    for (int e = 0; e < 16; ++e) bpart[(size_t)pb * Co + c0 + e] = 0.f;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(pl.cols));
    }
}

// dW[co][t][ci] += sum over the nk chunks of part[chunk][t * Ci + ci][co] in a
// fixed order: 32 elements per block (threadIdx.x), thread row j = threadIdx.y
// adds the chunks c = j, j + 8, j + 16, ... in turn, and the eight row sums are
// then added in row order, so the result does not depend on scheduling.
constexpr int kSumLanes = 8;
__global__ void __launch_bounds__(32 * kSumLanes) k_wgrad_sum(const float *__restrict__ part, int nk, int rows_pad,
                                                              int rows, int Co, int KV, int Ci,
                                                              float *__restrict__ dW) {
    __shared__ float sh[kSumLanes][32];
    const long long e = (long long)blockIdx.x * 32 + threadIdx.x;
    const bool in = e < (long long)rows * Co;
    const int row = in ? (int)(e / Co) : 0, co = in ? (int)(e - (long long)row * Co) : 0;
    float s = 0.f;
    if (in)
        for (int c = threadIdx.y; c < nk; c += kSumLanes) s += part[((size_t)c * rows_pad + row) * Co + co];
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && in) {
        float t = 0.f;
        for (int j = 0; j < kSumLanes; ++j) t += sh[j][threadIdx.x];
        const int tap = row / Ci, ci = row - tap * Ci;
        dW[((long long)co * KV + tap) * Ci + ci] += t;
    }
}

// bpart[block][co] = this block's sum of dY[p][co]; k_bias_sum adds the blocks in order
__global__ void k_bias_grad(const bf16 *__restrict__ dY, int ldy, float *__restrict__ bpart, long long P, int Co) {
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
        bpart[(size_t)blockIdx.x * Co + co] = t;
    }
}

__global__ void k_bias_sum(const float *__restrict__ bpart, int nblk, int Co, float *__restrict__ db) {
    const int co = blockIdx.x * blockDim.x + threadIdx.x;
    if (co >= Co) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += bpart[(size_t)b * Co + co];
    db[co] += s;
}

// Library-held scratch for the weight-gradient partials, grown on demand
// (the stream is drained before a smaller buffer is replaced).
float *grad_workspace(size_t bytes, cudaStream_t s) {
    static float *buf = nullptr;
    static size_t have = 0;
    if (bytes <= have) return buf;
    if (buf) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return nullptr;
        cudaFree(buf);
        buf = nullptr;
        have = 0;
    }
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        buf = nullptr;
        return nullptr;
    }
    have = bytes;
    return buf;
}

}  // namespace ws

using namespace ws;

static bool bad_channels(int c) { return c < 16 || (c % 16) != 0; }

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            n = 0;
        if (n <= 0) n = 1;
    }
    return n;
}

// forward kernel choice: 0 automatic, 1 gathered tiles (k_conv_fwd_tc), 2 resident tiles
// (k_conv3_fwd_pers or k_conv3_fwd_res, as measured faster), 3 resident tiles, one block per tile
// (k_conv3_fwd_res only), 4 resident tiles, persistent wherever its buffers fit
static int g_fwd_algo = 0;

// cuTensorMapEncodeTiled from the driver, fetched through the runtime (no libcuda link)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 128-row tiles that cover lt output lines of pitch W + 2
static int res_tiles(int lt, int pitch, int W) { return ((lt - 1) * pitch + W + 127) / 128; }

// Tile plan of k_conv3_fwd_res: the line count `by` with the fewest computed
// rows per output (discarded halo columns and ragged tiles), among those whose
// accumulators fit the tensor memory (tiles x Co <= 512 columns) and whose
// ring of at least two stages fits shared memory (a plan that leaves one block
// per SM counts 15 % slower).  Then blocks per SM and stages as measured best
// on the U-Net's layers (batch 4): for Co >= 64 one block per SM with up to 4
// stages (32^3 64->64: 521 TFLOP/s against 418 with two blocks of 3 stages;
// 160->64: 625 against 466), for narrower outputs two blocks per SM with 2
// stages each (64^3 96->32: 628 against 572 with 3 stages; 32->32: 484
// against 470), and ties broken toward fewer lines.  That choice is made for
// lines of 32 columns or more, where it was measured; at 16^3 it left a
// nearly empty second wave (96->96: 164 against 243 TFLOP/s), so narrower lines
// keep the search's stages and blocks per SM.  Returns false if none fits.
static constexpr int kSmemPerSM = 233472, kSmemPerBlockMax = 232448, kSmemReserved = 1024;
static size_t res_smem(const ResPlan &p) { return (size_t)p.stages * p.stage_bytes + 1024 + 8 * (2 * p.stages + 2) + 16; }
static bool res_plan(int W, int H, int Co, ResPlan &best) {
    const int pitch = W + 2;
    if (pitch > 256 || Co > 256) return false;
    const bool tuned = W >= 32;  // the measured choice below; narrower lines keep the search's own
    double best_eff = -1.0;
    for (int by = 1; by <= H && by <= 254; ++by) {
        const int nt = res_tiles(by, pitch, W);
        if (nt * Co > 512) break;
        int cols = 32;
        while (cols < nt * Co) cols *= 2;
        int per_sm = 512 / cols;
        int R = 128 * nt + 2 * pitch + 2;
        if (R < (by + 2) * pitch) R = (by + 2) * pitch;
        R = (R + 7) / 8 * 8;
        ResPlan p;
        p.by = by;
        p.nyt = (H + by - 1) / by;
        p.pitch = pitch;
        p.ntiles = nt;
        p.cols = cols;
        p.a_half = (uint32_t)R * 16u;
        p.stage_bytes = 2 * p.a_half + 18u * (uint32_t)Co * 16u;
        p.tx_bytes = 2u * (uint32_t)((by + 2) * pitch) * 16u + 18u * (uint32_t)Co * 16u;
        // the most stages (2 .. 6) at the most blocks per SM that still fit two
        int ns = 1;
        for (; per_sm >= 1; --per_sm) {
            long long budget = (long long)kSmemPerSM / per_sm - kSmemReserved;
            if (budget > kSmemPerBlockMax) budget = kSmemPerBlockMax;
            for (ns = 6; ns >= 2; --ns) {
                p.stages = ns;
                if ((long long)res_smem(p) <= budget) break;
            }
            if (ns >= 2) break;
        }
        if (ns < 2) continue;
        long long rows = 0;
        for (int y = 0; y < H; y += by) rows += 128LL * res_tiles(by < H - y ? by : H - y, pitch, W);
        const double eff = (double)H * W / (double)rows * (per_sm >= 2 ? 1.0 : 0.85);
        if (tuned ? eff > best_eff + 1e-9 : eff >= best_eff) {  // ties: the fewer lines where tuned
            best_eff = eff;
            best = p;
        }
    }
    if (best_eff <= 0.0) return false;
    if (!tuned) {
        best.per_sm = 512 / best.cols;
        while (best.per_sm > 1 &&
               (long long)res_smem(best) > (long long)kSmemPerSM / best.per_sm - kSmemReserved)
            --best.per_sm;
        return true;
    }
    // blocks per SM and stages of the chosen tiles: one block with up to 4
    // stages for Co >= 64, else up to two blocks with 2 stages each (two
    // stages fit one block per SM whenever the search above found a plan)
    const int ns_max = Co >= 64 ? 4 : 2;
    best.stages = 0;
    for (int per_sm = Co >= 64 ? 1 : std::min(512 / best.cols, 2); per_sm >= 1 && !best.stages; --per_sm) {
        long long budget = (long long)kSmemPerSM / per_sm - kSmemReserved;
        if (budget > kSmemPerBlockMax) budget = kSmemPerBlockMax;
        for (int ns = ns_max; ns >= 2; --ns) {
            best.stages = ns;
            if ((long long)res_smem(best) <= budget) {
                best.per_sm = per_sm;
                break;
            }
            best.stages = 0;
        }
    }
    return best.stages >= 2;
}

// shared memory to request so that no more blocks share an SM than the plan's
// blocks per SM (which the tensor memory holds)
static size_t res_smem_request(const ResPlan &p) {
    size_t s = res_smem(p);
    const int per_sm = p.per_sm;
    const size_t floor_bytes = (size_t)kSmemPerSM / (size_t)(per_sm + 1) - kSmemReserved + 16;
    if (s < floor_bytes) s = floor_bytes;
    if (s > (size_t)kSmemPerBlockMax) s = kSmemPerBlockMax;
    return s;
}

static bool act_map(CUtensorMap *map, const void *t, int ld, const Act &a, int C, int box_x, int box_y) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dim[5] = {(cuuint64_t)C, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D, (cuuint64_t)a.N};
    const cuuint64_t row = (cuuint64_t)ld * 2;
    const cuuint64_t str[4] = {row, row * a.W, row * a.W * a.H, row * a.W * a.H * a.D};
    const cuuint32_t box[5] = {8, (cuuint32_t)box_x, (cuuint32_t)box_y, 1, 1};
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(t), dim, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Persistent variant of a resident-tile plan: the same tiles with two
// accumulator buffers (each a power of two of at least tiles x Co columns, the
// pair within the 512 columns), one block per SM, the most stages (2 ..
// kPersStages) that fit.  False where the buffers do not fit.
constexpr int kPersStages = 4;
static size_t pers_smem(const ResPlan &p) { return (size_t)p.stages * p.stage_bytes + 1024 + 8 * (2 * p.stages + 5) + 16; }
static bool pers_plan(const ResPlan &res, int Co, ResPlan &p, uint32_t &buf_cols) {
    p = res;
    buf_cols = 32;
    while (buf_cols < (uint32_t)(p.ntiles * Co)) buf_cols *= 2;
    if (2 * buf_cols > 512) return false;
    p.cols = (int)(2 * buf_cols);
    p.per_sm = 1;
    for (p.stages = kPersStages; p.stages >= 2; --p.stages)
        if (pers_smem(p) <= (size_t)kSmemPerBlockMax) return true;
    return false;
}

// The persistent forward kernel where it measured faster (U-Net layers at 64^3,
// 32^3, 16^3, batch 4): Co >= 64 (32^3 64->64: 517 against 466 TFLOP/s) and
// 16-channel inputs (3 K-steps a tile; 64^3 16->32: 381 against 321); one
// block per tile for narrower outputs of wider inputs (64^3 96->32: 617
// against 478, 32->32: 440 against 433).
static bool want_persistent(int Ci, int Co) {
    return g_fwd_algo == 4 || (g_fwd_algo != 3 && (Co >= 64 || Ci <= 16));
}

static int conv3_fwd_res(const void *x, int ldx, const void *w, const float *bias, void *y, int ldy, int y_f32,
                         const Act &a, int Ci, int Co, int relu, cudaStream_t s, const ResPlan &pl) {
    EncodeTiledFn enc = encode_tiled();
    CUtensorMap xmap, wmap;
    if (!enc || !act_map(&xmap, x, ldx, a, Ci, pl.pitch, pl.by + 2)) return 2;
    const cuuint32_t ones[3] = {1, 1, 1};
    const cuuint64_t wdim[3] = {(cuuint64_t)Ci, 27, (cuuint64_t)Co};
    const cuuint64_t wstr[2] = {(cuuint64_t)Ci * 2, (cuuint64_t)Ci * 2 * 27};
    const cuuint32_t wbox[3] = {8, 1, (cuuint32_t)Co};
    if (enc(&wmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(w), wdim, wstr, wbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return 2;
    const size_t smem = res_smem_request(pl);
    static size_t attr[2] = {0, 0};
    const int which = y_f32 ? 1 : 0;
    if (attr[which] < smem) {
        const cudaError_t e = y_f32 ? cudaFuncSetAttribute(k_conv3_fwd_res<true>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                                    : cudaFuncSetAttribute(k_conv3_fwd_res<false>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return 2;
        attr[which] = smem;
    }
    const long long blocks = (long long)a.N * a.D * pl.nyt;
    if (blocks > 0x7FFFFFFFLL) return 1;
    ResPlan pp;
    uint32_t buf_cols = 0;
    if (want_persistent(Ci, Co) && pers_plan(pl, Co, pp, buf_cols)) {
        // one persistent block per SM (at most one per tile)
        const size_t psmem = std::max(pers_smem(pp), (size_t)kSmemPerSM / 2 - kSmemReserved + 16);
        static size_t pattr[2] = {0, 0};
        if (pattr[which] < psmem) {
            const cudaError_t e = y_f32 ? cudaFuncSetAttribute(k_conv3_fwd_pers<true>,
                                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem)
                                        : cudaFuncSetAttribute(k_conv3_fwd_pers<false>,
                                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
            if (e != cudaSuccess) return 2;
            pattr[which] = psmem;
        }
        const unsigned grid = (unsigned)std::min<long long>(blocks, sm_count());
        if (y_f32)
            k_conv3_fwd_pers<true><<<grid, PTHREADS, psmem, s>>>(xmap, wmap, bias, y, ldy, a, Ci, Co, relu, pp,
                                                                 (int)blocks, buf_cols);
        else
            k_conv3_fwd_pers<false><<<grid, PTHREADS, psmem, s>>>(xmap, wmap, bias, y, ldy, a, Ci, Co, relu, pp,
                                                                  (int)blocks, buf_cols);
        return cudaGetLastError() == cudaSuccess ? 0 : 2;
    }
    if (y_f32)
        k_conv3_fwd_res<true><<<(unsigned)blocks, RTHREADS, smem, s>>>(xmap, wmap, bias, y, ldy, a, Ci, Co, relu, pl);
    else
        k_conv3_fwd_res<false><<<(unsigned)blocks, RTHREADS, smem, s>>>(xmap, wmap, bias, y, ldy, a, Ci, Co, relu, pl);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// weight-gradient kernel choice: 0 automatic, 1 gathered rows (k_conv_wgrad_tc), 2 resident tiles
// (k_conv3_wgrad_dz where it applies, else k_conv3_wgrad_res), 3 resident tiles without the dz slots
// (k_conv3_wgrad_res only)
static int g_wgrad_algo = 0;


// blocks of a weight-gradient launch: at most this many full waves (resident
// blocks x SMs).  One wave measured best on the U-Net's layers (64^3 32->32:
// 314 TFLOP/s against 262 with two waves and 196 with four): fewer partials to
// add and no block waiting for a second wave.
constexpr int kWgWaves = 1;

static size_t wg_smem(const WgPlan &p) { return (size_t)p.stages * p.stage_bytes + 1024 + 8 * (2 * p.stages + 2) + 16; }

// Plan of k_conv3_wgrad_res: the widest channel block (128, 64, 32 or 16
// channels dividing Ci; M = 128 rows hold 128 / ci_blk tap pairs), K-blocks
// of at most 132 rows (whole lines of W + 2 columns; the best of 2 .. 12 lines
// measured on the U-Net's 64^3, 32^3 and 16^3 layers within 5 %), the most
// stages (2 .. 4) at the most blocks per SM that the tensor memory (3 Co
// columns) allows, and kWgWaves full waves of blocks in all.  Returns false
// where no plan fits (W > 254, Co > 160, or not even two stages).
static bool wg_plan(const Act &a, int Ci, int Co, WgPlan &p) {
    const int pitch = a.W + 2;
    if (pitch > 256 || 3 * Co > 512) return false;
    int cb = 128;
    while (cb > 16 && Ci % cb) cb /= 2;
    if (Ci % cb) return false;
    p.ci_blk = cb;
    p.J = 128 / cb;
    p.ntile = (9 + p.J - 1) / p.J;
    p.pitch = pitch;
    p.cols = 32;
    while (p.cols < 3 * Co) p.cols *= 2;
    bool found = false;
    int resident = 1;
    for (int by = std::max(1, std::min(a.H, 132 / pitch)); by >= 1 && !found; --by) {
        p.by = by;
        p.ksteps = (by * pitch + 15) / 16;
        const int rb = (p.ksteps * 16 + 2 + 7) / 8 * 8;
        p.region = (uint32_t)rb * 16u;
        p.stage_bytes = (uint32_t)(16 + Co / 8) * p.region;
        for (int per_sm = 512 / p.cols; per_sm >= 1 && !found; --per_sm) {
            long long budget = (long long)kSmemPerSM / per_sm - kSmemReserved;
            if (budget > kSmemPerBlockMax) budget = kSmemPerBlockMax;
            for (int ns = 4; ns >= 2; --ns) {
                p.stages = ns;
                if ((long long)wg_smem(p) <= budget) {
                    found = true;
                    resident = per_sm;
                    break;
                }
            }
        }
    }
    if (!found) return false;
    p.nyb = (a.H + p.by - 1) / p.by;
    const long long nkb = (long long)a.N * a.D * p.nyb;
    if (nkb > 0x7FFFFFFFLL) return false;
    const int by_blocks = (Ci / cb) * p.ntile;
    long long npb = (long long)kWgWaves * resident * sm_count() / by_blocks;  // no partial last wave
    if (npb < 1) npb = 1;
    if (npb > nkb) npb = nkb;
    p.kpb = (int)((nkb + npb - 1) / npb);
    p.npb = (int)((nkb + p.kpb - 1) / p.kpb);
    return by_blocks <= 65535;
}

// Plan of k_conv3_wgrad_dz (Ci a multiple of 32, Co <= 48): K-blocks of at
// most 132 rows as for k_conv3_wgrad_res, regions holding the X box with its
// two halo lines and the rows the dy, dx shifts reach past the last K-step,
// the most stages (2 .. 4) that fit at the blocks per SM the tensor memory
// (9 Co columns) allows, kWgWaves full waves of blocks in all.
static bool wg_dz_plan(const Act &a, int Ci, int Co, WgPlan &p) {
    const int pitch = a.W + 2;
    if (pitch > 256 || Ci % 32 || Co > 48) return false;
    p.ci_blk = 32;
    p.J = 4;
    p.ntile = 1;
    p.pitch = pitch;
    p.cols = 32;
    while (p.cols < 9 * Co) p.cols *= 2;
    const int nreg = std::max(16, 13 + Co / 8);
    bool found = false;
    int resident = 1;
    for (int by = std::max(1, std::min(a.H, 132 / pitch)); by >= 1 && !found; --by) {
        if (by + 2 > 256) continue;
        p.by = by;
        p.ksteps = (by * pitch + 15) / 16;
        const int rb = (std::max((by + 2) * pitch, p.ksteps * 16 + 2 * pitch + 2) + 7) / 8 * 8;
        p.region = (uint32_t)rb * 16u;
        p.stage_bytes = (uint32_t)nreg * p.region;
        for (int per_sm = 512 / p.cols; per_sm >= 1 && !found; --per_sm) {
            long long budget = (long long)kSmemPerSM / per_sm - kSmemReserved;
            if (budget > kSmemPerBlockMax) budget = kSmemPerBlockMax;
            for (int ns = 4; ns >= 2; --ns) {
                p.stages = ns;
                if ((long long)wg_smem(p) <= budget) {
                    found = true;
                    resident = per_sm;
                    break;
                }
            }
        }
    }
    if (!found) return false;
    p.nyb = (a.H + p.by - 1) / p.by;
    const long long nkb = (long long)a.N * a.D * p.nyb;
    if (nkb > 0x7FFFFFFFLL) return false;
    const int by_blocks = Ci / 32;
    long long npb = (long long)kWgWaves * resident * sm_count() / by_blocks;  // no partial last wave
    if (npb < 1) npb = 1;
    if (npb > nkb) npb = nkb;
    p.kpb = (int)((nkb + npb - 1) / npb);
    p.npb = (int)((nkb + p.kpb - 1) / p.kpb);
    return by_blocks <= 65535;
}

static size_t wg_smem_request(const WgPlan &p) {
    size_t s = wg_smem(p);
    const int per_sm = 512 / p.cols;
    const size_t floor_bytes = (size_t)kSmemPerSM / (size_t)(per_sm + 1) - kSmemReserved + 16;
    if (s < floor_bytes) s = floor_bytes;
    if (s > (size_t)kSmemPerBlockMax) s = kSmemPerBlockMax;
    return s;
}

// the weight-gradient partials of k_conv3_wgrad_res into part [npb][27 Ci][Co]
static int conv3_wgrad_res(const void *x, int ldx, const void *dy, int ldy, float *part, float *bpart, const Act &a,
                           int Ci, int Co, cudaStream_t s, const WgPlan &pl, bool dz_slots) {
    CUtensorMap xmap, dymap;
    if (!act_map(&xmap, x, ldx, a, Ci, pl.pitch, dz_slots ? pl.by + 2 : pl.by) ||
        !act_map(&dymap, dy, ldy, a, Co, pl.pitch, pl.by))
        return 2;
    const size_t smem = wg_smem_request(pl);
    static size_t attr[2] = {0, 0};
    if (attr[dz_slots] < smem) {
        if (cudaFuncSetAttribute(dz_slots ? k_conv3_wgrad_dz : k_conv3_wgrad_res,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return 2;
        attr[dz_slots] = smem;
    }
    const dim3 grid((unsigned)pl.npb, (unsigned)((Ci / pl.ci_blk) * pl.ntile), 1);
    if (dz_slots)
        k_conv3_wgrad_dz<<<grid, RTHREADS, smem, s>>>(xmap, dymap, part, bpart, a, Ci, Co, pl);
    else
        k_conv3_wgrad_res<<<grid, RTHREADS, smem, s>>>(xmap, dymap, part, bpart, a, Ci, Co, pl);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// byte offsets of the weight gradient's MN-major operand descriptors: between
// the two core matrices of a K chunk (leading) and between 8-row groups (stride)
constexpr uint32_t kWgradLbo = 128, kWgradSbo = 256;


extern "C" {

int ws_conv3d_fwd(const void *x, int ldx, const void *w, const float *bias, void *y, int ldy, int y_f32, int N, int D,
                  int H, int W, int Ci, int Co, int k, int relu, void *stream) {
    if (!x || !w || !y || N < 1 || D < 1 || H < 1 || W < 1 || (k != 1 && k != 3)) return 1;
    if (bad_channels(Ci) || bad_channels(Co) || ldx < Ci || ldy < Co || (ldx % 8) || (ldy % 2)) return 1;
    if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(w) & 15)) return 1;
    // one CTA per 128 positions and all Co channels (N = Co <= 256 in one MMA)
    if (Co > 256 || (ldy % (y_f32 ? 4 : 8)) || (reinterpret_cast<uintptr_t>(y) & 15)) return 1;
    Act a{N, D, H, W};
    const long long P = (long long)N * D * H * W;
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 3 && g_fwd_algo != 1) {
        ResPlan pl;
        if (res_plan(W, H, Co, pl)) return conv3_fwd_res(x, ldx, w, bias, y, ldy, y_f32, a, Ci, Co, relu, s, pl);
        if (g_fwd_algo >= 2) return 1;
    }
    const int cols = Co <= 32 ? 32 : (Co <= 64 ? 64 : (Co <= 128 ? 128 : 256));
    const size_t smem = 2 * (size_t)TKC * (TBM * 32 + (size_t)Co * 32) + 2 * sizeof(uint64_t) + 16;
    static bool attr[2] = {false, false};
    if (!attr[y_f32 ? 1 : 0]) {
        const cudaError_t e = y_f32 ? cudaFuncSetAttribute(k_conv_fwd_tc<true>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024)
                                    : cudaFuncSetAttribute(k_conv_fwd_tc<false>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        if (e != cudaSuccess) return 2;
        attr[y_f32 ? 1 : 0] = true;
    }
    const dim3 grid((unsigned)((P + TBM - 1) / TBM), 1, 1);
    if (y_f32)
        k_conv_fwd_tc<true><<<grid, TTHREADS, smem, s>>>((const bf16 *)x, ldx, (const bf16 *)w, bias, y, ldy, a, Ci,
                                                         Co, k, relu, cols);
    else
        k_conv_fwd_tc<false><<<grid, TTHREADS, smem, s>>>((const bf16 *)x, ldx, (const bf16 *)w, bias, y, ldy, a,
                                                          Ci, Co, k, relu, cols);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_conv3d_fwd_algo(int algo) {
    if (algo < 0 || algo > 4) return -1;
    const int prev = g_fwd_algo;
    g_fwd_algo = algo;
    return prev;
}

int ws_conv3d_plan(int which, int N, int D, int H, int W, int Ci, int Co, long long *out, int nout) {
    if (!out || nout < 0 || N < 1 || D < 1 || H < 1 || W < 1 || bad_channels(Ci) || bad_channels(Co) || Co > 256 ||
        (which != 0 && which != 1))
        return -2;
    long long v[16] = {0};
    int n = 0;
    const Act a{N, D, H, W};
    if (which == 0) {
        ResPlan pl, pp;
        uint32_t buf_cols = 0;
        if (g_fwd_algo == 1 || !res_plan(W, H, Co, pl)) return -1;
        const long long tiles = (long long)N * D * pl.nyt;
        const bool pers = want_persistent(Ci, Co) && pers_plan(pl, Co, pp, buf_cols);
        const ResPlan &q = pers ? pp : pl;
        const size_t smem = pers ? std::max(pers_smem(pp), (size_t)kSmemPerSM / 2 - kSmemReserved + 16)
                                 : res_smem_request(pl);
        const long long f[14] = {pers ? 1 : 0, q.by, q.nyt, q.pitch, q.ntiles, q.stages, q.cols, q.per_sm,
                                 q.a_half, q.stage_bytes, q.tx_bytes, (long long)smem,
                                 pers ? std::min<long long>(tiles, sm_count()) : tiles,
                                 pers ? (long long)buf_cols : 0};
        for (; n < 14; ++n) v[n] = f[n];
    } else {
        WgPlan pl;
        if (g_wgrad_algo == 1) return -1;
        const bool dz = g_wgrad_algo != 3 && wg_dz_plan(a, Ci, Co, pl);
        if (!dz && !wg_plan(a, Ci, Co, pl)) return -1;
        const long long f[16] = {dz ? 1 : 0, pl.by, pl.nyb, pl.pitch, pl.ksteps, pl.J, pl.ci_blk, pl.ntile,
                                 pl.npb, pl.kpb, pl.stages, pl.cols, pl.region, pl.stage_bytes,
                                 (long long)wg_smem_request(pl), (long long)(Ci / pl.ci_blk) * pl.ntile};
        for (; n < 16; ++n) v[n] = f[n];
    }
    for (int i = 0; i < n && i < nout; ++i) out[i] = v[i];
    return n;
}

int ws_conv3d_bwd_weight_algo(int algo) {
    if (algo < 0 || algo > 3) return -1;
    const int prev = g_wgrad_algo;
    g_wgrad_algo = algo;
    return prev;
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
    if ((reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(dy) & 15) || Co > 256) return 1;
    Act a{N, D, H, W};
    const long long P = (long long)N * D * H * W;
    const int KV = k * k * k;
    // rows (tap, channel) in tiles of 128, one block per (row tile, chunk of 4096 positions)
    const long long chunk = 4096;
    const long long nk = (P + chunk - 1) / chunk;
    if (nk > 65535) return 1;
    const int cols = Co <= 32 ? 32 : (Co <= 64 ? 64 : (Co <= 128 ? 128 : 256));
    const size_t smem = 2 * 4 * (size_t)(128 * 32 + Co * 32) + 2 * sizeof(uint64_t) + 16;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024) !=
            cudaSuccess)
            return 2;
        attr = true;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long bias_blocks = (P + 8 * 64 - 1) / (8 * 64);
    const int nbb = (int)(bias_blocks < 1024 ? bias_blocks : 1024);
    if (k == 3 && g_wgrad_algo != 1) {
        WgPlan pl;
        // Ci a multiple of 32 and Co <= 48: the dz-slot kernel (each X line loaded 3 times, not 9)
        const bool dz_slots = g_wgrad_algo != 3 && wg_dz_plan(a, Ci, Co, pl);
        if (dz_slots || wg_plan(a, Ci, Co, pl)) {
            // the kernel sums the bias gradient too when it has a free slot for a row of ones
            const bool fold = db && (dz_slots || pl.J * pl.ntile > 9);
            const size_t wpart = (size_t)pl.npb * 27 * Ci * Co;
            const size_t bparts = fold ? (size_t)pl.npb : (size_t)nbb;
            float *ws_buf = grad_workspace((wpart + bparts * Co) * sizeof(float), s);
            if (!ws_buf) return 2;
            float *bpart = ws_buf + wpart;
            const int rc = conv3_wgrad_res(x, ldx, dy, ldy, ws_buf, fold ? bpart : nullptr, a, Ci, Co, s, pl, dz_slots);
            if (rc) return rc;
            const long long elems = 27LL * Ci * Co;
            k_wgrad_sum<<<(unsigned)((elems + 31) / 32), dim3(32, kSumLanes), 0, s>>>(ws_buf, pl.npb, 27 * Ci,
                                                                                      27 * Ci, Co, 27, Ci, dw);
            if (db) {
                if (!fold) {
                    const dim3 g2((unsigned)nbb, (unsigned)((Co + 31) / 32), 1);
                    k_bias_grad<<<g2, 256, 0, s>>>((const bf16 *)dy, ldy, bpart, P, Co);
                }
                k_bias_sum<<<(Co + 255) / 256, 256, 0, s>>>(bpart, (int)bparts, Co, db);
            }
            return cudaGetLastError() == cudaSuccess ? 0 : 2;
        }
        if (g_wgrad_algo >= 2) return 1;
    }
    const int rows = KV * Ci, tiles = (rows + 127) / 128;
    // partial tiles [nk][tiles * 128][Co], then the bias partials [nbb][Co]
    const size_t wpart = (size_t)nk * tiles * 128 * Co;
    float *ws_buf = grad_workspace((wpart + (size_t)nbb * Co) * sizeof(float), s);
    if (!ws_buf) return 2;
    const dim3 grid((unsigned)tiles, (unsigned)nk, 1);
    k_conv_wgrad_tc<<<grid, WTTHREADS, smem, s>>>((const bf16 *)x, ldx, (const bf16 *)dy, ldy, ws_buf, a, Ci, Co, k,
                                                  chunk, cols, kWgradLbo, kWgradSbo);
    const long long elems = (long long)rows * Co;
    k_wgrad_sum<<<(unsigned)((elems + 31) / 32), dim3(32, kSumLanes), 0, s>>>(ws_buf, (int)nk, tiles * 128, rows, Co,
                                                                              KV, Ci, dw);
    if (db) {
        float *bpart = ws_buf + wpart;
        const dim3 g2((unsigned)nbb, (unsigned)((Co + 31) / 32), 1);
        k_bias_grad<<<g2, 256, 0, s>>>((const bf16 *)dy, ldy, bpart, P, Co);
        k_bias_sum<<<(Co + 255) / 256, 256, 0, s>>>(bpart, nbb, Co, db);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int ws_tc_status(void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int flag = 0;
    const int zero = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return 2;
    if (cudaMemcpyFromSymbol(&flag, g_tc_timeout, sizeof(int)) != cudaSuccess) return 2;
    if (flag && cudaMemcpyToSymbol(g_tc_timeout, &zero, sizeof(int)) != cudaSuccess) return 2;
    return flag ? 5 : 0;
}

}  // extern "C"
