/*
 * ws.h - C ABI of the warm-start surrogate kernels (BF16 tensor-core 3-D
 * convolutions with FP32 accumulation, and the elementwise pieces of a 3-D
 * U-Net).  The surrogate maps (geometry mask, wall potential, viscosity ratio,
 * inclination, body force) to initial fields for the lattice Boltzmann solver;
 * the paper has no counterpart (it is a systems layer on top of the method).
 *
 * Conventions
 *  - Tensor pointers are DEVICE pointers owned by the caller.  The library
 *    allocates only the weight gradient's workspace (ws_conv3d_bwd_weight);
 *    ws_conv3d_plan writes a HOST array.
 *  - Activations are channels-last BF16: element (n, z, y, x, c) of a tensor
 *    with row stride ld (>= channels) is at ((((n*D + z)*H + y)*W + x)*ld + c);
 *    a channel offset is applied by passing a pointer into the row.  Channel
 *    counts are multiples of 16; ld is a multiple of 8 and the base 16-byte
 *    aligned for BF16 tensors read by the convolutions.
 *  - Convolution weights are BF16 [Co][k][k][k][Ci] (k = 1 or 3, "same" zero
 *    padding, stride 1); biases and weight gradients are FP32.
 *  - Work is queued on `stream` (cudaStream_t, NULL = legacy default) without
 *    synchronisation.  Return value: 0 ok, 1 invalid argument (nothing
 *    launched), 2 CUDA launch error; the kernel-choice and plan queries
 *    document their own.
 */
#ifndef WS_H
#define WS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y = act(conv(x, w) + bias); y is BF16 (y_f32 = 0) or FP32 (y_f32 = 1) with
 * row stride ldy; relu != 0 applies max(., 0); bias may be NULL.  Runs as an
 * implicit GEMM on the tcgen05 tensor cores (M = output positions, N = Co,
 * K = taps x Ci), accumulated in tensor memory.  Two kernels:
 *  - resident tiles (k = 3, W <= 254): a run of output lines of one plane is
 *    one tile; TMA loads its input one padded plane at a time and the 9 taps
 *    of the plane are shifted views of that tile.  For Co >= 64 or Ci = 16,
 *    where two accumulator buffers fit the tensor memory, one persistent
 *    block per SM strides over the tiles (the epilogue of a tile overlapping
 *    the next tile's MMAs); otherwise each block computes one tile.  Both give
 *    the same bits;
 *  - gathered tiles (k = 1, and k = 3 where no resident plan fits): 128
 *    positions per block, each tap's rows gathered with 16-byte copies.
 * Additional argument rules: Co <= 256, y 16-byte aligned, ldy a multiple of
 * 8 (BF16) or 4 (FP32).  Errors: 1 bad argument (also when the resident
 * kernel is forced and no plan fits), 2 launch failure or no TMA encoder in
 * the driver. */
int ws_conv3d_fwd(const void *x, int ldx, const void *w, const float *bias, void *y, int ldy, int y_f32, int N,
                  int D, int H, int W, int Ci, int Co, int k, int relu, void *stream);

/* Selects the forward kernel of later ws_conv3d_fwd calls (process-wide):
 * 0 automatic (resident tiles where a plan fits, else gathered), 1 gathered
 * tiles always, 2 resident tiles always for k = 3, 3 as 2 but one block per
 * tile (never the persistent kernel), 4 as 2 but persistent wherever its
 * buffers fit.  Returns the previous choice, or -1 for an unknown value
 * (nothing changes). */
int ws_conv3d_fwd_algo(int algo);

/* wf[ci][t][co] = w[co][k^3-1-t][ci]: weights for the data gradient, which is
 * then ws_conv3d_fwd(dy, wf) with Ci and Co exchanged. */
int ws_conv3d_flip_weights(const void *w, void *wf, int Co, int Ci, int k, void *stream);

/* dw[co][t][ci] += sum_p dy[p][co] x[p + t - k/2][ci] and db[co] += sum_p dy[p][co]
 * (db may be NULL).  Accumulates: clear dw and db first.  Runs on the tcgen05
 * tensor cores with N = Co <= 256; x and dy 16-byte aligned.  Two kernels:
 *  - resident tiles (k = 3, W <= 254, Co <= 160): K = the positions of runs of
 *    whole lines, M = 128 rows of (tap pair (dz, dy), channel) loaded by TMA
 *    as line boxes, the three dx taps as shifted views of the same boxes; for
 *    Ci a multiple of 32 and Co <= 48, M = (dz, channel) rows of boxes with
 *    halo lines instead, and all nine (dy, dx) taps are shifted views;
 *  - gathered rows (k = 1, and k = 3 where no resident plan fits): rows
 *    (tap, ci) in tiles of 128, K = chunks of 4096 positions gathered with
 *    16-byte copies.
 * Each block writes its partial sums into a workspace the library holds
 * (grown on demand with cudaMalloc, after draining the stream); the partials
 * are then added into dw in a fixed order, so repeated calls give identical
 * bits.  The workspace is one per process: calls that
 * could overlap on the GPU (other streams, other host threads) race on it, so
 * issue them on one stream.  Errors: 1 bad argument, 2 allocation or launch
 * failure. */
int ws_conv3d_bwd_weight(const void *x, int ldx, const void *dy, int ldy, float *dw, float *db, int N, int D, int H,
                         int W, int Ci, int Co, int k, void *stream);

/* Selects the weight-gradient kernel of later ws_conv3d_bwd_weight calls
 * (process-wide): 0 automatic (resident tiles where a plan fits, else
 * gathered rows), 1 gathered rows always, 2 resident tiles always for k = 3
 * (a call that no plan fits then returns 1), 3 as 2 but with tap-pair rows
 * only (never the (dz, channel) rows).  Returns the previous choice, or -1
 * for an unknown value (nothing changes). */
int ws_conv3d_bwd_weight_algo(int algo);

/* The tiling the resident-tile kernels would use for a 3x3x3 convolution of
 * this shape under the current kernel choice (host only: no GPU work, no
 * allocation).  which = 0: forward (also the data gradient with Ci and Co
 * exchanged); out[0..13] = persistent kernel (0/1), lines per tile, tiles per
 * plane, line pitch (W + 2), 128-row M tiles per tile, stages, tensor-memory
 * columns, blocks per SM, bytes of one K half of a stage's input, stage bytes,
 * TMA bytes per stage, dynamic shared memory requested, blocks in the grid,
 * columns per accumulator buffer (persistent kernel, else 0).  which = 1:
 * weight gradient; out[0..15] = dz-slot kernel (0/1), lines per K-block,
 * K-blocks per plane, line pitch, K-steps per K-block, tap slots per M tile,
 * channels per M group, M tiles per channel block, position blocks, K-blocks
 * per position block, stages, tensor-memory columns, region bytes, stage
 * bytes, dynamic shared memory requested, blocks per position block (grid y).
 * The block counts follow the SM count of the current device (1 where no
 * device is visible).  Writes min(nout, count) values and returns the count;
 * -1 when the gathered kernel would run (no resident plan fits, or it is
 * selected), -2 for invalid arguments. */
int ws_conv3d_plan(int which, int N, int D, int H, int W, int Ci, int Co, long long *out, int nout);

/* 2x2x2 average pooling (D, H, W even) and its adjoint; nearest-neighbour 2x
 * upsampling and its adjoint (sum of the 8 children).  BF16 in and out.  The
 * adjoints of pool/upsample accumulate into dx when accumulate != 0.  D, H, W
 * are the sizes of the finer tensor for the pooling calls and of the coarser
 * one for the upsampling calls. */
int ws_avgpool2(const void *x, int ldx, void *y, int ldy, int N, int D, int H, int W, int C, void *stream);
int ws_avgpool2_bwd(const void *dy, int ldy, void *dx, int ldx, int N, int D, int H, int W, int C, int accumulate,
                    void *stream);
int ws_upsample2(const void *x, int ldx, void *y, int ldy, int N, int D, int H, int W, int C, void *stream);
int ws_upsample2_bwd(const void *dy, int ldy, void *dx, int ldx, int N, int D, int H, int W, int C, int accumulate,
                     void *stream);

/* ReLU adjoint in place: dy[p][c] = 0 where y[p][c] <= 0 (y is the BF16
 * activation the forward pass produced). */
int ws_relu_bwd(const void *y, int ldy, void *dy, int lddy, long long P, int C, void *stream);

/* Masked mean-squared error between prediction pred (FP32, [P][ldp], first C
 * channels) and target (FP32 [P][C]) over cells with mask[p] != 0, weighted per
 * channel by wch[C]; writes the BF16 gradient d(loss)/d(pred) into dpred
 * ([P][lddp], channels beyond C zeroed) and adds the loss to *loss (FP32,
 * device). */
int ws_mse_loss(const float *pred, int ldp, const float *target, const uint8_t *mask, const float *wch, void *dpred,
                int lddp, float *loss, long long P, int C, void *stream);

/* Adam with FP32 master weights w, moments m and v, gradient g (n values);
 * writes the BF16 copy wb used by the convolutions (wb may be NULL) and
 * clears g for the next accumulation.  lr_t is the bias-corrected step size
 * of this iteration. */
int ws_adam(float *w, float *m, float *v, float *g, void *wb, long long n, float lr_t, float beta1, float beta2,
            float eps, float weight_decay, void *stream);

/* Waits for `stream`, then reports whether a tensor-core convolution since the
 * last call gave up on a bounded wait for its matrix units (5; the affected
 * outputs are not written) or not (0); clears the record.  2 on a CUDA error. */
int ws_tc_status(void *stream);

/* FP32 -> BF16 copy into a channel slice: y[p][c] = x[p*ldx + c], c < C. */
int ws_to_bf16(const float *x, int ldx, void *y, int ldy, long long P, int C, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WS_H */
