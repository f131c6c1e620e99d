// Two-pass update on the compact layout (LBM_KERNEL_COMPACT).
//
// Only the non-solid cells of an instance are stored, in cell order (x
// fastest); the compact index k of a cell is the number of non-solid cells
// before it.  The two components of a value are stored side by side, so one
// 4-byte (FP16/BF16), 8-byte (FP32) or 16-byte (FP64) access moves both.
// Per instance b (stride kmax = the largest non-solid count):
//   f[b][i][k][alpha], ref[b][k][alpha], psi[b][k][alpha],
//   cxyz[b][k] (packed coordinates), clink[b][k] (geometry word),
//   rowtab[b][row][word] = {rank of the word's first cell, non-solid mask}.
// On porous geometries the dense layout wastes most of each 32-byte sector on
// SOLID cells and writes sectors only in part; here a warp's 32 cells read and
// write contiguous runs of every plane, and the component pairs halve the
// load, store and address instructions.
//
//   k_psi_c            S1-S3 as k_psi: pull, sum to rho_alpha, store psi.
//   k_collide_c        S1-S7 as k_collide (FP64: the scalar device code of
//                      the dense kernels, so both layouts give identical bits).
//   k_collide_c2       S1-S7 for the FP32-arithmetic storages, both components
//                      as packed FP32 pairs (lbm_pair2.cuh).
#include "lbm_compact_update.cuh"

namespace lbm {

// instantiated in lbm_update_*.cu
extern template cudaError_t launch_compact_t<double>(const StepArgs &, int);
extern template cudaError_t launch_compact_t<float>(const StepArgs &, int);
extern template cudaError_t launch_compact_t<__half>(const StepArgs &, int);
extern template cudaError_t launch_compact_t<__nv_bfloat16>(const StepArgs &, int);
extern template cudaError_t launch_persist_t<double>(const StepArgs &, int);
extern template cudaError_t launch_persist_t<float>(const StepArgs &, int);
extern template cudaError_t launch_persist_t<__half>(const StepArgs &, int);
extern template cudaError_t launch_persist_t<__nv_bfloat16>(const StepArgs &, int);

__global__ void k_compact_links(const uint32_t *__restrict__ list, const int *__restrict__ count,
                                const uint32_t *__restrict__ link, uint32_t *__restrict__ clink, long long n,
                                uint32_t kmax) {
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)count[b]) return;
    clink[(size_t)b * kmax + k] = link[(size_t)b * n + list[(size_t)b * n + k]];
}

// one thread per (instance, component, non-solid cell); all 19 planes.
// dense f[b][alpha][i][cell], ref[b][alpha][cell] <-> compact f[b][i][k][alpha], ref[b][k][alpha]
template <class S>
__global__ void k_layout(bool to_compact, const S *__restrict__ fin, S *__restrict__ fout, const Ref *__restrict__ rin,
                         Ref *__restrict__ rout, const uint32_t *__restrict__ list, const int *__restrict__ count,
                         long long n, uint32_t kmax) {
    const int bc = blockIdx.y;  // b * 2 + alpha
    const int b = bc >> 1, al = bc & 1;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)count[b]) return;
    const size_t cell = list[(size_t)b * n + k];
    for (int i = 0; i < kQ; ++i) {
        const size_t d = ((size_t)bc * kQ + i) * (size_t)n + cell;
        const size_t c = (((size_t)b * kQ + i) * kmax + k) * 2 + al;
        if (to_compact)
            fout[c] = fin[d];
        else
            fout[d] = fin[c];
    }
    if (rin) {
        const size_t d = (size_t)bc * n + cell, c = ((size_t)b * kmax + k) * 2 + al;
        if (to_compact)
            rout[c] = rin[d];
        else
            rout[d] = rin[c];
    }
}


cudaError_t launch_compact(const StepArgs &a, int parts) {
    switch (a.precision) {
    case LBM_FP64: return launch_compact_t<double>(a, parts);
    case LBM_FP32: return launch_compact_t<float>(a, parts);
    case LBM_FP32_F16S: return launch_compact_t<__half>(a, parts);
    case LBM_FP32_BF16S: return launch_compact_t<__nv_bfloat16>(a, parts);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_persist(const StepArgs &a, int nsteps) {
    switch (a.precision) {
    case LBM_FP64: return launch_persist_t<double>(a, nsteps);
    case LBM_FP32: return launch_persist_t<float>(a, nsteps);
    case LBM_FP32_F16S: return launch_persist_t<__half>(a, nsteps);
    case LBM_FP32_BF16S: return launch_persist_t<__nv_bfloat16>(a, nsteps);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_compact_links(const uint32_t *list, const int *count, const uint32_t *link, uint32_t *clink,
                                 const Grid &g, int batch, uint32_t kmax, cudaStream_t s) {
    const dim3 grid((kmax + 255) / 256 > 0 ? (kmax + 255) / 256 : 1, (unsigned)batch, 1);
    k_compact_links<<<grid, 256, 0, s>>>(list, count, link, clink, g.n, kmax);
    return cudaGetLastError();
}

template <class S>
static cudaError_t launch_layout_t(bool to_compact, const void *fin, void *fout, const Ref *rin, Ref *rout,
                                   const uint32_t *list, const int *count, const Grid &g, int batch, uint32_t kmax,
                                   cudaStream_t s) {
    const dim3 grid((kmax + 255) / 256 > 0 ? (kmax + 255) / 256 : 1, (unsigned)batch * 2, 1);
    k_layout<S><<<grid, 256, 0, s>>>(to_compact, (const S *)fin, (S *)fout, rin, rout, list, count, g.n, kmax);
    return cudaGetLastError();
}

cudaError_t launch_layout(lbm_precision prec, bool to_compact, const void *fin, void *fout, const Ref *rin, Ref *rout,
                          const uint32_t *list, const int *count, const Grid &g, int batch, uint32_t kmax,
                          cudaStream_t s) {
    switch (prec) {
    case LBM_FP64: return launch_layout_t<double>(to_compact, fin, fout, nullptr, nullptr, list, count, g, batch, kmax, s);
    case LBM_FP32: return launch_layout_t<float>(to_compact, fin, fout, rin, rout, list, count, g, batch, kmax, s);
    case LBM_FP32_F16S: return launch_layout_t<__half>(to_compact, fin, fout, rin, rout, list, count, g, batch, kmax, s);
    case LBM_FP32_BF16S:
        return launch_layout_t<__nv_bfloat16>(to_compact, fin, fout, rin, rout, list, count, g, batch, kmax, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
