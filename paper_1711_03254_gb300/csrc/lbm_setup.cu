// Geometry set-up on the device: validation of uploaded cell types, and the
// per-instance lists of the non-solid cells in cell order (x fastest) with
// the compact layout's packed coordinates and per-row occupancy words.
//
// One warp walks one row (y, z) of an instance in 32-cell words and finds the
// non-solid cells of each word with a ballot.  A first pass counts the cells
// of every row, one block per instance turns the counts into exclusive row
// offsets, and a second pass writes every cell's list entry at its rank
// (row offset + cells before it in the row).
#include "lbm_internal.h"
#include "lbm_device.cuh"

namespace lbm {

namespace {

constexpr int kRowThreads = 256, kScanThreads = 1024;

// flags[0] = 1 if a type is above 3; flags[1 + b] = 1 if instance b has a FLUID cell
__global__ void k_check_types(const uint8_t *__restrict__ type, long long n, int batch, int *flags) {
    for (int b = blockIdx.y; b < batch; b += gridDim.y) {
        const uint8_t *t = type + (size_t)b * n;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const uint8_t v = t[i];
            const unsigned act = __activemask();
            const bool bad = __any_sync(act, v > 3), fluid = __any_sync(act, v == 0);
            if ((threadIdx.x & 31) == __ffs(act) - 1) {
                if (bad) flags[0] = 1;
                if (fluid) flags[1 + b] = 1;
            }
        }
    }
}

// FILL = false: rowcnt[b][r] = non-solid cells of row r.  FILL = true:
// rowcnt holds the exclusive row offsets; writes list[b][rank] (cell index,
// stride n), cxyz[b][rank] (packed x | y << 11 | z << 22, stride kmax) and
// tab[b][r][w] = {rank of the word's first cell, mask} (cxyz, tab may be NULL).
template <bool FILL>
__global__ void __launch_bounds__(kRowThreads) k_rows(const uint32_t *__restrict__ link, Grid g, int batch,
                                                      uint32_t *rowcnt, uint32_t *list, uint32_t *cxyz, uint2 *tab,
                                                      uint32_t kmax) {
    const int lane = threadIdx.x & 31;
    const long long rows = (long long)g.ny * g.nz;
    const int W = (g.nx + 31) / 32;
    const long long nwarps = (long long)gridDim.x * (kRowThreads / 32);
    // gr is the same for the 32 lanes of a warp, so the loops and ballots are warp-uniform
    for (long long gr = blockIdx.x * (long long)(kRowThreads / 32) + threadIdx.x / 32; gr < rows * batch;
         gr += nwarps) {
        const int b = (int)(gr / rows);
        const long long r = gr - (long long)b * rows;
        const uint32_t *lk = link + (size_t)b * g.n + (size_t)r * g.nx;
        uint32_t c = FILL ? rowcnt[gr] : 0u;
        for (int w = 0; w < W; ++w) {
            const int x = w * 32 + lane;
            const bool ns = x < g.nx && cell_type(lk[x]) != kSolid;
            const uint32_t mask = __ballot_sync(0xffffffffu, ns);
            if (FILL) {
                if (tab && lane == 0) tab[((size_t)b * (rows + 1) + r) * W + w] = make_uint2(c, mask);
                if (ns) {
                    const uint32_t at = c + __popc(mask & ((1u << lane) - 1u));
                    list[(size_t)b * g.n + at] = (uint32_t)(r * g.nx + x);
                    if (cxyz)
                        cxyz[(size_t)b * kmax + at] =
                            (uint32_t)x | ((uint32_t)(r % g.ny) << 11) | ((uint32_t)(r / g.ny) << 22);
                }
            }
            c += (uint32_t)__popc(mask);
        }
        if (!FILL && lane == 0) rowcnt[gr] = c;
    }
}

// In place: row counts -> exclusive row offsets of each instance; count[b] =
// the instance's non-solid cells, which the closing row of the table (row
// `rows`) holds for every word.
__global__ void __launch_bounds__(kScanThreads) k_scan_rows(uint32_t *rowcnt, long long rows, int batch, int *count,
                                                            uint2 *tab, int W) {
    __shared__ uint32_t part[kScanThreads];
    const int tid = threadIdx.x;
    for (int b = blockIdx.x; b < batch; b += gridDim.x) {
        uint32_t *rc = rowcnt + (size_t)b * rows;
        const long long per = (rows + kScanThreads - 1) / kScanThreads;
        const long long lo = tid * per < rows ? tid * per : rows;
        const long long hi = lo + per < rows ? lo + per : rows;
        uint32_t s = 0;
        for (long long r = lo; r < hi; ++r) s += rc[r];
        part[tid] = s;
        __syncthreads();
        for (int o = 1; o < kScanThreads; o <<= 1) {  // inclusive scan of the chunk sums
            const uint32_t v = tid >= o ? part[tid - o] : 0u;
            __syncthreads();
            part[tid] += v;
            __syncthreads();
        }
        uint32_t run = tid ? part[tid - 1] : 0u;
        for (long long r = lo; r < hi; ++r) {
            const uint32_t v = rc[r];
            rc[r] = run;
            run += v;
        }
        const uint32_t total = part[kScanThreads - 1];
        if (tid == 0) count[b] = (int)total;
        if (tab)
            for (int w = tid; w < W; w += kScanThreads) tab[((size_t)b * (rows + 1) + rows) * W + w] = make_uint2(total, 0u);
        __syncthreads();  // part[] is reused by the next instance
    }
}

unsigned row_blocks(const Grid &g, int batch) {
    const long long warps = (long long)g.ny * g.nz * batch;
    const long long blocks = (warps + kRowThreads / 32 - 1) / (kRowThreads / 32);
    return (unsigned)(blocks < 152 * 16 ? blocks : 152 * 16);
}

}  // namespace

cudaError_t launch_check_types(const uint8_t *type, const Grid &g, int batch, int *flags, cudaStream_t s) {
    long long bx = (g.n + 255) / 256;
    if (bx > 1024) bx = 1024;
    const unsigned by = (unsigned)(batch < 65535 ? batch : 65535);
    k_check_types<<<dim3((unsigned)bx, by, 1), 256, 0, s>>>(type, g.n, batch, flags);
    return cudaGetLastError();
}

cudaError_t launch_row_counts(const uint32_t *link, const Grid &g, int batch, uint32_t *rowcnt, int *count,
                              uint2 *tab, cudaStream_t s) {
    k_rows<false><<<row_blocks(g, batch), kRowThreads, 0, s>>>(link, g, batch, rowcnt, nullptr, nullptr, nullptr, 0u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned sb = (unsigned)(batch < 65535 ? batch : 65535);
    k_scan_rows<<<sb, kScanThreads, 0, s>>>(rowcnt, (long long)g.ny * g.nz, batch, count, tab, (g.nx + 31) / 32);
    return cudaGetLastError();
}

cudaError_t launch_row_fill(const uint32_t *link, const Grid &g, int batch, uint32_t *rowstart, uint32_t *list,
                            uint32_t *cxyz, uint2 *tab, uint32_t kmax, cudaStream_t s) {
    k_rows<true><<<row_blocks(g, batch), kRowThreads, 0, s>>>(link, g, batch, rowstart, list, cxyz, tab, kmax);
    return cudaGetLastError();
}

}  // namespace lbm
