// Internal interfaces between the host runtime (lbm_api.cu) and the kernel
// launchers.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_types.h"

namespace lbm {

struct StepArgs {
    lbm_precision precision;
    int eq_order, wall_model, write_macro;
    int reg_order;     // 2 or 3 (0 is taken as 2)
    int slip;          // 1: some instance has wall slip (the pulls blend in specular reflection)
    unsigned *bar = nullptr;  // persistent update: barrier counter and give-up flag (2 words)
    long long bar_cycles = 0; // its barriers' bound on a wait, in SM clock cycles
    unsigned bar_missing = 0; // arrivals its barriers wait for beyond the grid (failure test: > 0)
    int batch;
    Grid g;
    const void *f_in;
    void *f_out;
    const uint32_t *link;
    void *psi;
    void *macro;
    const void *par;   // InstParam<T>[batch] on the device
    const Ref *ref_in; // reference densities of the current state (unused in FP64)
    Ref *ref_out;      // reference densities written with f_out
    const uint32_t *list = nullptr;  // non-solid cells per instance [batch][n] (two-pass), or NULL
    const int *list_count = nullptr; // entries per instance (device)
    long long list_max = 0;          // largest entry count
    // compact layout (LBM_KERNEL_COMPACT): arrays indexed by the compact index k
    // (k-th non-solid cell of the instance), instance stride kmax
    const uint32_t *cxyz = nullptr;  // packed coordinates x | y << 11 | z << 22
    const uint32_t *clink = nullptr; // geometry words of the non-solid cells
    const uint2 *rowtab = nullptr;   // [batch][rows + 1][words] {rank of the word's first cell, non-solid mask}
    int words = 0;                   // 32-cell words per row
    uint32_t kmax = 0;
    cudaStream_t stream;
    // when non-NULL: events recorded before the first kernel and after each
    // kernel of the launch (two-pass: 3 events, fused and cluster: 2)
    cudaEvent_t *ev = nullptr;
};

// Variant EQ of the two-pass kernels (bit 0: eq_order 1, bit 1: reg_order 3,
// bit 2: wall slip), passed to f as a std::integral_constant.
inline int collide_variant(const StepArgs &a) {
    return (a.eq_order ? 1 : 0) | (a.reg_order == 3 ? 2 : 0) | (a.slip ? 4 : 0);
}

template <class F> inline void dispatch_variant(int v, F &&f) {
    switch (v) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    default: f(std::integral_constant<int, 7>{}); break;
    }
}

inline void record_event(const StepArgs &a, int k) {
    if (a.ev) cudaEventRecord(a.ev[k], a.stream);
}

struct InitArgs {
    lbm_precision precision;
    int eq_order;
    int batch;
    Grid g;
    const double *r1, *r2, *u;  // device FP64 fields (u interleaved)
    const uint32_t *link;
    void *f_out, *macro, *usnap;
    Ref *ref_out;
    const void *par;
    cudaStream_t stream;
};

struct ReduceArgs {
    bool fp64;
    int batch;
    Grid g;
    const void *macro;
    void *usnap;
    const uint32_t *link;
    double *partial;   // [batch][nblk][9]
    int nblk;
    double *out;       // [batch][9]: M1 M2 Px Py Pz |du|^2 |u|^2 max|u| non-finite count
    long long k;       // updates since the snapshot
    cudaStream_t stream;
};

cudaError_t launch_two_pass(const StepArgs &a);
cudaError_t launch_psi_solid(const uint32_t *link, void *psi, bool fp64, const Grid &g, int batch, const void *par,
                             cudaStream_t s);
// tile: 0 = 32x8, 1 = 32x4, 2 = 64x4, 3 = 32x16 cells per CTA; zchunk planes per CTA
cudaError_t launch_fused(const StepArgs &a, int tile, int zchunk);
int fused_tile_count();
// nsteps updates in one persistent launch, one thread-block cluster per instance
cudaError_t launch_cluster(const StepArgs &a, int nsteps);
cudaError_t launch_persist(const StepArgs &a, int nsteps);
int cluster_size_for(long long n);
cudaError_t launch_init(const InitArgs &a);
cudaError_t launch_links(const uint8_t *type, uint32_t *link, const Grid &g, int batch, cudaStream_t s);
cudaError_t launch_macro_to_f64(const void *macro, bool fp64, double *r1, double *r2, double *u, const Grid &g,
                                int batch, cudaStream_t s);
cudaError_t launch_reduce(const ReduceArgs &a, int *launches);
// out != NULL: expand f to FP64 into out; otherwise store `in` (FP64) into fo.
cudaError_t launch_f_convert(lbm_precision prec, const void *f, double *out, const double *in, void *fo,
                             const Ref *ref, const uint32_t *link, const Grid &g, int batch, cudaStream_t s);
int reduce_blocks(long long n);

// geometry set-up (lbm_setup.cu).  flags[0] = 1 if a type is above 3,
// flags[1 + b] = 1 if instance b has a FLUID cell (flags zeroed by the caller).
cudaError_t launch_check_types(const uint8_t *type, const Grid &g, int batch, int *flags, cudaStream_t s);
// rowcnt[b][row] = exclusive offsets of the non-solid cells of each row,
// count[b] = non-solid cells of instance b; closing table row = count[b].
cudaError_t launch_row_counts(const uint32_t *link, const Grid &g, int batch, uint32_t *rowcnt, int *count,
                              uint2 *tab, cudaStream_t s);
// list[b][rank] (stride n), cxyz[b][rank] (stride kmax) and the row table
// from the offsets of launch_row_counts; cxyz and tab may be NULL.
cudaError_t launch_row_fill(const uint32_t *link, const Grid &g, int batch, uint32_t *rowstart, uint32_t *list,
                            uint32_t *cxyz, uint2 *tab, uint32_t kmax, cudaStream_t s);

// compact layout
constexpr int kCompactMaxX = 2048, kCompactMaxY = 2048, kCompactMaxZ = 1024;

// single-read fused update on the compact layout (lbm_fusedc.cu)
struct FcPlan {
    int bands = 0, chunks = 0, units = 0;  // bands of rows x z chunks x instances
    int lag_cap = 0;                       // cells per lag slot
    int clusters = 0;                      // clusters launched (co-resident)
    size_t smem = 0;                       // dynamic shared memory per CTA
    bool ok = false;                       // fits this geometry and device
};
int fusedc_rows_per_cta();
cudaError_t fusedc_plan(lbm_precision prec, int eq_order, const Grid &g, int batch, int lag_cap, FcPlan &out);
cudaError_t launch_fusedc(const StepArgs &a, const FcPlan &p);
cudaError_t launch_compact(const StepArgs &a, int parts = 3);
// geometry words of the listed cells: clink[b][k] = link[b][list[b][k]]
cudaError_t launch_compact_links(const uint32_t *list, const int *count, const uint32_t *link, uint32_t *clink,
                                 const Grid &g, int batch, uint32_t kmax, cudaStream_t s);
// f and the reference densities between the dense and the compact layout
cudaError_t launch_layout(lbm_precision prec, bool to_compact, const void *fin, void *fout, const Ref *rin, Ref *rout,
                          const uint32_t *list, const int *count, const Grid &g, int batch, uint32_t kmax,
                          cudaStream_t s);

}  // namespace lbm
