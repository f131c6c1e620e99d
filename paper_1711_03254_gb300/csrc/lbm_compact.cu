// Two-pass update on the compact layout (LBM_KERNEL_COMPACT).
//
// Only the non-solid cells of an instance are stored, in cell order (x
// fastest); the compact index k of a cell is the number of non-solid cells
// before it.  Per instance b (stride kmax = the largest non-solid count):
//   f[b][alpha][i][k], ref[b][alpha][k], psi[b][alpha][k],
//   cxyz[b][k] (packed coordinates), clink[b][k] (geometry word),
//   rowtab[b][row][word] = {rank of the word's first cell, non-solid mask}.
// On porous geometries the dense layout wastes most of each 32-byte sector on
// SOLID cells and writes sectors only in part; here a warp's 32 cells read and
// write contiguous runs of every plane.
//
//   k_psi_c      S1-S3 as k_psi: pull, sum to rho_alpha, store psi.
//   k_collide_c  S1-S7 as k_collide.
// The arithmetic is the same device code as the dense kernels (pull_moments,
// sc_forces, relax, collide_store), so both layouts give identical bits.
#include "lbm_internal.h"
#include "lbm_device.cuh"

namespace lbm {

struct CompactCell {
    int x, y, z;
    uint32_t word;
};

__device__ __forceinline__ CompactCell compact_cell(const StepArgs &a, int b, uint32_t k) {
    CompactCell c;
    const uint32_t p = __ldg(a.cxyz + (size_t)b * a.kmax + k);
    c.x = (int)(p & 2047u);
    c.y = (int)((p >> 11) & 2047u);
    c.z = (int)(p >> 22);
    c.word = __ldg(a.clink + (size_t)b * a.kmax + k);
    return c;
}

__device__ __forceinline__ const uint2 *instance_tab(const StepArgs &a, int b) {
    return a.rowtab + (size_t)b * ((size_t)a.g.ny * a.g.nz + 1) * a.words;
}

// For an OUTLET cell whose upstream (-x) neighbour is neither SOLID nor
// OUTLET, the update pulls that neighbour's streamed values: returns true and
// its position, compact index and word.  False for every other cell.
__device__ __forceinline__ bool outlet_source(const StepArgs &a, int b, const CompactCell &c, const CNbr &own,
                                              int &xu, uint32_t &ku, uint32_t &wu) {
    if (cell_type(c.word) != kOutlet || ((c.word >> 2) & 1u)) return false;
    ku = own.nb[2];  // x - 1, not SOLID
    wu = __ldg(a.clink + (size_t)b * a.kmax + ku);
    if (cell_type(wu) == kOutlet) return false;
    xu = c.x == 0 ? a.g.nx - 1 : c.x - 1;
    return true;
}

template <class S>
__global__ void __launch_bounds__(256, 4) k_psi_c(StepArgs a) {
    using T = typename Storage<S>::T;
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)__ldg(a.list_count + b)) return;
    const CompactCell c = compact_cell(a, b, k);
    const InstParam<T> &p = ((const InstParam<T> *)a.par)[b];
    T *psi = (T *)a.psi + (size_t)b * 2 * a.kmax;
    T p0, p1;
    if (cell_type(c.word) == kInlet) {
        p0 = p.rho_in[0];
        p1 = p.rho_in[1];
    } else {
        const S *fb = (const S *)a.f_in + (size_t)b * 2 * kQ * a.kmax;
        const size_t rb = (size_t)b * 2 * a.kmax;
        auto pull = [&](const CNbr &nb, uint32_t sk, uint32_t sw) {
            T r0 = T(0), r1 = T(0);
            if constexpr (Storage<S>::shifted) {
                r0 = (T)__half2float(a.ref_in[rb + sk]);
                r1 = (T)__half2float(a.ref_in[rb + a.kmax + sk]);
            }
            p0 = pull_density<S, true, CNbr>(fb, a.kmax, (int)sk, nb, sw, r0);
            p1 = pull_density<S, true, CNbr>(fb + kQ * (size_t)a.kmax, a.kmax, (int)sk, nb, sw, r1);
        };
        CNbr own;
        own.init(c.x, c.y, c.z, k, instance_tab(a, b), a.words, a.g);
        int xu;
        uint32_t ku, wu;
        if (outlet_source(a, b, c, own, xu, ku, wu)) {
            CNbr up;
            up.init(xu, c.y, c.z, ku, instance_tab(a, b), a.words, a.g);
            pull(up, ku, wu);
        } else {
            pull(own, k, c.word);
        }
    }
    psi[k] = p0;
    psi[a.kmax + k] = p1;
}

template <class S, int EQ>
__global__ void __launch_bounds__(256, 2) k_collide_c(StepArgs a) {
    using T = typename Storage<S>::T;
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)__ldg(a.list_count + b)) return;
    const CompactCell c = compact_cell(a, b, k);
    const uint32_t word = c.word;
    const InstParam<T> &p = ((const InstParam<T> *)a.par)[b];
    const size_t n = a.kmax;
    const size_t fofs = (size_t)b * 2 * kQ * n;
    const size_t rb = (size_t)b * 2 * n;
    S *fo = (S *)a.f_out;
    const T *psi0 = (const T *)a.psi + rb;
    const T *psi1 = psi0 + n;
    const long long cell = c.x + (long long)a.g.nx * (c.y + (long long)a.g.ny * c.z);
    T *mac = (T *)a.macro + (long long)b * 5 * a.g.n;
    CNbr own;
    own.init(c.x, c.y, c.z, k, instance_tab(a, b), a.words, a.g);
    // psi of both components at the 18 neighbours (own cell where SOLID: masked
    // by the force and never used as a reference there)
    T q0[kQ], q1[kQ];
    auto load_psi = [&]() {
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            const uint32_t j = ((word >> i) & 1u) ? k : own.dst(i);
            q0[i] = __ldg(psi0 + j);
            q1[i] = __ldg(psi1 + j);
        }
    };
    if (cell_type(word) == kInlet) {
        load_psi();
        auto s0 = [&](int i) -> T { return ref_value((i == 0 || ((word >> i) & 1u)) ? p.rho_in[0] : q0[i]); };
        auto s1 = [&](int i) -> T { return ref_value((i == 0 || ((word >> i) & 1u)) ? p.rho_in[1] : q1[i]); };
        store_equilibrium<S, EQ>(fo + fofs, n, (int)k, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2], s0);
        store_equilibrium<S, EQ>(fo + fofs + kQ * n, n, (int)k, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2], s1);
        if constexpr (Storage<S>::shifted) {
            a.ref_out[rb + k] = __float2half_rn((float)p.rho_in[0]);
            a.ref_out[rb + n + k] = __float2half_rn((float)p.rho_in[1]);
        }
        if (a.write_macro) {
            mac[cell] = p.rho_in[0];
            mac[a.g.n + cell] = p.rho_in[1];
            mac[2 * a.g.n + cell] = p.u_in[0];
            mac[3 * a.g.n + cell] = p.u_in[1];
            mac[4 * a.g.n + cell] = p.u_in[2];
        }
        return;
    }
    const S *f = (const S *)a.f_in + fofs;
    Moments<T> m0, m1;
    auto pull = [&](const CNbr &nb, uint32_t sk, uint32_t sw) {
        T r0 = T(0), r1 = T(0);
        if constexpr (Storage<S>::shifted) {
            r0 = (T)__half2float(a.ref_in[rb + sk]);
            r1 = (T)__half2float(a.ref_in[rb + n + sk]);
        }
        m0 = pull_moments<S, true, CNbr>(f, n, (int)sk, nb, sw, r0);
        m1 = pull_moments<S, true, CNbr>(f + kQ * n, n, (int)sk, nb, sw, r1);
    };
    {
        int xu;
        uint32_t ku, wu;
        if (outlet_source(a, b, c, own, xu, ku, wu)) {
            CNbr up;
            up.init(xu, c.y, c.z, ku, instance_tab(a, b), a.words, a.g);
            pull(up, ku, wu);
        } else {
            pull(own, k, word);
        }
    }
    load_psi();
    auto psi_at = [&](int i, T &v0, T &v1) {
        v0 = q0[i];
        v1 = q1[i];
    };
    const Forces<T> F = sc_forces<T>(psi_at, word, m0.rho, m1.rho, p, a.wall_model);
    const Relax<T> R = relax<T>(m0, m1, F, p);
    auto sig0 = [&](int i) -> T { return ref_value((i == 0 || ((word >> i) & 1u)) ? m0.rho : q0[i]); };
    auto sig1 = [&](int i) -> T { return ref_value((i == 0 || ((word >> i) & 1u)) ? m1.rho : q1[i]); };
    collide_store<S, EQ>(fo + fofs, n, (int)k, m0, R.ux, R.uy, R.uz, F.F[0][0], F.F[0][1], F.F[0][2], R.omega,
                         R.fcoef, sig0);
    collide_store<S, EQ>(fo + fofs + kQ * n, n, (int)k, m1, R.ux, R.uy, R.uz, F.F[1][0], F.F[1][1], F.F[1][2],
                         R.omega, R.fcoef, sig1);
    if constexpr (Storage<S>::shifted) {
        a.ref_out[rb + k] = __float2half_rn((float)m0.rho);
        a.ref_out[rb + n + k] = __float2half_rn((float)m1.rho);
    }
    if (a.write_macro) {
        mac[cell] = m0.rho;
        mac[a.g.n + cell] = m1.rho;
        mac[2 * a.g.n + cell] = R.ux;
        mac[3 * a.g.n + cell] = R.uy;
        mac[4 * a.g.n + cell] = R.uz;
    }
}

__global__ void k_compact_links(const uint32_t *__restrict__ list, const int *__restrict__ count,
                                const uint32_t *__restrict__ link, uint32_t *__restrict__ clink, long long n,
                                uint32_t kmax) {
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)count[b]) return;
    clink[(size_t)b * kmax + k] = link[(size_t)b * n + list[(size_t)b * n + k]];
}

// one thread per (non-solid cell, instance x component); all 19 planes
template <class S>
__global__ void k_layout(bool to_compact, const S *__restrict__ fin, S *__restrict__ fout, const Ref *__restrict__ rin,
                         Ref *__restrict__ rout, const uint32_t *__restrict__ list, const int *__restrict__ count,
                         long long n, uint32_t kmax) {
    const int bc = blockIdx.y;  // b * 2 + alpha
    const int b = bc >> 1;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)count[b]) return;
    const size_t cell = list[(size_t)b * n + k];
    const size_t ds = (size_t)n, cs = (size_t)kmax;
    for (int i = 0; i < kQ; ++i) {
        const size_t d = ((size_t)bc * kQ + i) * ds + cell, c = ((size_t)bc * kQ + i) * cs + k;
        if (to_compact)
            fout[c] = fin[d];
        else
            fout[d] = fin[c];
    }
    if (rin) {
        const size_t d = (size_t)bc * n + cell, c = (size_t)bc * kmax + k;
        if (to_compact)
            rout[c] = rin[d];
        else
            rout[d] = rin[c];
    }
}

template <class S>
static cudaError_t launch_compact_t(const StepArgs &a) {
    const dim3 grid((unsigned)((a.list_max + 255) / 256 > 0 ? (a.list_max + 255) / 256 : 1), (unsigned)a.batch, 1);
    record_event(a, 0);
    k_psi_c<S><<<grid, 256, 0, a.stream>>>(a);
    record_event(a, 1);
    if (a.eq_order == 0)
        k_collide_c<S, 0><<<grid, 256, 0, a.stream>>>(a);
    else
        k_collide_c<S, 1><<<grid, 256, 0, a.stream>>>(a);
    record_event(a, 2);
    return cudaGetLastError();
}

cudaError_t launch_compact(const StepArgs &a) {
    switch (a.precision) {
    case LBM_FP64: return launch_compact_t<double>(a);
    case LBM_FP32: return launch_compact_t<float>(a);
    case LBM_FP32_F16S: return launch_compact_t<__half>(a);
    case LBM_FP32_BF16S: return launch_compact_t<__nv_bfloat16>(a);
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
