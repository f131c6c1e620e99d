// Two-pass update kernels, initialisation and geometry preprocessing.
//
//   k_psi      S1-S3: pull the 19 streamed values of each component, sum them
//              to rho_alpha and store the pseudo-potential psi (rho in fluid,
//              rho^s at SOLID cells, rho_in at INLET cells).
//   k_collide  S1-S7: pull again, reduce to moments, read psi of the 18
//              neighbours, forces, u_F, tau_mix, regularised collision, store.
//
// Layout in HBM (per instance b): f[b][alpha][i][cell], cell = x + nx (y + ny z);
// psi[b][alpha][cell]; macro[b][{rho1, rho2, ux, uy, uz}][cell]; reference
// densities ref[b][alpha][cell] (FP16, double-buffered with f); geometry word
// link[b][cell] (bits 0..18 SOLID neighbours, bits 24..25 cell type).
#include "lbm_twopass.cuh"

namespace lbm {

// instantiated in lbm_update_*.cu
extern template cudaError_t launch_two_pass_t<double>(const StepArgs &);
extern template cudaError_t launch_two_pass_t<float>(const StepArgs &);
extern template cudaError_t launch_two_pass_t<__half>(const StepArgs &);
extern template cudaError_t launch_two_pass_t<__nv_bfloat16>(const StepArgs &);

// Initial density of every cell as its neighbours see it (0 at SOLID cells,
// rho_in at INLET cells), rounded to the FP16 reference of the shifted
// storages: the reference densities of the initial state.
template <class T>
__global__ void k_init_ref(const double *__restrict__ r1, const double *__restrict__ r2,
                           const uint32_t *__restrict__ link, Ref *__restrict__ rout, Grid g,
                           const InstParam<T> *__restrict__ par) {
    const int b = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    const long long gk = (long long)b * g.n + k;
    const uint32_t t = cell_type(__ldg(link + gk));
    T a0 = T(0), a1 = T(0);
    if (t == kInlet) {
        a0 = par[b].rho_in[0];
        a1 = par[b].rho_in[1];
    } else if (t != kSolid) {
        a0 = (T)r1[gk];
        a1 = (T)r2[gk];
    }
    rout[(long long)b * 2 * g.n + k] = __float2half_rn((float)a0);
    rout[(long long)b * 2 * g.n + g.n + k] = __float2half_rn((float)a1);
}

// f := feq(rho_alpha, u) from FP64 fields (u interleaved [b][cell][3]).  The
// shifted storages store each value against the reference density of the
// cell it streams into: k_init_ref has written those (ref), and a value that
// bounces back off a SOLID neighbour takes the cell's own density.  Four
// blocks per SM (64 registers, some spilled): at the 86 registers the compiler
// chose unbounded, two blocks left the kernel waiting on memory latency (22 %
// of the warps active, 0.57 ms at 192^3); lbm_set_fields at 256^3 went from
// 5.17 to 4.68 ms with its copies (3 blocks: 4.79).
template <class S, int EQ>
__global__ void __launch_bounds__(256, 4) k_init(const double *__restrict__ r1, const double *__restrict__ r2, const double *__restrict__ u,
                       const uint32_t *__restrict__ link, S *__restrict__ fo, const Ref *__restrict__ ref,
                       typename Storage<S>::T *__restrict__ macro, typename Storage<S>::T *__restrict__ usnap, Grid g,
                       const InstParam<typename Storage<S>::T> *__restrict__ par) {
    using T = typename Storage<S>::T;
    const int b = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    const long long gk = (long long)b * g.n + k;
    const uint32_t word = link[gk];
    const uint32_t t = cell_type(word);
    const InstParam<T> &p = par[b];
    T a0, a1, ux, uy, uz;
    if (t == kSolid) {
        a0 = a1 = ux = uy = uz = T(0);
    } else if (t == kInlet) {
        a0 = p.rho_in[0]; a1 = p.rho_in[1];
        ux = p.u_in[0]; uy = p.u_in[1]; uz = p.u_in[2];
    } else {
        a0 = (T)r1[gk]; a1 = (T)r2[gk];
        ux = (T)u[3 * gk]; uy = (T)u[3 * gk + 1]; uz = (T)u[3 * gk + 2];
    }
    int x, y, z;
    cell_coords(k, g, x, y, z);
    Nbr nb;
    nb.init(x, y, z, g);
    const long long fofs = (long long)b * 2 * kQ * g.n;
    const Ref *ref0 = ref + (long long)b * 2 * g.n, *ref1 = ref0 + g.n;
    // (only the shifted storages call these)
    store_equilibrium<S, EQ>(fo + fofs, g.n, (int)k, a0, ux, uy, uz, [&](int i) -> T {
        return ((word >> i) & 1u) ? ref_value(a0) : (T)__half2float(__ldg(ref0 + nb.dst(i)));
    });
    store_equilibrium<S, EQ>(fo + fofs + kQ * g.n, g.n, (int)k, a1, ux, uy, uz, [&](int i) -> T {
        return ((word >> i) & 1u) ? ref_value(a1) : (T)__half2float(__ldg(ref1 + nb.dst(i)));
    });
    T *mac = macro + (long long)b * 5 * g.n;
    mac[k] = a0; mac[g.n + k] = a1;
    mac[2 * g.n + k] = ux; mac[3 * g.n + k] = uy; mac[4 * g.n + k] = uz;
    T *us = usnap + (long long)b * 3 * g.n;
    us[k] = ux; us[g.n + k] = uy; us[2 * g.n + k] = uz;
}

__global__ void k_links(const uint8_t *__restrict__ type, uint32_t *__restrict__ link, Grid g) {
    const int b = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    int x, y, z;
    cell_coords(k, g, x, y, z);
    Nbr nb;
    nb.init(x, y, z, g);
    const uint8_t *tb = type + (long long)b * g.n;
    uint32_t w = (uint32_t)tb[k] << 24;
#pragma unroll
    for (int i = 1; i < kQ; ++i)
        if (tb[nb.dst(i)] == kSolid) w |= 1u << i;
    link[(long long)b * g.n + k] = w;
}

// Macro fields (T) -> FP64 host layout (u interleaved).
template <class T>
__global__ void k_macro_to_f64(const T *__restrict__ macro, double *__restrict__ r1, double *__restrict__ r2,
                               double *__restrict__ u, Grid g) {
    const int b = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    const T *mac = macro + (long long)b * 5 * g.n;
    const long long gk = (long long)b * g.n + k;
    r1[gk] = (double)mac[k];
    r2[gk] = (double)mac[g.n + k];
    u[3 * gk] = (double)mac[2 * g.n + k];
    u[3 * gk + 1] = (double)mac[3 * g.n + k];
    u[3 * gk + 2] = (double)mac[4 * g.n + k];
}

// Distributions <-> FP64, one thread per cell and component: value i of cell x
// is stored relative to the reference density of x + c_i (or of x itself when
// x + c_i is SOLID).
template <class S>
__global__ void k_f_convert(const S *__restrict__ f, double *__restrict__ out, const double *__restrict__ in,
                            S *__restrict__ fo, const Ref *__restrict__ ref, const uint32_t *__restrict__ link,
                            Grid g) {
    using T = typename Storage<S>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int bc = blockIdx.y;  // b * 2 + alpha
    if (k >= g.n) return;
    const int b = bc >> 1;
    const uint32_t word = link[(long long)b * g.n + k];
    if (cell_type(word) == kSolid) {  // no distributions in SOLID cells
        if (out)
            for (int i = 0; i < kQ; ++i) out[((long long)bc * kQ + i) * g.n + k] = 0.0;
        return;
    }
    int x, y, z;
    cell_coords(k, g, x, y, z);
    Nbr nb;
    nb.init(x, y, z, g);
    const long long rb = (long long)bc * g.n;
#pragma unroll 1
    for (int i = 0; i < kQ; ++i) {
        T sh = T(0);
        if constexpr (Storage<S>::shifted) {
            const long long src = ((word >> i) & 1u) ? k : nb.dst(i);
            sh = wgt<T>(i) * (T)__half2float(ref[rb + src]);
        }
        const long long idx = ((long long)bc * kQ + i) * g.n + k;
        if (out)
            out[idx] = (double)Storage<S>::load(f + idx, sh);
        else
            Storage<S>::store(fo + idx, (T)in[idx], sh);
    }
}

// ------------------------------------------------------------------ launchers



// ψ of every SOLID cell (constant in time; the list kernels never visit them).
template <class T>
__global__ void k_psi_solid(const uint32_t *__restrict__ link, T *__restrict__ psi, Grid g,
                            const InstParam<T> *__restrict__ par) {
    const int b = blockIdx.y;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    if (cell_type(link[(long long)b * g.n + k]) != kSolid) return;
    psi[((long long)b * 2 + 0) * g.n + k] = par[b].rs[0];
    psi[((long long)b * 2 + 1) * g.n + k] = par[b].rs[1];
}

cudaError_t launch_psi_solid(const uint32_t *link, void *psi, bool fp64, const Grid &g, int batch, const void *par,
                             cudaStream_t s) {
    if (fp64)
        k_psi_solid<double><<<cell_grid(g, batch, 256), 256, 0, s>>>(link, (double *)psi, g,
                                                                     (const InstParam<double> *)par);
    else
        k_psi_solid<float><<<cell_grid(g, batch, 256), 256, 0, s>>>(link, (float *)psi, g,
                                                                    (const InstParam<float> *)par);
    return cudaGetLastError();
}

cudaError_t launch_two_pass(const StepArgs &a) {
    switch (a.precision) {
    case LBM_FP64: return launch_two_pass_t<double>(a);
    case LBM_FP32: return launch_two_pass_t<float>(a);
    case LBM_FP32_F16S: return launch_two_pass_t<__half>(a);
    case LBM_FP32_BF16S: return launch_two_pass_t<__nv_bfloat16>(a);
    }
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t launch_init_t(const InitArgs &a) {
    using T = typename Storage<S>::T;
    const dim3 grid = cell_grid(a.g, a.batch, 256);
    if constexpr (Storage<S>::shifted)
        k_init_ref<T><<<grid, 256, 0, a.stream>>>(a.r1, a.r2, a.link, a.ref_out, a.g, (const InstParam<T> *)a.par);
    if (a.eq_order == 0)
        k_init<S, 0><<<grid, 256, 0, a.stream>>>(a.r1, a.r2, a.u, a.link, (S *)a.f_out, a.ref_out, (T *)a.macro,
                                                 (T *)a.usnap, a.g, (const InstParam<T> *)a.par);
    else
        k_init<S, 1><<<grid, 256, 0, a.stream>>>(a.r1, a.r2, a.u, a.link, (S *)a.f_out, a.ref_out, (T *)a.macro,
                                                 (T *)a.usnap, a.g, (const InstParam<T> *)a.par);
    return cudaGetLastError();
}

cudaError_t launch_init(const InitArgs &a) {
    switch (a.precision) {
    case LBM_FP64: return launch_init_t<double>(a);
    case LBM_FP32: return launch_init_t<float>(a);
    case LBM_FP32_F16S: return launch_init_t<__half>(a);
    case LBM_FP32_BF16S: return launch_init_t<__nv_bfloat16>(a);
    }
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t launch_f_convert_t(const void *f, double *out, const double *in, void *fo, const Ref *ref,
                                      const uint32_t *link, const Grid &g, int batch, cudaStream_t s) {
    const dim3 grid((unsigned)((g.n + 255) / 256), (unsigned)(batch * 2), 1);
    k_f_convert<S><<<grid, 256, 0, s>>>((const S *)f, out, in, (S *)fo, ref, link, g);
    return cudaGetLastError();
}

cudaError_t launch_f_convert(lbm_precision prec, const void *f, double *out, const double *in, void *fo,
                             const Ref *ref, const uint32_t *link, const Grid &g, int batch, cudaStream_t s) {
    switch (prec) {
    case LBM_FP64: return launch_f_convert_t<double>(f, out, in, fo, ref, link, g, batch, s);
    case LBM_FP32: return launch_f_convert_t<float>(f, out, in, fo, ref, link, g, batch, s);
    case LBM_FP32_F16S: return launch_f_convert_t<__half>(f, out, in, fo, ref, link, g, batch, s);
    case LBM_FP32_BF16S: return launch_f_convert_t<__nv_bfloat16>(f, out, in, fo, ref, link, g, batch, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_links(const uint8_t *type, uint32_t *link, const Grid &g, int batch, cudaStream_t s) {
    k_links<<<cell_grid(g, batch, 256), 256, 0, s>>>(type, link, g);
    return cudaGetLastError();
}

cudaError_t launch_macro_to_f64(const void *macro, bool fp64, double *r1, double *r2, double *u, const Grid &g,
                                int batch, cudaStream_t s) {
    if (fp64)
        k_macro_to_f64<double><<<cell_grid(g, batch, 256), 256, 0, s>>>((const double *)macro, r1, r2, u, g);
    else
        k_macro_to_f64<float><<<cell_grid(g, batch, 256), 256, 0, s>>>((const float *)macro, r1, r2, u, g);
    return cudaGetLastError();
}

}  // namespace lbm
