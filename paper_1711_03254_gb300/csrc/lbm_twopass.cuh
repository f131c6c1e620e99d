// Kernels of the two-pass update on the dense layout (k_psi, k_collide) and
// their launcher, instantiated once per storage format in lbm_update_*.cu
// (one translation unit each, so that the variants compile in parallel).
// Layout and steps: see lbm_kernels.cu.
#pragma once

#include "lbm_internal.h"
#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ void cell_coords(long long k, const Grid &g, int &x, int &y, int &z) {
    const int kk = (int)k;
    const int t = kk / g.nx;
    x = kk - t * g.nx;
    z = t / g.ny;
    y = t - z * g.ny;
}

// OUTLET cells stream the values of their upstream (-x) neighbour unless that
// neighbour is SOLID or OUTLET itself.
__device__ __forceinline__ void source_cell(const uint32_t *__restrict__ link_b, uint32_t word, int &x, int y, int z,
                                            const Grid &g, uint32_t &src_word) {
    src_word = word;
    if (cell_type(word) == kOutlet) {
        const int xu = x == 0 ? g.nx - 1 : x - 1;
        const uint32_t wu = __ldg(link_b + xu + y * g.nx + (long long)z * g.nxy);
        const uint32_t tu = cell_type(wu);
        if (tu != kSolid && tu != kOutlet) {
            x = xu;
            src_word = wu;
        }
    }
}

template <class S>
__device__ __forceinline__ typename Storage<S>::T ref_at(const Ref *__restrict__ r, long long idx) {
    if constexpr (Storage<S>::shifted)
        return (typename Storage<S>::T)__half2float(r[idx]);
    else
        return typename Storage<S>::T(0);
}

// Cell handled by this thread: the thread index itself, or (with a list) the
// j-th non-solid cell of the instance, so that warps only carry cells that
// do work.  Returns false when the thread has no cell.
__device__ __forceinline__ bool my_cell(const uint32_t *__restrict__ list, const int *__restrict__ count, int b,
                                        const Grid &g, long long &k) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (list) {
        if (j >= count[b]) return false;
        k = __ldg(list + (long long)b * g.n + j);
        return true;
    }
    k = j;
    return j < g.n;
}

template <class S, bool SLIP>
__global__ void __launch_bounds__(256) k_psi(const S *__restrict__ f, const Ref *__restrict__ rin,
                                             const uint32_t *__restrict__ link, typename Storage<S>::T *__restrict__ psi,
                                             Grid g, const InstParam<typename Storage<S>::T> *__restrict__ par,
                                             const uint32_t *__restrict__ list, const int *__restrict__ count) {
    using T = typename Storage<S>::T;
    const int b = blockIdx.y;
    long long k;
    if (!my_cell(list, count, b, g, k)) return;
    const uint32_t *link_b = link + (long long)b * g.n;
    const uint32_t word = __ldg(link_b + k);
    const uint32_t t = cell_type(word);
    const InstParam<T> &p = par[b];
    T p0, p1;
    if (t == kSolid) {
        p0 = p.rs[0];
        p1 = p.rs[1];
    } else if (t == kInlet) {
        p0 = p.rho_in[0];
        p1 = p.rho_in[1];
    } else {
        int x, y, z;
        cell_coords(k, g, x, y, z);
        uint32_t sw;
        source_cell(link_b, word, x, y, z, g, sw);
        Nbr nb;
        nb.init(x, y, z, g);
        const int self = x + y * g.nx + z * g.nxy;
        const S *fb = f + (long long)b * 2 * kQ * g.n;
        const long long rb = (long long)b * 2 * g.n;
        p0 = pull_density<S, true, Nbr, SLIP>(fb, g.n, self, nb, sw, ref_at<S>(rin, rb + self), {p.slip, Storage<S>::shifted ? rin + rb : nullptr});
        p1 = pull_density<S, true, Nbr, SLIP>(fb + kQ * g.n, g.n, self, nb, sw, ref_at<S>(rin, rb + g.n + self),
                                             {p.slip, Storage<S>::shifted ? rin + rb + g.n : nullptr});
    }
    psi[((long long)b * 2 + 0) * g.n + k] = p0;
    psi[((long long)b * 2 + 1) * g.n + k] = p1;
}

template <class S, int EQ>
__global__ void __launch_bounds__(256, 2) k_collide(const S *__restrict__ f, S *__restrict__ fo,
                                                 const Ref *__restrict__ rin, Ref *__restrict__ rout,
                                                 const uint32_t *__restrict__ link,
                                                 const typename Storage<S>::T *__restrict__ psi,
                                                 typename Storage<S>::T *__restrict__ macro, Grid g,
                                                 const InstParam<typename Storage<S>::T> *__restrict__ par,
                                                 int wall_model, int write_macro, const uint32_t *__restrict__ list,
                                                 const int *__restrict__ count) {
    using T = typename Storage<S>::T;
    const int b = blockIdx.y;
    long long k;
    if (!my_cell(list, count, b, g, k)) return;
    const uint32_t *link_b = link + (long long)b * g.n;
    const uint32_t word = __ldg(link_b + k);
    const uint32_t t = cell_type(word);
    const InstParam<T> &p = par[b];
    const long long fofs = (long long)b * 2 * kQ * g.n;
    const long long rb = (long long)b * 2 * g.n;
    T *mac = macro + (long long)b * 5 * g.n;
    if (t == kSolid) {
        if (write_macro)
            for (int c = 0; c < 5; ++c) mac[c * g.n + k] = T(0);
        return;
    }
    int x, y, z;
    cell_coords(k, g, x, y, z);
    Nbr own;
    own.init(x, y, z, g);
    const T *psi0 = psi + (long long)b * 2 * g.n;
    const T *psi1 = psi0 + g.n;
    // reference density of the cell each value streams into (own cell when the
    // neighbour is SOLID and the value bounces back)
    auto sig_for = [&](const T *ps, T own_rho) {
        return [=, &own](int i) -> T {
            return ref_value(((word >> i) & 1u) ? own_rho : __ldg(ps + own.dst(i)));
        };
    };
    if (t == kInlet) {
        store_equilibrium<S, EQ>(fo + fofs, g.n, (int)k, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2],
                                 sig_for(psi0, p.rho_in[0]));
        store_equilibrium<S, EQ>(fo + fofs + kQ * g.n, g.n, (int)k, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2],
                                 sig_for(psi1, p.rho_in[1]));
        if constexpr (Storage<S>::shifted) {
            rout[rb + k] = __float2half_rn((float)p.rho_in[0]);
            rout[rb + g.n + k] = __float2half_rn((float)p.rho_in[1]);
        }
        if (write_macro) {
            mac[k] = p.rho_in[0];
            mac[g.n + k] = p.rho_in[1];
            mac[2 * g.n + k] = p.u_in[0];
            mac[3 * g.n + k] = p.u_in[1];
            mac[4 * g.n + k] = p.u_in[2];
        }
        return;
    }
    int sx = x;
    uint32_t sw;
    source_cell(link_b, word, sx, y, z, g, sw);
    Moments<T> m0, m1;
    if (sx == x) {
        m0 = pull_moments<S, true, Nbr, has_slip(EQ)>(f + fofs, g.n, (int)k, own, sw, ref_at<S>(rin, rb + k),
                                                      {p.slip, Storage<S>::shifted ? rin + rb : nullptr});
        m1 = pull_moments<S, true, Nbr, has_slip(EQ)>(f + fofs + kQ * g.n, g.n, (int)k, own, sw,
                                                      ref_at<S>(rin, rb + g.n + k), {p.slip, Storage<S>::shifted ? rin + rb + g.n : nullptr});
    } else {
        Nbr up;
        up.init(sx, y, z, g);
        const int self = sx + y * g.nx + z * g.nxy;
        m0 = pull_moments<S, true, Nbr, has_slip(EQ)>(f + fofs, g.n, self, up, sw, ref_at<S>(rin, rb + self),
                                                      {p.slip, Storage<S>::shifted ? rin + rb : nullptr});
        m1 = pull_moments<S, true, Nbr, has_slip(EQ)>(f + fofs + kQ * g.n, g.n, self, up, sw,
                                                      ref_at<S>(rin, rb + g.n + self), {p.slip, Storage<S>::shifted ? rin + rb + g.n : nullptr});
    }
    // psi of both components at the 18 neighbours, loaded once: they feed the
    // forces and (shifted storage) the reference densities of the stores
    T q0[kQ], q1[kQ];
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const int j = own.dst(i);
        q0[i] = __ldg(psi0 + j);
        q1[i] = __ldg(psi1 + j);
    }
    auto psi_at = [&](int i, T &a, T &c) {
        a = q0[i];
        c = q1[i];
    };
    const Forces<T> F = sc_forces<T>(psi_at, word, m0.rho, m1.rho, p, wall_model);
    const Relax<T> R = relax<T>(m0, m1, F, p);
    const T ux = R.ux, uy = R.uy, uz = R.uz, omega = R.omega, fcoef = R.fcoef;
    // reference density of the cell each value streams into (own cell when the
    // neighbour is SOLID and the value bounces back)
    auto sig0 = [&](int i) -> T { return ref_value((i == 0 || ((word >> i) & 1u)) ? m0.rho : q0[i]); };
    auto sig1 = [&](int i) -> T { return ref_value((i == 0 || ((word >> i) & 1u)) ? m1.rho : q1[i]); };
    collide_store<S, EQ>(fo + fofs, g.n, (int)k, m0, ux, uy, uz, F.F[0][0], F.F[0][1], F.F[0][2], omega, fcoef,
                         sig0);
    collide_store<S, EQ>(fo + fofs + kQ * g.n, g.n, (int)k, m1, ux, uy, uz, F.F[1][0], F.F[1][1], F.F[1][2], omega,
                         fcoef, sig1);
    if constexpr (Storage<S>::shifted) {
        rout[rb + k] = __float2half_rn((float)m0.rho);
        rout[rb + g.n + k] = __float2half_rn((float)m1.rho);
    }
    if (write_macro) {
        mac[k] = m0.rho;
        mac[g.n + k] = m1.rho;
        mac[2 * g.n + k] = ux;
        mac[3 * g.n + k] = uy;
        mac[4 * g.n + k] = uz;
    }
}

inline dim3 cell_grid(const Grid &g, int batch, int threads) {
    return dim3((unsigned)((g.n + threads - 1) / threads), (unsigned)batch, 1);
}

template <class S>
cudaError_t launch_two_pass_t(const StepArgs &a) {
    using T = typename Storage<S>::T;
    // with cell lists only the non-solid cells get threads (ψ of SOLID cells is static)
    const long long span = a.list ? (a.list_max > 0 ? a.list_max : 1) : a.g.n;
    const dim3 grid((unsigned)((span + 255) / 256), (unsigned)a.batch, 1);
    record_event(a, 0);
    if (a.slip)
        k_psi<S, true><<<grid, 256, 0, a.stream>>>((const S *)a.f_in, a.ref_in, a.link, (T *)a.psi, a.g,
                                                   (const InstParam<T> *)a.par, a.list, a.list_count);
    else
        k_psi<S, false><<<grid, 256, 0, a.stream>>>((const S *)a.f_in, a.ref_in, a.link, (T *)a.psi, a.g,
                                                    (const InstParam<T> *)a.par, a.list, a.list_count);
    record_event(a, 1);
    dispatch_variant(collide_variant(a), [&](auto v) {
        constexpr int EQ = decltype(v)::value;
        k_collide<S, EQ><<<grid, 256, 0, a.stream>>>((const S *)a.f_in, (S *)a.f_out, a.ref_in, a.ref_out, a.link,
                                                     (const T *)a.psi, (T *)a.macro, a.g, (const InstParam<T> *)a.par,
                                                     a.wall_model, a.write_macro, a.list, a.list_count);
    });
    record_event(a, 2);
    return cudaGetLastError();
}

}  // namespace lbm
