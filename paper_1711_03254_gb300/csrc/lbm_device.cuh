// Device building blocks of the two-component Shan-Chen D3Q19 update
// (Otomo et al., arXiv:1711.03254, Sec. 2).  Everything here is inlined into
// the kernels of lbm_kernels.cu; nothing is shared with the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_types.h"

namespace lbm {

constexpr int kQ = 19;

// D3Q19 velocities: 0 rest, then opposite pairs (2k-1, 2k):
// +-x, +-y, +-z, (+x+y,-x-y), (+x-y,-x+y), (+x+z,-x-z), (+x-z,-x+z),
// (+y+z,-y-z), (+y-z,-y+z).
__host__ __device__ constexpr int cx(int i) {
    constexpr int v[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
}
__host__ __device__ constexpr int cy(int i) {
    constexpr int v[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
}
__host__ __device__ constexpr int cz(int i) {
    constexpr int v[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// lattice weights (1/3, 1/18, 1/36) as exact rationals num/36
__host__ __device__ constexpr int w36(int i) { return i == 0 ? 12 : (i <= 6 ? 2 : 1); }

template <class T> __device__ __forceinline__ constexpr T wgt(int i) { return T(w36(i)) / T(36); }

// Specular reflection at a voxel wall (partial slip, the surface scattering
// of Sec. 2).  For an edge direction i with non-zero components on axes a < b
// whose source x - c_i is SOLID: if the face neighbour x - c_ia e_a is open
// and x - c_ib e_b SOLID, the wall's normal is e_b and the particle came from
// x - c_ia e_a in the direction of c_i with its b component reversed (and
// likewise with a and b exchanged); at corners (both face neighbours SOLID, or
// neither) it bounces back.  The partner cell reflects this cell's value the
// same way, so blending the two conserves mass.
__host__ __device__ constexpr int dir_of(int x, int y, int z) {
    for (int k = 0; k < kQ; ++k)
        if (cx(k) == x && cy(k) == y && cz(k) == z) return k;
    return -1;
}
__host__ __device__ constexpr int comp(int i, int a) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }
// the m-th (0, 1) axis on which the edge direction i is non-zero
__host__ __device__ constexpr int edge_axis(int i, int m) {
    return m == 0 ? (cx(i) != 0 ? 0 : 1) : (cz(i) != 0 ? 2 : 1);
}
// direction from x to its face neighbour x - c_ia e_a (a = edge_axis(i, m))
__host__ __device__ constexpr int face_back(int i, int m) {
    return dir_of(edge_axis(i, m) == 0 ? -cx(i) : 0, edge_axis(i, m) == 1 ? -cy(i) : 0,
                  edge_axis(i, m) == 2 ? -cz(i) : 0);
}
// c_i with its component on edge_axis(i, m) reversed
__host__ __device__ constexpr int mirrored(int i, int m) {
    return dir_of(edge_axis(i, m) == 0 ? -cx(i) : cx(i), edge_axis(i, m) == 1 ? -cy(i) : cy(i),
                  edge_axis(i, m) == 2 ? -cz(i) : cz(i));
}
// For the edge direction i of a cell with SOLID-neighbour bits `links` and
// x - c_i SOLID: the direction from the cell to the reflection's source cell
// (`via`) and the direction of the reflected value there (`j`); false at
// corners.
__device__ __forceinline__ bool specular_source(int i, uint32_t links, int &via, int &j) {
    const bool sa = (links >> face_back(i, 0)) & 1u, sb = (links >> face_back(i, 1)) & 1u;
    if (sa == sb) return false;
    via = sa ? face_back(i, 1) : face_back(i, 0);
    j = sa ? mirrored(i, 0) : mirrored(i, 1);
    return true;
}
constexpr bool has_slip(int EQ) { return (EQ & 4) != 0; }

// Cell-type encoding of the per-cell geometry word: bits 0..18 flag the
// directions i whose neighbour x + c_i is SOLID, bits 24..25 hold the type.
constexpr uint32_t kFluid = 0, kSolid = 1, kInlet = 2, kOutlet = 3;
__device__ __forceinline__ uint32_t cell_type(uint32_t word) { return (word >> 24) & 3u; }

// -------------------------------------------------------------- storage
// How one distribution value is held in HBM.  FP32 and the 16-bit formats
// store the deviation from a rest equilibrium w_i R, where R is the density
// (rounded to FP16) that the cell the value streams into had at its last
// update: R is the same for all 19 values a cell pulls, so the reader adds
// w_i R(self) back.  A constant reference density would leave the minority
// phase (f ~ 0) stored as -w_i rho0, whose rounding error repeats every update
// and drifts the minority mass.
template <class S> struct Storage;
__device__ __forceinline__ float ref_value(float r) { return __half2float(__float2half_rn(r)); }
__device__ __forceinline__ double ref_value(double r) { return r; }
template <> struct Storage<double> {
    using T = double;
    static constexpr bool shifted = false;
    __device__ static __forceinline__ double load(const double *p, double) { return __ldg(p); }
    __device__ static __forceinline__ double load_rw(const double *p, double) { return __ldcg(p); }
    __device__ static __forceinline__ void store(double *p, double v, double) { *p = v; }
    __device__ static __forceinline__ void store_d(double *p, double d) { *p = d; }
};
template <> struct Storage<float> {
    using T = float;
    static constexpr bool shifted = true;
    __device__ static __forceinline__ float load(const float *p, float sh) { return __ldg(p) + sh; }
    __device__ static __forceinline__ float load_rw(const float *p, float sh) { return __ldcg(p) + sh; }
    __device__ static __forceinline__ void store(float *p, float v, float sh) { *p = v - sh; }
    __device__ static __forceinline__ void store_d(float *p, float d) { *p = d; }
};
// FP16 holds the deviations scaled by 2^12 (exactly: a power of two), which
// moves the typical deviations (1e-8 .. 1e-1) out of FP16's subnormal range
// (below 6.1e-5, where its relative precision falls off) while keeping room up
// to 65504 / 4096 = 16.  BF16 has FP32's exponent range and needs no scale.
constexpr float kF16Scale = 4096.f, kF16Unscale = 1.f / 4096.f;
template <> struct Storage<__half> {
    using T = float;
    static constexpr bool shifted = true;
    __device__ static __forceinline__ float load(const __half *p, float sh) {
        return __half2float(__ldg(p)) * kF16Unscale + sh;
    }
    __device__ static __forceinline__ float load_rw(const __half *p, float sh) {
        return __half2float(__ldcg(p)) * kF16Unscale + sh;
    }
    __device__ static __forceinline__ void store(__half *p, float v, float sh) {
        *p = __float2half_rn((v - sh) * kF16Scale);
    }
    __device__ static __forceinline__ void store_d(__half *p, float d) { *p = __float2half_rn(d * kF16Scale); }
};
template <> struct Storage<__nv_bfloat16> {
    using T = float;
    static constexpr bool shifted = true;
    __device__ static __forceinline__ float load(const __nv_bfloat16 *p, float sh) {
        return __bfloat162float(__ldg(p)) + sh;
    }
    __device__ static __forceinline__ float load_rw(const __nv_bfloat16 *p, float sh) {
        return __bfloat162float(__ldcg(p)) + sh;
    }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, float v, float sh) {
        *p = __float2bfloat16_rn(v - sh);
    }
    __device__ static __forceinline__ void store_d(__nv_bfloat16 *p, float d) { *p = __float2bfloat16_rn(d); }
};

// -------------------------------------------------------------- neighbours
// Wrapped coordinates x-1, x, x+1 (and y, z scaled to linear offsets).
struct Nbr {
    int X[3], Y[3], Z[3];
    __device__ __forceinline__ void init(int x, int y, int z, const Grid &g) {
        X[0] = x == 0 ? g.nx - 1 : x - 1;
        X[1] = x;
        X[2] = x == g.nx - 1 ? 0 : x + 1;
        Y[0] = (y == 0 ? g.ny - 1 : y - 1) * g.nx;
        Y[1] = y * g.nx;
        Y[2] = (y == g.ny - 1 ? 0 : y + 1) * g.nx;
        Z[0] = (z == 0 ? g.nz - 1 : z - 1) * g.nxy;
        Z[1] = z * g.nxy;
        Z[2] = (z == g.nz - 1 ? 0 : z + 1) * g.nxy;
    }
    // linear index of x - c_i (pull source)
    __device__ __forceinline__ int src(int i) const { return X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)]; }
    // linear index of x + c_i
    __device__ __forceinline__ int dst(int i) const { return X[1 + cx(i)] + Y[1 + cy(i)] + Z[1 + cz(i)]; }
};

// Neighbours in the compact layout, where only the non-solid cells of an
// instance are stored, in cell order: the compact index of a cell is the
// number of non-solid cells before it.  Each row (y, z) of the instance is
// described by 32-cell words {rank of the word's first cell, mask of its
// non-solid cells} (tab[row][word]; one extra row at the end holds the total).
// nb[j] is the compact index of x + c_j wherever that cell is not SOLID; at
// SOLID neighbours it is meaningless and must not be dereferenced.
struct CNbr {
    uint32_t nb[kQ];
    // linear offset of x - c_i / x + c_i within one plane of the compact layout
    __device__ __forceinline__ uint32_t src(int i) const { return nb[opp(i)]; }
    __device__ __forceinline__ uint32_t dst(int i) const { return nb[i]; }

    // (x, y, z) with compact index k; tb = the instance's row table.
    __device__ __forceinline__ void init(int x, int y, int z, uint32_t k, const uint2 *__restrict__ tb, int words,
                                         const Grid &g) {
        const int ys[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
        const int zs[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
        const int w = x >> 5, xb = x & 31;
        const uint32_t below = (1u << xb) - 1u;
        // own row: neighbours along x are the adjacent compact indices
        nb[0] = k;
        nb[1] = k + 1u;
        nb[2] = k - 1u;
#pragma unroll
        for (int j = 3; j < kQ; ++j) {
            if (cx(j) != 0) continue;  // filled with the x = 0 member of its row below
            const int r = zs[1 + cz(j)] * g.ny + ys[1 + cy(j)];
            const uint2 e = __ldg(tb + (size_t)r * words + w);
            const uint32_t at = e.x + __popc(e.y & below);  // rank of (x, row)
            nb[j] = at;
            // the +x and -x members of the same row (only the y or z face rows have
            // them): rank(x + 1) = rank(x) + [x non-solid], rank(x - 1) = rank(x) - 1
#pragma unroll
            for (int m = 7; m < kQ; ++m) {
                if (cy(m) != cy(j) || cz(m) != cz(j) || cx(m) == 0) continue;
                nb[m] = cx(m) > 0 ? at + ((e.y >> xb) & 1u) : at - 1u;
            }
        }
        // x = 0 or nx - 1: the members across the periodic x boundary are the
        // first (+x from nx - 1) or last (-x from 0) non-solid cell of their row
        if (x == 0 || x == g.nx - 1) wrap_x(x, ys, zs, tb, words, g);
    }

    __device__ __forceinline__ void wrap_x(int x, const int (&ys)[3], const int (&zs)[3], const uint2 *__restrict__ tb,
                                        int words, const Grid &g) {
        auto row_rank = [&](int r) -> uint32_t { return __ldg(tb + (size_t)r * words).x; };
#pragma unroll
        for (int m = 1; m < kQ; ++m) {
            if (cx(m) == 0) continue;
            const int r = zs[1 + cz(m)] * g.ny + ys[1 + cy(m)];
            if (cx(m) > 0 && x == g.nx - 1) nb[m] = row_rank(r);
            if (cx(m) < 0 && x == 0) nb[m] = row_rank(r + 1) - 1u;
        }
    }
};

// Moments of the streamed distributions of one component (S1-S2).  In the
// shifted storage formats they are summed over the stored deviations
// d_i = f_i - w_i R (no cancellation against the rest equilibrium):
//   rho = R + sum d,  rd = sum d,  j = sum c d,  p = sum c c d,
// so that Pi - rho T0 I = p - rd T0 I.  Unshifted: rd = rho, p = sum c c f.
template <class T> struct Moments {
    T rho, rd, jx, jy, jz;
    T pxx, pyy, pzz, pxy, pxz, pyz;
};

// Pull the 19 streamed values of component `comp` into cell `self` (linear
// index) whose neighbours are `nb` and whose solid-neighbour bits are `links`
// (bit k: x + c_k is SOLID, so the value travelling in direction i comes back
// from the cell itself when bit opp(i) is set), and reduce them to moments.
// `rref` is the reference density R of the pulling cell (see Storage).
// RO = true reads through the read-only data path (buffers not written by the
// same launch); RO = false uses coherent loads (persistent kernels).
// Moments of the 19 stored values v of one component (R = rref in the shifted
// formats, see Moments).
template <class T, bool SHIFTED>
__device__ __forceinline__ Moments<T> moments_of(const T (&v)[kQ], T rref) {
    Moments<T> m;
    T r = v[0];
#pragma unroll
    for (int i = 1; i < kQ; ++i) r += v[i];
    m.rd = r;
    m.rho = SHIFTED ? rref + r : r;
    m.jx = (v[1] - v[2]) + (v[7] - v[8]) + (v[9] - v[10]) + (v[11] - v[12]) + (v[13] - v[14]);
    m.jy = (v[3] - v[4]) + (v[7] - v[8]) + (v[10] - v[9]) + (v[15] - v[16]) + (v[17] - v[18]);
    m.jz = (v[5] - v[6]) + (v[11] - v[12]) + (v[14] - v[13]) + (v[15] - v[16]) + (v[18] - v[17]);
    const T e_xy = (v[7] + v[8]) + (v[9] + v[10]);
    const T e_xz = (v[11] + v[12]) + (v[13] + v[14]);
    const T e_yz = (v[15] + v[16]) + (v[17] + v[18]);
    m.pxx = (v[1] + v[2]) + e_xy + e_xz;
    m.pyy = (v[3] + v[4]) + e_xy + e_yz;
    m.pzz = (v[5] + v[6]) + e_xz + e_yz;
    m.pxy = (v[7] + v[8]) - (v[9] + v[10]);
    m.pxz = (v[11] + v[12]) - (v[13] + v[14]);
    m.pyz = (v[15] + v[16]) - (v[17] + v[18]);
    return m;
}

// Density of the 19 stored values v (same summation order as moments_of).
template <class T, bool SHIFTED> __device__ __forceinline__ T density_of(const T (&v)[kQ], T rref) {
    T r = v[0];
#pragma unroll
    for (int i = 1; i < kQ; ++i) r += v[i];
    return SHIFTED ? rref + r : r;
}

// Wall slip of one component's pulled values v (dense layout): every edge
// direction whose source is SOLID gets (1 - s) times the bounced-back value
// plus s times the specular reflection (specular_source).  In the shifted
// formats the reflected value is stored against its source cell's reference
// density, and is moved to this cell's (rref) with the source's entry of the
// component's reference plane rcomp.
template <class S, class NB>
__device__ __forceinline__ void slip_values(const S *__restrict__ fcomp, long long n, const NB &nb, uint32_t links,
                                            typename Storage<S>::T s, const Ref *__restrict__ rcomp,
                                            typename Storage<S>::T rref, typename Storage<S>::T (&v)[kQ]) {
    using T = typename Storage<S>::T;
    if (s == T(0)) return;
#pragma unroll
    for (int i = 7; i < kQ; ++i) {
        int via, j;
        if (!((links >> opp(i)) & 1u) || !specular_source(i, links, via, j)) continue;
        const uint32_t src = (uint32_t)nb.dst(via);
        T r = Storage<S>::load(fcomp + ((uint32_t)j * (uint32_t)n + src), T(0));
        if constexpr (Storage<S>::shifted) r += wgt<T>(i) * ((T)__half2float(__ldg(rcomp + src)) - rref);
        v[i] = (T(1) - s) * v[i] + s * r;
    }
}

// Optional wall slip of a pull: the instance's slip fraction and the pulled
// component's reference plane (shifted formats).
template <class T> struct SlipArgs {
    T s = T(0);
    const Ref *rcomp = nullptr;
};

template <class S, bool RO = true, class NB = Nbr, bool SLIP = false>
__device__ __forceinline__ Moments<typename Storage<S>::T>
pull_moments(const S *__restrict__ fcomp, long long n, int self, const NB &nb, uint32_t links,
             typename Storage<S>::T rref, SlipArgs<typename Storage<S>::T> sl = {}) {
    using T = typename Storage<S>::T;
    T v[kQ];  // stored values: deviations d_i in the shifted formats, f_i otherwise
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const bool bb = (links >> opp(i)) & 1u;
        // 32-bit offsets within one component's planes (19 n < 2^32 is checked at creation)
        const uint32_t idx = bb ? (uint32_t)opp(i) * (uint32_t)n + (uint32_t)self
                                : (uint32_t)i * (uint32_t)n + (uint32_t)nb.src(i);
        v[i] = RO ? Storage<S>::load(fcomp + idx, T(0)) : Storage<S>::load_rw(fcomp + idx, T(0));
    }
    if constexpr (SLIP) slip_values<S>(fcomp, n, nb, links, sl.s, sl.rcomp, rref, v);
    return moments_of<T, Storage<S>::shifted>(v, rref);
}

// Density only (for the pseudo-potential pass), same summation order.
template <class S, bool RO = true, class NB = Nbr, bool SLIP = false>
__device__ __forceinline__ typename Storage<S>::T pull_density(const S *__restrict__ fcomp, long long n, int self,
                                                              const NB &nb, uint32_t links,
                                                              typename Storage<S>::T rref,
                                                              SlipArgs<typename Storage<S>::T> sl = {}) {
    using T = typename Storage<S>::T;
    T v[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const bool bb = (links >> opp(i)) & 1u;
        // 32-bit offsets within one component's planes (19 n < 2^32 is checked at creation)
        const uint32_t idx = bb ? (uint32_t)opp(i) * (uint32_t)n + (uint32_t)self
                                : (uint32_t)i * (uint32_t)n + (uint32_t)nb.src(i);
        v[i] = RO ? Storage<S>::load(fcomp + idx, T(0)) : Storage<S>::load_rw(fcomp + idx, T(0));
    }
    if constexpr (SLIP) slip_values<S>(fcomp, n, nb, links, sl.s, sl.rcomp, rref, v);
    return density_of<T, Storage<S>::shifted>(v, rref);
}

// Collision variants EQ: bit 0 adds the quadratic terms to the equilibrium of
// Eq. 3 (eq_order 1); bit 1 adds the third-order Hermite terms to the
// regularised non-equilibrium part of Eq. 10 (reg_order 3).
constexpr bool eq_full(int EQ) { return (EQ & 1) != 0; }
constexpr bool reg_third(int EQ) { return (EQ & 2) != 0; }

// Equilibrium of Eq. 3 for direction i (bit 0 of EQ adds the quadratic terms).
template <class T, int EQ>
__device__ __forceinline__ T feq_dir(int i, T rho, T ux, T uy, T uz, T uu) {
    const T cu = T(cx(i)) * ux + T(cy(i)) * uy + T(cz(i)) * uz;
    // 1/T0 = 3, 1/(6 T0^3) = 1/(2 T0^2) = 9/2
    T e = T(1) + cu * (T(3) + T(4.5) * cu * cu - T(4.5) * uu);
    if (eq_full(EQ)) e += T(4.5) * cu * cu - T(1.5) * uu;
    return rho * wgt<T>(i) * e;
}

// S6-S7 for one component: writes f*_i = feq_i + w_i/(2 T0^2) H_i : A + w_i c_i.F/(2 T0)
// with A = (1 - 1/tau) Pi^neq + (1 - 1/(2 tau)) (u_F F + F u_F), plus, with the
// third-order regularisation, (1 - 1/tau) w_i times third_order_term.
// sig(i) is the reference density of the cell value i streams into.
//
// Directions come in opposite pairs (i, i+1) with c_{i+1} = -c_i: the parts of
// f*_i that are even in c (rest term of feq, the quadratic terms of Eq. 3 for
// eq_full, H_i : A) are shared, the odd parts (the c.u terms of feq, the
// first-order forcing, the third-order terms) change sign, so each pair costs
// one evaluation.
template <class T> struct CollidePrep {
    T rho, ux, uy, uz, Fx, Fy, Fz, uu, odd_k;
    T axx, ayy, azz, axy, axz, ayz, ktr;
    // relaxed third-order moments (1 - 1/tau) a3 (reg_third only)
    T bxxy, bxyy, bxxz, bxzz, byyz, byzz;
};

// Third-order part of the regularised f'_i / w_i for the odd direction i, from
// the relaxed recursive moments a3_abg = u_a Pi_bg + u_b Pi_ag + u_g Pi_ab
// (Pi = Pi^neq).  On D3Q19, H_aaa and H_xyz vanish at every velocity and the
// six other third-order Hermite polynomials alias pairwise (sum_i w_i H_xxy
// H_yzz = -T0^3); the lattice function whose moments over the six equal a3
// works out, per velocity class, to
//   face  c = s e_a:          -9 s (a_abb + a_acc)
//   edge  c = s e_a + t e_b:   9 (t a_aab + s a_abb)
// (with 1/T0^3 = 27; the same function as the general projection with the
// Gram matrix of the six polynomials).
template <class T, class V>
__device__ __forceinline__ V third_order_term(int i, V bxxy, V bxyy, V bxxz, V bxzz, V byyz, V byzz) {
    const int c0 = cx(i), c1 = cy(i), c2 = cz(i);
    if (c0 && c1) return T(9) * (T(c1) * bxxy + T(c0) * bxyy);
    if (c0 && c2) return T(9) * (T(c2) * bxxz + T(c0) * bxzz);
    if (c1 && c2) return T(9) * (T(c2) * byyz + T(c1) * byzz);
    if (c0) return T(-9 * c0) * (bxyy + bxzz);
    if (c1) return T(-9 * c1) * (bxxy + byzz);
    return T(-9 * c2) * (bxxz + byyz);
}

template <class T, int EQ>
__device__ __forceinline__ CollidePrep<T> collide_prep(const Moments<T> &m, T ux, T uy, T uz, T Fx, T Fy, T Fz,
                                                       T omega, T fcoef) {
    CollidePrep<T> c;
    const T T0 = T(1) / T(3);
    c.rho = m.rho;
    c.ux = ux, c.uy = uy, c.uz = uz, c.Fx = Fx, c.Fy = Fy, c.Fz = Fz;
    c.uu = ux * ux + uy * uy + uz * uz;
    // Pi^neq = Pi - Pi^eq with Pi^eq = rho T0 I (+ rho u u for EQ = 1)
    T nxx = m.pxx - m.rd * T0, nyy = m.pyy - m.rd * T0, nzz = m.pzz - m.rd * T0;
    T nxy = m.pxy, nxz = m.pxz, nyz = m.pyz;
    if (eq_full(EQ)) {
        nxx -= m.rho * ux * ux; nyy -= m.rho * uy * uy; nzz -= m.rho * uz * uz;
        nxy -= m.rho * ux * uy; nxz -= m.rho * ux * uz; nyz -= m.rho * uy * uz;
    }
    if (reg_third(EQ)) {
        c.bxxy = omega * (T(2) * ux * nxy + uy * nxx);
        c.bxyy = omega * (T(2) * uy * nxy + ux * nyy);
        c.bxxz = omega * (T(2) * ux * nxz + uz * nxx);
        c.bxzz = omega * (T(2) * uz * nxz + ux * nzz);
        c.byyz = omega * (T(2) * uy * nyz + uz * nyy);
        c.byzz = omega * (T(2) * uz * nyz + uy * nzz);
    }
    c.axx = omega * nxx + fcoef * (T(2) * ux * Fx);
    c.ayy = omega * nyy + fcoef * (T(2) * uy * Fy);
    c.azz = omega * nzz + fcoef * (T(2) * uz * Fz);
    c.axy = omega * nxy + fcoef * (ux * Fy + uy * Fx);
    c.axz = omega * nxz + fcoef * (ux * Fz + uz * Fx);
    c.ayz = omega * nyz + fcoef * (uy * Fz + uz * Fy);
    c.ktr = -T(1.5) * (c.axx + c.ayy + c.azz);  // -(T0/(2 T0^2)) tr A
    c.odd_k = T(3) - T(4.5) * c.uu;
    return c;
}

// Stored value of f*_0 (c = 0): its deviation f*_0 - w_0 R from the rest
// equilibrium of the reference density R of the cell it streams into (R = 0
// in the unshifted format).  Forming rho - R first keeps FP32 from cancelling
// two O(w rho) numbers.
template <class T, int EQ> __device__ __forceinline__ T collide_rest(const CollidePrep<T> &c, T R) {
    T e = c.rho - R;
    if (eq_full(EQ)) e = (c.rho - R) - T(1.5) * c.rho * c.uu;
    return wgt<T>(0) * (e + c.ktr);
}

// Stored values of f*_i and f*_{i+1} for the opposite pair (i, i+1), i odd,
// with reference densities Ri, Ro (see collide_rest).
template <class T, int EQ>
__device__ __forceinline__ void collide_pair(const CollidePrep<T> &c, int i, T Ri, T Ro, T &vi, T &vo) {
    const T c0 = T(cx(i)), c1 = T(cy(i)), c2 = T(cz(i));
    const T cu = c0 * c.ux + c1 * c.uy + c2 * c.uz;
    const T cAc = c0 * c0 * c.axx + c1 * c1 * c.ayy + c2 * c2 * c.azz +
                  T(2) * (c0 * c1 * c.axy + c0 * c2 * c.axz + c1 * c2 * c.ayz);
    const T cF = c0 * c.Fx + c1 * c.Fy + c2 * c.Fz;
    // w_i x (even part without the rest term, odd part) of f*_i
    T even = T(4.5) * cAc + c.ktr;
    if (eq_full(EQ)) even += c.rho * (T(4.5) * cu * cu - T(1.5) * c.uu);
    T odd = c.rho * cu * (c.odd_k + T(4.5) * cu * cu) + T(1.5) * cF;
    if (reg_third(EQ)) odd += third_order_term<T, T>(i, c.bxxy, c.bxyy, c.bxxz, c.bxzz, c.byyz, c.byzz);
    const T w = wgt<T>(i);
    vi = w * (((c.rho - Ri) + even) + odd);
    vo = w * (((c.rho - Ro) + even) - odd);
}

template <class S, int EQ, class Sig>
__device__ __forceinline__ void collide_store(S *__restrict__ fout, long long n, int self,
                                              const Moments<typename Storage<S>::T> &m,
                                              typename Storage<S>::T ux, typename Storage<S>::T uy,
                                              typename Storage<S>::T uz, typename Storage<S>::T Fx,
                                              typename Storage<S>::T Fy, typename Storage<S>::T Fz,
                                              typename Storage<S>::T omega, typename Storage<S>::T fcoef,
                                              const Sig &sig) {
    using T = typename Storage<S>::T;
    const CollidePrep<T> c = collide_prep<T, EQ>(m, ux, uy, uz, Fx, Fy, Fz, omega, fcoef);
    auto ref = [&](int i) -> T { return Storage<S>::shifted ? sig(i) : T(0); };
    Storage<S>::store_d(fout + (uint32_t)self, collide_rest<T, EQ>(c, ref(0)));
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
        T vi, vo;
        collide_pair<T, EQ>(c, i, ref(i), ref(i + 1), vi, vo);
        Storage<S>::store_d(fout + ((uint32_t)i * (uint32_t)n + (uint32_t)self), vi);
        Storage<S>::store_d(fout + ((uint32_t)(i + 1) * (uint32_t)n + (uint32_t)self), vo);
    }
}

template <class S, int EQ, class Sig>
__device__ __forceinline__ void store_equilibrium(S *__restrict__ fout, long long n, int self,
                                                  typename Storage<S>::T rho, typename Storage<S>::T ux,
                                                  typename Storage<S>::T uy, typename Storage<S>::T uz,
                                                  const Sig &sig) {
    using T = typename Storage<S>::T;
    const T uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < kQ; ++i)
        Storage<S>::store(fout + ((uint32_t)i * (uint32_t)n + (uint32_t)self), feq_dir<T, EQ>(i, rho, ux, uy, uz, uu),
                          Storage<S>::shifted ? wgt<T>(i) * sig(i) : T(0));
}

// S4: forces on both components from the pseudo-potential of the 18
// neighbours (psi_nb[beta] read through `psi_at`), the SOLID-neighbour bits
// and the body force.  Force-stencil weights are 2 w_i.
template <class T> struct Forces {
    T F[2][3];
};

// Bulk sums s[beta][axis] = sum_i ws_i c_i psi_beta(x + c_i) over the non-SOLID
// neighbours, accumulated one neighbour at a time (i = 1..18 in order).
template <class T> struct ForceSums {
    T s[2][3];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) s[b][a] = T(0);
    }
    __device__ __forceinline__ void add(int i, bool solid, T p0, T p1) {
        p0 = solid ? T(0) : p0;
        p1 = solid ? T(0) : p1;
        const T ws = T(2) * wgt<T>(i);
        if (cx(i)) { s[0][0] += T(cx(i)) * ws * p0; s[1][0] += T(cx(i)) * ws * p1; }
        if (cy(i)) { s[0][1] += T(cy(i)) * ws * p0; s[1][1] += T(cy(i)) * ws * p1; }
        if (cz(i)) { s[0][2] += T(cz(i)) * ws * p0; s[1][2] += T(cz(i)) * ws * p1; }
    }
};

// S4 from the bulk sums: F^alpha = G rho_alpha sum ws c psi_beta (beta != alpha),
// the wall part of Eq. 11 for the SOLID neighbours, and the body force.
template <class T>
__device__ __forceinline__ Forces<T> sc_forces_finish(const ForceSums<T> &bs, uint32_t links, T rho0, T rho1,
                                                      const InstParam<T> &p, int wall_model) {
    const T(&s)[2][3] = bs.s;
    Forces<T> out;
    const T r[2] = {rho0, rho1};
    // bulk part: F^alpha = G rho_alpha sum ws c psi_beta, beta != alpha
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out.F[0][a] = p.G * r[0] * s[1][a];
        out.F[1][a] = p.G * r[1] * s[0][a];
    }
    const uint32_t wl = links & 0x7FFFEu;
    if (wl) {
        // wall part (Eq. 11): psi_beta(SOLID) = rho^s_beta (models 0, 1), the
        // cell's own rho_beta plus rho^s_beta (model 2), or the cell's own
        // rho_beta with the wall potential's part added balanced (model 3)
        T d[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            if ((links >> i) & 1u) {
                const T ws = T(2) * wgt<T>(i);
                d[0] += T(cx(i)) * ws;
                d[1] += T(cy(i)) * ws;
                d[2] += T(cz(i)) * ws;
            }
        }
        T fw[2][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T w1 = wall_model == 2 ? r[1] + p.rs[1] : wall_model == 3 ? r[1] : p.rs[1];
            const T w0 = wall_model == 2 ? r[0] + p.rs[0] : wall_model == 3 ? r[0] : p.rs[0];
            fw[0][a] = p.G * r[0] * (w1 * d[a]);
            fw[1][a] = p.G * r[1] * (w0 * d[a]);
        }
        if (wall_model == 0) {
            const T rho = r[0] + r[1];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T net = fw[0][a] + fw[1][a];
                fw[0][a] -= r[0] / rho * net;
                fw[1][a] -= r[1] / rho * net;
            }
        } else if (wall_model == 3) {
            const T rho = r[0] + r[1];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T fs0 = p.G * r[0] * (p.rs[1] * d[a]);
                const T fs1 = p.G * r[1] * (p.rs[0] * d[a]);
                const T net = fs0 + fs1;
                fw[0][a] += fs0 - r[0] / rho * net;
                fw[1][a] += fs1 - r[1] / rho * net;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out.F[0][a] += fw[0][a];
            out.F[1][a] += fw[1][a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out.F[0][a] += r[0] * p.g[a];
        out.F[1][a] += r[1] * p.g[a];
    }
    return out;
}

template <class T, class PsiAt>
__device__ __forceinline__ Forces<T> sc_forces(const PsiAt &psi_at, uint32_t links, T rho0, T rho1,
                                               const InstParam<T> &p, int wall_model) {
    ForceSums<T> bs;
    bs.clear();
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        T p0, p1;
        psi_at(i, p0, p1);
        bs.add(i, (links >> i) & 1u, p0, p1);
    }
    return sc_forces_finish<T>(bs, links, rho0, rho1, p, wall_model);
}

// S5: tau_mix from the density-weighted viscosity, p = rho_1 / rho in [0, 1].
template <class T> __device__ __forceinline__ T tau_mix(T rho0, T rho1, const InstParam<T> &p) {
    T q = rho0 * (T(1) / (rho0 + rho1));
    q = q < T(0) ? T(0) : (q > T(1) ? T(1) : q);
    const T nu = q * p.nu[0] + (T(1) - q) * p.nu[1];
    return T(3) * nu + T(0.5);
}

// S5 for the cell: u_F = (j + F_tot / 2) / rho (Eq. 8) and the relaxation
// factors 1 - 1/tau and 1 - 1/(2 tau) of the collision (one reciprocal each).
template <class T> struct Relax {
    T ux, uy, uz, omega, fcoef;
};
template <class T>
__device__ __forceinline__ Relax<T> relax(const Moments<T> &m0, const Moments<T> &m1, const Forces<T> &F,
                                          const InstParam<T> &p) {
    const T inv = T(1) / (m0.rho + m1.rho);
    Relax<T> r;
    r.ux = (m0.jx + m1.jx + T(0.5) * (F.F[0][0] + F.F[1][0])) * inv;
    r.uy = (m0.jy + m1.jy + T(0.5) * (F.F[0][1] + F.F[1][1])) * inv;
    r.uz = (m0.jz + m1.jz + T(0.5) * (F.F[0][2] + F.F[1][2])) * inv;
    const T itau = T(1) / tau_mix<T>(m0.rho, m1.rho, p);
    r.omega = T(1) - itau;
    r.fcoef = T(1) - T(0.5) * itau;
    return r;
}

}  // namespace lbm
