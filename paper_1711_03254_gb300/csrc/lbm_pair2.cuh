// The update of Sec. 2 with both components as packed FP32 pairs
// (x = component 1, y = component 2 of the paper; alpha = 0, 1 here).
//
// Every step from the moments to the stored values applies the same formula
// to the two components, so it runs on the FP32x2 add / mul / fma of sm_100
// and later: one instruction for both components, each lane rounded exactly
// as the scalar FP32 operation.  Terms whose lattice coefficient c_i is zero
// are dropped at compile time.  Used by the compact update for the FP32 and
// 16-bit storages (FP32 arithmetic); the FP64 path keeps the scalar code of
// lbm_device.cuh.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b: b * (-1) is exact, so the single rounding is that of the subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// (component 1, component 0): the partner component of each lane
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

// ---------------------------------------------------------------- moments (S1-S2)
// Moments of both components from the 19 stored pairs v, in storage units
// (the FP16 storage holds deviations times 2^12).  `unscale` takes a sum back
// to FP32 units; it is a power of two, so scaling the sums equals scaling each
// value.  R is the pair of reference densities of the cell (shifted storage:
// rho = R + sum d, see Moments).  Summation order as moments_of.
struct Moments2 {
    float2 rho, rd, jx, jy, jz;
    float2 pxx, pyy, pzz, pxy, pxz, pyz;
};

template <bool SCALED>
__device__ __forceinline__ Moments2 moments2(const float2 (&v)[kQ], float2 R, float unscale) {
    Moments2 m;
    float2 r = v[0];
#pragma unroll
    for (int i = 1; i < kQ; ++i) r = add2(r, v[i]);
    m.rd = r;
    m.jx = add2(add2(add2(add2(sub2(v[1], v[2]), sub2(v[7], v[8])), sub2(v[9], v[10])), sub2(v[11], v[12])),
                sub2(v[13], v[14]));
    m.jy = add2(add2(add2(add2(sub2(v[3], v[4]), sub2(v[7], v[8])), sub2(v[10], v[9])), sub2(v[15], v[16])),
                sub2(v[17], v[18]));
    m.jz = add2(add2(add2(add2(sub2(v[5], v[6]), sub2(v[11], v[12])), sub2(v[14], v[13])), sub2(v[15], v[16])),
                sub2(v[18], v[17]));
    const float2 s78 = add2(v[7], v[8]), s910 = add2(v[9], v[10]);
    const float2 s1112 = add2(v[11], v[12]), s1314 = add2(v[13], v[14]);
    const float2 s1516 = add2(v[15], v[16]), s1718 = add2(v[17], v[18]);
    const float2 e_xy = add2(s78, s910), e_xz = add2(s1112, s1314), e_yz = add2(s1516, s1718);
    m.pxx = add2(add2(add2(v[1], v[2]), e_xy), e_xz);
    m.pyy = add2(add2(add2(v[3], v[4]), e_xy), e_yz);
    m.pzz = add2(add2(add2(v[5], v[6]), e_xz), e_yz);
    m.pxy = sub2(s78, s910);
    m.pxz = sub2(s1112, s1314);
    m.pyz = sub2(s1516, s1718);
    if (SCALED) {
        const float2 s = bc2(unscale);
        m.rd = mul2(m.rd, s);
        m.jx = mul2(m.jx, s), m.jy = mul2(m.jy, s), m.jz = mul2(m.jz, s);
        m.pxx = mul2(m.pxx, s), m.pyy = mul2(m.pyy, s), m.pzz = mul2(m.pzz, s);
        m.pxy = mul2(m.pxy, s), m.pxz = mul2(m.pxz, s), m.pyz = mul2(m.pyz, s);
    }
    m.rho = add2(R, m.rd);
    return m;
}

// Density pair only (the pseudo-potential pass), same summation order.
template <bool SCALED>
__device__ __forceinline__ float2 density2(const float2 (&v)[kQ], float2 R, float unscale) {
    float2 r = v[0];
#pragma unroll
    for (int i = 1; i < kQ; ++i) r = add2(r, v[i]);
    if (SCALED) r = mul2(r, bc2(unscale));
    return add2(R, r);
}

// ---------------------------------------------------------------- forces (S4)
// Sums sum_i ws_i c_i psi(x + c_i) for both components, over all 18
// neighbours.  At a SOLID neighbour the caller passes the cell's own psi pair
// (its densities: the same sum of the same pulled values).  For wall models 2
// and 3 those terms are the wall's neutral part (a SOLID neighbour carries
// the cell's own rho_beta); for models 0 and 1 forces2 removes them again
// (psi_own * sum over the SOLID directions of ws_i c_i), which leaves the bulk
// sum over the non-SOLID neighbours of Eq. 10 without a select per direction.
struct ForceSums2 {
    float2 x, y, z;
    __device__ __forceinline__ void clear() { x = y = z = bc2(0.f); }
    __device__ __forceinline__ void add(int i, float2 q) {
        const float ws = 2.f * wgt<float>(i);
        if (cx(i)) x = fma2(q, bc2(float(cx(i)) * ws), x);
        if (cy(i)) y = fma2(q, bc2(float(cy(i)) * ws), y);
        if (cz(i)) z = fma2(q, bc2(float(cz(i)) * ws), z);
    }
};

struct Forces2 {
    float2 x, y, z;  // total force on (component 0, component 1) per axis
};

// S4 from the sums: bulk part G rho_alpha sum ws c psi_beta (beta != alpha),
// the wall part of Eq. 11 at SOLID neighbours (models 0 to 3 as
// sc_forces_finish) and the body force rho_alpha g.  psi_own is read for
// models 0 and 1 only.
__device__ __forceinline__ Forces2 forces2(ForceSums2 s, float2 psi_own, uint32_t links, float2 rho,
                                           const InstParam<float> &p, int wall_model) {
    const float2 grho = mul2(bc2(p.G), rho);
    Forces2 F;
    const uint32_t wl = links & 0x7FFFEu;
    if (wl) {
        float d[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            if ((links >> i) & 1u) {
                const float ws = 2.f * wgt<float>(i);
                if (cx(i)) d[0] += float(cx(i)) * ws;
                if (cy(i)) d[1] += float(cy(i)) * ws;
                if (cz(i)) d[2] += float(cz(i)) * ws;
            }
        }
        if (wall_model < 2) {
            // the sums ran over the SOLID neighbours with the cell's own psi
            s.x = fma2(psi_own, bc2(-d[0]), s.x);
            s.y = fma2(psi_own, bc2(-d[1]), s.y);
            s.z = fma2(psi_own, bc2(-d[2]), s.z);
        }
        F.x = mul2(grho, swap2(s.x));
        F.y = mul2(grho, swap2(s.y));
        F.z = mul2(grho, swap2(s.z));
        // the wall potential's part G rho_alpha rho^s_beta d, balanced between
        // the components for models 0 and 3 (the net wall force is shared by
        // density); models 2 and 3 carry the neutral part in the sums already
        const float2 rsw = swap2(make_float2(p.rs[0], p.rs[1]));
        float2 fw[3] = {mul2(grho, mul2(rsw, bc2(d[0]))), mul2(grho, mul2(rsw, bc2(d[1]))),
                        mul2(grho, mul2(rsw, bc2(d[2])))};
        if (wall_model == 0 || wall_model == 3) {
            const float rt = rho.x + rho.y;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float net = fw[a].x + fw[a].y;
                fw[a].x -= rho.x / rt * net;
                fw[a].y -= rho.y / rt * net;
            }
        }
        F.x = add2(F.x, fw[0]);
        F.y = add2(F.y, fw[1]);
        F.z = add2(F.z, fw[2]);
    } else {
        F.x = mul2(grho, swap2(s.x));
        F.y = mul2(grho, swap2(s.y));
        F.z = mul2(grho, swap2(s.z));
    }
    F.x = fma2(rho, bc2(p.g[0]), F.x);
    F.y = fma2(rho, bc2(p.g[1]), F.y);
    F.z = fma2(rho, bc2(p.g[2]), F.z);
    return F;
}

// S5: u_F of Eq. 8 and the relaxation factors (as relax()).
__device__ __forceinline__ Relax<float> relax2(const Moments2 &m, const Forces2 &F, const InstParam<float> &p) {
    const float inv = 1.f / (m.rho.x + m.rho.y);
    Relax<float> r;
    r.ux = (m.jx.x + m.jx.y + 0.5f * (F.x.x + F.x.y)) * inv;
    r.uy = (m.jy.x + m.jy.y + 0.5f * (F.y.x + F.y.y)) * inv;
    r.uz = (m.jz.x + m.jz.y + 0.5f * (F.z.x + F.z.y)) * inv;
    const float itau = 1.f / tau_mix<float>(m.rho.x, m.rho.y, p);
    r.omega = 1.f - itau;
    r.fcoef = 1.f - 0.5f * itau;
    return r;
}

// ---------------------------------------------------------------- collision (S6-S7)
// As CollidePrep / collide_rest / collide_pair, for both components at once.
// The velocity terms (u_F is shared by the components) stay scalar.
struct Prep2 {
    float2 rho, Fx, Fy, Fz;
    float2 axx, ayy, azz, axy, axz, ayz, ktr;
    float2 bxxy, bxyy, bxxz, bxzz, byyz, byzz;  // reg_third only (as CollidePrep)
    float ux, uy, uz, uu, odd_k;
};

template <int EQ>
__device__ __forceinline__ Prep2 prep2(const Moments2 &m, const Relax<float> &R, const Forces2 &F) {
    Prep2 c;
    const float T0 = 1.f / 3.f;
    const float ux = R.ux, uy = R.uy, uz = R.uz;
    c.rho = m.rho;
    c.Fx = F.x, c.Fy = F.y, c.Fz = F.z;
    c.ux = ux, c.uy = uy, c.uz = uz;
    c.uu = ux * ux + uy * uy + uz * uz;
    // Pi^neq = Pi - rho T0 I (- rho u u for EQ = 1)
    const float2 mT0 = bc2(-T0);
    float2 nxx = fma2(m.rd, mT0, m.pxx), nyy = fma2(m.rd, mT0, m.pyy), nzz = fma2(m.rd, mT0, m.pzz);
    float2 nxy = m.pxy, nxz = m.pxz, nyz = m.pyz;
    if (eq_full(EQ)) {
        const float2 rx = mul2(m.rho, bc2(ux)), ry = mul2(m.rho, bc2(uy)), rz = mul2(m.rho, bc2(uz));
        nxx = fma2(rx, bc2(-ux), nxx);
        nyy = fma2(ry, bc2(-uy), nyy);
        nzz = fma2(rz, bc2(-uz), nzz);
        nxy = fma2(rx, bc2(-uy), nxy);
        nxz = fma2(rx, bc2(-uz), nxz);
        nyz = fma2(ry, bc2(-uz), nyz);
    }
    // A = omega Pi^neq + fcoef (u_F F + F u_F)
    const float2 om = bc2(R.omega), fc = bc2(R.fcoef);
    if (reg_third(EQ)) {
        // omega (2 u_a Pi_ab + u_b Pi_aa) and so on (third_order_term)
        c.bxxy = mul2(om, fma2(bc2(2.f * ux), nxy, mul2(bc2(uy), nxx)));
        c.bxyy = mul2(om, fma2(bc2(2.f * uy), nxy, mul2(bc2(ux), nyy)));
        c.bxxz = mul2(om, fma2(bc2(2.f * ux), nxz, mul2(bc2(uz), nxx)));
        c.bxzz = mul2(om, fma2(bc2(2.f * uz), nxz, mul2(bc2(ux), nzz)));
        c.byyz = mul2(om, fma2(bc2(2.f * uy), nyz, mul2(bc2(uz), nyy)));
        c.byzz = mul2(om, fma2(bc2(2.f * uz), nyz, mul2(bc2(uy), nzz)));
    }
    c.axx = fma2(om, nxx, mul2(fc, mul2(bc2(2.f * ux), F.x)));
    c.ayy = fma2(om, nyy, mul2(fc, mul2(bc2(2.f * uy), F.y)));
    c.azz = fma2(om, nzz, mul2(fc, mul2(bc2(2.f * uz), F.z)));
    c.axy = fma2(om, nxy, mul2(fc, fma2(bc2(ux), F.y, mul2(bc2(uy), F.x))));
    c.axz = fma2(om, nxz, mul2(fc, fma2(bc2(ux), F.z, mul2(bc2(uz), F.x))));
    c.ayz = fma2(om, nyz, mul2(fc, fma2(bc2(uy), F.z, mul2(bc2(uz), F.y))));
    c.ktr = mul2(bc2(-1.5f), add2(add2(c.axx, c.ayy), c.azz));  // -(T0/(2 T0^2)) tr A
    c.odd_k = 3.f - 4.5f * c.uu;
    return c;
}

// Stored pair of f*_0 (deviation from w_0 R, R the pair of reference
// densities of the cell it streams into), times `scale`.
template <int EQ> __device__ __forceinline__ float2 rest2(const Prep2 &c, float2 R, float scale) {
    float2 e = sub2(c.rho, R);
    if (eq_full(EQ)) e = fma2(mul2(bc2(-1.5f), c.rho), bc2(c.uu), e);
    return mul2(bc2(wgt<float>(0) * scale), add2(e, c.ktr));
}

// third_order_term of lbm_device.cuh on pairs
__device__ __forceinline__ float2 third_order_pair(int i, const Prep2 &c) {
    const int c0 = cx(i), c1 = cy(i), c2 = cz(i);
    if (c0 && c1) return fma2(bc2(9.f * c1), c.bxxy, mul2(bc2(9.f * c0), c.bxyy));
    if (c0 && c2) return fma2(bc2(9.f * c2), c.bxxz, mul2(bc2(9.f * c0), c.bxzz));
    if (c1 && c2) return fma2(bc2(9.f * c2), c.byyz, mul2(bc2(9.f * c1), c.byzz));
    if (c0) return mul2(bc2(-9.f * c0), add2(c.bxyy, c.bxzz));
    if (c1) return mul2(bc2(-9.f * c1), add2(c.bxxy, c.byzz));
    return mul2(bc2(-9.f * c2), add2(c.bxxz, c.byyz));
}

// Stored pairs of f*_i and f*_{i+1} (i odd, c_{i+1} = -c_i), times `scale`,
// with reference pairs Ri, Ro: the even part is shared, the odd part changes
// sign.  Every odd i has a positive first non-zero component of c_i.
template <int EQ>
__device__ __forceinline__ void pair2(const Prep2 &c, int i, float2 Ri, float2 Ro, float scale, float2 &vi,
                                      float2 &vo) {
    const int c0 = cx(i), c1 = cy(i), c2 = cz(i);
    // c.u (scalar) and c.F, c.A.c (pairs) over the non-zero components only
    float cu = 0.f;
    if (c0) cu = float(c0) * c.ux;
    if (c1) cu = c0 ? cu + float(c1) * c.uy : float(c1) * c.uy;
    if (c2) cu = (c0 || c1) ? cu + float(c2) * c.uz : float(c2) * c.uz;
    float2 cF, cAc;
    if (c0) {
        cF = c.Fx;
        cAc = c.axx;
        if (c1) {
            cF = c1 > 0 ? add2(cF, c.Fy) : sub2(cF, c.Fy);
            cAc = fma2(bc2(float(2 * c0 * c1)), c.axy, add2(cAc, c.ayy));
        } else if (c2) {
            cF = c2 > 0 ? add2(cF, c.Fz) : sub2(cF, c.Fz);
            cAc = fma2(bc2(float(2 * c0 * c2)), c.axz, add2(cAc, c.azz));
        }
    } else if (c1) {
        cF = c.Fy;
        cAc = c.ayy;
        if (c2) {
            cF = c2 > 0 ? add2(cF, c.Fz) : sub2(cF, c.Fz);
            cAc = fma2(bc2(float(2 * c1 * c2)), c.ayz, add2(cAc, c.azz));
        }
    } else {
        cF = c.Fz;
        cAc = c.azz;
    }
    float2 even = fma2(bc2(4.5f), cAc, c.ktr);
    if (eq_full(EQ)) even = fma2(c.rho, bc2(4.5f * cu * cu - 1.5f * c.uu), even);
    float2 odd = fma2(c.rho, bc2(cu * (c.odd_k + 4.5f * cu * cu)), mul2(bc2(1.5f), cF));
    if (reg_third(EQ)) odd = add2(odd, third_order_pair(i, c));
    const float2 w = bc2(wgt<float>(i) * scale);
    vi = mul2(w, add2(add2(sub2(c.rho, Ri), even), odd));
    vo = mul2(w, sub2(add2(sub2(c.rho, Ro), even), odd));
}

}  // namespace lbm
