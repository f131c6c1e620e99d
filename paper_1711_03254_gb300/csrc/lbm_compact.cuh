// Pieces of the compact-layout update shared by its kernels (lbm_compact.cu:
// the two-pass update; lbm_fusedc.cu: the single-read fused update).
//
// Only the non-solid cells of an instance are stored, in cell order (x
// fastest); the compact index k of a cell is the number of non-solid cells
// before it.  The two components of a value are stored side by side, so one
// 4-byte (FP16/BF16), 8-byte (FP32) or 16-byte (FP64) access moves both.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_pair2.cuh"

namespace lbm {

// Both components of one stored value.
template <class S> struct Pair;
template <> struct Pair<double> {
    using P = double2;
    __device__ static __forceinline__ void load(const P *p, double &a, double &b) {
        const P v = __ldg(p);
        a = v.x;
        b = v.y;
    }
    __device__ static __forceinline__ void load_cg(const P *p, double &a, double &b) {
        const P v = __ldcg(p);
        a = v.x;
        b = v.y;
    }
    __device__ static __forceinline__ void store(P *p, double a, double b, double, double) { *p = make_double2(a, b); }
    __device__ static __forceinline__ void store_d(P *p, double a, double b) { *p = make_double2(a, b); }
    __device__ static __forceinline__ void load_shared(const P *p, double &a, double &b) {
        const P v = *p;
        a = v.x;
        b = v.y;
    }
};
template <> struct Pair<float> {
    using P = float2;
    __device__ static __forceinline__ void load(const P *p, float &a, float &b) {
        const P v = __ldg(p);
        a = v.x + 0.f;  // as Storage<float>::load with a zero shift
        b = v.y + 0.f;
    }
    __device__ static __forceinline__ void store(P *p, float a, float b, float sa, float sb) {
        *p = make_float2(a - sa, b - sb);
    }
    __device__ static __forceinline__ void store_d(P *p, float a, float b) { *p = make_float2(a, b); }
    __device__ static __forceinline__ void load_shared(const P *p, float &a, float &b) {
        const P v = *p;
        a = v.x + 0.f;
        b = v.y + 0.f;
    }
};
template <> struct Pair<__half> {  // values scaled as in Storage<__half>
    using P = __half2;
    __device__ static __forceinline__ void load(const P *p, float &a, float &b) {
        const float2 v = __half22float2(__ldg(p));
        a = v.x * kF16Unscale + 0.f;
        b = v.y * kF16Unscale + 0.f;
    }
    __device__ static __forceinline__ void store(P *p, float a, float b, float sa, float sb) {
        *p = __floats2half2_rn((a - sa) * kF16Scale, (b - sb) * kF16Scale);
    }
    __device__ static __forceinline__ void store_d(P *p, float a, float b) {
        *p = __floats2half2_rn(a * kF16Scale, b * kF16Scale);
    }
    __device__ static __forceinline__ void load_shared(const P *p, float &a, float &b) {
        const float2 v = __half22float2(*p);
        a = v.x * kF16Unscale + 0.f;
        b = v.y * kF16Unscale + 0.f;
    }
};
template <> struct Pair<__nv_bfloat16> {
    using P = __nv_bfloat162;
    __device__ static __forceinline__ void load(const P *p, float &a, float &b) {
        const float2 v = __bfloat1622float2(__ldg(p));
        a = v.x + 0.f;
        b = v.y + 0.f;
    }
    __device__ static __forceinline__ void store(P *p, float a, float b, float sa, float sb) {
        *p = __floats2bfloat162_rn(a - sa, b - sb);
    }
    __device__ static __forceinline__ void store_d(P *p, float a, float b) { *p = __floats2bfloat162_rn(a, b); }
    __device__ static __forceinline__ void load_shared(const P *p, float &a, float &b) {
        const float2 v = __bfloat1622float2(*p);
        a = v.x + 0.f;
        b = v.y + 0.f;
    }
};

template <class T> struct Vec2;
template <> struct Vec2<double> { using V = double2; };
template <> struct Vec2<float> { using V = float2; };

// Both components of a stored value as one FP32 pair in storage units, for
// the packed-pair arithmetic (FP32 and 16-bit storages).  kUnscale takes a
// sum of stored values to FP32 units and kScale a result back (2^-12 and 2^12
// for the scaled FP16 deviations, exact powers of two).
template <class S> struct Pair2;
template <> struct Pair2<float> {
    using P = float2;
    static constexpr bool kScaled = false;
    static constexpr float kUnscale = 1.f, kScale = 1.f;
    __device__ static __forceinline__ float2 load(const P *p) { return __ldg(p); }
    __device__ static __forceinline__ float2 load_cg(const P *p) { return __ldcg(p); }
    __device__ static __forceinline__ float2 load_shared(const P *p) { return *p; }
    __device__ static __forceinline__ void store(P *p, float2 v) { *p = v; }
};
template <> struct Pair2<__half> {
    using P = __half2;
    static constexpr bool kScaled = true;
    static constexpr float kUnscale = kF16Unscale, kScale = kF16Scale;
    __device__ static __forceinline__ float2 load(const P *p) { return __half22float2(__ldg(p)); }
    __device__ static __forceinline__ float2 load_cg(const P *p) { return __half22float2(__ldcg(p)); }
    __device__ static __forceinline__ float2 load_shared(const P *p) { return __half22float2(*p); }
    __device__ static __forceinline__ void store(P *p, float2 v) { *p = __float22half2_rn(v); }
};
template <> struct Pair2<__nv_bfloat16> {
    using P = __nv_bfloat162;
    static constexpr bool kScaled = false;
    static constexpr float kUnscale = 1.f, kScale = 1.f;
    __device__ static __forceinline__ float2 load(const P *p) { return __bfloat1622float2(__ldg(p)); }
    __device__ static __forceinline__ float2 load_cg(const P *p) { return __bfloat1622float2(__ldcg(p)); }
    __device__ static __forceinline__ float2 load_shared(const P *p) { return __bfloat1622float2(*p); }
    __device__ static __forceinline__ void store(P *p, float2 v) { *p = __float22bfloat162_rn(v); }
};
// FP32 arithmetic (packed pairs) for every storage but FP64
template <class S> constexpr bool packed_pairs() { return sizeof(S) < 8; }

struct CompactCell {
    int x, y, z;
    uint32_t word;
};

// cell from its packed coordinates p and geometry word
__device__ __forceinline__ CompactCell unpack_cell(uint32_t p, uint32_t word) {
    CompactCell c;
    c.x = (int)(p & 2047u);
    c.y = (int)((p >> 11) & 2047u);
    c.z = (int)(p >> 22);
    c.word = word;
    return c;
}

__device__ __forceinline__ CompactCell compact_cell(const StepArgs &a, int b, uint32_t k) {
    return unpack_cell(__ldg(a.cxyz + (size_t)b * a.kmax + k), __ldg(a.clink + (size_t)b * a.kmax + k));
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

// Pull the 19 stored pairs of the cell with compact index sk (neighbours nb,
// geometry word sw) into v0, v1 (bounce-back from SOLID neighbours).
template <class S, bool COH = false>
__device__ __forceinline__ void pull_pairs(const typename Pair<S>::P *__restrict__ f, uint32_t n, uint32_t sk,
                                           const CNbr &nb, uint32_t sw, typename Storage<S>::T (&v0)[kQ],
                                           typename Storage<S>::T (&v1)[kQ]) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const bool bb = (sw >> opp(i)) & 1u;
        const uint32_t idx = bb ? (uint32_t)opp(i) * n + sk : (uint32_t)i * n + nb.src(i);
        if constexpr (COH)
            Pair<S>::load_cg(f + idx, v0[i], v1[i]);
        else
            Pair<S>::load(f + idx, v0[i], v1[i]);
    }
}

template <class S>
__device__ __forceinline__ void ref_pair(const StepArgs &a, int b, uint32_t sk, typename Storage<S>::T &r0,
                                         typename Storage<S>::T &r1) {
    r0 = r1 = typename Storage<S>::T(0);
    if constexpr (Storage<S>::shifted) {
        const __half2 r = __ldg((const __half2 *)a.ref_in + (size_t)b * a.kmax + sk);
        r0 = __low2float(r);
        r1 = __high2float(r);
    }
}

// Loads of data written earlier in the same launch (the persistent update)
// go through L2 (COH = true): the read-only L1 path could still hold the
// lines of two updates before.
template <bool COH, class T> __device__ __forceinline__ T ld_data(const T *p) { return COH ? __ldcg(p) : __ldg(p); }

// pull_pairs for the packed-pair path: the 19 stored pairs in storage units.
template <class S, bool COH = false>
__device__ __forceinline__ void pull_pairs2(const typename Pair2<S>::P *__restrict__ f, uint32_t n, uint32_t sk,
                                            const CNbr &nb, uint32_t sw, float2 (&v)[kQ]) {
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const bool bb = (sw >> opp(i)) & 1u;
        const uint32_t idx = bb ? (uint32_t)opp(i) * n + sk : (uint32_t)i * n + nb.src(i);
        v[i] = COH ? Pair2<S>::load_cg(f + idx) : Pair2<S>::load(f + idx);
    }
}

template <bool COH = false> __device__ __forceinline__ float2 ref_pair2(const StepArgs &a, int b, uint32_t sk) {
    return __half22float2(ld_data<COH>((const __half2 *)a.ref_in + (size_t)b * a.kmax + sk));
}

// Wall slip of the pulled pairs v of cell sk (the compact form of
// slip_values): each edge direction whose source is SOLID gets (1 - s) times
// the bounced-back pair plus s times the specular reflection, in storage
// units.  The reflected pair is stored against its source cell's reference
// pair; it is moved to this cell's with both entries of the instance's
// reference table `ref` (FP32 and 16-bit storages all hold deviations).
template <class S, bool COH = false>
__device__ __forceinline__ void slip_pairs2(const typename Pair2<S>::P *__restrict__ f, uint32_t n, uint32_t sk,
                                            const CNbr &nb, uint32_t sw, float s, const __half2 *__restrict__ ref,
                                            float2 (&v)[kQ]) {
    if (s == 0.f) return;
    const float2 rown = __half22float2(ld_data<COH>(ref + sk));
    const float2 sv = bc2(s), kv = bc2(1.f - s);
#pragma unroll
    for (int i = 7; i < kQ; ++i) {
        int via, j;
        if (!((sw >> opp(i)) & 1u) || !specular_source(i, sw, via, j)) continue;
        const uint32_t src = nb.dst(via);
        float2 r = COH ? Pair2<S>::load_cg(f + ((size_t)j * n + src)) : Pair2<S>::load(f + ((size_t)j * n + src));
        r = fma2(sub2(__half22float2(ld_data<COH>(ref + src)), rown), bc2(wgt<float>(i) * Pair2<S>::kScale), r);
        v[i] = fma2(sv, r, mul2(kv, v[i]));
    }
}

// slip_pairs2 for the FP64 pairs (no reference densities).
template <class S>
__device__ __forceinline__ void slip_pairs(const typename Pair<S>::P *__restrict__ f, uint32_t n, const CNbr &nb,
                                           uint32_t sw, typename Storage<S>::T s, typename Storage<S>::T (&v0)[kQ],
                                           typename Storage<S>::T (&v1)[kQ]) {
    using T = typename Storage<S>::T;
    static_assert(!Storage<S>::shifted, "slip_pairs serves the unshifted FP64 storage");
    if (s == T(0)) return;
#pragma unroll
    for (int i = 7; i < kQ; ++i) {
        int via, j;
        if (!((sw >> opp(i)) & 1u) || !specular_source(i, sw, via, j)) continue;
        T r0, r1;
        Pair<S>::load(f + ((size_t)j * n + nb.dst(via)), r0, r1);
        v0[i] = (T(1) - s) * v0[i] + s * r0;
        v1[i] = (T(1) - s) * v1[i] + s * r1;
    }
}

// ---------------------------------------------------------------- cp.async helpers
template <int BYTES> __device__ __forceinline__ void cp_async_ca(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace lbm
