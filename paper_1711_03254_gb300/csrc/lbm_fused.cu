// Fused single-read update: each CTA owns a TX x TY column of cells and
// marches it through a chunk of z planes.  For every plane it pulls the
// streamed distributions once, keeps the moments of its own cells in shared
// memory, and writes the pseudo-potential of the plane plus a one-cell ring
// around it into a 3-plane ring buffer in shared memory (the ring cells are
// recomputed from their streamed values rather than read back from a separate
// density pass).  One plane behind, it evaluates the interaction forces from
// shared memory and collides (S4-S7).
//
// HBM traffic per fluid cell is the algorithmic minimum (f in, f out, one
// geometry word, the reference densities) plus halo re-reads, which mostly hit
// L2 because neighbouring columns march in step, and the unused parts of
// 32-byte sectors shared with SOLID cells.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int TX, int TY> struct Tile {
    static constexpr int EX = TX + 2, EY = TY + 2;
    static constexpr int NT = TX * TY;  // threads = interior cells per plane
    static constexpr int NE = EX * EY;  // extended cells per plane
};

constexpr int kMom = 11;  // moments kept per component (see Moments)

// ring-buffer slot of the plane at z offset cz(i) from the colliding plane
__device__ __forceinline__ int cz_slot(int i, int sl, int sm, int su) {
    return cz(i) < 0 ? sl : (cz(i) > 0 ? su : sm);
}

// Pull one component of one cell (x, y, z): returns its density and, when
// `mom` is non-null, stores its moments at mom[q * stride].  Components are
// pulled one after the other so that only 19 loads are in flight per thread.
template <class S>
__device__ __forceinline__ typename Storage<S>::T cell_pull(const S *__restrict__ fb, const uint32_t *__restrict__ link_b,
                                                           const Grid &g, int x, int y, int z, uint32_t word, int comp,
                                                           typename Storage<S>::T *mom, int stride,
                                                           const Ref *__restrict__ rin_b) {
    using T = typename Storage<S>::T;
    uint32_t sw = word;
    if (cell_type(word) == kOutlet) {
        const int xu = x == 0 ? g.nx - 1 : x - 1;
        const uint32_t wu = __ldg(link_b + xu + y * g.nx + (long long)z * g.nxy);
        const uint32_t tu = cell_type(wu);
        if (tu != kSolid && tu != kOutlet) {
            x = xu;
            sw = wu;
        }
    }
    Nbr nb;
    nb.init(x, y, z, g);
    const int self = x + y * g.nx + z * g.nxy;
    T rr = T(0);
    if constexpr (Storage<S>::shifted) rr = (T)__half2float(rin_b[comp * g.n + self]);
    const S *fc = fb + (long long)comp * kQ * g.n;
    if (mom) {
        const Moments<T> m = pull_moments<S>(fc, g.n, self, nb, sw, rr);
        mom[0] = m.rho; mom[stride] = m.rd; mom[2 * stride] = m.jx; mom[3 * stride] = m.jy;
        mom[4 * stride] = m.jz; mom[5 * stride] = m.pxx; mom[6 * stride] = m.pyy; mom[7 * stride] = m.pzz;
        mom[8 * stride] = m.pxy; mom[9 * stride] = m.pxz; mom[10 * stride] = m.pyz;
        return m.rho;
    }
    return pull_density<S>(fc, g.n, self, nb, sw, rr);
}

template <class T>
__device__ __forceinline__ Moments<T> read_moments(const T *mom, int stride) {
    Moments<T> m;
    m.rho = mom[0]; m.rd = mom[stride]; m.jx = mom[2 * stride]; m.jy = mom[3 * stride]; m.jz = mom[4 * stride];
    m.pxx = mom[5 * stride]; m.pyy = mom[6 * stride]; m.pzz = mom[7 * stride];
    m.pxy = mom[8 * stride]; m.pxz = mom[9 * stride]; m.pyz = mom[10 * stride];
    return m;
}

// Shared-memory layout of the fused kernel.
template <class T, int TX, int TY> struct FusedSmem {
    using TL = Tile<TX, TY>;
    T sp[3][2][TL::EY][TL::EX];        // pseudo-potential ring of three planes
    T mom[2][2 * kMom][TL::NT];        // moments of the interior cells, by plane parity
    uint32_t word[2][TL::NT];          // geometry words of the interior cells, by plane parity
};

constexpr uint32_t kNoCollide = 1u << 30;  // interior slot outside the domain or on a halo plane

template <class S, int EQ, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, (TX * TY <= 256 ? 2 : 1))
    k_fused(const S *__restrict__ f, S *__restrict__ fo, const Ref *__restrict__ rin, Ref *__restrict__ rout,
            const uint32_t *__restrict__ link, typename Storage<S>::T *__restrict__ macro, Grid g,
            const InstParam<typename Storage<S>::T> *__restrict__ par, int wall_model, int write_macro, int tiles_x,
            int tiles_y, int zchunk, int nchunks) {
    using T = typename Storage<S>::T;
    using TL = Tile<TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<T, TX, TY> &sm = *reinterpret_cast<FusedSmem<T, TX, TY> *>(smem_raw);

    // block -> (tile x, tile y, z chunk, instance)
    int bid = blockIdx.x;
    const int tx0 = (bid % tiles_x) * TX;
    bid /= tiles_x;
    const int ty0 = (bid % tiles_y) * TY;
    bid /= tiles_y;
    const int zc = bid % nchunks;
    const int b = bid / nchunks;
    const int z0 = zc * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);
    const int tid = threadIdx.x;

    const uint32_t *link_b = link + (long long)b * g.n;
    const S *fb = f + (long long)b * 2 * kQ * g.n;
    S *fob = fo + (long long)b * 2 * kQ * g.n;
    T *mac = macro + (long long)b * 5 * g.n;
    const InstParam<T> &p = par[b];
    const Ref *rin_b = rin + (long long)b * 2 * g.n;
    Ref *rout_b = rout + (long long)b * 2 * g.n;

    for (int pz = z0 - 1; pz <= z1; ++pz) {
        const int zz = pz < 0 ? pz + g.nz : (pz >= g.nz ? pz - g.nz : pz);
        const int slot = (pz + 3) % 3;
        const int par2 = pz & 1;
        const bool inner = pz >= z0 && pz < z1;

        // ---- extended plane: pseudo-potential of every cell, moments of own cells
        for (int e = tid; e < TL::NE; e += TL::NT) {
            const int ey = e / TL::EX, ex = e - ey * TL::EX;
            int x = tx0 - 1 + ex, y = ty0 - 1 + ey;
            x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
            y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
            if (g.nx < TL::EX) x %= g.nx;  // grids narrower than a tile wrap more than once
            if (g.ny < TL::EY) y %= g.ny;
            const uint32_t w = __ldg(link_b + x + y * g.nx + (long long)zz * g.nxy);
            const uint32_t t = cell_type(w);
            const bool interior = ex >= 1 && ex <= TX && ey >= 1 && ey <= TY;
            const bool mine = interior && inner && tx0 + ex - 1 < g.nx && ty0 + ey - 1 < g.ny;
            const int s = interior ? (ey - 1) * TX + (ex - 1) : 0;
            if (interior) sm.word[par2][s] = mine ? w : kNoCollide;
            if (t == kSolid) {
                sm.sp[slot][0][ey][ex] = p.rs[0];
                sm.sp[slot][1][ey][ex] = p.rs[1];
            } else if (t == kInlet) {
                sm.sp[slot][0][ey][ex] = p.rho_in[0];
                sm.sp[slot][1][ey][ex] = p.rho_in[1];
            } else {
#pragma unroll 1
                for (int comp = 0; comp < 2; ++comp) {
                    T *mom = mine ? &sm.mom[par2][comp * kMom][s] : nullptr;
                    sm.sp[slot][comp][ey][ex] = cell_pull<S>(fb, link_b, g, x, y, zz, w, comp, mom, TL::NT, rin_b);
                }
            }
        }
        __syncthreads();

        // ---- collide the previous plane
        const int cz = pz - 1;
        if (cz >= z0 && cz < z1) {
            const int cpar = cz & 1;
            const int sm_ = (cz + 3) % 3, sl = (cz + 2) % 3, su = (cz + 4) % 3;  // planes cz, cz-1, cz+1
            const int s = tid;
            const uint32_t word = sm.word[cpar][s];
            const int lx = s % TX, ly = s / TX;
            const long long k = (long long)(tx0 + lx) + (long long)(ty0 + ly) * g.nx + (long long)cz * g.nxy;
            const uint32_t t = cell_type(word);
            auto sig_for = [&](int comp, T own_rho) {
                return [&, comp, own_rho](int i) -> T {
                    return ref_value(((word >> i) & 1u)
                                         ? own_rho
                                         : sm.sp[cz_slot(i, sl, sm_, su)][comp][ly + 1 + cy(i)][lx + 1 + cx(i)]);
                };
            };
            if (word & kNoCollide) {
                // outside the domain: nothing to do
            } else if (t == kFluid || t == kOutlet) {
                const Moments<T> a0 = read_moments<T>(&sm.mom[cpar][0][s], TL::NT);
                const Moments<T> a1 = read_moments<T>(&sm.mom[cpar][kMom][s], TL::NT);
                auto psi_at = [&](int i, T &v0, T &v1) {
                    const int sl_ = cz_slot(i, sl, sm_, su);
                    v0 = sm.sp[sl_][0][ly + 1 + cy(i)][lx + 1 + cx(i)];
                    v1 = sm.sp[sl_][1][ly + 1 + cy(i)][lx + 1 + cx(i)];
                };
                const Forces<T> F = sc_forces<T>(psi_at, word, a0.rho, a1.rho, p, wall_model);
                const Relax<T> R = relax<T>(a0, a1, F, p);
                const T ux = R.ux, uy = R.uy, uz = R.uz, omega = R.omega, fcoef = R.fcoef;
                collide_store<S, EQ>(fob, g.n, (int)k, a0, ux, uy, uz, F.F[0][0], F.F[0][1], F.F[0][2], omega, fcoef,
                                     sig_for(0, a0.rho));
                collide_store<S, EQ>(fob + kQ * g.n, g.n, (int)k, a1, ux, uy, uz, F.F[1][0], F.F[1][1], F.F[1][2],
                                     omega, fcoef, sig_for(1, a1.rho));
                if constexpr (Storage<S>::shifted) {
                    rout_b[k] = __float2half_rn((float)a0.rho);
                    rout_b[g.n + k] = __float2half_rn((float)a1.rho);
                }
                if (write_macro) {
                    mac[k] = a0.rho;
                    mac[g.n + k] = a1.rho;
                    mac[2 * g.n + k] = ux;
                    mac[3 * g.n + k] = uy;
                    mac[4 * g.n + k] = uz;
                }
            } else if (t == kInlet) {
                store_equilibrium<S, EQ>(fob, g.n, (int)k, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2],
                                         sig_for(0, p.rho_in[0]));
                store_equilibrium<S, EQ>(fob + kQ * g.n, g.n, (int)k, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2],
                                         sig_for(1, p.rho_in[1]));
                if constexpr (Storage<S>::shifted) {
                    rout_b[k] = __float2half_rn((float)p.rho_in[0]);
                    rout_b[g.n + k] = __float2half_rn((float)p.rho_in[1]);
                }
                if (write_macro) {
                    mac[k] = p.rho_in[0];
                    mac[g.n + k] = p.rho_in[1];
                    mac[2 * g.n + k] = p.u_in[0];
                    mac[3 * g.n + k] = p.u_in[1];
                    mac[4 * g.n + k] = p.u_in[2];
                }
            } else if (write_macro) {  // SOLID
                for (int c = 0; c < 5; ++c) mac[c * g.n + k] = T(0);
            }
        }
        __syncthreads();
    }
}

template <class T, int TX, int TY> constexpr int fused_smem_bytes() {
    return (int)((sizeof(FusedSmem<T, TX, TY>) + 15) / 16 * 16);
}

template <class S, int EQ, int TX, int TY>
static cudaError_t launch_fused_tile(const StepArgs &a, int zchunk) {
    using T = typename Storage<S>::T;
    const int tiles_x = (a.g.nx + TX - 1) / TX, tiles_y = (a.g.ny + TY - 1) / TY;
    const int nchunks = (a.g.nz + zchunk - 1) / zchunk;
    const long long blocks = (long long)tiles_x * tiles_y * nchunks * a.batch;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    constexpr int smem = fused_smem_bytes<T, TX, TY>();
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    static bool attr_set = false;  // once per instantiation
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_fused<S, EQ, TX, TY>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    record_event(a, 0);
    k_fused<S, EQ, TX, TY><<<(unsigned)blocks, TX * TY, smem, a.stream>>>(
        (const S *)a.f_in, (S *)a.f_out, a.ref_in, a.ref_out, a.link, (T *)a.macro, a.g,
        (const InstParam<T> *)a.par, a.wall_model, a.write_macro, tiles_x, tiles_y, zchunk, nchunks);
    record_event(a, 1);
    return cudaGetLastError();
}

template <class S, int EQ>
static cudaError_t launch_fused_eq(const StepArgs &a, int tile, int zchunk) {
    switch (tile) {
    case 0: return launch_fused_tile<S, EQ, 32, 8>(a, zchunk);
    case 1: return launch_fused_tile<S, EQ, 32, 4>(a, zchunk);
    case 2: return launch_fused_tile<S, EQ, 64, 4>(a, zchunk);
    case 3: return launch_fused_tile<S, EQ, 32, 16>(a, zchunk);
    }
    return cudaErrorInvalidValue;
}

template <class S> static cudaError_t launch_fused_s(const StepArgs &a, int tile, int zchunk) {
    return a.eq_order == 0 ? launch_fused_eq<S, 0>(a, tile, zchunk) : launch_fused_eq<S, 1>(a, tile, zchunk);
}

cudaError_t launch_fused(const StepArgs &a, int tile, int zchunk) {
    if (zchunk < 1) return cudaErrorInvalidValue;
    switch (a.precision) {
    case LBM_FP64: return launch_fused_s<double>(a, tile, zchunk);
    case LBM_FP32: return launch_fused_s<float>(a, tile, zchunk);
    case LBM_FP32_F16S: return launch_fused_s<__half>(a, tile, zchunk);
    case LBM_FP32_BF16S: return launch_fused_s<__nv_bfloat16>(a, tile, zchunk);
    }
    return cudaErrorInvalidValue;
}

int fused_tile_count() { return 4; }

}  // namespace lbm
