// Fused single-read update: each CTA owns a TX x TY column of cells and
// marches it through a chunk of z planes.  For every plane it pulls the
// streamed distributions once, keeps the 10 moments per component of its own
// cells in registers, and writes the pseudo-potential of the plane plus a
// one-cell ring around it into a 3-plane ring buffer in shared memory (the
// ring cells are recomputed from their streamed values rather than read
// back from a separate density pass).  One plane behind, it evaluates the
// interaction forces from shared memory and collides (S4-S7).
//
// HBM traffic per fluid cell is the algorithmic minimum (f in, f out, one
// geometry word) plus the halo re-reads, which hit L2 because neighbouring
// columns march in step.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int TX, int TY> struct Tile {
    static constexpr int EX = TX + 2, EY = TY + 2;
    static constexpr int NT = TX * TY;
    static constexpr int HALO = 2 * EX + 2 * TY;  // ring cells of the extended tile
};

// ring-buffer slot of the plane at z offset cz(i) from the colliding plane
__device__ __forceinline__ int cz_slot(int i, int sl, int sm, int su) {
    return cz(i) < 0 ? sl : (cz(i) > 0 ? su : sm);
}

// Pull one cell (x, y, z) -> density (and moments when `want_moments`);
// returns the pseudo-potential pair via psi0/psi1.
template <class S>
__device__ __forceinline__ void cell_pull(const S *__restrict__ fb, const uint32_t *__restrict__ link_b,
                                          const Grid &g, const InstParam<typename Storage<S>::T> &p, int x, int y,
                                          int z, uint32_t word, bool want_moments,
                                          Moments<typename Storage<S>::T> &m0, Moments<typename Storage<S>::T> &m1,
                                          typename Storage<S>::T &psi0, typename Storage<S>::T &psi1,
                                          typename Storage<S>::T r00, typename Storage<S>::T r01) {
    using T = typename Storage<S>::T;
    const uint32_t t = cell_type(word);
    if (t == kSolid) {
        psi0 = p.rs[0];
        psi1 = p.rs[1];
        return;
    }
    if (t == kInlet) {
        psi0 = p.rho_in[0];
        psi1 = p.rho_in[1];
        return;
    }
    uint32_t sw = word;
    if (t == kOutlet) {
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
    if (want_moments) {
        m0 = pull_moments<S>(fb, g.n, self, nb, sw, r00);
        m1 = pull_moments<S>(fb + kQ * g.n, g.n, self, nb, sw, r01);
        psi0 = m0.rho;
        psi1 = m1.rho;
    } else {
        psi0 = pull_density<S>(fb, g.n, self, nb, sw, r00);
        psi1 = pull_density<S>(fb + kQ * g.n, g.n, self, nb, sw, r01);
    }
}

template <class T, int TX, int TY> __host__ __device__ constexpr int fused_psi_bytes() {
    return (int)(((3 * 2 * (TX + 2) * (TY + 2) * sizeof(T)) + 15) / 16 * 16);
}
template <class T, int TX, int TY> __host__ __device__ constexpr int fused_smem_bytes() {
    return fused_psi_bytes<T, TX, TY>() + (int)(2 * 20 * TX * TY * sizeof(T));
}

template <class S, int EQ, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_fused(const S *__restrict__ f, S *__restrict__ fo,
                                                  const uint32_t *__restrict__ link,
                                                  typename Storage<S>::T *__restrict__ macro, Grid g,
                                                  const InstParam<typename Storage<S>::T> *__restrict__ par,
                                                  typename Storage<S>::T r00, typename Storage<S>::T r01,
                                                  int wall_model, int write_macro, int tiles_x, int tiles_y,
                                                  int zchunk, int nchunks) {
    using T = typename Storage<S>::T;
    using TL = Tile<TX, TY>;
    // dynamic shared memory: pseudo-potential ring of 3 planes [3][2][EY][EX],
    // then the moments of the own cells of the last two planes [2][20][NT]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*sp)[2][TL::EY][TL::EX] = reinterpret_cast<T(*)[2][TL::EY][TL::EX]>(smem_raw);
    T(*sm_mom)[20][TL::NT] = reinterpret_cast<T(*)[20][TL::NT]>(smem_raw + fused_psi_bytes<T, TX, TY>());

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

    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    const int x = tx0 + lx, y = ty0 + ly;
    const bool mine = x < g.nx && y < g.ny;
    const int xw = x % g.nx, yw = y % g.ny;  // wrapped (only for ragged tiles)

    const uint32_t *link_b = link + (long long)b * g.n;
    const S *fb = f + (long long)b * 2 * kQ * g.n;
    S *fob = fo + (long long)b * 2 * kQ * g.n;
    T *mac = macro + (long long)b * 5 * g.n;
    const InstParam<T> &p = par[b];

    // halo cell assigned to this thread (ring of the extended tile)
    const int h = threadIdx.x;
    int hex = -1, hey = -1;
    if (h < TL::HALO) {
        if (h < TL::EX) {
            hex = h; hey = 0;
        } else if (h < 2 * TL::EX) {
            hex = h - TL::EX; hey = TL::EY - 1;
        } else if (h < 2 * TL::EX + TY) {
            hex = 0; hey = 1 + (h - 2 * TL::EX);
        } else {
            hex = TL::EX - 1; hey = 1 + (h - 2 * TL::EX - TY);
        }
    }
    int hx = 0, hy = 0;
    if (hex >= 0) {
        hx = tx0 - 1 + hex;
        hy = ty0 - 1 + hey;
        hx = ((hx % g.nx) + g.nx) % g.nx;
        hy = ((hy % g.ny) + g.ny) % g.ny;
    }

    uint32_t word_prev = 0, word_cur = 0;

    for (int pz = z0 - 1; pz <= z1; ++pz) {
        const int zz = pz < 0 ? pz + g.nz : (pz >= g.nz ? pz - g.nz : pz);
        const int slot = (pz + 3) % 3;
        const bool inner = pz >= z0 && pz < z1;
        // own cell of this plane
        {
            const uint32_t w = __ldg(link_b + xw + yw * g.nx + (long long)zz * g.nxy);
            T q0, q1;
            Moments<T> c0, c1;
            const bool want = inner && mine;
            cell_pull<S>(fb, link_b, g, p, xw, yw, zz, w, want, c0, c1, q0, q1, r00, r01);
            sp[slot][0][ly + 1][lx + 1] = q0;
            sp[slot][1][ly + 1][lx + 1] = q1;
            if (want && cell_type(w) != kSolid && cell_type(w) != kInlet) {
                T *ms = &sm_mom[pz & 1][0][threadIdx.x];
                const T v[20] = {c0.rho, c0.jx, c0.jy, c0.jz, c0.pxx, c0.pyy, c0.pzz, c0.pxy, c0.pxz, c0.pyz,
                                 c1.rho, c1.jx, c1.jy, c1.jz, c1.pxx, c1.pyy, c1.pzz, c1.pxy, c1.pxz, c1.pyz};
#pragma unroll
                for (int q = 0; q < 20; ++q) ms[q * TL::NT] = v[q];
            }
            word_cur = w;
        }
        if (hex >= 0) {
            const uint32_t w = __ldg(link_b + hx + hy * g.nx + (long long)zz * g.nxy);
            T q0, q1;
            Moments<T> d0, d1;
            cell_pull<S>(fb, link_b, g, p, hx, hy, zz, w, false, d0, d1, q0, q1, r00, r01);
            sp[slot][0][hey][hex] = q0;
            sp[slot][1][hey][hex] = q1;
        }
        __syncthreads();
        // collide the previous plane
        const int cz = pz - 1;
        if (cz >= z0 && cz < z1 && mine) {
            const uint32_t word = word_prev;
            const uint32_t t = cell_type(word);
            const long long k = (long long)x + (long long)y * g.nx + (long long)cz * g.nxy;
            if (t == kInlet) {
                store_equilibrium<S, EQ>(fob, g.n, (int)k, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2], r00);
                store_equilibrium<S, EQ>(fob + kQ * g.n, g.n, (int)k, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2],
                                         r01);
                if (write_macro) {
                    mac[k] = p.rho_in[0];
                    mac[g.n + k] = p.rho_in[1];
                    mac[2 * g.n + k] = p.u_in[0];
                    mac[3 * g.n + k] = p.u_in[1];
                    mac[4 * g.n + k] = p.u_in[2];
                }
            } else if (t == kSolid) {
                if (write_macro)
                    for (int c = 0; c < 5; ++c) mac[c * g.n + k] = T(0);
            } else {
                Moments<T> a0, a1;
                {
                    const T *ms = &sm_mom[cz & 1][0][threadIdx.x];
                    a0.rho = ms[0]; a0.jx = ms[1 * TL::NT]; a0.jy = ms[2 * TL::NT]; a0.jz = ms[3 * TL::NT];
                    a0.pxx = ms[4 * TL::NT]; a0.pyy = ms[5 * TL::NT]; a0.pzz = ms[6 * TL::NT];
                    a0.pxy = ms[7 * TL::NT]; a0.pxz = ms[8 * TL::NT]; a0.pyz = ms[9 * TL::NT];
                    a1.rho = ms[10 * TL::NT]; a1.jx = ms[11 * TL::NT]; a1.jy = ms[12 * TL::NT];
                    a1.jz = ms[13 * TL::NT]; a1.pxx = ms[14 * TL::NT]; a1.pyy = ms[15 * TL::NT];
                    a1.pzz = ms[16 * TL::NT]; a1.pxy = ms[17 * TL::NT]; a1.pxz = ms[18 * TL::NT];
                    a1.pyz = ms[19 * TL::NT];
                }
                const int sm = (cz + 3) % 3, sl = (cz + 2) % 3, su = (cz + 4) % 3;  // planes cz, cz-1, cz+1
                auto psi_at = [&](int i, T &v0, T &v1) {
                    const int s = cz_slot(i, sl, sm, su);
                    v0 = sp[s][0][ly + 1 + cy(i)][lx + 1 + cx(i)];
                    v1 = sp[s][1][ly + 1 + cy(i)][lx + 1 + cx(i)];
                };
                const Forces<T> F = sc_forces<T>(psi_at, word, a0.rho, a1.rho, p, wall_model);
                const T rho = a0.rho + a1.rho;
                const T Fx = F.F[0][0] + F.F[1][0], Fy = F.F[0][1] + F.F[1][1], Fz = F.F[0][2] + F.F[1][2];
                const T ux = (a0.jx + a1.jx) / rho + T(0.5) * (Fx / rho);
                const T uy = (a0.jy + a1.jy) / rho + T(0.5) * (Fy / rho);
                const T uz = (a0.jz + a1.jz) / rho + T(0.5) * (Fz / rho);
                const T tau = tau_mix<T>(a0.rho, a1.rho, p);
                const T omega = T(1) - T(1) / tau;
                const T fcoef = T(1) - T(1) / (T(2) * tau);
                collide_store<S, EQ>(fob, g.n, (int)k, a0, ux, uy, uz, F.F[0][0], F.F[0][1], F.F[0][2], omega, fcoef,
                                     r00);
                collide_store<S, EQ>(fob + kQ * g.n, g.n, (int)k, a1, ux, uy, uz, F.F[1][0], F.F[1][1], F.F[1][2],
                                     omega, fcoef, r01);
                if (write_macro) {
                    mac[k] = a0.rho;
                    mac[g.n + k] = a1.rho;
                    mac[2 * g.n + k] = ux;
                    mac[3 * g.n + k] = uy;
                    mac[4 * g.n + k] = uz;
                }
            }
        }
        word_prev = word_cur;
        __syncthreads();
    }
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
    k_fused<S, EQ, TX, TY><<<(unsigned)blocks, TX * TY, smem, a.stream>>>(
        (const S *)a.f_in, (S *)a.f_out, a.link, (T *)a.macro, a.g, (const InstParam<T> *)a.par, (T)a.rho0[0],
        (T)a.rho0[1], a.wall_model, a.write_macro, tiles_x, tiles_y, zchunk, nchunks);
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
