// Batched persistent update for many small instances (parameter sweeps):
// one thread-block cluster per instance advances it by n updates inside a
// single launch.  Each update is the two-phase sequence of the two-pass path
// (pseudo-potential pass, then stream + collide), separated by hardware
// cluster barriers (barrier.cluster arrive/wait: release/acquire at cluster
// scope), so no grid-wide software barrier and no spin-wait is involved.
// The instance's distributions stay resident in L2 between updates.
#include <cooperative_groups.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace cg = cooperative_groups;

namespace lbm {

__device__ __forceinline__ void cl_coords(int k, const Grid &g, int &x, int &y, int &z) {
    const int t = k / g.nx;
    x = k - t * g.nx;
    z = t / g.ny;
    y = t - z * g.ny;
}

template <class S>
__device__ __forceinline__ void cl_source(const uint32_t *__restrict__ link_b, uint32_t word, int &x, int y, int z,
                                          const Grid &g, uint32_t &sw) {
    sw = word;
    if (cell_type(word) == kOutlet) {
        const int xu = x == 0 ? g.nx - 1 : x - 1;
        const uint32_t wu = link_b[xu + y * g.nx + z * g.nxy];
        const uint32_t tu = cell_type(wu);
        if (tu != kSolid && tu != kOutlet) {
            x = xu;
            sw = wu;
        }
    }
}

template <class S, int EQ>
__global__ void __launch_bounds__(256) k_cluster(S *__restrict__ fa, S *__restrict__ fb, Ref *__restrict__ ra,
                                                 Ref *__restrict__ rbuf, const uint32_t *__restrict__ link,
                                                 typename Storage<S>::T *__restrict__ psi,
                                                 typename Storage<S>::T *__restrict__ macro, Grid g,
                                                 const InstParam<typename Storage<S>::T> *__restrict__ par,
                                                 int wall_model, int nsteps) {
    using T = typename Storage<S>::T;
    cg::cluster_group cluster = cg::this_cluster();
    const int csize = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int b = blockIdx.x / csize;
    const int ncell = (int)g.n;
    const int stride = csize * blockDim.x;
    const int first = crank * blockDim.x + threadIdx.x;

    const uint32_t *link_b = link + (long long)b * g.n;
    const InstParam<T> &p = par[b];
    T *psi0 = psi + (long long)b * 2 * g.n;
    T *psi1 = psi0 + g.n;
    T *mac = macro + (long long)b * 5 * g.n;
    const long long fofs = (long long)b * 2 * kQ * g.n;
    const long long rofs = (long long)b * 2 * g.n;
    // coherent read of a reference density written by this launch
    auto ref_rd = [&](const Ref *r, long long idx) -> T {
        if constexpr (Storage<S>::shifted) {
            const unsigned short bits = __ldcg(reinterpret_cast<const unsigned short *>(r) + idx);
            return (T)__half2float(__ushort_as_half(bits));
        } else {
            return T(0);
        }
    };

    for (int s = 0; s < nsteps; ++s) {
        const S *fin = ((s & 1) ? fb : fa) + fofs;
        S *fout = ((s & 1) ? fa : fb) + fofs;
        const Ref *rin = ((s & 1) ? rbuf : ra) + rofs;
        Ref *rout = ((s & 1) ? ra : rbuf) + rofs;
        const bool last = s == nsteps - 1;
        // phase 1: pseudo-potential of every cell (S1-S3)
        for (int k = first; k < ncell; k += stride) {
            const uint32_t word = link_b[k];
            const uint32_t t = cell_type(word);
            T q0, q1;
            if (t == kSolid) {
                q0 = p.rs[0];
                q1 = p.rs[1];
            } else if (t == kInlet) {
                q0 = p.rho_in[0];
                q1 = p.rho_in[1];
            } else {
                int x, y, z;
                cl_coords(k, g, x, y, z);
                uint32_t sw;
                cl_source<S>(link_b, word, x, y, z, g, sw);
                Nbr nb;
                nb.init(x, y, z, g);
                const int self = x + y * g.nx + z * g.nxy;
                q0 = pull_density<S, false>(fin, g.n, self, nb, sw, ref_rd(rin, self));
                q1 = pull_density<S, false>(fin + kQ * g.n, g.n, self, nb, sw, ref_rd(rin, g.n + self));
            }
            psi0[k] = q0;
            psi1[k] = q1;
        }
        cluster.sync();
        // phase 2: stream, forces, collide (S1-S7)
        for (int k = first; k < ncell; k += stride) {
            const uint32_t word = link_b[k];
            const uint32_t t = cell_type(word);
            if (t == kSolid) {
                if (last)
                    for (int c = 0; c < 5; ++c) mac[c * g.n + k] = T(0);
                continue;
            }
            int x, y, z;
            cl_coords(k, g, x, y, z);
            Nbr own;
            own.init(x, y, z, g);
            auto sig_for = [&](const T *ps, T own_rho) {
                return [=, &own](int i) -> T {
                    return ref_value(((word >> i) & 1u) ? own_rho : __ldcg(ps + own.dst(i)));
                };
            };
            if (t == kInlet) {
                store_equilibrium<S, EQ>(fout, g.n, k, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2],
                                         sig_for(psi0, p.rho_in[0]));
                store_equilibrium<S, EQ>(fout + kQ * g.n, g.n, k, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2],
                                         sig_for(psi1, p.rho_in[1]));
                if constexpr (Storage<S>::shifted) {
                    rout[k] = __float2half_rn((float)p.rho_in[0]);
                    rout[g.n + k] = __float2half_rn((float)p.rho_in[1]);
                }
                if (last) {
                    mac[k] = p.rho_in[0];
                    mac[g.n + k] = p.rho_in[1];
                    mac[2 * g.n + k] = p.u_in[0];
                    mac[3 * g.n + k] = p.u_in[1];
                    mac[4 * g.n + k] = p.u_in[2];
                }
                continue;
            }
            int sx = x;
            uint32_t sw;
            cl_source<S>(link_b, word, sx, y, z, g, sw);
            Moments<T> m0, m1;
            if (sx == x) {
                m0 = pull_moments<S, false>(fin, g.n, k, own, sw, ref_rd(rin, k));
                m1 = pull_moments<S, false>(fin + kQ * g.n, g.n, k, own, sw, ref_rd(rin, g.n + k));
            } else {
                Nbr up;
                up.init(sx, y, z, g);
                const int self = sx + y * g.nx + z * g.nxy;
                m0 = pull_moments<S, false>(fin, g.n, self, up, sw, ref_rd(rin, self));
                m1 = pull_moments<S, false>(fin + kQ * g.n, g.n, self, up, sw, ref_rd(rin, g.n + self));
            }
            auto psi_at = [&](int i, T &a, T &c) {
                const int j = own.dst(i);
                a = __ldcg(psi0 + j);
                c = __ldcg(psi1 + j);
            };
            const Forces<T> F = sc_forces<T>(psi_at, word, m0.rho, m1.rho, p, wall_model);
            const Relax<T> R = relax<T>(m0, m1, F, p);
            const T ux = R.ux, uy = R.uy, uz = R.uz, omega = R.omega, fcoef = R.fcoef;
            collide_store<S, EQ>(fout, g.n, k, m0, ux, uy, uz, F.F[0][0], F.F[0][1], F.F[0][2], omega, fcoef,
                                 sig_for(psi0, m0.rho));
            collide_store<S, EQ>(fout + kQ * g.n, g.n, k, m1, ux, uy, uz, F.F[1][0], F.F[1][1], F.F[1][2], omega,
                                 fcoef, sig_for(psi1, m1.rho));
            if constexpr (Storage<S>::shifted) {
                rout[k] = __float2half_rn((float)m0.rho);
                rout[g.n + k] = __float2half_rn((float)m1.rho);
            }
            if (last) {
                mac[k] = m0.rho;
                mac[g.n + k] = m1.rho;
                mac[2 * g.n + k] = ux;
                mac[3 * g.n + k] = uy;
                mac[4 * g.n + k] = uz;
            }
        }
        cluster.sync();
    }
}

int cluster_size_for(long long n) {
    long long cs = (n + 255) / 256;
    if (cs < 1) cs = 1;
    if (cs > 8) cs = 8;
    // power of two cluster sizes schedule best
    int c = 1;
    while (c < cs) c <<= 1;
    return c;
}

template <class S, int EQ>
static cudaError_t launch_cluster_t(const StepArgs &a, int nsteps, int csize) {
    using T = typename Storage<S>::T;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.batch * csize), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    record_event(a, 0);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_cluster<S, EQ>, (S *)a.f_in, (S *)a.f_out, (Ref *)a.ref_in,
                                             a.ref_out, a.link, (T *)a.psi, (T *)a.macro, a.g,
                                             (const InstParam<T> *)a.par, a.wall_model, nsteps);
    record_event(a, 1);
    return e;
}

template <class S> static cudaError_t launch_cluster_s(const StepArgs &a, int nsteps, int csize) {
    return a.eq_order == 0 ? launch_cluster_t<S, 0>(a, nsteps, csize) : launch_cluster_t<S, 1>(a, nsteps, csize);
}

// f_in holds the state; after an even number of updates the result is back in
// f_in, after an odd number in f_out.
cudaError_t launch_cluster(const StepArgs &a, int nsteps) {
    if (nsteps <= 0) return cudaSuccess;
    const int csize = cluster_size_for(a.g.n);
    switch (a.precision) {
    case LBM_FP64: return launch_cluster_s<double>(a, nsteps, csize);
    case LBM_FP32: return launch_cluster_s<float>(a, nsteps, csize);
    case LBM_FP32_F16S: return launch_cluster_s<__half>(a, nsteps, csize);
    case LBM_FP32_BF16S: return launch_cluster_s<__nv_bfloat16>(a, nsteps, csize);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
