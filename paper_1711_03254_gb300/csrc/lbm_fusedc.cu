// Single-read fused update on the compact layout (LBM_KERNEL_FUSED_COMPACT).
//
// The compact two-pass update (lbm_compact.cu) reads f twice per update: the
// density pass pulls every cell's 19 values to form psi (Eq. 7), and the
// collision pass pulls them again together with psi of the 18 neighbours.
// Here f is pulled once, and psi never goes through HBM.
//
// Work decomposition.  A thread-block cluster of kFcCluster CTAs owns a band of
// kFcCluster * kFcRows rows (y) of one instance and marches a chunk of planes
// [za, zb) along z.  CTA r of the cluster owns rows y0 + r kFcRows ... of the
// band.  For every plane p = za - 1 ... zb:
//   A  pull the 19 stored pairs of every non-solid cell of the CTA's rows in
//      plane p (S1), sum them to the density pair (S2, S3) and write it to a
//      ring of psi planes in shared memory; the pulled pairs, the reference
//      densities, the coordinates and the geometry word go to a lag buffer in
//      shared memory (planes za ... zb - 1 only).  The two rows just outside the
//      band (y0 - 1 and the row after the band, wrapped) are pulled for their
//      densities only, shared out over the cluster's CTAs and written into the
//      ring of the CTA that borders them (distributed shared memory).
//   -- cluster barrier: psi of plane p is complete in every CTA --
//   B  collide plane p - 1 (S4-S7): moments from the lag buffer, psi of the 18
//      neighbours from the ring (rows of the neighbouring CTAs through
//      distributed shared memory), and store f* and the reference densities.
// Planes za - 1 and zb are recomputed halos (their densities only); the
// recompute costs 2 / (zb - za) of a chunk's pulls.  The rows just outside a
// band cost 2 / (kFcCluster kFcRows) of a plane's pulls.
//
// Synchronisation.  The ring holds kFcSlots = 4 planes, so the plane written by
// A(p + 1) is none of the three read by B(p), and one cluster barrier per plane
// suffices: the slot A(p + 2) overwrites was last read in B(p), which every CTA
// finished before arriving at the barrier of plane p + 1.  The lag buffer has
// two slots and is private to each thread: thread t pulls cells t, t + T, ...
// of a plane in A and collides the same cells in B.  A barrier ends every
// chunk (the next chunk restarts the ring) and the kernel, so no CTA leaves
// while another can still read its shared memory.  The barriers are the
// hardware cluster barrier (no software spin-wait).
//
// The arithmetic is that of k_collide_c2 (same operations in the same order:
// at a SOLID neighbour the cell's own psi pair enters the force sums and
// forces2 takes it out again), so both strategies give identical bits.
#include <cooperative_groups.h>

#include "lbm_compact.cuh"

namespace cg = cooperative_groups;

namespace lbm {

constexpr int kFcThreads = 256;  // threads per CTA
constexpr int kFcCluster = 8;    // CTAs per cluster (the portable maximum)
constexpr int kFcRows = 2;       // rows of the band per CTA
constexpr int kFcSlots = 4;      // planes of the psi ring
constexpr int kFcBand = kFcCluster * kFcRows;
constexpr int kFcExtra = 3;      // lag words besides the pairs: reference pair, coordinates, geometry word

int fusedc_rows_per_cta() { return kFcRows; }

template <class S> __host__ __device__ constexpr size_t fusedc_lag_cell_bytes() {
    return kQ * sizeof(typename Pair2<S>::P) + kFcExtra * 4;
}

// One lag slot, rounded up to 16 bytes so that the second slot's pairs stay
// aligned for every pair size.
template <class S> __host__ __device__ constexpr size_t fusedc_lag_slot_bytes(int lag_cap) {
    return ((size_t)lag_cap * fusedc_lag_cell_bytes<S>() + 15) & ~(size_t)15;
}

template <class S> size_t fusedc_smem_bytes(int nx, int lag_cap) {
    const size_t ring = (size_t)kFcSlots * (kFcRows + 2) * (size_t)(nx + 2) * sizeof(float2);
    return ring + 2 * fusedc_lag_slot_bytes<S>(lag_cap);
}

// First compact index of row y of plane p (y == ny: the first cell of the next
// plane, or the instance's total after the last plane).
__device__ __forceinline__ uint32_t fc_row_start(const uint2 *__restrict__ tab, int words, const Grid &g, int p,
                                                 int y) {
    const size_t r = (size_t)p * g.ny + y;
    return __ldg(tab + r * words).x;
}

// A: pull the cell with compact index k; returns its density pair and, for the
// lag buffer, its stored pairs, reference pair, coordinates and word.
template <class S>
__device__ __forceinline__ float2 fc_pull(const StepArgs &a, int b, const uint2 *__restrict__ tab,
                                          const typename Pair2<S>::P *__restrict__ f,
                                          const __half2 *__restrict__ rin, const InstParam<float> &prm, uint32_t k,
                                          typename Pair2<S>::P (&raw)[kQ], __half2 &R, uint32_t &pxyz,
                                          uint32_t &word) {
    pxyz = __ldg(a.cxyz + (size_t)b * a.kmax + k);
    word = __ldg(a.clink + (size_t)b * a.kmax + k);
    const CompactCell c = unpack_cell(pxyz, word);
    if (cell_type(word) == kInlet) {
        R = __floats2half2_rn(prm.rho_in[0], prm.rho_in[1]);
        return make_float2(prm.rho_in[0], prm.rho_in[1]);
    }
    const uint32_t n = a.kmax;
    auto pull = [&](const CNbr &nb, uint32_t sk, uint32_t sw) -> float2 {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const bool bb = (sw >> opp(i)) & 1u;
            const uint32_t idx = bb ? (uint32_t)opp(i) * n + sk : (uint32_t)i * n + nb.src(i);
            raw[i] = __ldg(f + idx);
        }
        R = __ldg(rin + sk);
        float2 v[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) v[i] = Pair2<S>::load_shared(&raw[i]);
        return density2<Pair2<S>::kScaled>(v, __half22float2(R), Pair2<S>::kUnscale);
    };
    CNbr own;
    own.init(c.x, c.y, c.z, k, tab, a.words, a.g);
    int xu;
    uint32_t ku, wu;
    if (outlet_source(a, b, c, own, xu, ku, wu)) {
        CNbr up;
        up.init(xu, c.y, c.z, ku, tab, a.words, a.g);
        return pull(up, ku, wu);
    }
    return pull(own, k, word);
}

// psi pair of cell x (plus its periodic images at x = -1 and x = nx) into one
// ring row (generic pointer to the row's x = -1 entry; local or remote).
__device__ __forceinline__ void fc_ring_store(float2 *row, int x, int nx, float2 v) {
    row[x + 1] = v;
    if (x == 0) row[nx + 1] = v;
    if (x == nx - 1) row[0] = v;
}

// 16-bit storage: two CTAs per SM within the registers (128; a few bytes of
// spill); FP32 storage keeps one, its lag buffer fills most of an SM's shared
// memory anyway
template <class S> constexpr int fc_min_blocks() { return sizeof(S) == 2 ? 2 : 1; }

template <class S, int EQ>
__global__ void __launch_bounds__(kFcThreads, fc_min_blocks<S>()) k_fused_c(StepArgs a, FcPlan fp) {
    using P = typename Pair2<S>::P;
    extern __shared__ __align__(16) unsigned char fc_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank();
    const int cid = blockIdx.x / kFcCluster;
    const int nclusters = gridDim.x / kFcCluster;
    const int tid = threadIdx.x;
    const Grid g = a.g;
    const int nx = g.nx;
    const int ringw = nx + 2;
    const size_t slot_elems = (size_t)(kFcRows + 2) * ringw;  // float2 per ring slot
    float2 *ring = (float2 *)fc_smem;
    unsigned char *lag_base = fc_smem + kFcSlots * slot_elems * sizeof(float2);
    const int cap = fp.lag_cap;
    const size_t lag_slot_bytes = fusedc_lag_slot_bytes<S>(cap);
    auto lag_pairs = [&](int s) { return (P *)(lag_base + s * lag_slot_bytes); };
    auto lag_words = [&](int s) { return (uint32_t *)(lag_base + s * lag_slot_bytes + (size_t)kQ * cap * sizeof(P)); };
    // ring row `lr` (-1 ... kFcRows) of slot 0 in this CTA
    auto ring_row = [&](int lr) { return ring + (size_t)(lr + 1) * ringw; };
    const uint32_t n = a.kmax;

    for (int u = cid; u < fp.units; u += nclusters) {
        const int b = u / (fp.bands * fp.chunks);
        const int rem = u - b * fp.bands * fp.chunks;
        const int band = rem / fp.chunks, chunk = rem - (rem / fp.chunks) * fp.chunks;
        const int y0 = band * kFcBand;
        const int band_end = min(y0 + kFcBand, g.ny);
        const int yc0 = y0 + crank * kFcRows;
        const int rows_c = max(0, min(yc0 + kFcRows, band_end) - yc0);
        const int last_rank = (band_end - 1 - y0) / kFcRows;  // owns the band's last row
        const int last_rows = band_end - (y0 + last_rank * kFcRows);
        const int za = (int)((long long)chunk * g.nz / fp.chunks);
        const int zb = (int)((long long)(chunk + 1) * g.nz / fp.chunks);
        const int y_lo = y0 == 0 ? g.ny - 1 : y0 - 1;
        const int y_hi = band_end == g.ny ? 0 : band_end;
        const uint2 *tab = instance_tab(a, b);
        const InstParam<float> &prm = ((const InstParam<float> *)a.par)[b];
        const P *f = (const P *)a.f_in + (size_t)b * kQ * n;
        P *fo = (P *)a.f_out + (size_t)b * kQ * n;
        const __half2 *rin = (const __half2 *)a.ref_in + (size_t)b * n;
        __half2 *rout = (__half2 *)a.ref_out + (size_t)b * n;
        float *mac = (float *)a.macro + (long long)b * 5 * g.n;
        // the band's outside rows live in CTA 0 (row -1) and in the CTA that owns
        // the last row (row last_rows)
        float2 *lo_row = cl.map_shared_rank(ring_row(-1), 0);
        float2 *hi_row = cl.map_shared_rank(ring_row(last_rows), (unsigned)last_rank);
        // rows y - 1 and y + 1 of this CTA's first and last rows
        float2 *below0 = crank > 0 ? cl.map_shared_rank(ring_row(kFcRows - 1), (unsigned)(crank - 1)) : ring_row(-1);
        float2 *above_last = crank == last_rank ? ring_row(rows_c)
                                                : cl.map_shared_rank(ring_row(0), (unsigned)min(crank + 1, kFcCluster - 1));
        uint32_t k0_prev = 0;
        int n_prev = 0;
        const int Z = zb - za;
        for (int it = 0; it < Z + 2; ++it) {
            int p = za - 1 + it;
            p = p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p);
            const int slot = it & (kFcSlots - 1);
            const bool halo_plane = it == 0 || it == Z + 1;
            const size_t soff = (size_t)slot * slot_elems;
            // ---------------------------------------------------------------- A
            const uint32_t k0 = rows_c > 0 ? fc_row_start(tab, a.words, g, p, yc0) : 0u;
            const uint32_t k1 = rows_c > 0 ? fc_row_start(tab, a.words, g, p, yc0 + rows_c) : 0u;
            const int n_own = (int)(k1 - k0);
            P *lp = lag_pairs(it & 1);
            uint32_t *lw = lag_words(it & 1);
            for (int j = tid; j < n_own; j += kFcThreads) {
                P raw[kQ];
                __half2 R;
                uint32_t pxyz, word;
                const float2 rho = fc_pull<S>(a, b, tab, f, rin, prm, k0 + (uint32_t)j, raw, R, pxyz, word);
                const CompactCell c = unpack_cell(pxyz, word);
                fc_ring_store(ring + soff + (size_t)(c.y - yc0 + 1) * ringw, c.x, nx, rho);
                if (!halo_plane) {
#pragma unroll
                    for (int i = 0; i < kQ; ++i) lp[(size_t)i * cap + j] = raw[i];
                    lw[j] = *(const uint32_t *)&R;
                    lw[cap + j] = pxyz;
                    lw[2 * cap + j] = word;
                }
            }
            {
                // the two rows outside the band, shared out over the cluster
                const uint32_t l0 = fc_row_start(tab, a.words, g, p, y_lo);
                const uint32_t l1 = y_lo + 1 < g.ny ? fc_row_start(tab, a.words, g, p, y_lo + 1)
                                                    : fc_row_start(tab, a.words, g, p, g.ny);
                const uint32_t h0 = fc_row_start(tab, a.words, g, p, y_hi);
                const uint32_t h1 = y_hi + 1 < g.ny ? fc_row_start(tab, a.words, g, p, y_hi + 1)
                                                    : fc_row_start(tab, a.words, g, p, g.ny);
                const int nl = (int)(l1 - l0), nh = (int)(h1 - h0);
                for (int h = crank * kFcThreads + tid; h < nl + nh; h += kFcCluster * kFcThreads) {
                    const bool low = h < nl;
                    const uint32_t k = low ? l0 + (uint32_t)h : h0 + (uint32_t)(h - nl);
                    P raw[kQ];
                    __half2 R;
                    uint32_t pxyz, word;
                    const float2 rho = fc_pull<S>(a, b, tab, f, rin, prm, k, raw, R, pxyz, word);
                    const CompactCell c = unpack_cell(pxyz, word);
                    fc_ring_store((low ? lo_row : hi_row) + soff, c.x, nx, rho);
                }
            }
            cl.sync();
            // ---------------------------------------------------------------- B
            if (it >= 2) {
                const size_t off_m = (size_t)((it - 2) & (kFcSlots - 1)) * slot_elems;
                const size_t off_0 = (size_t)((it - 1) & (kFcSlots - 1)) * slot_elems;
                const size_t off_p = soff;
                const P *qp = lag_pairs((it - 1) & 1);
                const uint32_t *qw = lag_words((it - 1) & 1);
                for (int j = tid; j < n_prev; j += kFcThreads) {
                    const uint32_t k = k0_prev + (uint32_t)j;
                    const uint32_t pxyz = qw[cap + j], word = qw[2 * cap + j];
                    const CompactCell c = unpack_cell(pxyz, word);
                    const int r = c.y - yc0;
                    const float2 *rows[3] = {r > 0 ? ring_row(r - 1) : below0, ring_row(r),
                                             r < rows_c - 1 ? ring_row(r + 1) : above_last};
                    const size_t offs[3] = {off_m, off_0, off_p};
                    // psi pair at x + c_i (i >= 1)
                    auto psi_at = [&](int i) -> float2 {
                        return rows[1 + cy(i)][offs[1 + cz(i)] + (size_t)(c.x + 1 + cx(i))];
                    };
                    const float2 own_psi = rows[1][off_0 + (size_t)(c.x + 1)];
                    const long long cell = c.x + (long long)nx * (c.y + (long long)g.ny * c.z);
                    if (cell_type(word) == kInlet) {
                        using PP = typename Pair<S>::P;
                        PP *fo1 = (PP *)fo;
                        const float uu = prm.u_in[0] * prm.u_in[0] + prm.u_in[1] * prm.u_in[1] + prm.u_in[2] * prm.u_in[2];
#pragma unroll
                        for (int i = 0; i < kQ; ++i) {
                            const bool self_ref = i == 0 || ((word >> i) & 1u);
                            const float2 q = self_ref ? make_float2(prm.rho_in[0], prm.rho_in[1]) : psi_at(i);
                            Pair<S>::store(fo1 + (size_t)i * n + k,
                                           feq_dir<float, EQ>(i, prm.rho_in[0], prm.u_in[0], prm.u_in[1], prm.u_in[2], uu),
                                           feq_dir<float, EQ>(i, prm.rho_in[1], prm.u_in[0], prm.u_in[1], prm.u_in[2], uu),
                                           wgt<float>(i) * ref_value(q.x), wgt<float>(i) * ref_value(q.y));
                        }
                        rout[k] = __floats2half2_rn(prm.rho_in[0], prm.rho_in[1]);
                        if (a.write_macro) {
                            mac[cell] = prm.rho_in[0];
                            mac[g.n + cell] = prm.rho_in[1];
                            mac[2 * g.n + cell] = prm.u_in[0];
                            mac[3 * g.n + cell] = prm.u_in[1];
                            mac[4 * g.n + cell] = prm.u_in[2];
                        }
                        continue;
                    }
                    float2 v[kQ];
#pragma unroll
                    for (int i = 0; i < kQ; ++i) v[i] = Pair2<S>::load_shared(qp + (size_t)i * cap + j);
                    const uint32_t rbits = qw[j];
                    const Moments2 m =
                        moments2<Pair2<S>::kScaled>(v, __half22float2(*(const __half2 *)&rbits), Pair2<S>::kUnscale);
                    const __half2 rho_h = __float22half2_rn(m.rho);
                    ForceSums2 bs;
                    bs.clear();
                    __half2 Rp[kQ];
                    Rp[0] = rho_h;
#pragma unroll
                    for (int i = 1; i < kQ; ++i) {
                        const bool solid = (word >> i) & 1u;
                        const float2 q = solid ? own_psi : psi_at(i);
                        bs.add(i, q);
                        Rp[i] = solid ? rho_h : __float22half2_rn(q);
                    }
                    const float2 psi_own = (word & 0x7FFFEu) ? own_psi : bc2(0.f);
                    const Forces2 F = forces2(bs, psi_own, word, m.rho, prm, a.wall_model);
                    const Relax<float> Rx = relax2(m, F, prm);
                    const Prep2 cp = prep2<EQ>(m, Rx, F);
                    constexpr float sc = Pair2<S>::kScale;
                    Pair2<S>::store(fo + k, rest2<EQ>(cp, __half22float2(Rp[0]), sc));
#pragma unroll
                    for (int i = 1; i < kQ; i += 2) {
                        float2 vi, vo;
                        pair2<EQ>(cp, i, __half22float2(Rp[i]), __half22float2(Rp[i + 1]), sc, vi, vo);
                        Pair2<S>::store(fo + (size_t)i * n + k, vi);
                        Pair2<S>::store(fo + (size_t)(i + 1) * n + k, vo);
                    }
                    rout[k] = rho_h;
                    if (a.write_macro) {
                        mac[cell] = m.rho.x;
                        mac[g.n + cell] = m.rho.y;
                        mac[2 * g.n + cell] = Rx.ux;
                        mac[3 * g.n + cell] = Rx.uy;
                        mac[4 * g.n + cell] = Rx.uz;
                    }
                }
            }
            k0_prev = k0;
            n_prev = halo_plane ? 0 : n_own;
        }
        // the next chunk restarts the ring; no CTA may still read it
        cl.sync();
    }
}

template <class S, int EQ> static const void *fc_kernel() { return (const void *)k_fused_c<S, EQ>; }

static const void *fc_kernel_for(lbm_precision prec, int eq) {
    switch (prec) {
    case LBM_FP32: return eq ? fc_kernel<float, 1>() : fc_kernel<float, 0>();
    case LBM_FP32_F16S: return eq ? fc_kernel<__half, 1>() : fc_kernel<__half, 0>();
    case LBM_FP32_BF16S: return eq ? fc_kernel<__nv_bfloat16, 1>() : fc_kernel<__nv_bfloat16, 0>();
    default: return nullptr;
    }
}

static size_t fc_smem_for(lbm_precision prec, int nx, int lag_cap) {
    switch (prec) {
    case LBM_FP32: return fusedc_smem_bytes<float>(nx, lag_cap);
    case LBM_FP32_F16S: return fusedc_smem_bytes<__half>(nx, lag_cap);
    case LBM_FP32_BF16S: return fusedc_smem_bytes<__nv_bfloat16>(nx, lag_cap);
    default: return 0;
    }
}

// Plan for a geometry: shared memory, co-resident clusters and the z chunks.
// Chunks are chosen to minimise (rounds of clusters) x (planes per chunk + the
// halo planes' share), the time of the slowest cluster.
cudaError_t fusedc_plan(lbm_precision prec, int eq_order, const Grid &g, int batch, int lag_cap, FcPlan &out) {
    out = FcPlan{};
    const void *kern = fc_kernel_for(prec, eq_order);
    if (!kern || lag_cap < 1) return cudaSuccess;
    int dev = 0, max_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = fc_smem_for(prec, g.nx, lag_cap);
    if (smem > (size_t)max_optin) return cudaSuccess;  // does not fit: not eligible
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kFcCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kFcCluster, 1, 1);
    cfg.blockDim = dim3(kFcThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (active < 1) return cudaSuccess;
    const int bands = (g.ny + kFcBand - 1) / kFcBand;
    long long best_nc = 1;
    double best = 1e300;
    for (long long nc = 1; nc <= g.nz; ++nc) {
        const long long units = (long long)batch * bands * nc;
        const long long rounds = (units + active - 1) / active;
        const long long zmax = (g.nz + nc - 1) / nc;
        const double t = (double)rounds * ((double)zmax + 0.7);
        if (t < best - 1e-9) {
            best = t;
            best_nc = nc;
        }
    }
    const long long units = (long long)batch * bands * best_nc;
    if (units > (1LL << 30)) return cudaSuccess;
    out.bands = bands;
    out.chunks = (int)best_nc;
    out.units = (int)units;
    out.lag_cap = lag_cap;
    out.smem = smem;
    out.clusters = (int)std::min<long long>(units, active);
    out.ok = true;
    return cudaSuccess;
}

cudaError_t launch_fusedc(const StepArgs &a, const FcPlan &fp) {
    const void *kern = fc_kernel_for(a.precision, a.eq_order);
    if (!kern || !fp.ok) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kFcCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(fp.clusters * kFcCluster), 1, 1);
    cfg.blockDim = dim3(kFcThreads, 1, 1);
    cfg.dynamicSmemBytes = fp.smem;
    cfg.stream = a.stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    StepArgs args = a;
    FcPlan plan = fp;
    void *params[] = {(void *)&args, (void *)&plan};
    record_event(a, 0);
    cudaError_t e = cudaLaunchKernelExC(&cfg, kern, params);
    record_event(a, 1);
    return e;
}

}  // namespace lbm
