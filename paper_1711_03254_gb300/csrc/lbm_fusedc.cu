// Single-read fused update on the compact layout (LBM_KERNEL_FUSED_COMPACT).
//
// The compact two-pass update (lbm_compact.cu) reads f twice per update: the
// density pass pulls every cell's 19 values to form psi (Eq. 7), and the
// collision pass pulls them again together with psi of the 18 neighbours.
// Here f is pulled once, and psi never goes through HBM.
//
// Work decomposition.  A thread-block cluster of kFcCluster CTAs owns a band of
// kFcCluster rows (y) of one instance, one row per CTA, and marches a chunk of
// planes [za, zb) along z; planes za - 1 and zb are recomputed halos (their
// densities only).  The two rows just outside the band are pulled for their
// densities too, their cells shared out over the cluster's CTAs.
//
// Pipeline.  Iteration `it` handles plane p = za - 1 + it:
//   S1  wait for the copies issued in the previous iteration; CTA barrier.
//   S2  densities (S2, S3 of the update) of plane p's cells from their pulled
//       pairs in the lag buffer, into the ring of psi planes in shared memory;
//       the outside rows' densities go into the ring of the CTA that borders
//       them (distributed shared memory).
//   S3  cluster barrier: psi of plane p is complete in every CTA.
//   S4  issue the pulls of plane p + 1 (S1 of the update) as asynchronous
//       copies (cp.async) straight into the lag buffer; the neighbour indices
//       come from the row table staged in shared memory.
//   S5  stage the coordinates and geometry words of plane p + 2's cells and
//       the row table of plane p + 3 (asynchronous copies).
//   S6  collide plane p - 1 (S4-S7): moments from the lag buffer, psi of the
//       18 neighbours from the ring (rows of the neighbouring CTAs through
//       distributed shared memory), store f* and the reference densities.
// The copies of S4 and S5 are in flight while S6 computes, so the collision
// hides the memory latency of the next plane, and every memory access of a
// cell's pull is issued at once (no chain of dependent loads).
//
// Synchronisation.  The psi ring holds 4 planes, so the plane S2 writes is none
// of the three S6 of the previous iteration read; the slot S2 overwrites two
// iterations later was last read before the cluster barrier in between.  The
// lag buffer has 3 slots (plane p + 1 in flight, plane p waiting for its
// collision, plane p - 1 being collided) and is private to each thread: thread
// t pulls cells t, t + T, ... of its row in every plane and collides the same
// cells.  Staged row tables and geometry are shared and published by the CTA
// barrier of S1.  A cluster barrier ends every chunk and the kernel, so no CTA
// leaves while another can still read its shared memory.  All barriers are
// hardware barriers (no software spin-wait).
//
// The arithmetic is that of k_collide_c2 (same operations in the same order:
// at a SOLID neighbour the cell's own psi pair enters the force sums and
// forces2 takes it out again), so both strategies give identical bits.
#include <cooperative_groups.h>

#include "lbm_compact.cuh"

namespace cg = cooperative_groups;

namespace lbm {

constexpr int kFcThreads = 128;  // threads per CTA
constexpr int kFcCluster = 8;    // CTAs per cluster = rows per band
constexpr int kFcSlots = 4;      // planes of the psi ring
constexpr int kFcLag = 3;        // lag slots of the own row's cells
constexpr int kFcHLag = 2;       // lag slots of the outside rows' cells
constexpr int kFcTabPlanes = 4;  // planes of the staged row table
constexpr int kFcTabRows = 9;    // staged rows per plane: y-1..y+1 around the own row and both outside rows

int fusedc_rows_per_cta() { return 1; }

__host__ __device__ constexpr size_t fc_align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared-memory layout of one CTA (the same arithmetic on host and device).
template <class S> struct FcLayout {
    using P = typename Pair2<S>::P;
    int nx, words, cap, hcap;
    __host__ __device__ FcLayout(int nx_, int words_, int cap_)
        : nx(nx_), words(words_), cap(cap_), hcap((2 * cap_ + kFcCluster - 1) / kFcCluster) {}
    // psi ring: [slot][row: outside-low, own, outside-high][x = -1 .. nx]
    __host__ __device__ size_t ring_bytes() const { return fc_align16((size_t)kFcSlots * 3 * (nx + 2) * 8); }
    // own lag slot: pairs [kQ][cap], then reference pair, geometry word, coordinates [cap]
    __host__ __device__ size_t lag_bytes() const { return fc_align16((size_t)cap * (kQ * sizeof(P) + 12)); }
    // outside-row lag slot: pairs [kQ][hcap], then reference pair, coordinates [hcap]
    __host__ __device__ size_t hlag_bytes() const { return fc_align16((size_t)hcap * (kQ * sizeof(P) + 8)); }
    // geometry stage slot: coordinates, then words, of the own and outside cells [cap + hcap]
    __host__ __device__ size_t geo_bytes() const { return fc_align16((size_t)(cap + hcap) * 8); }
    __host__ __device__ size_t tab_bytes() const { return fc_align16((size_t)kFcTabPlanes * kFcTabRows * words * 8); }
    __host__ __device__ size_t total() const {
        return ring_bytes() + kFcLag * lag_bytes() + kFcHLag * hlag_bytes() + 2 * geo_bytes() + tab_bytes();
    }
};

template <class S> size_t fusedc_smem_bytes(int nx, int lag_cap) {
    return FcLayout<S>(nx, (nx + 31) / 32, lag_cap).total();
}

// Neighbour indices of a cell from the staged row table (as CNbr::init, which
// reads the table in global memory).  p[dz + 1] points at the staged words of
// row y - 1 of plane z + dz; rows y and y + 1 follow, `words` apart.
struct FcRows {
    const uint2 *p[3];
    __device__ __forceinline__ const uint2 *row(int dz, int dy, int words) const {
        return p[1 + dz] + (1 + dy) * words;
    }
};

__device__ __forceinline__ uint32_t fc_rank_end(const uint2 *row, int words) {
    const uint2 e = row[words - 1];
    return e.x + __popc(e.y);
}

__device__ __forceinline__ void fc_nbr(CNbr &nb, int x, uint32_t k, const FcRows &R, int words, int nx) {
    const int w = x >> 5, xb = x & 31;
    const uint32_t below = (1u << xb) - 1u;
    nb.nb[0] = k;
    nb.nb[1] = k + 1u;
    nb.nb[2] = k - 1u;
#pragma unroll
    for (int j = 3; j < kQ; ++j) {
        if (cx(j) != 0) continue;
        const uint2 e = R.row(cz(j), cy(j), words)[w];
        const uint32_t at = e.x + __popc(e.y & below);
        nb.nb[j] = at;
#pragma unroll
        for (int m = 7; m < kQ; ++m) {
            if (cy(m) != cy(j) || cz(m) != cz(j) || cx(m) == 0) continue;
            nb.nb[m] = cx(m) > 0 ? at + ((e.y >> xb) & 1u) : at - 1u;
        }
    }
    if (x == 0 || x == nx - 1) {
#pragma unroll
        for (int m = 1; m < kQ; ++m) {
            if (cx(m) == 0) continue;
            const uint2 *row = R.row(cz(m), cy(m), words);
            if (cx(m) > 0 && x == nx - 1) nb.nb[m] = row[0].x;
            if (cx(m) < 0 && x == 0) nb.nb[m] = fc_rank_end(row, words) - 1u;
        }
    }
}

// Issue the pull of one cell (S1 of the update) as asynchronous copies of its
// 19 stored pairs and its reference pair into lag entries dst_pairs[i * stride]
// and dst_ref.  OUTLET cells pull their upstream neighbour's values (as
// outlet_source); INLET cells pull nothing.
template <class S>
__device__ __forceinline__ void fc_issue_pull(const StepArgs &a, int b, const typename Pair2<S>::P *f,
                                              const __half2 *rin, uint32_t k, int x, uint32_t word,
                                              const FcRows &R, typename Pair2<S>::P *dst_pairs, size_t stride,
                                              uint32_t *dst_ref) {
    using P = typename Pair2<S>::P;
    if (cell_type(word) == kInlet) return;
    const int nx = a.g.nx;
    CNbr nb;
    fc_nbr(nb, x, k, R, a.words, nx);
    uint32_t sk = k, sw = word;
    if (cell_type(word) == kOutlet && !((word >> 2) & 1u)) {
        const uint32_t ku = nb.nb[2];
        const uint32_t wu = __ldg(a.clink + (size_t)b * a.kmax + ku);
        if (cell_type(wu) != kOutlet) {
            fc_nbr(nb, x == 0 ? nx - 1 : x - 1, ku, R, a.words, nx);
            sk = ku;
            sw = wu;
        }
    }
    const uint32_t n = a.kmax;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const bool bb = (sw >> opp(i)) & 1u;
        const uint32_t idx = bb ? (uint32_t)opp(i) * n + sk : (uint32_t)i * n + nb.src(i);
        cp_async_ca<sizeof(P)>(dst_pairs + (size_t)i * stride, f + idx);
    }
    cp_async_ca<4>(dst_ref, rin + sk);
}

// Density pair of a pulled cell from its lag entry (as density2 over the same
// stored values, in the same order).
template <class S>
__device__ __forceinline__ float2 fc_density(const typename Pair2<S>::P *pairs, size_t stride, uint32_t ref_bits) {
    float2 v[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) v[i] = Pair2<S>::load_shared(pairs + (size_t)i * stride);
    __half2 R;
    memcpy(&R, &ref_bits, 4);
    return density2<Pair2<S>::kScaled>(v, __half22float2(R), Pair2<S>::kUnscale);
}

// psi pair of cell x (plus its periodic images at x = -1 and x = nx) into one
// ring row (generic pointer to the row's x = -1 entry; local or remote).
__device__ __forceinline__ void fc_ring_store(float2 *row, int x, int nx, float2 v) {
    row[x + 1] = v;
    if (x == 0) row[nx + 1] = v;
    if (x == nx - 1) row[0] = v;
}

// 16-bit storage: two CTAs per SM within the shared memory; FP32 storage: one
// (its lag buffer takes most of an SM's shared memory)
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
    const int nx = g.nx, ny = g.ny, nz = g.nz, words = a.words;
    const FcLayout<S> L(nx, words, fp.lag_cap);
    const int cap = L.cap, hcap = L.hcap;
    const int ringw = nx + 2;
    unsigned char *sp = fc_smem;
    float2 *ring = (float2 *)sp;
    sp += L.ring_bytes();
    unsigned char *lag0 = sp;
    sp += kFcLag * L.lag_bytes();
    unsigned char *hlag0 = sp;
    sp += kFcHLag * L.hlag_bytes();
    uint32_t *geo0 = (uint32_t *)sp;
    sp += 2 * L.geo_bytes();
    uint2 *tab0 = (uint2 *)sp;
    // lag slot s: pairs [kQ][cap], then fields f = 0 reference pair, 1 word, 2 coordinates [cap]
    auto lag_pairs = [&](int s) { return (P *)(lag0 + s * L.lag_bytes()); };
    auto lag_u32 = [&](int s, int fld) {
        return (uint32_t *)(lag0 + s * L.lag_bytes() + (size_t)kQ * cap * sizeof(P)) + (size_t)fld * cap;
    };
    auto hlag_pairs = [&](int s) { return (P *)(hlag0 + s * L.hlag_bytes()); };
    auto hlag_u32 = [&](int s, int fld) {
        return (uint32_t *)(hlag0 + s * L.hlag_bytes() + (size_t)kQ * hcap * sizeof(P)) + (size_t)fld * hcap;
    };
    // geometry stage slot s: field 0 coordinates, 1 words [cap + hcap]
    auto geo = [&](int s, int fld) { return geo0 + (size_t)s * (L.geo_bytes() / 4) + (size_t)fld * (cap + hcap); };
    // staged row table: [plane slot][row 0..8][word]
    auto tab_row = [&](int pslot, int r) { return tab0 + ((size_t)pslot * kFcTabRows + r) * words; };
    auto ring_row = [&](int slot, int ri) { return ring + ((size_t)slot * 3 + ri) * ringw; };
    const size_t slot_elems = (size_t)3 * ringw;
    const uint32_t n = a.kmax;

    for (int u = cid; u < fp.units; u += nclusters) {
        const int b = u / (fp.bands * fp.chunks);
        const int rem = u - b * fp.bands * fp.chunks;
        const int band = rem / fp.chunks, chunk = rem - (rem / fp.chunks) * fp.chunks;
        const int y0 = band * kFcCluster;
        const int band_end = min(y0 + kFcCluster, ny);
        const int y = y0 + crank;
        const bool has_row = y < band_end;
        const int last = band_end - 1 - y0;  // rank owning the band's last row
        const int za = (int)((long long)chunk * nz / fp.chunks);
        const int zb = (int)((long long)(chunk + 1) * nz / fp.chunks);
        const int Z = zb - za;
        const int y_lo = y0 == 0 ? ny - 1 : y0 - 1;
        const int y_hi = band_end == ny ? 0 : band_end;
        const uint2 *tab = instance_tab(a, b);
        const InstParam<float> &prm = ((const InstParam<float> *)a.par)[b];
        const P *f = (const P *)a.f_in + (size_t)b * kQ * n;
        P *fo = (P *)a.f_out + (size_t)b * kQ * n;
        const __half2 *rin = (const __half2 *)a.ref_in + (size_t)b * n;
        __half2 *rout = (__half2 *)a.ref_out + (size_t)b * n;
        const uint32_t *cxyz = a.cxyz + (size_t)b * n, *clink = a.clink + (size_t)b * n;
        float *mac = (float *)a.macro + (long long)b * 5 * g.n;
        // psi rows y - 1 and y + 1: the neighbouring CTAs' own rows, or the
        // band's outside rows kept by CTA 0 (low) and the last CTA (high)
        float2 *row_lo = crank > 0 ? cl.map_shared_rank(ring_row(0, 1), (unsigned)(crank - 1)) : ring_row(0, 0);
        float2 *row_hi = crank < last ? cl.map_shared_rank(ring_row(0, 1), (unsigned)min(crank + 1, kFcCluster - 1))
                                      : ring_row(0, 2);
        float2 *out_lo = cl.map_shared_rank(ring_row(0, 0), 0);
        float2 *out_hi = cl.map_shared_rank(ring_row(0, 2), (unsigned)last);
        auto plane_of = [&](int it) {
            int p = (za - 1 + it) % nz;
            return p < 0 ? p + nz : p;
        };
        auto wrap_y = [&](int yy) { return yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy); };
        auto tslot = [](int it) { return (it + 1) & (kFcTabPlanes - 1); };
        // rows staged per plane: own y-1, y, y+1 (0..2), outside-low (3..5), outside-high (6..8)
        auto stage_tab = [&](int it) {
            const int p = plane_of(it);
            const int ps = tslot(it);
            const int ys[3] = {y, y_lo, y_hi};
            for (int e = tid; e < kFcTabRows * words; e += kFcThreads) {
                const int r = e / words, w = e - r * words;
                const int yy = wrap_y(ys[r / 3] + (r % 3) - 1);
                cp_async_ca<8>(tab_row(ps, r) + w, tab + ((size_t)p * ny + yy) * words + w);
            }
        };
        // cells of plane `it`: own row [k0, k0 + n_own), outside rows [l0, l0 + nl) and [h0, h0 + nh)
        struct Range {
            uint32_t k0, l0, h0;
            int n_own, nl, nh;
        };
        auto ranges = [&](int it) {
            const int ps = tslot(it);
            Range r;
            r.k0 = has_row ? tab_row(ps, 1)[0].x : 0u;
            r.n_own = has_row ? (int)(fc_rank_end(tab_row(ps, 1), words) - r.k0) : 0;
            r.l0 = tab_row(ps, 4)[0].x;
            r.nl = (int)(fc_rank_end(tab_row(ps, 4), words) - r.l0);
            r.h0 = tab_row(ps, 7)[0].x;
            r.nh = (int)(fc_rank_end(tab_row(ps, 7), words) - r.h0);
            return r;
        };
        auto stage_geo = [&](int it) {
            const Range r = ranges(it);
            uint32_t *gx = geo(it & 1, 0), *gw = geo(it & 1, 1);
            for (int j = tid; j < r.n_own; j += kFcThreads) {
                cp_async_ca<4>(gx + j, cxyz + r.k0 + j);
                cp_async_ca<4>(gw + j, clink + r.k0 + j);
            }
            for (int m = 0, h = crank + kFcCluster * tid; h < r.nl + r.nh; ++m, h += kFcCluster * kFcThreads) {
                const uint32_t k = h < r.nl ? r.l0 + (uint32_t)h : r.h0 + (uint32_t)(h - r.nl);
                const int e = cap + m * kFcThreads + tid;
                cp_async_ca<4>(gx + e, cxyz + k);
                cp_async_ca<4>(gw + e, clink + k);
            }
        };
        // the staged row pointers around row index `mid` (1: own, 4: low, 7: high) for plane `it`
        auto rows_at = [&](int it, int mid) {
            FcRows R;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz) R.p[dz] = tab_row(tslot(it - 1 + dz), mid - 1);
            return R;
        };
        auto issue_pulls = [&](int it, const Range &r) {
            const uint32_t *gx = geo(it & 1, 0), *gw = geo(it & 1, 1);
            const int ls = it % kFcLag, hs = it & 1;
            P *lp = lag_pairs(ls);
            uint32_t *lref = lag_u32(ls, 0), *lword = lag_u32(ls, 1), *lxyz = lag_u32(ls, 2);
            const FcRows Ro = rows_at(it, 1);
            for (int j = tid; j < r.n_own; j += kFcThreads) {
                const uint32_t pxyz = gx[j], word = gw[j];
                lword[j] = word;
                lxyz[j] = pxyz;
                fc_issue_pull<S>(a, b, f, rin, r.k0 + (uint32_t)j, (int)(pxyz & 2047u), word, Ro, lp + j, cap,
                                 lref + j);
            }
            P *hp = hlag_pairs(hs);
            uint32_t *href = hlag_u32(hs, 0), *hxyz = hlag_u32(hs, 1);
            const FcRows Rl = rows_at(it, 4), Rh = rows_at(it, 7);
            // (Rh is Rl shifted by three staged rows in every plane)
            for (int m = 0, h = crank + kFcCluster * tid; h < r.nl + r.nh; ++m, h += kFcCluster * kFcThreads) {
                const bool low = h < r.nl;
                const uint32_t k = low ? r.l0 + (uint32_t)h : r.h0 + (uint32_t)(h - r.nl);
                const int e = m * kFcThreads + tid;
                const uint32_t pxyz = gx[cap + e], word = gw[cap + e];
                hxyz[e] = pxyz | (low ? 0u : 0x80000000u);
                fc_issue_pull<S>(a, b, f, rin, k, (int)(pxyz & 2047u), word, low ? Rl : Rh, hp + e, hcap,
                                 href + e);
            }
        };

        // prologue: row tables of planes -1 .. 2, geometry of planes 0 and 1, pulls of plane 0
        for (int it = -1; it <= 2; ++it) stage_tab(it);
        cp_async_commit_group();
        cp_async_wait_all();
        __syncthreads();
        stage_geo(0);
        stage_geo(1);
        cp_async_commit_group();
        cp_async_wait_all();
        __syncthreads();
        Range rng_cur = ranges(0), rng_prev{};
        issue_pulls(0, rng_cur);
        cp_async_commit_group();
        for (int it = 0; it < Z + 2; ++it) {
            const int slot = it & (kFcSlots - 1);
            // ---------------------------------------------------------------- S1
            cp_async_wait_all();
            __syncthreads();
            // ---------------------------------------------------------------- S2
            {
                const Range &r = rng_cur;
                const int ls = it % kFcLag, hs = it & 1;
                const P *lp = lag_pairs(ls);
                const uint32_t *lref = lag_u32(ls, 0), *lword = lag_u32(ls, 1), *lxyz = lag_u32(ls, 2);
                float2 *own = ring_row(slot, 1);
                for (int j = tid; j < r.n_own; j += kFcThreads) {
                    const uint32_t word = lword[j];
                    const float2 rho = cell_type(word) == kInlet ? make_float2(prm.rho_in[0], prm.rho_in[1])
                                                                 : fc_density<S>(lp + j, cap, lref[j]);
                    fc_ring_store(own, (int)(lxyz[j] & 2047u), nx, rho);
                }
                const P *hp = hlag_pairs(hs);
                const uint32_t *href = hlag_u32(hs, 0), *hxyz = hlag_u32(hs, 1);
                const uint32_t *gw = geo(it & 1, 1);
                for (int m = 0, h = crank + kFcCluster * tid; h < r.nl + r.nh; ++m, h += kFcCluster * kFcThreads) {
                    const int e = m * kFcThreads + tid;
                    const uint32_t word = gw[cap + e], hx = hxyz[e];
                    const float2 rho = cell_type(word) == kInlet ? make_float2(prm.rho_in[0], prm.rho_in[1])
                                                                 : fc_density<S>(hp + e, hcap, href[e]);
                    fc_ring_store(((hx >> 31) ? out_hi : out_lo) + (size_t)slot * slot_elems, (int)(hx & 2047u), nx,
                                  rho);
                }
            }
            // ---------------------------------------------------------------- S3
            cl.sync();
            // ---------------------------------------------------------------- S4, S5
            Range rng_next{};
            if (it + 1 <= Z + 1) {
                rng_next = ranges(it + 1);
                issue_pulls(it + 1, rng_next);
            }
            if (it + 2 <= Z + 1) stage_geo(it + 2);
            if (it + 3 <= Z + 2) stage_tab(it + 3);
            cp_async_commit_group();
            // ---------------------------------------------------------------- S6
            if (it >= 2) {
                const size_t offs[3] = {(size_t)((it - 2) & (kFcSlots - 1)) * slot_elems,
                                        (size_t)((it - 1) & (kFcSlots - 1)) * slot_elems, (size_t)slot * slot_elems};
                const int ls = (it - 1) % kFcLag;
                const P *qp = lag_pairs(ls);
                const uint32_t *qref = lag_u32(ls, 0), *qword = lag_u32(ls, 1), *qxyz = lag_u32(ls, 2);
                const float2 *rows[3] = {row_lo, ring_row(0, 1), row_hi};
                for (int j = tid; j < rng_prev.n_own; j += kFcThreads) {
                    const uint32_t k = rng_prev.k0 + (uint32_t)j;
                    const uint32_t pxyz = qxyz[j], word = qword[j];
                    const CompactCell c = unpack_cell(pxyz, word);
                    auto psi_at = [&](int i) -> float2 {
                        return rows[1 + cy(i)][offs[1 + cz(i)] + (size_t)(c.x + 1 + cx(i))];
                    };
                    const float2 own_psi = rows[1][offs[1] + (size_t)(c.x + 1)];
                    const long long cell = c.x + (long long)nx * (c.y + (long long)ny * c.z);
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
                    const uint32_t rbits = qref[j];
                    __half2 Rref;
                    memcpy(&Rref, &rbits, 4);
                    const Moments2 m = moments2<Pair2<S>::kScaled>(v, __half22float2(Rref), Pair2<S>::kUnscale);
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
                    const float2 psi_own = ((word & 0x7FFFEu) && a.wall_model < 2) ? own_psi : bc2(0.f);
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
            rng_prev = rng_cur;
            if (it == 0 || it == Z + 1) rng_prev.n_own = 0;  // halo planes are not collided
            rng_cur = rng_next;
        }
        // the next chunk restarts the ring and the stages; no CTA may still read them
        cp_async_wait_all();
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
    const int bands = (g.ny + kFcCluster - 1) / kFcCluster;
    long long best_nc = 1;
    double best = 1e300;
    for (long long nc = 1; nc <= g.nz; ++nc) {
        const long long units = (long long)batch * bands * nc;
        const long long rounds = (units + active - 1) / active;
        const long long zmax = (g.nz + nc - 1) / nc;
        const double t = (double)rounds * ((double)zmax + 1.0);
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
