// Kernels of the two-pass update on the compact layout (k_psi_c,
// k_collide_c, k_collide_c2) and their launcher, instantiated once per
// storage format in lbm_update_*.cu (one translation unit each, so that the
// variants compile in parallel).  Layout and steps: see lbm_compact.cu.
#pragma once

#include "lbm_compact.cuh"

namespace lbm {

// Occupancy, measured on GB300 (256^3 packed spheres, ms per update).  The
// update runs 128-thread blocks, 6 per SM for the FP32 and 16-bit storages
// (80 registers, no spills) and 4 for FP64: FP16 0.297 against 0.317 at 5 and
// 0.310 at 7 (72 registers, spilling), 256-thread blocks 3 per SM 0.322; FP32
// 0.380 against 0.401 at 5, 0.415 at 7 and 0.441 at 4; FP64 the same at 3 to 5.
// The psi pass runs 256-thread blocks, 6 per SM (40 registers): 16-bit
// storage 0.139 ms against 0.159 at 4 and 0.192 at 3 per SM (5 and 8: 0.139),
// and 0.163 for a persistent variant that prefetched each thread's next cell
// with cp.async; FP32 0.186 against 0.218 at 3 per SM.
constexpr int kPsiThreads = 256, kPsiBlocks = 6, kCollideThreads = 128;
template <class S> constexpr int collide_min_blocks() { return sizeof(S) == 2 ? 6 : (sizeof(S) == 4 ? 6 : 4); }

// S1-S3 for the non-solid cell k of instance b: pull, sum to rho_alpha, store
// the psi pair.  COH: f and the reference densities were written earlier in
// the same launch (the persistent update), so they are read through L2.
// PRE: the caller holds the cell (cell_pre) and its neighbour indices
// (nbr_pre) from an earlier update (the persistent update with one cell per
// thread).
template <class S, bool SLIP, bool COH, bool PRE = false>
__device__ __forceinline__ void psi_cell(const StepArgs &a, int b, uint32_t k, const CompactCell *cell_pre = nullptr,
                                         const CNbr *nbr_pre = nullptr) {
    using T = typename Storage<S>::T;
    using V = typename Vec2<T>::V;
    const CompactCell c = PRE ? *cell_pre : compact_cell(a, b, k);
    const InstParam<T> &p = ((const InstParam<T> *)a.par)[b];
    V *psi = (V *)a.psi + (size_t)b * a.kmax;
    T p0, p1;
    if (cell_type(c.word) == kInlet) {
        p0 = p.rho_in[0];
        p1 = p.rho_in[1];
    } else {
        const typename Pair<S>::P *f = (const typename Pair<S>::P *)a.f_in + (size_t)b * kQ * a.kmax;
        auto pull = [&](const CNbr &nb, uint32_t sk, uint32_t sw) {
            if constexpr (packed_pairs<S>()) {
                float2 v[kQ];
                pull_pairs2<S, COH>(f, a.kmax, sk, nb, sw, v);
                if constexpr (SLIP)
                    slip_pairs2<S, COH>(f, a.kmax, sk, nb, sw, p.slip,
                                        (const __half2 *)a.ref_in + (size_t)b * a.kmax, v);
                const float2 d = density2<Pair2<S>::kScaled>(v, ref_pair2<COH>(a, b, sk), Pair2<S>::kUnscale);
                p0 = d.x;
                p1 = d.y;
            } else {
                T v0[kQ], v1[kQ], r0, r1;
                pull_pairs<S, COH>(f, a.kmax, sk, nb, sw, v0, v1);
                if constexpr (SLIP) slip_pairs<S>(f, a.kmax, nb, sw, p.slip, v0, v1);
                ref_pair<S>(a, b, sk, r0, r1);
                p0 = density_of<T, Storage<S>::shifted>(v0, r0);
                p1 = density_of<T, Storage<S>::shifted>(v1, r1);
            }
        };
        CNbr own_l;
        if constexpr (!PRE) own_l.init(c.x, c.y, c.z, k, instance_tab(a, b), a.words, a.g);
        const CNbr &own = PRE ? *nbr_pre : own_l;
        int xu;
        uint32_t ku, wu;
        if (outlet_source(a, b, c, own, xu, ku, wu)) {
            CNbr up;
            up.init(xu, c.y, c.z, ku, instance_tab(a, b), a.words, a.g);
            pull(up, ku, wu);
        } else {
            pull(own, k, c.word);
        }
    }
    V out;
    out.x = p0;
    out.y = p1;
    psi[k] = out;
}

template <class S, bool SLIP>
__global__ void __launch_bounds__(kPsiThreads, kPsiBlocks) k_psi_c(StepArgs a) {
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)__ldg(a.list_count + b)) return;
    psi_cell<S, SLIP, false>(a, b, k);
}

// The body of k_collide_c for the non-solid cell k of instance b (COH and
// PRE as for collide_cell2).
template <class S, int EQ, bool COH, bool PRE = false>
__device__ __forceinline__ void collide_cell(const StepArgs &a, int b, uint32_t k, int write_macro,
                                             const CompactCell *cell_pre = nullptr, const CNbr *nbr_pre = nullptr) {
    using T = typename Storage<S>::T;
    using V = typename Vec2<T>::V;
    using P = typename Pair<S>::P;
    const CompactCell c = PRE ? *cell_pre : compact_cell(a, b, k);
    const uint32_t word = c.word;
    const InstParam<T> &p = ((const InstParam<T> *)a.par)[b];
    const uint32_t n = a.kmax;
    P *fo = (P *)a.f_out + (size_t)b * kQ * n;
    const V *psi = (const V *)a.psi + (size_t)b * n;
    __half2 *rout = (__half2 *)a.ref_out + (size_t)b * n;
    const long long cell = c.x + (long long)a.g.nx * (c.y + (long long)a.g.ny * c.z);
    T *mac = (T *)a.macro + (long long)b * 5 * a.g.n;
    CNbr own_l;
    if constexpr (!PRE) own_l.init(c.x, c.y, c.z, k, instance_tab(a, b), a.words, a.g);
    const CNbr &own = PRE ? *nbr_pre : own_l;
    // psi of both components at the 18 neighbours (own cell where SOLID: masked
    // by the force and never used as a reference there)
    T q0[kQ], q1[kQ];
    auto load_psi = [&]() {
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            const uint32_t j = ((word >> i) & 1u) ? k : own.dst(i);
            const V q = ld_data<COH>(psi + j);
            q0[i] = q.x;
            q1[i] = q.y;
        }
    };
    if (cell_type(word) == kInlet) {
        load_psi();
        const T uu = p.u_in[0] * p.u_in[0] + p.u_in[1] * p.u_in[1] + p.u_in[2] * p.u_in[2];
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const bool self_ref = i == 0 || ((word >> i) & 1u);
            const T s0 = Storage<S>::shifted ? wgt<T>(i) * ref_value(self_ref ? p.rho_in[0] : q0[i]) : T(0);
            const T s1 = Storage<S>::shifted ? wgt<T>(i) * ref_value(self_ref ? p.rho_in[1] : q1[i]) : T(0);
            Pair<S>::store(fo + (size_t)i * n + k, feq_dir<T, EQ>(i, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2], uu),
                           feq_dir<T, EQ>(i, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2], uu), s0, s1);
        }
        if constexpr (Storage<S>::shifted) rout[k] = __floats2half2_rn((float)p.rho_in[0], (float)p.rho_in[1]);
        if (write_macro) {
            mac[cell] = p.rho_in[0];
            mac[a.g.n + cell] = p.rho_in[1];
            mac[2 * a.g.n + cell] = p.u_in[0];
            mac[3 * a.g.n + cell] = p.u_in[1];
            mac[4 * a.g.n + cell] = p.u_in[2];
        }
        return;
    }
    const P *f = (const P *)a.f_in + (size_t)b * kQ * n;
    Moments<T> m0, m1;
    auto pull = [&](const CNbr &nb, uint32_t sk, uint32_t sw) {
        T v0[kQ], v1[kQ], r0, r1;
        pull_pairs<S, COH>(f, n, sk, nb, sw, v0, v1);
        if constexpr (has_slip(EQ)) slip_pairs<S>(f, n, nb, sw, p.slip, v0, v1);
        ref_pair<S>(a, b, sk, r0, r1);
        m0 = moments_of<T, Storage<S>::shifted>(v0, r0);
        m1 = moments_of<T, Storage<S>::shifted>(v1, r1);
    };
    {
        int xu;
        uint32_t ku, wu;
        if (outlet_source(a, b, c, own, xu, ku, wu)) {
            CNbr up;
            up.init(xu, c.y, c.z, ku, instance_tab(a, b), a.words, a.g);
            pull(up, ku, wu);
        } else {
            pull(own, k, word);
        }
    }
    // psi of both components at the 18 neighbours, streamed into the force sums;
    // what the stores need of it is kept as FP16 reference pairs (the reference
    // density of the cell each value streams into; own cell where SOLID)
    ForceSums<T> bs;
    bs.clear();
    __half2 Rp[kQ];
    Rp[0] = __floats2half2_rn((float)m0.rho, (float)m1.rho);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const bool solid = (word >> i) & 1u;
        const V q = __ldg(psi + (solid ? k : own.dst(i)));
        bs.add(i, solid, q.x, q.y);
        if constexpr (Storage<S>::shifted)
            Rp[i] = __floats2half2_rn((float)(solid ? m0.rho : q.x), (float)(solid ? m1.rho : q.y));
    }
    const Forces<T> F = sc_forces_finish<T>(bs, word, m0.rho, m1.rho, p, a.wall_model);
    const Relax<T> R = relax<T>(m0, m1, F, p);
    const CollidePrep<T> c0 =
        collide_prep<T, EQ>(m0, R.ux, R.uy, R.uz, F.F[0][0], F.F[0][1], F.F[0][2], R.omega, R.fcoef);
    const CollidePrep<T> c1 =
        collide_prep<T, EQ>(m1, R.ux, R.uy, R.uz, F.F[1][0], F.F[1][1], F.F[1][2], R.omega, R.fcoef);
    auto ref0 = [&](int i) -> T { return Storage<S>::shifted ? (T)__low2float(Rp[i]) : T(0); };
    auto ref1 = [&](int i) -> T { return Storage<S>::shifted ? (T)__high2float(Rp[i]) : T(0); };
    Pair<S>::store_d(fo + k, collide_rest<T, EQ>(c0, ref0(0)), collide_rest<T, EQ>(c1, ref1(0)));
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
        T a_i, a_o, b_i, b_o;
        collide_pair<T, EQ>(c0, i, ref0(i), ref0(i + 1), a_i, a_o);
        collide_pair<T, EQ>(c1, i, ref1(i), ref1(i + 1), b_i, b_o);
        Pair<S>::store_d(fo + (size_t)i * n + k, a_i, b_i);
        Pair<S>::store_d(fo + (size_t)(i + 1) * n + k, a_o, b_o);
    }
    if constexpr (Storage<S>::shifted) rout[k] = __floats2half2_rn((float)m0.rho, (float)m1.rho);
    if (write_macro) {
        mac[cell] = m0.rho;
        mac[a.g.n + cell] = m1.rho;
        mac[2 * a.g.n + cell] = R.ux;
        mac[3 * a.g.n + cell] = R.uy;
        mac[4 * a.g.n + cell] = R.uz;
    }
}

template <class S, int EQ>
__global__ void __launch_bounds__(kCollideThreads, collide_min_blocks<S>()) k_collide_c(StepArgs a) {
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)__ldg(a.list_count + b)) return;
    collide_cell<S, EQ, false>(a, b, k, a.write_macro);
}

// k_collide_c2: the update of k_collide_c with both components as packed FP32
// pairs (lbm_pair2.cuh), for the FP32 and 16-bit storages.  Same steps and
// memory accesses; the neighbour psi pairs enter the force sums unselected
// (the cell's own pair at SOLID neighbours, removed in forces2), and the
// storage scale of FP16 is folded into the moment sums and the weights.
// The body of k_collide_c2 for the non-solid cell k of instance b; qs is the
// block's shared-memory slots of the neighbour psi pairs (one column per
// thread).  COH: psi, f and the reference densities were written earlier in
// the same launch (the persistent update) and are read through L2.
template <class S, int EQ, bool COH, bool PRE = false>
__device__ __forceinline__ void collide_cell2(const StepArgs &a, int b, uint32_t k, int write_macro,
                                              float2 (&qs)[kQ - 1][kCollideThreads],
                                              const CompactCell *cell_pre = nullptr, const CNbr *nbr_pre = nullptr) {
    using P = typename Pair2<S>::P;
    const CompactCell c = PRE ? *cell_pre : compact_cell(a, b, k);
    const uint32_t word = c.word;
    const InstParam<float> &p = ((const InstParam<float> *)a.par)[b];
    const uint32_t n = a.kmax;
    const float2 *psi = (const float2 *)a.psi + (size_t)b * n;
    __half2 *rout = (__half2 *)a.ref_out + (size_t)b * n;
    const long long cell = c.x + (long long)a.g.nx * (c.y + (long long)a.g.ny * c.z);
    float *mac = (float *)a.macro + (long long)b * 5 * a.g.n;
    CNbr own_l;
    if constexpr (!PRE) own_l.init(c.x, c.y, c.z, k, instance_tab(a, b), a.words, a.g);
    const CNbr &own = PRE ? *nbr_pre : own_l;
    if (cell_type(word) == kInlet) {
        // equilibrium at (rho_in, u_in) as deviations from the reference pairs
        typename Pair<S>::P *fo = (typename Pair<S>::P *)a.f_out + (size_t)b * kQ * n;
        const float uu = p.u_in[0] * p.u_in[0] + p.u_in[1] * p.u_in[1] + p.u_in[2] * p.u_in[2];
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const bool self_ref = i == 0 || ((word >> i) & 1u);
            const float2 q = self_ref ? make_float2(p.rho_in[0], p.rho_in[1]) : ld_data<COH>(psi + own.dst(i));
            Pair<S>::store(fo + (size_t)i * n + k, feq_dir<float, EQ>(i, p.rho_in[0], p.u_in[0], p.u_in[1], p.u_in[2], uu),
                           feq_dir<float, EQ>(i, p.rho_in[1], p.u_in[0], p.u_in[1], p.u_in[2], uu),
                           wgt<float>(i) * ref_value(q.x), wgt<float>(i) * ref_value(q.y));
        }
        rout[k] = __floats2half2_rn(p.rho_in[0], p.rho_in[1]);
        if (write_macro) {
            mac[cell] = p.rho_in[0];
            mac[a.g.n + cell] = p.rho_in[1];
            mac[2 * a.g.n + cell] = p.u_in[0];
            mac[3 * a.g.n + cell] = p.u_in[1];
            mac[4 * a.g.n + cell] = p.u_in[2];
        }
        return;
    }
    // the psi pairs of the 18 neighbours (the cell's own at SOLID ones) start
    // on their way into this thread's shared-memory slots now, so that their
    // latency overlaps the pull of f; no other thread reads the slots (the
    // persistent update loads them through L2 into the same slots)
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const bool solid = (word >> i) & 1u;
        if constexpr (COH)
            qs[i - 1][tid] = __ldcg(psi + (solid ? k : own.dst(i)));
        else
            cp_async_ca<8>(&qs[i - 1][tid], psi + (solid ? k : own.dst(i)));
    }
    if constexpr (!COH) cp_async_commit_group();
    const P *f = (const P *)a.f_in + (size_t)b * kQ * n;
    P *fo = (P *)a.f_out + (size_t)b * kQ * n;
    Moments2 m;
    auto pull = [&](const CNbr &nb, uint32_t sk, uint32_t sw) {
        float2 v[kQ];
        pull_pairs2<S, COH>(f, n, sk, nb, sw, v);
        if constexpr (has_slip(EQ))
            slip_pairs2<S, COH>(f, n, sk, nb, sw, p.slip, (const __half2 *)a.ref_in + (size_t)b * n, v);
        m = moments2<Pair2<S>::kScaled>(v, ref_pair2<COH>(a, b, sk), Pair2<S>::kUnscale);
    };
    {
        int xu;
        uint32_t ku, wu;
        if (outlet_source(a, b, c, own, xu, ku, wu)) {
            CNbr up;
            up.init(xu, c.y, c.z, ku, instance_tab(a, b), a.words, a.g);
            pull(up, ku, wu);
        } else {
            pull(own, k, word);
        }
    }
    // psi pairs of the 18 neighbours into the force sums; the stores keep the
    // FP16 reference pair of each direction (the density of the cell the
    // value streams into; the cell's own at SOLID neighbours)
    const __half2 rho_h = __float22half2_rn(m.rho);
    ForceSums2 bs;
    bs.clear();
    __half2 Rp[kQ];
    Rp[0] = rho_h;
    if constexpr (!COH) cp_async_wait_all();
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const bool solid = (word >> i) & 1u;
        const float2 q = qs[i - 1][tid];
        bs.add(i, q);
        Rp[i] = solid ? rho_h : __float22half2_rn(q);
    }
    const float2 psi_own = ((word & 0x7FFFEu) && a.wall_model < 2) ? ld_data<COH>(psi + k) : bc2(0.f);
    const Forces2 F = forces2(bs, psi_own, word, m.rho, p, a.wall_model);
    const Relax<float> R = relax2(m, F, p);
    const Prep2 cp = prep2<EQ>(m, R, F);
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
    if (write_macro) {
        mac[cell] = m.rho.x;
        mac[a.g.n + cell] = m.rho.y;
        mac[2 * a.g.n + cell] = R.ux;
        mac[3 * a.g.n + cell] = R.uy;
        mac[4 * a.g.n + cell] = R.uz;
    }
}

template <class S, int EQ>
__global__ void __launch_bounds__(kCollideThreads, collide_min_blocks<S>()) k_collide_c2(StepArgs a) {
    __shared__ float2 qs[kQ - 1][kCollideThreads];
    const int b = blockIdx.y;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (uint32_t)__ldg(a.list_count + b)) return;
    collide_cell2<S, EQ, false>(a, b, k, a.write_macro, qs);
}

// ---------------------------------------------------------------- persistent update
// LBM_KERNEL_PERSISTENT: one cooperative launch runs n updates of the compact
// two-pass update.  Every block strides over all (instance, cell) items of the
// batch: the density pass, a grid-wide barrier, the collision pass, a barrier,
// and so on; the ping-pong buffers swap every update.  Data written earlier in
// the launch (f, psi, the reference densities) is read through L2.  It serves
// small instances and batches of them, where two launches per update cost more
// than the work.
constexpr int kPersistThreads = kCollideThreads;
constexpr int kPersistMaxUpdates = 1 << 20;      // per launch: the barrier counter stays below 2^32
constexpr long long kBarrierCycles = 4000000000LL;  // about 2 s of SM clock

// Grid-wide barrier of a cooperative launch, with a bound on the wait.  Thread
// 0 of every block arrives on bar[0] and waits until all blocks of this phase
// have arrived (and `missing` more, which the failure test sets), until
// another block has given up (bar[1] set), or for `cycles` of its SM clock,
// after which it sets bar[1] itself.  Returns false when the launch must end
// (the host then reports LBM_ERR_TIMEOUT).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned phase, long long cycles, unsigned missing) {
    __shared__ int go;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = phase * gridDim.x + missing;
        const long long t0 = clock64();
        int ok = 1;
        while (*(volatile unsigned *)bar < target) {
            if (*(volatile unsigned *)(bar + 1)) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > cycles) {
                atomicExch(bar + 1, 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        go = ok;
    }
    __syncthreads();
    return go != 0;
}

// a0: the buffers of the first update (f_in -> f_out), a1: swapped.  OWNED:
// every thread has at most one item, whose cell and neighbour indices it
// finds once and keeps in registers for all n updates (then each pass waits
// on one chain of loads, f and psi, instead of three); 4 blocks per SM at 128
// registers (16^3: 5.6 us per update against 7.5 looking the indices up).
template <class S, int EQ, bool OWNED>
__global__ void __launch_bounds__(kPersistThreads, OWNED ? (sizeof(S) == 8 ? 3 : 4) : 1)
    k_persist_c(StepArgs a0, StepArgs a1, int n, int write_macro, unsigned *bar) {
    __shared__ float2 qs[kQ - 1][kPersistThreads];
    // both argument sets in shared memory, read by every thread
    __shared__ __align__(16) unsigned char sa_raw[2 * sizeof(StepArgs)];
    StepArgs *sa = reinterpret_cast<StepArgs *>(sa_raw);
    if (threadIdx.x == 0) {
        memcpy(&sa[0], &a0, sizeof(StepArgs));
        memcpy(&sa[1], &a1, sizeof(StepArgs));
    }
    __syncthreads();
    const long long items = (long long)a0.batch * a0.kmax;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned phase = 0;
    if constexpr (OWNED) {
        int b = 0;
        uint32_t k = 0;
        bool has = false;
        CompactCell c{};
        CNbr own;
        if (first < items) {
            b = (int)(first / a0.kmax);
            k = (uint32_t)(first - (long long)b * a0.kmax);
            has = k < (uint32_t)__ldg(a0.list_count + b);
            if (has) {
                c = compact_cell(sa[0], b, k);
                own.init(c.x, c.y, c.z, k, instance_tab(sa[0], b), a0.words, a0.g);
            }
        }
        for (int u = 0; u < n; ++u) {
            const StepArgs &a = sa[u & 1];
            if (has) psi_cell<S, false, true, true>(a, b, k, &c, &own);
            if (!grid_barrier(bar, ++phase, a.bar_cycles, a.bar_missing)) return;
            const int wm = (write_macro && u == n - 1) ? 1 : 0;
            if (has) {
                if constexpr (packed_pairs<S>())
                    collide_cell2<S, EQ, true, true>(a, b, k, wm, qs, &c, &own);
                else
                    collide_cell<S, EQ, true, true>(a, b, k, wm, &c, &own);
            }
            if (!grid_barrier(bar, ++phase, a.bar_cycles, a.bar_missing)) return;
        }
        return;
    }
    for (int u = 0; u < n; ++u) {
        const StepArgs &a = sa[u & 1];
        for (long long j = first; j < items; j += stride) {
            const int b = (int)(j / a.kmax);
            const uint32_t k = (uint32_t)(j - (long long)b * a.kmax);
            if (k < (uint32_t)__ldg(a.list_count + b)) psi_cell<S, false, true>(a, b, k);
        }
        if (!grid_barrier(bar, ++phase, a.bar_cycles, a.bar_missing)) return;
        const int wm = (write_macro && u == n - 1) ? 1 : 0;
        for (long long j = first; j < items; j += stride) {
            const int b = (int)(j / a.kmax);
            const uint32_t k = (uint32_t)(j - (long long)b * a.kmax);
            if (k < (uint32_t)__ldg(a.list_count + b)) {
                if constexpr (packed_pairs<S>())
                    collide_cell2<S, EQ, true>(a, b, k, wm, qs);
                else
                    collide_cell<S, EQ, true>(a, b, k, wm);
            }
        }
        if (!grid_barrier(bar, ++phase, a.bar_cycles, a.bar_missing)) return;
    }
}

// n updates in cooperative launches of at most kPersistMaxUpdates each, as
// many blocks as fit on the GPU at once (none idle waiting for a slot, which
// the barriers need) but no more than the items.  Variants: eq_order and
// reg_order (wall slip is refused on the host).
template <class S>
cudaError_t launch_persist_t(const StepArgs &a, int n) {
    {
        cudaError_t e = cudaSuccess;
        auto run = [&](auto v) {
            constexpr int EQ = decltype(v)::value;
            int dev = 0, sms = 0, per_sm = 0;
            e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_persist_c<S, EQ, true>,
                                                                  kPersistThreads, 0);
            if (e != cudaSuccess) return;
            const long long items = (long long)a.batch * a.kmax;
            const long long need = (items + kPersistThreads - 1) / kPersistThreads;
            // one item per thread when the whole batch fits in one wave
            const bool owned = per_sm >= 1 && need <= (long long)per_sm * sms;
            if (!owned && e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_persist_c<S, EQ, false>,
                                                                  kPersistThreads, 0);
            if (e != cudaSuccess) return;
            if (per_sm < 1) {
                e = cudaErrorLaunchOutOfResources;
                return;
            }
            long long want = need;
            if (want > (long long)per_sm * sms) want = (long long)per_sm * sms;
            if (want < 1) want = 1;
            StepArgs sw = a;
            sw.f_in = a.f_out;
            sw.f_out = const_cast<void *>(a.f_in);
            sw.ref_in = a.ref_out;
            sw.ref_out = const_cast<Ref *>(a.ref_in);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)want, 1, 1);
            cfg.blockDim = dim3(kPersistThreads, 1, 1);
            cfg.stream = a.stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            record_event(a, 0);
            for (int done = 0; done < n && e == cudaSuccess;) {
                const int chunk = n - done < kPersistMaxUpdates ? n - done : kPersistMaxUpdates;
                const int wm = done + chunk == n ? a.write_macro : 0;
                e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), a.stream);
                if (e == cudaSuccess) {
                    const StepArgs &x0 = (done & 1) ? sw : a, &x1 = (done & 1) ? a : sw;
                    e = owned ? cudaLaunchKernelEx(&cfg, k_persist_c<S, EQ, true>, x0, x1, chunk, wm, a.bar)
                              : cudaLaunchKernelEx(&cfg, k_persist_c<S, EQ, false>, x0, x1, chunk, wm, a.bar);
                }
                done += chunk;
            }
            record_event(a, 1);
        };
        switch (collide_variant(a) & 3) {
        case 0: run(std::integral_constant<int, 0>{}); break;
        case 1: run(std::integral_constant<int, 1>{}); break;
        case 2: run(std::integral_constant<int, 2>{}); break;
        default: run(std::integral_constant<int, 3>{}); break;
        }
        return e;
    }
}

// parts: bit 0 the density pass, bit 1 the collision pass (both: one update;
// one at a time: the split update of a domain decomposition, with the ghost
// planes exchanged in between)
template <class S>
cudaError_t launch_compact_t(const StepArgs &a, int parts) {
    const long long m = a.list_max > 0 ? a.list_max : 1;
    const dim3 gp((unsigned)((m + kPsiThreads - 1) / kPsiThreads), (unsigned)a.batch, 1);
    const dim3 gc((unsigned)((m + kCollideThreads - 1) / kCollideThreads), (unsigned)a.batch, 1);
    record_event(a, 0);
    if (parts & 1) {
        if (a.slip)
            k_psi_c<S, true><<<gp, kPsiThreads, 0, a.stream>>>(a);
        else
            k_psi_c<S, false><<<gp, kPsiThreads, 0, a.stream>>>(a);
    }
    record_event(a, 1);
    // (a persistent variant that prefetches the next cell with cp.async, as the
    // psi pass does, measured 10 % slower here: the update is issue-bound, and
    // the prefetch buffers cost occupancy and registers)
    if (parts & 2) {
        dispatch_variant(collide_variant(a), [&](auto v) {
            constexpr int EQ = decltype(v)::value;
            if constexpr (packed_pairs<S>())
                k_collide_c2<S, EQ><<<gc, kCollideThreads, 0, a.stream>>>(a);
            else
                k_collide_c<S, EQ><<<gc, kCollideThreads, 0, a.stream>>>(a);
        });
    }
    record_event(a, 2);
    return cudaGetLastError();
}

}  // namespace lbm
