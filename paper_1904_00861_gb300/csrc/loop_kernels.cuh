// The device code of the pseudo-time loop of Algorithm 2 (particles frozen in
// pseudo-time) and of the end of the real step, shared by the translation units
// that instantiate its kernels (iterate.cu: the pair-cache form; iterate_fa.cu:
// the form that recomputes the pair geometry).
//
// One iteration k, for every fluid particle at once (Jacobi: reads only the
// iterate k buffers, writes the k+1 buffers):
//   rates at (V^k, p^{k+1/2}) from the pair cache       Eqs. (dp-dtau-frozen-edac,
//                                                        mom-sph-frozen)
//   dV/dtau = {F - (3 V^k - 4 V^n + V^{n-1})/(2 dt)} 2 dt / (2 dt + 3 dtau)
//                                                        Eq. (dv_dtau_exact)
//   V^{k+1} = V^k + dtau dV/dtau                         Eq. (vkp1_frozen)
//   p^{k+1} = p^{k+1/2} + dtau/2 dp/dtau                 Eq. (pkp1_frozen)
//   p^{k+3/2} = p^{k+1} + dtau/2 dp/dtau                 Eq. (pkstar_frozen), the
//                                                        next half step with the
//                                                        rate just computed
// The pressure is carried as p-hat^k = p^{k+1/2}, so p-hat^{k+1} = p-hat^k +
// dtau dp/dtau and p^{k+1} = (p-hat^k + p-hat^{k+1}) / 2.
// Residuals of Eq. (conv): R_p = mean|dp/dtau| dt / (rho0 c^2) and
// R_v = mean|dt dV/dtau| / v_ref over the fluid particles.
//
// Two drivers run the same per-tile arithmetic (so they give bit-identical
// results):
//  - k_iterate: one launch per iteration; the last block to finish reduces the
//    per-tile residual partials in a fixed order, applies the stop rules of
//    Sec. 3.4 and sets the condition of the graph's while node.
//  - k_loop: one cooperative launch runs every iteration of the real step; the
//    blocks meet at a grid barrier after each iteration, and every block reduces
//    the same partials in the same order and takes the same stop decision.
#pragma once

#include <algorithm>

#include "bulk.cuh"
#include "geometry.cuh"
#include "loop_rules.cuh"
#include "pair_terms.cuh"

namespace dtsph {

namespace {

inline int blocks(int n) { return (n + kBlock - 1) / kBlock; }

// Lanes per wall slot in the wall phase of an iteration (a warp serves
// 32 / kWallLanes wall slots).
constexpr int kWallLanes = 8;

// Wall values of wall slot s for the iteration whose iterate sits in buffer
// cur, from the cached fluid neighbours of the slot, by the kWallLanes lanes of
// a group (sub: lane in the group; gmask: the group's lanes in the warp). Lane
// sub takes entries sub, sub + kWallLanes, ..., R of them in flight (their
// coefficients, then their neighbour gathers); the lanes' partial sums then
// merge in a fixed order, so every run gives the same bits. Adami et al.:
// p_w = sum_f (p_f W + rho0 (g . r_wf) W) / sum_f W (the second term cached as
// Wg), ghost velocity 2 v_w - sum_f V_f W / sum_f W.
template <int D, bool F32>
__device__ __forceinline__ void wall_slot(const Buffers &B, int s, int cur, int sub, unsigned gmask)
{
    constexpr int R = 2;
    const int cnt = B.pcount[s];
    const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
    double acc[5] = {0, 0, 0, 0, 0};    // sum W, sum (p W + Wg), sum V W
    for (int k0 = sub; k0 < cnt; k0 += kWallLanes * R) {
        double W[R], Wg[R];
        uint32_t jb[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const size_t e = base + (size_t)min(k0 + r * kWallLanes, cnt - 1) * kWarp;
            if (F32) {
                const float4 c = B.pc32[e];
                W[r] = c.x;
                Wg[r] = c.y;
                jb[r] = D == 2 ? __float_as_uint(c.w) : B.pj[e];
            } else {
                const double4_32a c = B.pc64[e];
                W[r] = c.x;
                Wg[r] = c.y;
                jb[r] = B.pj[e];
            }
        }
        double q[R][4];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = (int)(jb[r] & ~kWallBit);     // a wall entry's slot is read and not used
            if (F32) {
                const float4 v = B.nb32[cur][j];
                q[r][0] = v.x; q[r][1] = v.y; q[r][2] = v.z; q[r][3] = v.w;
            } else {
                const double4_32a v = B.nb64[cur][j];
                q[r][0] = v.x; q[r][1] = v.y; q[r][2] = v.z; q[r][3] = v.w;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (k0 + r * kWallLanes >= cnt || (jb[r] & kWallBit)) continue;   // fluid neighbours only
            acc[0] += W[r];
            acc[1] += q[r][3] * W[r] + Wg[r];
            acc[2] += q[r][0] * W[r];
            acc[3] += q[r][1] * W[r];
            acc[4] += q[r][2] * W[r];
        }
    }
#pragma unroll
    for (int o = kWallLanes / 2; o > 0; o >>= 1)
#pragma unroll
        for (int t = 0; t < 5; ++t) acc[t] += __shfl_xor_sync(gmask, acc[t], o);
    if (sub != 0) return;
    const double sw = acc[0];
    double gv[3];
    for (int a = 0; a < 3; ++a) {
        const double vw = a < D ? B.vn_a[(size_t)a * B.n + s] : 0.0;
        gv[a] = 2.0 * vw - (sw > 0 ? acc[2 + a] / sw : 0.0);
    }
    double pw = sw > 0 ? acc[1] / sw : 0.0;
    if (pw < 0.0 && B.phys[B.inst_of[s]].free_surface) pw = 0.0;   // free-surface runs (Sec. 3.2)
    if (F32) B.nb32[cur][s] = make_float4((float)gv[0], (float)gv[1], (float)gv[2], (float)pw);
    else B.nb64[cur][s] = make_double4_32a(gv[0], gv[1], gv[2], pw);
}

// The lanes of thread t's wall group: its lane in the group and the group's mask.
__device__ __forceinline__ void wall_group(int t, int &sub, unsigned &gmask)
{
    const int lane = t & 31;
    sub = lane & (kWallLanes - 1);
    gmask = ((1u << kWallLanes) - 1u) << (lane & ~(kWallLanes - 1));
}

// Wall values for iteration k (one launch per iteration), kWallLanes lanes per
// wall particle of the wall list.
template <int D, bool F32>
__global__ void __launch_bounds__(kBlock) k_walls_iter(Buffers B)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = t / kWallLanes;                        // the same for the whole group
    if (w >= B.nw) return;
    const int s = B.wslot_a[w];
    const LoopState *ls = B.ls + B.inst_of[s];
    if (ls->done) return;
    int sub;
    unsigned gmask;
    wall_group(t, sub, gmask);
    wall_slot<D, F32>(B, s, ls->iter & 1, sub, gmask);
}

// One entry of the pair cache in registers.
template <typename T, int D, bool F32>
struct CacheEntry {
    T g[3];
    T F;
    uint32_t jb;
    __device__ __forceinline__ void load(const Buffers &B, size_t e)
    {
        if (F32) {
            const float4 c = B.pc32[e];
            g[0] = (T)c.x;
            g[1] = (T)c.y;
            if (D == 3) {
                g[2] = (T)c.z;
                F = (T)c.w;
                jb = B.pj[e];
            } else {
                g[2] = T(0);
                F = (T)c.z;
                jb = __float_as_uint(c.w);
            }
        } else {
            const double4_32a c = B.pc64[e];
            g[0] = (T)c.x;
            g[1] = (T)c.y;
            g[2] = (T)c.z;
            F = (T)c.w;
            jb = B.pj[e];
        }
    }
};

// Pair-cache rows of one warp in shared memory (one lane per slot). The 32 slots
// of the warp form one slice of the sliced cache, so their entries k = 0, 1, ...
// are consecutive rows (32 coefficient records, then, where the index is kept
// apart, 32 indices). Chunks of kRows rows arrive by bulk copies into a ring of
// S stages (S - 1 chunks in flight while one is used), each completing on its
// stage's mbarrier. The ring of warp w sits at w * stride(S) in dynamic shared
// memory: S stages, then S barriers.
template <int D, bool F32>
struct RowFmt {
    static constexpr int kCoef = F32 ? 16 : 32;                 // bytes of one coefficient record
    static constexpr bool kSepJ = !(F32 && D == 2);             // index in pj (2D FP32C: in .w)
    static constexpr int kRows = F32 ? 4 : 2;                   // rows per chunk
    static constexpr int kCoefRow = kWarp * kCoef;
    static constexpr int kJRow = kSepJ ? kWarp * 4 : 0;
    static constexpr int kStageBytes = kRows * (kCoefRow + kJRow);
    static __host__ __device__ constexpr size_t stride(int S)
    {
        return ((size_t)S * kStageBytes + (size_t)S * 8 + 127) / 128 * 128;
    }
};

// Dynamic shared memory of the one-lane kernels for S stages: one ring per warp.
template <int D, bool F32>
__host__ __device__ constexpr size_t ring_bytes(int S)
{
    return RowFmt<D, F32>::stride(S) * (kBlock / kWarp);
}

template <int D, bool F32>
struct WarpRing {
    unsigned char *buf;    // stage st at buf + st * kStageBytes
    uint64_t *bar;         // S barriers
    int S;
};

template <typename T, int D, int L>
struct TileShared {
    T part[D + 1][kBlock / L];
    double red[2][kBlock / kWarp];
};

extern __shared__ __align__(128) unsigned char dyn_smem[];

// Bulk-copy state of a warp's ring, kept across tiles: chunks consumed so far
// (stage = pos % S, phase parity = (pos / S) & 1), and whether every
// wait so far completed.
struct RingPos {
    uint32_t pos = 0;
    bool ok = true;
};

// This warp's ring in dynamic shared memory (one-lane kernels only).
template <int D, bool F32>
__device__ __forceinline__ WarpRing<D, F32> warp_ring(int S)
{
    using RF = RowFmt<D, F32>;
    unsigned char *base = dyn_smem + (size_t)(threadIdx.x >> 5) * RF::stride(S);
    return WarpRing<D, F32>{base, reinterpret_cast<uint64_t *>(base + (size_t)S * RF::kStageBytes), S};
}

// Initialises the mbarriers of every warp's ring (whole block, then syncs).
template <int D, bool F32, int L>
__device__ __forceinline__ void ring_init(int S)
{
    if constexpr (L == 1) {
        if ((threadIdx.x & 31) == 0) {
            const WarpRing<D, F32> rg = warp_ring<D, F32>(S);
            for (int st = 0; st < S; ++st) mbar_init(&rg.bar[st], 1);
            mbar_fence_init();
        }
    }
    __syncthreads();
}

// The prescribed velocity of list entry jb's particle if it is a wall particle
// (the V_j of the divergence term; the packed copy of V^n of order A, in the
// working precision), else zeros. Issued with the neighbour-state gathers.
template <int D, bool F32, typename T>
__device__ __forceinline__ void wall_velocity(const Buffers &B, uint32_t jb, T *vw)
{
    vw[0] = vw[1] = vw[2] = T(0);
    if (!(jb & kWallBit)) return;
    const int j = (int)(jb & ~kWallBit);
    if constexpr (F32) {
        if (D == 2) {
            const float2 w = *reinterpret_cast<const float2 *>(&B.wv32[j]);
            vw[0] = (T)w.x;
            vw[1] = (T)w.y;
        } else {
            const float4 w = B.wv32[j];
            vw[0] = (T)w.x;
            vw[1] = (T)w.y;
            vw[2] = (T)w.z;
        }
    } else {
        if (D == 2) {
            const double2 w = *reinterpret_cast<const double2 *>(&B.wv64[j]);
            vw[0] = (T)w.x;
            vw[1] = (T)w.y;
        } else {
            const double4_32a w = B.wv64[j];
            vw[0] = (T)w.x;
            vw[1] = (T)w.y;
            vw[2] = (T)w.z;
        }
    }
}

// The working precision of the pair sums: FP32 on the FP32C path, else FP64.
template <bool F32>
using Real = typename std::conditional<F32, float, double>::type;

// Phase 1 of an iteration for slot s: L lanes per particle split its cached pair
// list (lane l takes entries l, l+L, ...), accumulate the two rates
// (Kahan-compensated FP32 on the FP32C path) and merge their partial sums with
// warp shuffles; with one lane the warp's rows stream through the warp's
// shared-memory ring. The rates, in the working precision, are valid on lane
// lane_in = 0 of the particle's group.
template <int D, bool F32, bool WALLS, int L, bool FA = false>
__device__ __forceinline__ void pair_sums(const Buffers &B, const Phys &P, const Geom &G, int cur, int s, int lane_in,
                                          bool active, RingPos &rp, Real<F32> &apT, Real<F32> *FT)
{
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    const PairConst<T> k = pair_const<T>(P);
    T vi[3] = {T(0), T(0), T(0)}, pi = T(0);
    int cnt = 0;
    if (active) {
        if (F32) {
            float4 q = B.nb32[cur][s];
            vi[0] = q.x; vi[1] = q.y; vi[2] = q.z; pi = q.w;
        } else {
            double4_32a q = B.nb64[cur][s];
            vi[0] = (T)q.x; vi[1] = (T)q.y; vi[2] = (T)q.z; pi = (T)q.w;
        }
        cnt = B.pcount[s];
    }
    Acc ap, Fa[3];
    // the pair terms of one cache entry with its gathered neighbour state
    using Q = typename std::conditional<F32, float4, double4_32a>::type;
    const Q *nbq = F32 ? (const Q *)(const void *)B.nb32[cur] : (const Q *)(const void *)B.nb64[cur];
    // vw: the prescribed velocity of a wall neighbour (the divergence term's
    // V_j), gathered with the neighbour states
    // (one call for both kinds of neighbour: a warp whose lanes hold both runs
    // the pair arithmetic once)
    auto pair = [&](const CacheEntry<T, D, F32> &ce, const Q &q, const T *vw) {
        const T vj[3] = {(T)q.x, (T)q.y, (T)q.z};
        const T pj = (T)q.w;
        if constexpr (WALLS) {
            const bool wall = (ce.jb & kWallBit) != 0;
            const T vd[3] = {wall ? vw[0] : vj[0], wall ? vw[1] : vj[1], wall ? vw[2] : vj[2]};
            pair_accumulate<D, T, Acc>(k, ce.g, ce.F, vi, pi, vd, vj, pj, ap, Fa);
        } else {
            pair_accumulate<D, T, Acc>(k, ce.g, ce.F, vi, pi, vj, vj, pj, ap, Fa);
        }
    };
    if constexpr (FA) {
        // Form A: the geometry of every pair recomputed from the lists at r^0
        // with k_pair_cache's operations (offset_sep or listed_sep, then
        // grad_coef), so every coefficient has the bits the cache would hold and
        // both forms give the same results; the entries keep the order of the
        // cached rows (lane l takes l, l + L, ..., R in flight per round)
        static_assert(!WALLS, "the wall values come from the cache");
        const uint32_t *lst = slot_list(B, s);
        const float4 oi = F32 && active ? B.off[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        constexpr int R = 4;
        for (int q0 = lane_in; q0 < cnt; q0 += L * R) {
            uint32_t jbv[R];
            if constexpr (L == 1) {
                // four consecutive entries in one 16-byte load; an entry past the
                // count repeats entry q0, so its gathers stay in bounds
                const uint4 v = *reinterpret_cast<const uint4 *>(lst + q0);
                jbv[0] = v.x;
                jbv[1] = q0 + 1 < cnt ? v.y : v.x;
                jbv[2] = q0 + 2 < cnt ? v.z : v.x;
                jbv[3] = q0 + 3 < cnt ? v.w : v.x;
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) jbv[r] = lst[min(q0 + r * L, cnt - 1)];
            }
            float4 ov[R];
            Q qv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = entry_slot(jbv[r]);
                ov[r] = F32 ? B.off[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                qv[r] = nbq[j];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (q0 + r * L >= cnt) break;
                const int code = entry_code(jbv[r]);
                T d[3], r2;
                if constexpr (F32) {
                    offset_sep<D, T>(G, oi, ov[r], code, d, r2);
                } else {
                    int dx, dy, dz;
                    decode_shift(code, dx, dy, dz);
                    listed_sep<D, F32, T>(G, B.xp_a, B.off, B.n, s, entry_slot(jbv[r]), oi, dx, dy, dz, d, r2);
                }
                T g[3], F;
                grad_coef<D, T>(P, d, r2, g, F);
                CacheEntry<T, D, F32> ce;
                ce.g[0] = g[0];
                ce.g[1] = g[1];
                ce.g[2] = D == 3 ? g[2] : T(0);
                ce.F = F;
                ce.jb = jbv[r] & ~kCodeMask;
                pair(ce, qv[r], nullptr);
            }
        }
    } else if constexpr (L == 1) {
        // the warp's rows stream through its shared-memory ring; the
        // neighbour states of a chunk's rows are gathered together
        using RF = RowFmt<D, F32>;
        constexpr int R = RF::kRows;
        const int S = B.stages;
        constexpr unsigned full = 0xffffffffu;
        const int lane = threadIdx.x & 31;
        const WarpRing<D, F32> rg = warp_ring<D, F32>(S);
        const int cmax = __reduce_max_sync(full, cnt);
        const int nch = rp.ok ? (cmax + R - 1) / R : 0;
        const size_t row0 = (size_t)(s >> 5) * B.K;      // first row of the warp's slice
        const unsigned char *gcoef =
            (F32 ? (const unsigned char *)B.pc32 : (const unsigned char *)B.pc64) + row0 * RF::kCoefRow;
        const unsigned char *gj = (const unsigned char *)B.pj + row0 * (kWarp * 4);
        // a cache larger than L2 streams through it once per pass (first to
        // leave); a smaller one stays like the rest; the neighbour states,
        // gathered again every pass, stay
        const uint64_t pol_stream = B.l2_stream ? l2_policy_evict_first() : l2_policy_evict_normal();
        const uint64_t pol_keep = l2_policy_evict_last();
        auto issue = [&](int c) {        // lane 0: chunk c into its stage
            const int st = (int)((rp.pos + (uint32_t)c) % (uint32_t)S);
            const int r0 = c * R, nr = min(R, cmax - r0);
            const uint32_t bc = (uint32_t)(nr * RF::kCoefRow), bj = (uint32_t)(nr * RF::kJRow);
            unsigned char *stg = rg.buf + (size_t)st * RF::kStageBytes;
            mbar_arrive_expect_tx(&rg.bar[st], bc + bj);
            bulk_g2s_hint(stg, gcoef + (size_t)r0 * RF::kCoefRow, bc, &rg.bar[st], pol_stream);
            if (RF::kSepJ)
                bulk_g2s_hint(stg + R * RF::kCoefRow, gj + (size_t)r0 * RF::kJRow, bj, &rg.bar[st], pol_stream);
        };
        if (lane == 0)
            for (int c = 0; c < S && c < nch; ++c) issue(c);
        int c = 0;
        for (; c < nch; ++c) {
            const uint32_t q = rp.pos + (uint32_t)c;
            const int st = (int)(q % (uint32_t)S);
            if (!mbar_wait(&rg.bar[st], (q / (uint32_t)S) & 1u)) break;
            const int r0 = c * R, nr = min(R, cmax - r0);
            const unsigned char *stg = rg.buf + (size_t)st * RF::kStageBytes;
            // gather the neighbour states of the chunk's rows first (R loads
            // in flight per lane), then run the pair terms
            uint32_t jbv[R];
            Q qv[R];
            T wv[R][3];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr && r0 + r < cnt) {
                    jbv[r] = RF::kSepJ
                                 ? ((const uint32_t *)(stg + R * RF::kCoefRow + r * RF::kJRow))[lane]
                                 : __float_as_uint(((const float4 *)(stg + r * RF::kCoefRow))[lane].w);
                    if constexpr (F32)
                        qv[r] = ld_f4_hint(reinterpret_cast<const float4 *>(nbq) + (jbv[r] & ~kWallBit), pol_keep);
                    else
                        qv[r] = nbq[jbv[r] & ~kWallBit];
                    if constexpr (WALLS) wall_velocity<D, F32, T>(B, jbv[r], wv[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < nr && r0 + r < cnt) {
                    CacheEntry<T, D, F32> ce;
                    if (F32) {
                        const float4 v = ((const float4 *)(stg + r * RF::kCoefRow))[lane];
                        ce.g[0] = (T)v.x;
                        ce.g[1] = (T)v.y;
                        ce.g[2] = D == 3 ? (T)v.z : T(0);
                        ce.F = D == 3 ? (T)v.w : (T)v.z;
                    } else {
                        const double4_32a v = ((const double4_32a *)(stg + r * RF::kCoefRow))[lane];
                        ce.g[0] = (T)v.x;
                        ce.g[1] = (T)v.y;
                        ce.g[2] = (T)v.z;
                        ce.F = (T)v.w;
                    }
                    ce.jb = jbv[r];
                    pair(ce, qv[r], wv[r]);
                }
            }
            __syncwarp();
            if (lane == 0 && c + S < nch) {
                fence_proxy_async_smem();
                issue(c + S);
            }
        }
        if (c < nch) {
            // a wait gave up: drain what is still in flight, the chunk
            // whose wait gave up included (each wait bounded), stop using
            // the ring and report
            for (int d = c; d < nch && d < c + S; ++d) {
                const uint32_t q = rp.pos + (uint32_t)d;
                mbar_wait(&rg.bar[q % (uint32_t)S], (q / (uint32_t)S) & 1u);
            }
            rp.ok = false;
            if (lane == 0) atomicOr(B.err, kErrCopy);
        }
        rp.pos += (uint32_t)nch;
    } else {
        const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
        // R entries per round: their cache entries, then their neighbour
        // gathers, then the pair terms, so R loads of each kind are in flight
        // per lane (the entries keep the order lane_in, lane_in + L, ...)
        constexpr int R = 4;
        for (int k0 = lane_in; k0 < cnt; k0 += L * R) {
            CacheEntry<T, D, F32> ce[R];
#pragma unroll
            for (int r = 0; r < R; ++r) ce[r].load(B, base + (size_t)min(k0 + r * L, cnt - 1) * kWarp);
            Q qv[R];
            T wv[R][3];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                qv[r] = nbq[ce[r].jb & ~kWallBit];
                if constexpr (WALLS) wall_velocity<D, F32, T>(B, ce[r].jb, wv[r]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (k0 + r * L < cnt) pair(ce[r], qv[r], wv[r]);
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        ap.shfl_merge(o);
#pragma unroll
        for (int a = 0; a < D; ++a) Fa[a].shfl_merge(o);
    }
    apT = (T)ap.value();
#pragma unroll
    for (int a = 0; a < D; ++a) FT[a] = (T)Fa[a].value();
}

// Phase 2 of an iteration: the BDF2 pseudo-acceleration and update, FP64
// kappa (F + g - (3 V^k - 4 V^n + V^{n-1}) / (2 dt)), with the state-n part
// kappa ((V^{n-1} - 4 V^n) / (2 dt) - g) precomputed in s_a; V^{k+1} in FP64.
// On the FP32C path everything past the FP64 velocity update (the FP32
// copies, p-hat, the residual terms) stays in FP32, to keep conversions off
// the FP64 pipe: the residual terms are summed per warp with error-free
// two-sum compensation (a double-float sum, accurate to ~1e-12 of the total)
// and the warp totals are carried on in FP64. The FP64 path sums in FP64.
// For slot s2 (fl: a fluid slot) with its rates apT, FT from phase 1, by every
// lane of the warp; the warp's residual sums come back on lane 0.
template <int D, bool F32>
__device__ __forceinline__ void update_and_residuals(const Buffers &B, const Phys &P, int cur, int s2, bool fl,
                                                     Real<F32> apT, const Real<F32> *FT, double &w_ap, double &w_av)
{
    const int nxt = cur ^ 1;
    const int n = B.n;
    if (F32) {
        float r_ap = 0.f, r_av = 0.f;
        if (fl) {
            const float apf = (float)apT;
            float vnf[3] = {0.f, 0.f, 0.f};
            float av2 = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const size_t q = (size_t)a * n + s2;
                const double vk = B.vk[cur][q];
                const double Fv = (double)FT[a];
                const double av = __fma_rn(P.kappa, Fv, -__fma_rn(P.kc3, vk, B.s_a[q]));
                const double vnew = __fma_rn(P.dtau, av, vk);
                B.vk[nxt][q] = vnew;
                vnf[a] = (float)vnew;
                const float avf = (float)av;
                av2 = __fmaf_rn(avf, avf, av2);
            }
            const float pnew = __fmaf_rn(P.dtau_f, apf, B.nb32[cur][s2].w);
            B.nb32[nxt][s2] = make_float4(vnf[0], vnf[1], vnf[2], pnew);
            r_av = sqrtf(av2);
            r_ap = fabsf(apf);
        }
        float sa = r_ap, ea = 0.f, sb = r_av, eb = 0.f;
        warp_sum2(sa, ea);
        warp_sum2(sb, eb);
        w_ap = (threadIdx.x & 31) == 0 ? (double)sa + (double)ea : 0.0;
        w_av = (threadIdx.x & 31) == 0 ? (double)sb + (double)eb : 0.0;
    } else {
        double r_ap = 0.0, r_av = 0.0;
        if (fl) {
            const double apv = (double)apT;
            double vnew[3] = {0, 0, 0};
            double av2 = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const size_t q = (size_t)a * n + s2;
                const double vk = B.vk[cur][q];
                const double Fv = (double)FT[a];
                const double av = __fma_rn(P.kappa, Fv, -__fma_rn(P.kc3, vk, B.s_a[q]));
                vnew[a] = __fma_rn(P.dtau, av, vk);
                B.vk[nxt][q] = vnew[a];
                av2 = __fma_rn(av, av, av2);
            }
            const double pnew = __fma_rn(P.dtau, apv, B.nb64[cur][s2].w);
            B.nb64[nxt][s2] = make_double4_32a(vnew[0], vnew[1], vnew[2], pnew);
            r_av = sqrt(av2);
            r_ap = fabs(apv);
        }
        w_ap = warp_sum<double>(r_ap);
        w_av = warp_sum<double>(r_av);
    }
}

// One iteration over tile `tile` (slots tile*PPB .. tile*PPB+PPB-1, PPB = 256/L),
// by the whole block. Writes iterate k+1 of the tile's fluid particles and
// returns, on thread 0, the tile's residual sums (sum |dp/dtau|, sum |dV/dtau|):
// the warps' sums added in warp order. The tile's particles are a contiguous run
// of slots, so the warp reads of the sliced pair cache stay coalesced. Phase 2
// runs one thread per particle (the first PPB threads, whole warps, so the FP64
// work runs with every lane busy); with one lane per particle that thread is the
// particle's phase-1 lane, so the rates stay in registers.
template <int D, bool F32, bool WALLS, int L, bool FA = false>
__device__ __forceinline__ void tile_iteration(const Buffers &B, const Phys &P, const Geom &G, int cur, int tile,
                                               TileShared<typename std::conditional<F32, float, double>::type, D, L> &sh,
                                               RingPos &rp, double &blk_ap, double &blk_av)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int PPB = kBlock / L;
    static_assert(PPB % kWarp == 0, "whole warps in phase 2");
    const int n = B.n;
    const int grp = threadIdx.x / L, lane_in = threadIdx.x % L;
    const int s = tile * PPB + grp;
    const bool active = s < n && B.gid_a[s] < (uint32_t)B.nf;   // fluid (not wall, not padding)
    T apT = T(0), FT[3] = {T(0), T(0), T(0)};
    pair_sums<D, F32, WALLS, L, FA>(B, P, G, cur, s, lane_in, active, rp, apT, FT);
    double w_ap = 0, w_av = 0;
    if constexpr (L == 1) {
        update_and_residuals<D, F32>(B, P, cur, s, active, apT, FT, w_ap, w_av);
    } else {
        if (lane_in == 0) {
            sh.part[0][grp] = apT;
#pragma unroll
            for (int a = 0; a < D; ++a) sh.part[1 + a][grp] = FT[a];
        }
        __syncthreads();
        if (threadIdx.x < PPB) {
            const int s2 = tile * PPB + threadIdx.x;
            const bool fl = s2 < n && B.gid_a[s2] < (uint32_t)B.nf;
            T fq[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int a = 0; a < D; ++a) fq[a] = sh.part[1 + a][threadIdx.x];
            update_and_residuals<D, F32>(B, P, cur, s2, fl, sh.part[0][threadIdx.x], fq, w_ap, w_av);
        }
    }
    if (threadIdx.x < PPB && (threadIdx.x & 31) == 0) {
        sh.red[0][threadIdx.x >> 5] = w_ap;
        sh.red[1][threadIdx.x >> 5] = w_av;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < PPB / kWarp; ++w) {
            a += sh.red[0][w];
            b += sh.red[1][w];
        }
        blk_ap = a;
        blk_av = b;
    }
    __syncthreads();   // sh is reused by the next tile
}

// One pseudo-time iteration over all slots; one tile per block. The last block
// of an instance's tiles reduces that instance's partials in a fixed order and
// applies its stop rules; the last block of all sets the while-node condition
// (some instance still iterating).
template <int D, bool F32, bool WALLS, int L, bool FA = false>
__global__ void __launch_bounds__(kBlock, L == 1 && !FA ? (F32 ? (D == 2 ? 4 : 3) : 1) : (F32 ? 3 : 1))
    k_iterate(Buffers B, unsigned long long cond, int use_cond)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int PPB = kBlock / L;
    __shared__ TileShared<T, D, L> sh;
    __shared__ Phys P;
    __shared__ Geom G;
    __shared__ int last, tlo_sh;
    if (!use_cond && B.ctrl->active == 0) return;     // whole grid agrees: nothing to do
    // (ring_init ends with the barrier that publishes thread 0's set-up of the
    // block's shared state; without the ring the barrier stays)
    if constexpr (!FA) ring_init<D, F32, L>(B.stages);
    else __syncthreads();
    RingPos rp;
    const int inst = block_instance(B, blockIdx.x * PPB);
    LoopState *ls = B.ls + inst;
    int tlo, thi;
    instance_tiles(B.inst[inst], PPB, tlo, thi);
    const bool mine = (int)blockIdx.x < thi;          // false: a tile made of padding only
    const int it = ls->iter;
    const bool work = mine && !ls->done;
    if (work) {
        for (int w = threadIdx.x; w < (int)(sizeof(Phys) / 4); w += blockDim.x)
            reinterpret_cast<int *>(&P)[w] = reinterpret_cast<const int *>(B.phys + inst)[w];
        if constexpr (FA)
            for (int w = threadIdx.x; w < (int)(sizeof(Geom) / 4); w += blockDim.x)
                reinterpret_cast<int *>(&G)[w] = reinterpret_cast<const int *>(B.geo + inst)[w];
        __syncthreads();
        double a = 0, b = 0;
        tile_iteration<D, F32, WALLS, L, FA>(B, P, G, it & 1, blockIdx.x, sh, rp, a, b);
        if (threadIdx.x == 0) {
            B.blk[2 * blockIdx.x] = a;
            B.blk[2 * blockIdx.x + 1] = b;
            __threadfence();
            const unsigned int t = atomicAdd(&ls->ticket, 1u);
            last = (t == (unsigned int)(thi - tlo - 1));
            tlo_sh = tlo;
        }
        __syncthreads();
        if (last) {
            // last tile of this instance: fixed-order reduction of its partials
            __threadfence();
            double sa = 0, sb = 0;
            reduce_tiles(B.blk + 2 * tlo_sh, thi - tlo_sh, sh.red, sa, sb);
            if (threadIdx.x == 0) {
                const int r = finish_iteration(ls, P, it, sa, sb);
                ls->ticket = 0;
                if (r != -1) atomicSub(&B.ctrl->active, 1);
                __threadfence();
            }
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(&B.ctrl->ticket, 1u);
        if (t == gridDim.x - 1) {
            B.ctrl->ticket = 0;
            __threadfence();
            const int active = *(volatile int *)&B.ctrl->active;
            if (use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, active > 0 ? 1u : 0u);
        }
    }
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier for a cooperative launch (all blocks resident): arrival counter
// `bar`, reset to 0 before the launch; the epoch-th barrier waits for
// epoch * gridDim.x arrivals. The wait gives up after limit_ns (one second
// unless a test shortens it), raises kErrBarrier and returns false (the caller
// then stops iterating).
__device__ bool grid_barrier(unsigned int *bar, unsigned int epoch, uint32_t *err, int &ok_sh,
                             unsigned long long limit_ns)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = epoch * gridDim.x;
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        const unsigned long long t0 = global_ns();
        while (*(volatile unsigned int *)bar < target) {
            __nanosleep(32);
            if (global_ns() - t0 > limit_ns) {
                atomicOr(err, kErrBarrier);
                ok = 0;
                break;
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Exclusive prefix of the active (not yet converged) tiles of every instance,
// by the whole block: pre[i] = active tiles of instances 0 .. i-1, pre[ninst] =
// all of them. Reads the instances' done flags, so call it after the barrier
// that publishes them.
__device__ void active_tile_prefix(const Buffers &B, int ppb, int *pre)
{
    constexpr int E = (kDealMaxInst + kBlock - 1) / kBlock;
    __shared__ int wsum[kBlock / kWarp];
    const int ni = B.ninst;
    const int base = threadIdx.x * E;
    int cnt[E];
    int sum = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = base + e;
        int c = 0;
        if (i < ni && !*(volatile int *)&B.ls[i].done) {
            int lo, hi;
            instance_tiles(B.inst[i], ppb, lo, hi);
            c = hi - lo;
        }
        cnt[e] = c;
        sum += c;
    }
    // exclusive scan of the per-thread sums: within the warp, then over warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < wid; ++w) off += wsum[w];
    int run = off + incl - sum;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = base + e;
        if (i <= ni) pre[i] = run;
        run += cnt[e];
    }
    __syncthreads();
}

// The instance whose active tiles hold position k of the dealt order
// (pre[0] = 0 <= k < pre[ni]).
__device__ __forceinline__ int dealt_instance(const int *pre, int ni, int k)
{
    int lo = 0, hi = ni;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= k) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Every pseudo-time iteration of one real step in one cooperative launch. Tiles
// are dealt to blocks round robin: with one instance all tiles, with several
// (up to kDealMaxInst) the tiles of the instances still iterating, so that
// every block keeps an even share while converged instances drop out; after
// each iteration the blocks meet at a grid barrier. With one instance every block then reduces the per-tile
// partials (double-buffered on the iteration parity) in the fixed order of
// k_iterate and all blocks take the same stop decision. With several, block b
// finishes instances b, b + grid, ... and a second barrier publishes the
// decisions; tiles of finished instances are skipped. Walls get their own phase
// and barrier before the fluid phase.
template <int D, bool F32, bool WALLS, int L, bool FA = false>
__global__ void __launch_bounds__(kBlock, L == 1 && !FA ? ((F32 && D == 2 && !WALLS) ? 4 : 3) : (F32 ? 3 : 2))
    k_loop(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int PPB = kBlock / L;
    __shared__ TileShared<T, D, L> sh;
    __shared__ LoopState st;
    __shared__ Phys P;
    __shared__ Geom G;
    __shared__ int stop, ok_sh, p_inst;
    __shared__ int act_pre[kDealMaxInst + 1];
    if constexpr (!WALLS) {
        if (skip_form(B)) return;         // the step runs the other pair-term form
    }
    const int ntiles = (B.n + PPB - 1) / PPB;
    const bool single = B.ninst == 1;
    const bool deal = !single && B.ninst <= kDealMaxInst;
    if (threadIdx.x == 0) {
        if (single) st = *B.ls;
        stop = 0;
        p_inst = -1;
    }
    // (ring_init ends with the barrier that publishes thread 0's set-up of the
    // block's shared state; without the ring the barrier stays)
    if constexpr (!FA) ring_init<D, F32, L>(B.stages);
    else __syncthreads();
    RingPos rp;
    unsigned int epoch = 0;
    // (one instance: from the loop state's iteration, 0 at the start of a step,
    // the pause count when a loop without the cache goes on with it)
    int r = -1, it = single ? st.iter : 0;
    for (;; ++it) {
        const int cur = it & 1;
        if (WALLS) {
            // the wall list, kWallLanes lanes per wall particle
            int sub;
            unsigned gmask;
            wall_group(threadIdx.x, sub, gmask);
            constexpr int GPB = kBlock / kWallLanes;
            for (int w = blockIdx.x * GPB + (int)threadIdx.x / kWallLanes; w < B.nw; w += gridDim.x * GPB) {
                const int s = B.wslot_a[w];
                // (one instance: it is iterating, no need to look)
                if (single || !B.ls[B.inst_of[s]].done) wall_slot<D, F32>(B, s, cur, sub, gmask);
            }
            if (!grid_barrier(&B.ctrl->bar, ++epoch, B.err, ok_sh, B.barrier_ns)) break;
        }
        double *blk = B.blk + (size_t)(it & 1) * 2 * ntiles;
        int nwork = ntiles;
        if (deal) {
            active_tile_prefix(B, PPB, act_pre);
            nwork = act_pre[B.ninst];
        }
        for (int k = blockIdx.x; k < nwork; k += gridDim.x) {
            int inst, t, tlo, thi;
            if (deal) {
                inst = dealt_instance(act_pre, B.ninst, k);
                instance_tiles(B.inst[inst], PPB, tlo, thi);
                t = tlo + (k - act_pre[inst]);
            } else {
                t = k;
                inst = block_instance(B, t * PPB);
                instance_tiles(B.inst[inst], PPB, tlo, thi);
                if (t >= thi || (!single && *(volatile int *)&B.ls[inst].done)) continue;
            }
            if (inst != p_inst) {
                __syncthreads();
                for (int w = threadIdx.x; w < (int)(sizeof(Phys) / 4); w += blockDim.x)
                    reinterpret_cast<int *>(&P)[w] = reinterpret_cast<const int *>(B.phys + inst)[w];
                if constexpr (FA)
                    for (int w = threadIdx.x; w < (int)(sizeof(Geom) / 4); w += blockDim.x)
                        reinterpret_cast<int *>(&G)[w] = reinterpret_cast<const int *>(B.geo + inst)[w];
                __syncthreads();
                if (threadIdx.x == 0) p_inst = inst;
            }
            double a = 0, b = 0;
            tile_iteration<D, F32, WALLS, L, FA>(B, P, G, cur, t, sh, rp, a, b);
            if (threadIdx.x == 0) {
                blk[2 * t] = a;
                blk[2 * t + 1] = b;
            }
        }
        if (!grid_barrier(&B.ctrl->bar, ++epoch, B.err, ok_sh, B.barrier_ns)) break;
        if (single) {
            double sa = 0, sb = 0;
            int tlo, thi;
            instance_tiles(B.inst[0], PPB, tlo, thi);
            reduce_tiles(blk + 2 * tlo, thi - tlo, sh.red, sa, sb);
            if (threadIdx.x == 0) {
                const int k1 = it + 1;
                st.rp = sa * B.phys[0].rp_scale;
                st.rv = sb * B.phys[0].rv_scale;
                st.hist_p[it & 15] = st.rp;
                st.hist_v[it & 15] = st.rv;
                r = stop_or_pause(st, k1);
                stop = r != -1;
            }
            __syncthreads();
            if (stop) break;
        } else {
            for (int i = blockIdx.x; i < B.ninst; i += gridDim.x) {
                if (B.ls[i].done) continue;
                int tlo, thi;
                instance_tiles(B.inst[i], PPB, tlo, thi);
                double sa = 0, sb = 0;
                reduce_tiles(blk + 2 * tlo, thi - tlo, sh.red, sa, sb);
                if (threadIdx.x == 0) {
                    if (finish_iteration(B.ls + i, B.phys[i], it, sa, sb) != -1) atomicSub(&B.ctrl->active, 1);
                }
                __syncthreads();
            }
            if (!grid_barrier(&B.ctrl->bar, ++epoch, B.err, ok_sh, B.barrier_ns)) break;
            if (threadIdx.x == 0) stop = *(volatile int *)&B.ctrl->active == 0;
            __syncthreads();
            if (stop) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (single) {
            LoopState *ls = B.ls;
            const bool finished = stop != 0;
            ls->rp = st.rp;
            ls->rv = st.rv;
            for (int q = 0; q < 16; ++q) {
                ls->hist_p[q] = st.hist_p[q];
                ls->hist_v[q] = st.hist_v[q];
            }
            ls->iter = finished ? it + 1 : it;
            ls->reason = finished ? r : 3;
            ls->done = 1;
        } else if (!stop) {
            // a barrier gave up: close every instance still open
            for (int i = 0; i < B.ninst; ++i)
                if (!B.ls[i].done) {
                    B.ls[i].reason = 3;
                    B.ls[i].done = 1;
                }
        }
    }
}

// The block-wide minimum of v (every thread gets it).
__device__ __forceinline__ int block_min(int v, int *scratch)
{
    v = __reduce_min_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    int m = scratch[0];
    for (int w = 1; w < kBlock / kWarp; ++w) m = min(m, scratch[w]);
    __syncthreads();
    return m;
}

// The pseudo-time loop of a batch without walls with the instances decoupled:
// each instance advances through its iterations on its own, so the long
// iteration chains of the instances that converge slowly run beside the heavy
// iterations of the large instances instead of after them. Instance i's tiles
// of iteration k are handed out by a counter holding (k << 32) | next tile; the
// block that finishes the iteration's last tile reduces the instance's per-tile
// partials in the fixed order of k_iterate, applies the stop rules, and then
// opens iteration k + 1 or retires the instance. A block looks for an open tile
// from the smallest instances up (they take the most iterations) and waits,
// bounded by the barrier give-up time, while every open tile is taken. Every
// tile and every decision is computed as in k_loop, so the results are the
// same bits.
template <int D, bool F32, int L, bool FA = false>
__global__ void __launch_bounds__(kBlock, L == 1 && !FA ? ((F32 && D == 2) ? 4 : 3) : (F32 ? 3 : 2))
    k_loop_async(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int PPB = kBlock / L;
    __shared__ TileShared<T, D, L> sh;
    __shared__ Phys P;
    __shared__ Geom G;
    __shared__ int p_inst, w_inst, w_tile, w_it, last_sh, quit;
    __shared__ int mins[kBlock / kWarp];
    if (skip_form(B)) return;         // the step runs the other pair-term form
    const int ntiles = (B.n + PPB - 1) / PPB;
    const int ni = B.ninst;
    if (threadIdx.x == 0) p_inst = -1;
    // (ring_init ends with the barrier that publishes thread 0's set-up of the
    // block's shared state; without the ring the barrier stays)
    if constexpr (!FA) ring_init<D, F32, L>(B.stages);
    else __syncthreads();
    RingPos rp;
    unsigned long long wait_from = 0;
    bool waiting = false;
    for (;;) {
        // the first instance in search order with a tile left to hand out
        int cand = 0x7fffffff;
        for (int q = threadIdx.x; q < ni; q += kBlock) {
            const int i = B.sched[q];
            if (*(volatile int *)&B.ls[i].done) continue;
            const unsigned long long cl = *(volatile unsigned long long *)&B.il[i].claim;
            int tlo, thi;
            instance_tiles(B.inst[i], PPB, tlo, thi);
            if ((int)(cl & 0xffffffffull) < thi - tlo) {
                cand = q;
                break;
            }
        }
        cand = block_min(cand, mins);
        if (threadIdx.x == 0) {
            w_inst = -1;
            quit = 0;
            if (cand != 0x7fffffff) {
                const int i = B.sched[cand];
                int tlo, thi;
                instance_tiles(B.inst[i], PPB, tlo, thi);
                const unsigned long long old = atomicAdd(&B.il[i].claim, 1ull);
                const int t = (int)(old & 0xffffffffull);
                if (t < thi - tlo) {
                    w_inst = i;
                    w_tile = tlo + t;
                    w_it = (int)(old >> 32);
                    __threadfence();
                }
            } else if (*(volatile int *)&B.ctrl->active == 0) {
                quit = 1;
            }
            // every open tile is taken: wait, bounded, for an iteration to open
            // (thread 0 alone keeps the clock, so the block decides as one)
            if (w_inst >= 0) {
                waiting = false;
            } else if (!quit) {
                const unsigned long long now = global_ns();
                if (!waiting) {
                    waiting = true;
                    wait_from = now;
                } else if (now - wait_from > B.barrier_ns) {
                    atomicOr(B.err, kErrBarrier);
                    quit = 1;
                }
            }
        }
        __syncthreads();
        if (quit) break;
        const int inst = w_inst;
        if (inst < 0) {
            __nanosleep(128);
            continue;
        }
        const int t = w_tile, it = w_it;
        if (inst != p_inst) {
            for (int w = threadIdx.x; w < (int)(sizeof(Phys) / 4); w += blockDim.x)
                reinterpret_cast<int *>(&P)[w] = reinterpret_cast<const int *>(B.phys + inst)[w];
            if constexpr (FA)
                for (int w = threadIdx.x; w < (int)(sizeof(Geom) / 4); w += blockDim.x)
                    reinterpret_cast<int *>(&G)[w] = reinterpret_cast<const int *>(B.geo + inst)[w];
            __syncthreads();
            if (threadIdx.x == 0) p_inst = inst;
        }
        double a = 0, b = 0;
        tile_iteration<D, F32, false, L, FA>(B, P, G, it & 1, t, sh, rp, a, b);
        int tlo, thi;
        instance_tiles(B.inst[inst], PPB, tlo, thi);
        double *blk = B.blk + (size_t)(it & 1) * 2 * ntiles;
        if (threadIdx.x == 0) {
            blk[2 * t] = a;
            blk[2 * t + 1] = b;
            __threadfence();
            last_sh = atomicAdd(&B.il[inst].done_tiles, 1u) == (unsigned int)(thi - tlo - 1);
        }
        __syncthreads();
        if (last_sh) {
            // the iteration's last tile: the instance's decision, then the next
            // iteration opens (or the instance retires)
            __threadfence();
            double sa = 0, sb = 0;
            reduce_tiles(blk + 2 * tlo, thi - tlo, sh.red, sa, sb);
            if (threadIdx.x == 0) {
                const int r = finish_iteration(B.ls + inst, P, it, sa, sb);
                B.il[inst].done_tiles = 0u;
                __threadfence();
                if (r != -1) atomicSub(&B.ctrl->active, 1);   // stopped, or paused
                else atomicExch(&B.il[inst].claim, (unsigned long long)(it + 1) << 32);
            }
            __syncthreads();
        }
    }
    // A block leaves after a wait gave up only when it found nothing to claim:
    // every claimed tile belongs to a block still working, and the block that
    // completes an iteration opens the next and looks for work again, so the
    // blocks that stay finish every instance; the host sees kErrBarrier.
}

// Eq. (r-update): r^{n+1} = r^n + dt/2 (V^n + V^{n+1}) for fluid slots, then
// V^{n-1} <- V^n, V^n <- V^K, p^n <- p^K = (p-hat^K + p-hat^{K-1}) / 2; the
// instance's first slot logs the step, and the step's max|V^{n+1}| is folded in
// per warp (a block never straddles two instances), then by one atomic max per
// warp on the bits (non-negative doubles order as integers).
template <int D, bool F32>
__global__ void __launch_bounds__(kBlock) k_outer(Buffers B)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = block_instance(B, blockIdx.x * blockDim.x);
    LoopState *ls = B.ls + inst;
    StatRec *rec = B.stats + (size_t)ls->stat_slot * B.ninst + inst;
    const bool fluid = s < B.n && B.gid_a[s] < (uint32_t)B.nf;   // not a wall, not padding
    double vmag = 0.0;
    if (s < B.n) {
        const int K = ls->iter;
        const int fin = K & 1, prev = fin ^ 1;
        const int n = B.n;
        if (s == B.inst[inst].slot_off) {
            rec->iters = K;
            rec->reason = ls->reason;
            rec->rp = ls->rp;
            rec->rv = ls->rv;
            rec->form = B.form_sel ? *B.form_sel + 1 : (B.form_a ? 2 : 1);
            ls->last_iters = K;
            ls->step = ls->step + 1;
        }
        if (fluid) {
            const Geom &G = B.geo[inst];
            const double dt = B.phys[inst].dt;
            const bool move = !B.phys[inst].steady;               // steady mode: the particles stay
            double v2 = 0.0, d2 = 0.0;
            for (int a = 0; a < D; ++a) {
                const size_t q = (size_t)a * n + s;
                const double vn = B.vn_a[q];
                const double vK = B.vk[fin][q];
                v2 = __fma_rn(vK, vK, v2);
                if (move) {
                    double x = __fma_rn(0.5 * dt, __dadd_rn(vn, vK), B.x_a[q]);
                    if (G.periodic[a]) {
                        if (x >= G.hi[a]) x = __dsub_rn(x, G.L[a]);
                        else if (x < G.lo[a]) x = __dadd_rn(x, G.L[a]);
                    }
                    B.x_a[q] = x;
                    if (B.reuse_lists) {
                        // distance of r^{n+1} from r^0 (nearest image)
                        double dx = x - B.xp_a[q];
                        if (G.periodic[a]) {
                            if (dx > G.halfL[a]) dx -= G.L[a];
                            else if (dx < -G.halfL[a]) dx += G.L[a];
                        }
                        d2 += dx * dx;
                    }
                }
                B.vnm1_a[q] = vn;
                B.vn_a[q] = vK;
            }
            // the lists built at r^0 serve the next step only within list_skin / 2;
            // beyond, the next step bins and lists at r^n itself
            if (B.reuse_lists && !(d2 < B.phys[inst].disp2_reuse)) *(volatile int *)B.relist = 1;
            double p1, p0;
            if (F32) {
                p1 = B.nb32[fin][s].w;
                p0 = B.nb32[prev][s].w;
            } else {
                p1 = B.nb64[fin][s].w;
                p0 = B.nb64[prev][s].w;
            }
            B.pn_a[s] = __dmul_rn(0.5, __dadd_rn(p0, p1));
            vmag = sqrt(v2);
        }
    }
    // a NaN speed has larger bits than any finite one, so it shows as the maximum
    unsigned long long bits = (unsigned long long)__double_as_longlong(vmag);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((threadIdx.x & 31) == 0 && bits != 0ull)
        atomicMax((unsigned long long *)&rec->vmax, bits);
}

// The pair-term form of the step (form = 0, in the step graph): without the
// cache when the latest finished step's iterations, averaged over the
// instances with their fluid counts as weights, are at most kstar (an
// instance with no finished step since the allocation counts one iteration).
// Sums in a fixed order; one block.
__device__ void select_form(const Buffers &B)
{
    __shared__ double kw[kBlock], w[kBlock];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < B.ninst; i += blockDim.x) {
        const double nf = (double)B.inst[i].nf;
        const int k = B.ls[i].last_iters;
        a = __fma_rn(nf, (double)(k > 0 ? k : 1), a);
        b = __dadd_rn(b, nf);
    }
    kw[threadIdx.x] = a;
    w[threadIdx.x] = b;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            kw[threadIdx.x] = __dadd_rn(kw[threadIdx.x], kw[threadIdx.x + h]);
            w[threadIdx.x] = __dadd_rn(w[threadIdx.x], w[threadIdx.x + h]);
        }
        __syncthreads();
    }
    __shared__ int f_sh;
    if (threadIdx.x == 0) {
        const int f = kw[0] <= B.kstar * w[0] ? 1 : 0;
        *B.form_sel = f;
        B.form_count[f] += 1ull;
        f_sh = f;
    }
    __syncthreads();
    // without the cache the loop pauses after floor(kstar) iterations, where the
    // cache would have paid for itself; the step then builds it and goes on, so
    // a wrong guess costs about one cache pass
    const int m = f_sh && B.kstar >= 1.0 && B.kstar < 1e6 ? (int)B.kstar : 0;
    for (int i = threadIdx.x; i < B.ninst; i += blockDim.x) B.ls[i].pause_at = m;
}

__global__ void __launch_bounds__(kBlock) k_loop_reset(Buffers B)
{
    if (B.form_sel) select_form(B);
    reset_loops(B);
}

// A new particle state: every instance's step log starts again at step 0.
__global__ void __launch_bounds__(kBlock) k_restart_steps(Buffers B)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.ninst; i += gridDim.x * blockDim.x) B.ls[i].step = 0;
}

// After a loop without the pair cache (form_run 1): the instances it paused
// are reopened at their iteration for the cached loop that follows, and the
// step's form becomes 2 (recomputed, then cached), which runs the cache pass
// (without a loop reset) and that loop. One block.
__global__ void __launch_bounds__(kBlock) k_loop_resume(Buffers B)
{
    __shared__ int cnt;
    if (skip_form(B)) return;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < B.ninst; i += blockDim.x) {
        LoopState *ls = B.ls + i;
        if (ls->reason == kPaused) {
            ls->done = 0;
            ls->reason = -1;
            ls->ticket = 0;
            if (B.il) {
                B.il[i].claim = (unsigned long long)ls->iter << 32;
                B.il[i].done_tiles = 0u;
            }
            atomicAdd(&cnt, 1);
        }
        ls->pause_at = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0 && cnt > 0) {
        B.ctrl->ticket = 0;
        B.ctrl->bar = 0;
        B.ctrl->active = cnt;
        __threadfence();
        *B.form_sel = 2;
        B.form_count[1] -= 1ull;
        B.form_count[2] += 1ull;
    }
}

template <int D, bool F, bool W, int L, bool FA = false>
const void *loop_kernel() { return (const void *)k_loop<D, F, W, L, FA>; }

template <int D, bool F, int L, bool FA = false>
const void *async_kernel() { return (const void *)k_loop_async<D, F, L, FA>; }


}  // namespace

}  // namespace dtsph
