// The kernels that walk the neighbour lists (built in lists.cu): the wall
// extrapolation and the pair pass at the state n, the pair-coefficient cache
// that the pseudo-time loop reads (geometry frozen for the whole loop, Sec. 2.2;
// caching kernel gradients across pseudo-iterations is the speed-up the paper
// points at in Sec. 4.7 but did not implement), and particle shifting. The
// lists hold only pairs within the cutoff, so the pair arithmetic never runs
// under the distance test, which most candidates fail.
#include "geometry.cuh"
#include "loop_rules.cuh"

namespace dtsph {

namespace {

// ---------------------------------------------------------------- walls, state n

// The list walkers below give each slot a group of L lanes; lane l of a group
// takes the list entries l, l + L, ... Summing kernels merge the lanes' partial
// sums by shuffles, so their summation order depends on L alone: they use the
// fixed kSumLanes, which keeps every context (solo or batched, any size) on
// the same order. One lane per slot measured fastest on large problems and
// costs little on small ones. Block b covers slots b * (kBlock / L) ...

constexpr int kSumLanes = 1;

// Adami et al. wall values at state n in order B: p_w = (sum_f p_f W + rho0 g .
// sum_f r_wf W) / sum_f W, ghost velocity 2 v_w - sum_f V_f W / sum_f W; written
// into the packed (V, p) of the wall slot, from its neighbour list at r^n.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_walls_state_n(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int SPB = kBlock / L;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * SPB);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int s = blockIdx.x * SPB + threadIdx.x / L, lane_in = threadIdx.x % L;
    // every lane stays to the end: the partial sums are merged by full-warp shuffles
    const uint32_t gs = s < B.n ? B.gid_b[s] : kNoParticle;
    const bool wall = gs != kNoParticle && gs >= (uint32_t)B.nf;
    const auto *nb = nb_ptr<T>(B, 1);
    const float4 oi = wall && F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    double acc[6] = {0, 0, 0, 0, 0, 0};   // sum W, sum p W, sum rho0 (g . r) W, sum V W
    const double sigma = P.sig_h * P.h;
    const uint32_t *lst = slot_list(B, s);
    const int cnt = wall ? B.pcount[s] : 0;
    for (int k = lane_in; k < cnt; k += L) {
        const uint32_t jb = lst[k];
        if (jb & kWallBit) continue;                    // fluid neighbours only
        const int j = entry_slot(jb);
        int dx, dy, dz;
        decode_shift(entry_code(jb), dx, dy, dz);
        T d[3], r2;
        listed_sep<D, F32, T>(G, B.x_b, B.off, B.n, s, j, oi, dx, dy, dz, d, r2);
        const double W = sigma * (double)quintic_w<T>(Ar<T>::mul(sqrt(r2), (T)P.inv_h));
        const auto q = nb[j];
        double gr = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) gr += P.g[a] * (double)d[a];
        acc[0] += W;
        acc[1] += (double)q.w * W;
        acc[2] += P.rho0 * gr * W;
        acc[3] += (double)q.x * W;
        acc[4] += (double)q.y * W;
        acc[5] += (double)q.z * W;
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
        for (int t = 0; t < 6; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    if (!wall || lane_in != 0) return;
    const double sw = acc[0];
    double gv[3];
    for (int a = 0; a < 3; ++a) {
        const double vw = a < D ? B.vn_b[(size_t)a * B.n + s] : 0.0;
        gv[a] = 2.0 * vw - (sw > 0 ? acc[3 + a] / sw : 0.0);
    }
    double pw = sw > 0 ? (acc[1] + acc[2]) / sw : 0.0;
    if (pw < 0.0 && P.free_surface) pw = 0.0;     // free-surface runs keep it >= 0 (Sec. 3.2)
    if (F32) B.nb32[1][s] = make_float4((float)gv[0], (float)gv[1], (float)gv[2], (float)pw);
    else B.nb64[1][s] = make_double4_32a(gv[0], gv[1], gv[2], pw);
}

// ------------------------------------------------------------------ state n pass

// Rates at (r^n, V^n, p^n) in order B over the neighbour lists at r^n. With
// PRED, also the predictor of Eqs. (v0, r0): V^0 = V^n + dt F^n, r^0 = r^n +
// dt V^n + dt^2/2 F^n; the first pressure half step p-hat^0 = p^n + dtau/2
// dp^n/dtau (Eq. pkstar_frozen with the state-n rate); and the BDF2 source
// (V^{n-1} - 4 V^n) / (2 dt) of Eq. (dv_dtau_exact), all in FP64.
template <int D, bool F32, bool PRED, bool WALLS, int L>
__global__ void __launch_bounds__(kBlock, F32 ? (D == 2 ? 4 : 3) : 1) k_state_n(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    constexpr int SPB = kBlock / L;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * SPB);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int n = B.n;
    const int s = blockIdx.x * SPB + threadIdx.x / L, lane_in = threadIdx.x % L;
    // every lane stays to the end: the partial sums are merged by full-warp shuffles
    const uint32_t gs = s < n ? B.gid_b[s] : kNoParticle;
    const bool fluid = gs < (uint32_t)B.nf;
    const auto *nb = nb_ptr<T>(B, 1);
    const PairConst<T> k = pair_const<T>(P);
    Acc ap, Fa[3];
    {
        const typename Packed<T>::type qi = fluid ? nb[s] : typename Packed<T>::type{};
        const T vi[3] = {(T)qi.x, (T)qi.y, (T)qi.z};
        const T pi = (T)qi.w;
        const float4 oi = F32 && fluid ? B.off[s] : make_float4(0, 0, 0, 0);
        const uint32_t *lst = slot_list(B, s);
        const int cnt = fluid ? B.pcount[s] : 0;
        // R entries per round: their indices, then their gathers (neighbour
        // state and, FP32C, offset), then the pair terms, so that R loads are in
        // flight per lane; the entries keep their order
        constexpr int R = 4;
        using Q = typename Packed<T>::type;
        for (int q0 = lane_in; q0 < cnt; q0 += L * R) {
            uint32_t jbv[R];
            int cv[R];
            if constexpr (L == 1) {
                // four consecutive entries in one 16-byte load (rows start on
                // 32-byte boundaries and q0 is a multiple of four); an entry
                // past the count repeats entry q0, so its gathers stay in bounds
                const uint4 v = *reinterpret_cast<const uint4 *>(lst + q0);
                jbv[0] = v.x;
                jbv[1] = q0 + 1 < cnt ? v.y : v.x;
                jbv[2] = q0 + 2 < cnt ? v.z : v.x;
                jbv[3] = q0 + 3 < cnt ? v.w : v.x;
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) jbv[r] = lst[min(q0 + r * L, cnt - 1)];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) cv[r] = entry_code(jbv[r]);
            Q qv[R];
            float4 ov[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = entry_slot(jbv[r]);
                qv[r] = nb[j];
                ov[r] = F32 ? B.off[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (q0 + r * L >= cnt) break;
                const uint32_t jb = jbv[r];
                const int j = entry_slot(jb);
                T d[3], r2;
                if (F32) {
                    offset_sep<D, T>(G, oi, ov[r], cv[r], d, r2);
                } else {
                    int dx, dy, dz;
                    decode_shift(cv[r], dx, dy, dz);
                    listed_sep<D, F32, T>(G, B.x_b, B.off, n, s, j, oi, dx, dy, dz, d, r2);
                }
                T g[3], F;
                grad_coef<D, T>(P, d, r2, g, F);
                const auto qj = qv[r];
                const T vv[3] = {(T)qj.x, (T)qj.y, (T)qj.z};
                T vd[3] = {vv[0], vv[1], vv[2]};
                if (WALLS && (jb & kWallBit)) {
                    for (int a = 0; a < D; ++a) vd[a] = (T)B.vn_b[(size_t)a * n + j];
                }
                pair_accumulate<D, T, Acc>(k, g, F, vi, pi, vd, vv, (T)qj.w, ap, Fa);
            }
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        ap.shfl_merge(o);
#pragma unroll
        for (int a = 0; a < D; ++a) Fa[a].shfl_merge(o);
    }
    if (gs == kNoParticle || lane_in != 0) return;
    if (!fluid) {
        if (PRED) {
            for (int a = 0; a < D; ++a) B.xp_b[(size_t)a * n + s] = B.x_b[(size_t)a * n + s];
        }
        return;
    }
    const double apv = (double)(T)ap.value();
    double Fv[3];
    for (int a = 0; a < D; ++a) Fv[a] = __dadd_rn((double)(T)Fa[a].value(), P.g[a]);
    B.ap_b[s] = apv;
    for (int a = 0; a < D; ++a) B.f_b[(size_t)a * n + s] = Fv[a];
    if (PRED && P.steady) {
        // steady mode: the iteration starts from the state itself, the particles
        // stay, and the source is -g (the loop forms F + g - 0)
        for (int a = 0; a < D; ++a) {
            const size_t q = (size_t)a * n + s;
            B.xp_b[q] = B.x_b[q];
            B.v0_b[q] = B.vn_b[q];
            B.s_b[q] = -P.g[a];
        }
        B.ph0_b[s] = __fma_rn(0.5 * P.dtau, apv, B.pn_b[s]);
    } else if (PRED) {
        for (int a = 0; a < D; ++a) {
            const size_t q = (size_t)a * n + s;
            // explicit roundings: the same bits in every kernel variant
            const double V = B.vn_b[q];
            double xp = __fma_rn(0.5 * P.dt * P.dt, Fv[a], __fma_rn(P.dt, V, B.x_b[q]));
            if (G.periodic[a]) {
                if (xp >= G.hi[a]) xp = __dsub_rn(xp, G.L[a]);
                else if (xp < G.lo[a]) xp = __dadd_rn(xp, G.L[a]);
            }
            B.xp_b[q] = xp;
            B.v0_b[q] = __fma_rn(P.dt, Fv[a], V);
            B.s_b[q] = __dmul_rn(P.kappa, __fma_rn(__fma_rn(-4.0, V, B.vnm1_b[q]), P.inv_2dt, -P.g[a]));
        }
        B.ph0_b[s] = __fma_rn(0.5 * P.dtau, apv, B.pn_b[s]);
    }
}

// --------------------------------------------------------------- pair cache

// The cache entries of slot s (its list, in the sliced layout); lane threadIdx.x % L
// of the slot's group takes entries lane, lane + L, ...
template <int D, bool F32, int L>
__device__ __forceinline__ void pair_cache_slot(const Buffers &B, const Geom &G, const Phys &P,
                                                const double *__restrict__ xpos, const uint32_t *__restrict__ gid,
                                                int s)
{
    using T = typename std::conditional<F32, float, double>::type;
    const int lane_in = threadIdx.x % L;
    const int n = B.n;
    const bool wall_s = gid[s] >= (uint32_t)B.nf;
    const uint32_t *lst = slot_list(B, s);                    // the list, per slot
    const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);   // the cache rows, sliced
    const float4 oi = F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    const T sigma = (T)(P.sig_h * P.h);
    const int cnt = B.pcount[s];
    // R entries per round, their offsets gathered together (as in k_state_n)
    constexpr int R = 4;
    for (int q0 = lane_in; q0 < cnt; q0 += L * R) {
        uint32_t jbv[R];
        int cv[R];
#pragma unroll
        if constexpr (L == 1) {
            // four consecutive entries in one 16-byte load (as in k_state_n);
            // an entry past the count repeats entry q0
            const uint4 v = *reinterpret_cast<const uint4 *>(lst + q0);
            jbv[0] = v.x;
            jbv[1] = q0 + 1 < cnt ? v.y : v.x;
            jbv[2] = q0 + 2 < cnt ? v.z : v.x;
            jbv[3] = q0 + 3 < cnt ? v.w : v.x;
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) jbv[r] = lst[min(q0 + r * L, cnt - 1)];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) cv[r] = entry_code(jbv[r]);
        float4 ov[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ov[r] = F32 ? B.off[entry_slot(jbv[r])] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = q0 + r * L;
            if (q >= cnt) break;
            const size_t e = base + (size_t)q * kWarp;
            const uint32_t jb = jbv[r] & ~kCodeMask;      // what the pseudo-time loop reads
            const int j = entry_slot(jb);
            T d[3], r2;
            if (F32) {
                offset_sep<D, T>(G, oi, ov[r], cv[r], d, r2);
            } else {
                int dx, dy, dz;
                decode_shift(cv[r], dx, dy, dz);
                listed_sep<D, F32, T>(G, xpos, B.off, n, s, j, oi, dx, dy, dz, d, r2);
            }
            T c4[4] = {T(0), T(0), T(0), T(0)};
            if (wall_s) {
                const T W = Ar<T>::mul(sigma, quintic_w<T>(Ar<T>::mul(sqrt(r2), (T)P.inv_h)));
                T gr = T(0);
                for (int a = 0; a < D; ++a) gr += (T)P.g[a] * d[a];
                c4[0] = W;
                c4[1] = (T)P.rho0 * gr * W;
            } else {
                // layout (gradW, F_ij); FP32C in 2D packs (gx, gy, F_ij, index bits)
                T g[3], F;
                grad_coef<D, T>(P, d, r2, g, F);
                c4[0] = g[0];
                c4[1] = g[1];
                if (F32 && D == 2) {
                    c4[2] = F;
                } else {
                    c4[2] = D == 3 ? g[2] : T(0);
                    c4[3] = F;
                }
            }
            if (F32) {
                float4 v = make_float4((float)c4[0], (float)c4[1], (float)c4[2], (float)c4[3]);
                if (D == 2) v.w = __uint_as_float(jb);
                B.pc32[e] = v;
            } else {
                B.pc64[e] = make_double4_32a((double)c4[0], (double)c4[1], (double)c4[2], (double)c4[3]);
            }
            if (!(F32 && D == 2)) B.pj[e] = jb;           // the loop reads the index from pj
        }
    }
}

// The pair coefficients of every list entry (order of the latest binning):
// gradW_ij and F_ij for a fluid slot, W_wf and rho0 (g . r_wf) W_wf for a wall
// slot, at the entry's place in the sliced layout. Entries are independent, so
// L only sets the parallelism. Block 0 also resets the pseudo-time loop state.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_pair_cache(Buffers B, const double *__restrict__ xpos,
                                                       const uint32_t *__restrict__ gid)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int SPB = kBlock / L;
    __shared__ Geom G;
    __shared__ Phys P;
    if (skip_form(B)) return;            // the step runs the other pair-term form
    if (blockIdx.x == 0 && B.form_run != 2) {    // (2: a paused loop goes on with the cache)
        reset_loops(B);
    }
    // tiles of SPB slots, grid-stride (a launch with one block per tile takes
    // one each; a launch in a graph that may skip it takes one wave of blocks,
    // so that skipping costs little)
    const int ntile = (B.n + SPB - 1) / SPB;
    int p_inst = -1;
    for (int bt = blockIdx.x; bt < ntile; bt += gridDim.x) {
        const int inst = block_instance(B, bt * SPB);
        if (inst != p_inst) {
            __syncthreads();                 // the previous tile is done with G and P
            block_copy(G, B.geo[inst]);
            block_copy(P, B.phys[inst]);
            p_inst = inst;
        }
        const int s = bt * SPB + threadIdx.x / L;
        if (s < B.n && gid[s] != kNoParticle) pair_cache_slot<D, F32, L>(B, G, P, xpos, gid, s);
    }
}

// ---------------------------------------------------------------- shifting

// Particle shifting after the real step (Sec. 3.5), in order B at r^{n+1}, one
// lane per slot; the displacement over every neighbour (wall particles continue
// the particle distribution), the gradients of the correction over fluid
// neighbours (free-surface runs: particles with div r_i < dim - 1/2, fluid and
// wall neighbours counted, stay where they are):
//   dr_i = -(h^2/2) sum_j V_j (1 + W_ij / W(h)) gradW_ij          Eq. (shift-deltar)
//   f_i <- f_i + (grad f)_i . dr_i, (grad f)_i = sum_j V_j (f_j - f_i) gradW_ij
//                                                      for f = p, V   Eq. (shift-correct)
//   r_i <- r_i + dr_i (wrapped on periodic axes)
// with V_j = m / rho0 and W(h) the kernel at r = h. Every gradient uses the
// unshifted fields (reads order B); the shifted r, V, p go to the particle's
// slot in order A (perm), which the next step bins again.
template <int D, bool F32>
__global__ void __launch_bounds__(kBlock) k_shift(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * kBlock);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int n = B.n;
    const int s = blockIdx.x * kBlock + threadIdx.x;
    if (s >= n) return;
    if (B.gid_b[s] >= (uint32_t)B.nf) return;            // walls and padding stay
    const auto *nb = nb_ptr<T>(B, 1);                     // (V, p) at r^{n+1}, order B
    const auto qi = nb[s];
    const T vi[3] = {(T)qi.x, (T)qi.y, (T)qi.z};
    const T pi = (T)qi.w;
    const float4 oi = F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    const T vol = (T)(P.m / P.rho0);
    const T sigma = (T)(P.sig_h * P.h);
    const T w_h = sigma * quintic_w<T>(T(1));
    Acc dr[3], gp[3], gv[3][3];
    double divr = 0.0;            // div r_i = -sum_j V_j r_ij . gradW_ij, walls included
    const uint32_t *lst = slot_list(B, s);
    const int cnt = B.pcount[s];
    for (int k = 0; k < cnt; ++k) {
        const uint32_t jb = lst[k];
        const int j = entry_slot(jb);
        int dx, dy, dz;
        decode_shift(entry_code(jb), dx, dy, dz);
        T d[3], r2;
        listed_sep<D, F32, T>(G, B.x_b, B.off, n, s, j, oi, dx, dy, dz, d, r2);
        const T r = sqrt(r2);
        const T q = r * (T)P.inv_h;
        const T a = r > T(0) ? (T)P.sig_h * quintic_dwdq<T>(q) / r : T(0);
        divr -= (double)(vol * a * r2);                   // r_ij . gradW_ij = (dW/dr / r) r^2
        // the displacement counts every neighbour, wall particles included
        // (they continue the particle distribution)
        const T fdr = vol * (T(1) + sigma * quintic_w<T>(q) / w_h);
#pragma unroll
        for (int c = 0; c < D; ++c) dr[c].add(fdr * (a * d[c]));
        if (jb & kWallBit) continue;                      // the gradients: fluid neighbours only

        const auto qj = nb[j];
        const T vj[3] = {(T)qj.x, (T)qj.y, (T)qj.z};
        const T dp = vol * ((T)qj.w - pi);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const T gw = a * d[c];
            gp[c].add(dp * gw);
#pragma unroll
            for (int b2 = 0; b2 < D; ++b2) gv[b2][c].add(vol * (vj[b2] - vi[b2]) * gw);
        }
    }
    // a free-surface particle (Lind et al.'s test, Sec. 3.5) is not shifted
    const bool surface = P.free_surface && divr < (double)D - 0.5;
    const double dmul = surface ? 0.0 : -0.5 * P.h * P.h;
    double drv[3] = {0, 0, 0};
    for (int c = 0; c < D; ++c) drv[c] = dmul * (double)(T)dr[c].value();
    const int o = B.perm[s];
    double pnew = B.pn_b[s];
    for (int c = 0; c < D; ++c) pnew += (double)(T)gp[c].value() * drv[c];
    B.pn_a[o] = pnew;
    for (int b2 = 0; b2 < D; ++b2) {
        double v = B.vn_b[(size_t)b2 * n + s];
        for (int c = 0; c < D; ++c) v += (double)(T)gv[b2][c].value() * drv[c];
        B.vn_a[(size_t)b2 * n + o] = v;
        double x = B.x_b[(size_t)b2 * n + s] + drv[b2];
        if (G.periodic[b2]) {
            if (x >= G.hi[b2]) x -= G.L[b2];
            else if (x < G.lo[b2]) x += G.L[b2];
        }
        B.x_a[(size_t)b2 * n + o] = x;
    }
}

}  // namespace

// Lanes per slot of the pair-coefficient pass: enough warps to fill the GPU on
// small problems (each slot's chain of entries is latency-bound), one lane per
// slot on large ones.
int nlist_lanes(int n)
{
    int L = 1;
    while (L < 8 && (long long)n * L < 400000) L *= 2;
    return L;
}

// Neighbour lists at r^n (order B), then the wall values and the state-n pass.
int launch_state_n(const Buffers &B, bool predictor, cudaStream_t st, bool build_lists)
{
    constexpr int L = kSumLanes;
    const int nb = (int)(((long long)B.n * L + kBlock - 1) / kBlock);
    int k = 0;
    if (build_lists) {
        launch_nlist(B, B.x_b, B.cell_b, B.gid_b, st, false);
        k = 1;
    }
    if (B.nw > 0) {
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_walls_state_n<D, F32, L><<<nb, kBlock, 0, st>>>(B)));
        ++k;
    }
    const bool w = B.nw > 0;
    if (predictor && w)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, true, true, L><<<nb, kBlock, 0, st>>>(B)));
    else if (predictor)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, true, false, L><<<nb, kBlock, 0, st>>>(B)));
    else if (w)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, false, true, L><<<nb, kBlock, 0, st>>>(B)));
    else
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, false, false, L><<<nb, kBlock, 0, st>>>(B)));
    return k + 1;
}

// Neighbour lists at xpos, then the pair coefficients.
int launch_pair_cache(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st)
{
    launch_nlist(B, xpos, cell, gid, st, false);
    return 1 + launch_pair_cache_pass(B, xpos, gid, st);
}

int launch_pair_cache_pass(const Buffers &B, const double *xpos, const uint32_t *gid, cudaStream_t st)
{
    const int L = nlist_lanes(B.n);
    int nb = (int)(((long long)B.n * L + kBlock - 1) / kBlock);
    // in a graph that may skip the pass (the per-step form choice), one wave of
    // blocks striding over the tiles, so that a skipped launch costs little
    if (B.form_sel) nb = std::min(nb, kPassWaveBlocksPerSm * std::max(B.nsm, 1));
    if (L == 1) DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 1><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    else if (L == 2) DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 2><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    else if (L == 4) DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 4><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    else DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 8><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    return 1;
}

int launch_shift(const Buffers &B, cudaStream_t st)
{
    int k = launch_binning(B, B.x_a, B.gid_a, st);            // cells at r^{n+1}
    k += launch_permute_a_to_b(B, st);
    launch_nlist(B, B.x_b, B.cell_b, B.gid_b, st, false);
    DTSPH_DISPATCH(B.dim, B.fp32c, (k_shift<D, F32><<<(B.n + kBlock - 1) / kBlock, kBlock, 0, st>>>(B)));
    return k + 2;
}

}  // namespace dtsph
