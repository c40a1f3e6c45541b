// Neighbour traversal kernels: the wall extrapolation and the pair pass at the
// state n (geometry computed on the fly), and the pair-coefficient cache that the
// pseudo-time loop reads (geometry frozen for the whole loop, Sec. 2.2; caching
// kernel gradients across pseudo-iterations is the speed-up the paper points at
// in Sec. 5 but did not implement).
//
// Neighbour test: j != i and |r_ij|^2 < (3h)^2 in IEEE double, squares summed in
// axis order without FMA, minimum image on periodic axes. The FP32C path first
// tests an FP32 separation built from per-cell FP32 offsets and falls back to the
// FP64 test only inside a thin band around 3h, so both paths give the same sets.
#include "pair_terms.cuh"

namespace dtsph {

namespace {

// Candidate traversal by a group of L lanes that serve one particle. The 3^D
// cells around `cell` are taken row by row (a row = the three cells along x at
// fixed y, z offsets); inside a row the candidates of the three cells are
// numbered consecutively and lane l takes numbers l, l+L, ... Every lane of the
// group runs the same number of rounds, so `body` may use group ballots; it is
// called as body(valid, j, dx, dy, dz) where (dx, dy, dz) is the unwrapped cell
// shift of candidate j (r_ij = off_i - off_j - shift * s).
template <int D, int L, class Body>
__device__ __forceinline__ void group_candidates(const Geom &G, const int *__restrict__ start, int cell_off, int cell,
                                                 int lane_in, Body &&body)
{
    start += cell_off;            // the instance's cells, numbered from 0
    cell -= cell_off;
    const int c0 = cell % G.nc[0];
    const int c1 = (cell / G.nc[0]) % G.nc[1];
    const int c2 = cell / (G.nc[0] * G.nc[1]);
    const int zlo = D == 3 ? -1 : 0, zhi = D == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int z = c2 + dz;
        if (D == 3 && (z < 0 || z >= G.nc[2])) {
            if (!G.periodic[2]) continue;
            z = z < 0 ? z + G.nc[2] : z - G.nc[2];
        }
        for (int dy = -1; dy <= 1; ++dy) {
            int y = c1 + dy;
            if (y < 0 || y >= G.nc[1]) {
                if (!G.periodic[1]) continue;
                y = y < 0 ? y + G.nc[1] : y - G.nc[1];
            }
            const int row = (z * G.nc[1] + y) * G.nc[0];
            int b[3], m[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                int x = c0 + k - 1;
                bool ok = true;
                if (x < 0 || x >= G.nc[0]) {
                    if (G.periodic[0]) x = x < 0 ? x + G.nc[0] : x - G.nc[0];
                    else ok = false;
                }
                b[k] = ok ? start[row + x] : 0;
                m[k] = ok ? start[row + x + 1] - b[k] : 0;
            }
            const int m01 = m[0] + m[1];
            const int tot = m01 + m[2];
            for (int r = 0; r < tot; r += L) {
                const int v = r + lane_in;
                int j, dx;
                if (v < m[0]) { j = b[0] + v; dx = -1; }
                else if (v < m01) { j = b[1] + v - m[0]; dx = 0; }
                else { j = b[2] + v - m01; dx = 1; }
                body(v < tot, j, dx, dy, dz);
            }
        }
    }
}

// r_ij in FP64 with the minimum image; returns |r_ij|^2 (no FMA contraction).
template <int D>
__device__ __forceinline__ double sep64(const Geom &G, const double *__restrict__ x, int n, int i, int j, double *d)
{
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double v = __dsub_rn(x[(size_t)a * n + i], x[(size_t)a * n + j]);
        if (G.periodic[a]) {
            if (v > G.halfL[a]) v = __dsub_rn(v, G.L[a]);
            else if (v < -G.halfL[a]) v = __dadd_rn(v, G.L[a]);
        }
        d[a] = v;
    }
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    if (D == 3) r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    return r2;
}

// Neighbour test plus the separation in the working precision T.
// Returns true when j is a neighbour of i; d and r2 hold r_ij and |r_ij|^2.
template <int D, bool F32, typename T>
__device__ __forceinline__ bool neighbour(const Geom &G, const double *__restrict__ x, const float4 *__restrict__ off,
                                          int n, int i, int j, float4 oi, int dx, int dy, int dz, T *d, T &r2)
{
    if (F32) {
        float4 oj = off[j];
        using A = Ar<float>;
        const float f0 = A::fma(-(float)dx, G.s_f[0], A::sub(oi.x, oj.x));
        const float f1 = A::fma(-(float)dy, G.s_f[1], A::sub(oi.y, oj.y));
        const float f2 = D == 3 ? A::fma(-(float)dz, G.s_f[2], A::sub(oi.z, oj.z)) : 0.f;
        float q2 = A::fma(f1, f1, A::mul(f0, f0));
        if (D == 3) q2 = A::fma(f2, f2, q2);
        if (q2 >= G.rc2_hi) return false;
        if (q2 >= G.rc2_lo) {
            double e[3];
            if (!(sep64<D>(G, x, n, i, j, e) < G.rc2)) return false;
        }
        d[0] = (T)f0;
        d[1] = (T)f1;
        if (D == 3) d[2] = (T)f2;
        r2 = (T)q2;
        return true;
    } else {
        double e[3];
        double q2 = sep64<D>(G, x, n, i, j, e);
        if (!(q2 < G.rc2)) return false;
#pragma unroll
        for (int a = 0; a < D; ++a) d[a] = (T)e[a];
        r2 = (T)q2;
        return true;
    }
}

// Reciprocal square root and division in the working precision: the fast
// single-precision forms (a few ulp) on the FP32C path, IEEE double otherwise.
template <typename T> struct F32Math;
template <> struct F32Math<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
};
template <> struct F32Math<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
};

// gradW_ij and F_ij = (r_ij . gradW_ij) / (r^2 + eta h^2) from r_ij, with one
// reciprocal square root: r = r^2 / r, q = r / h, gradW = (dW/dr / r) r_ij.
template <int D, typename T>
__device__ __forceinline__ void grad_coef(const Phys &P, const T *d, T r2, T *g, T &F)
{
    using A = Ar<T>;
    if (r2 > T(0)) {
        const T rinv = F32Math<T>::rsqrt(r2);
        const T r = A::mul(r2, rinv);
        const T dwdr = A::mul((T)P.sig_h, quintic_dwdq<T>(A::mul(r, (T)P.inv_h)));
        const T a = A::mul(dwdr, rinv);
#pragma unroll
        for (int k = 0; k < D; ++k) g[k] = A::mul(a, d[k]);
        F = F32Math<T>::div(A::mul(dwdr, r), A::add(r2, (T)P.eta_h2));
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) g[k] = T(0);
        F = T(0);
    }
}

template <typename T> struct Packed;
template <> struct Packed<double> { using type = double4_32a; };
template <> struct Packed<float> { using type = float4; };

template <typename T>
__device__ __forceinline__ const typename Packed<T>::type *nb_ptr(const Buffers &B, int buf);
template <>
__device__ __forceinline__ const double4_32a *nb_ptr<double>(const Buffers &B, int buf) { return B.nb64[buf]; }
template <>
__device__ __forceinline__ const float4 *nb_ptr<float>(const Buffers &B, int buf) { return B.nb32[buf]; }

// Copies a table entry into shared memory with the whole block (then syncs).
template <typename T>
__device__ __forceinline__ void block_copy(T &dst, const T &src)
{
    static_assert(sizeof(T) % 4 == 0, "word copy");
    for (int w = threadIdx.x; w < (int)(sizeof(T) / 4); w += blockDim.x)
        reinterpret_cast<int *>(&dst)[w] = reinterpret_cast<const int *>(&src)[w];
    __syncthreads();
}

// ---------------------------------------------------------------- walls, state n

// Adami et al. wall values at state n in order B: p_w = (sum_f p_f W + rho0 g .
// sum_f r_wf W) / sum_f W, ghost velocity 2 v_w - sum_f V_f W / sum_f W; written
// into the packed (V, p) of the wall slot. L lanes per wall particle.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_walls_state_n(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * (kBlock / L));
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int cell_off = B.inst[inst].cell_off;
    const int grp = threadIdx.x / L, lane_in = threadIdx.x % L;
    const int s = blockIdx.x * (kBlock / L) + grp;
    // every lane stays to the end: the partial sums are merged by full-warp shuffles
    const uint32_t gs = s < B.n ? B.gid_b[s] : kNoParticle;
    const bool wall = gs != kNoParticle && gs >= (uint32_t)B.nf;
    const auto *nb = nb_ptr<T>(B, 1);
    const float4 oi = wall && F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    double acc[6] = {0, 0, 0, 0, 0, 0};   // sum W, sum p W, sum rho0 (g . r) W, sum V W
    const double sigma = P.sig_h * P.h;
    if (wall) group_candidates<D, L>(G, B.cell_start, cell_off, B.cell_b[s], lane_in, [&](bool valid, int j, int dx, int dy, int dz) {
        if (!valid || j == s || B.gid_b[j] >= (uint32_t)B.nf) return;
        T d[3], r2;
        if (!neighbour<D, F32, T>(G, B.x_b, B.off, B.n, s, j, oi, dx, dy, dz, d, r2)) return;
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
    });
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
    const double pw = sw > 0 ? (acc[1] + acc[2]) / sw : 0.0;
    if (F32) B.nb32[1][s] = make_float4((float)gv[0], (float)gv[1], (float)gv[2], (float)pw);
    else B.nb64[1][s] = make_double4_32a(gv[0], gv[1], gv[2], pw);
}

// ------------------------------------------------------------------ state n pass

// Rates at (r^n, V^n, p^n) in order B, L lanes per particle (partial sums
// merged by shuffles). With PRED, also the predictor of Eqs. (v0, r0):
// V^0 = V^n + dt F^n, r^0 = r^n + dt V^n + dt^2/2 F^n; the first pressure half
// step p-hat^0 = p^n + dtau/2 dp^n/dtau (Eq. pkstar_frozen with the state-n
// rate); and the BDF2 source (V^{n-1} - 4 V^n) / (2 dt) of Eq. (dv_dtau_exact),
// all in FP64, one thread per particle in whole warps.
template <int D, bool F32, bool PRED, int L, bool WALLS>
__global__ void __launch_bounds__(kBlock) k_state_n(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    constexpr int PPB = kBlock / L;
    __shared__ T part[D + 1][PPB];
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * PPB);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int cell_off = B.inst[inst].cell_off;
    const int n = B.n;
    const int grp = threadIdx.x / L, lane_in = threadIdx.x % L;
    const int s = blockIdx.x * PPB + grp;
    const bool fluid = s < n && B.gid_b[s] < (uint32_t)B.nf;
    {
        const auto *nb = nb_ptr<T>(B, 1);
        const PairConst<T> k = pair_const<T>(P);
        Acc ap, Fa[3];
        if (fluid) {
            const auto qi = nb[s];
            const T vi[3] = {(T)qi.x, (T)qi.y, (T)qi.z};
            const T pi = (T)qi.w;
            const float4 oi = F32 ? B.off[s] : make_float4(0, 0, 0, 0);
            group_candidates<D, L>(G, B.cell_start, cell_off, B.cell_b[s], lane_in, [&](bool valid, int j, int dx, int dy, int dz) {
                if (!valid || j == s) return;
                T d[3], r2;
                if (!neighbour<D, F32, T>(G, B.x_b, B.off, n, s, j, oi, dx, dy, dz, d, r2)) return;
                T g[3], F;
                grad_coef<D, T>(P, d, r2, g, F);
                const auto qj = nb[j];
                const T vv[3] = {(T)qj.x, (T)qj.y, (T)qj.z};
                T vd[3] = {vv[0], vv[1], vv[2]};
                if (WALLS && B.gid_b[j] >= (uint32_t)B.nf) {
                    for (int a = 0; a < D; ++a) vd[a] = (T)B.vn_b[(size_t)a * n + j];
                }
                pair_accumulate<D, T, Acc>(k, g, F, vi, pi, vd, vv, (T)qj.w, ap, Fa);
            });
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            ap.shfl_merge(o);
#pragma unroll
            for (int a = 0; a < D; ++a) Fa[a].shfl_merge(o);
        }
        if (lane_in == 0) {
            part[0][grp] = (T)ap.value();
#pragma unroll
            for (int a = 0; a < D; ++a) part[1 + a][grp] = (T)Fa[a].value();
        }
    }
    __syncthreads();
    if (threadIdx.x >= PPB) return;
    const int s2 = blockIdx.x * PPB + threadIdx.x;
    if (s2 >= n || B.gid_b[s2] == kNoParticle) return;
    if (B.gid_b[s2] >= (uint32_t)B.nf) {
        if (PRED) {
            for (int a = 0; a < D; ++a) B.xp_b[(size_t)a * n + s2] = B.x_b[(size_t)a * n + s2];
        }
        return;
    }
    const double apv = (double)part[0][threadIdx.x];
    double Fv[3];
    for (int a = 0; a < D; ++a) Fv[a] = __dadd_rn((double)part[1 + a][threadIdx.x], P.g[a]);
    B.ap_b[s2] = apv;
    for (int a = 0; a < D; ++a) B.f_b[(size_t)a * n + s2] = Fv[a];
    if (PRED) {
        for (int a = 0; a < D; ++a) {
            const size_t q = (size_t)a * n + s2;
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
        B.ph0_b[s2] = __fma_rn(0.5 * P.dtau, apv, B.pn_b[s2]);
    }
}

// --------------------------------------------------------------- pair cache

// For every slot (order of the latest binning) the list of its neighbours with
// gradW_ij and F_ij (fluid slot), or W_wf and rho0 (g . r_wf) W_wf (wall slot),
// sliced by warp so that entry k of the 32 slots of a warp is contiguous. L lanes
// per slot test candidates side by side; a group ballot keeps the list in
// candidate order. Block 0 also resets the pseudo-time loop state.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_pair_cache(Buffers B, const double *__restrict__ xpos,
                                                       const int *__restrict__ cell, const uint32_t *__restrict__ gid)
{
    using T = typename std::conditional<F32, float, double>::type;
    __shared__ Geom G;
    __shared__ Phys P;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < B.ninst; i += blockDim.x) {
            LoopState *ls = B.ls + i;
            ls->iter = 0;
            ls->done = 0;
            ls->reason = -1;
            ls->ticket = 0;
            ls->rp = 0;
            ls->rv = 0;
        }
        if (threadIdx.x == 0) {
            B.ctrl->ticket = 0;
            B.ctrl->bar = 0;
            B.ctrl->active = B.ninst;
        }
    }
    const int inst = block_instance(B, blockIdx.x * (kBlock / L));
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int cell_off = B.inst[inst].cell_off;
    const int grp = threadIdx.x / L, lane_in = threadIdx.x % L;
    const int s = blockIdx.x * (kBlock / L) + grp;
    if (s >= B.n) return;                                  // whole group leaves together
    const int n = B.n, K = B.K;
    if (gid[s] == kNoParticle) {
        if (lane_in == 0) B.pcount[s] = 0;
        return;
    }
    const bool wall_s = gid[s] >= (uint32_t)B.nf;
    const size_t base = (size_t)(s >> 5) * K * kWarp + (s & 31);
    const float4 oi = F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    const unsigned gshift = (threadIdx.x & 31) - lane_in;   // first lane of the group in the warp
    const unsigned gmask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << gshift;
    int cnt = 0;
    const T sigma = (T)(P.sig_h * P.h);
    group_candidates<D, L>(G, B.cell_start, cell_off, cell[s], lane_in, [&](bool valid, int j, int dx, int dy, int dz) {
        T d[3], r2;
        const bool in = valid && j != s && neighbour<D, F32, T>(G, xpos, B.off, n, s, j, oi, dx, dy, dz, d, r2);
        const unsigned bal = __ballot_sync(gmask, in) >> gshift;
        const int pos = cnt + __popc(bal & ((1u << lane_in) - 1u));
        cnt += __popc(bal);
        if (!in || pos >= K) return;
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
        const uint32_t jb = (uint32_t)j | (gid[j] >= (uint32_t)B.nf ? kWallBit : 0u);
        const size_t e = base + (size_t)pos * kWarp;
        if (F32) {
            float4 v = make_float4((float)c4[0], (float)c4[1], (float)c4[2], (float)c4[3]);
            if (D == 2) v.w = __uint_as_float(jb);
            else B.pj[e] = jb;
            B.pc32[e] = v;
        } else {
            B.pc64[e] = make_double4_32a((double)c4[0], (double)c4[1], (double)c4[2], (double)c4[3]);
            B.pj[e] = jb;
        }
    });
    if (lane_in == 0) {
        if (cnt > K) {
            atomicOr(B.err, kErrCapacity);
            cnt = K;
        }
        B.pcount[s] = cnt;
    }
}

}  // namespace

#define DTSPH_DISPATCH(D_, F32_, ...)                                                  \
    do {                                                                               \
        if ((D_) == 2 && !(F32_)) { constexpr int D = 2; constexpr bool F32 = false; __VA_ARGS__; } \
        else if ((D_) == 2) { constexpr int D = 2; constexpr bool F32 = true; __VA_ARGS__; }        \
        else if (!(F32_)) { constexpr int D = 3; constexpr bool F32 = false; __VA_ARGS__; }         \
        else { constexpr int D = 3; constexpr bool F32 = true; __VA_ARGS__; }                       \
    } while (0)

constexpr int kTravLanes = 8;   // lanes per particle of the traversal kernels

inline int trav_blocks(int n) { return (n + kBlock / kTravLanes - 1) / (kBlock / kTravLanes); }

int launch_state_n(const Buffers &B, bool predictor, cudaStream_t st)
{
    int k = 0;
    const int nb = trav_blocks(B.n);
    if (B.nw > 0) {
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_walls_state_n<D, F32, kTravLanes><<<nb, kBlock, 0, st>>>(B)));
        ++k;
    }
    const bool w = B.nw > 0;
    if (predictor && w)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, true, kTravLanes, true><<<nb, kBlock, 0, st>>>(B)));
    else if (predictor)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, true, kTravLanes, false><<<nb, kBlock, 0, st>>>(B)));
    else if (w)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, false, kTravLanes, true><<<nb, kBlock, 0, st>>>(B)));
    else
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, false, kTravLanes, false><<<nb, kBlock, 0, st>>>(B)));
    return k + 1;
}

int launch_pair_cache(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st)
{
    DTSPH_DISPATCH(B.dim, B.fp32c,
                   (k_pair_cache<D, F32, kTravLanes><<<trav_blocks(B.n), kBlock, 0, st>>>(B, xpos, cell, gid)));
    return 1;
}

}  // namespace dtsph
