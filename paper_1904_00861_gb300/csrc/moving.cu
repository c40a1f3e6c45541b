// The pseudo-time loop with the particles moving in pseudo-time (Algorithm 1,
// Sec. 2.1 and the "moving" SPH forms of Sec. 3).
//
// One iteration k for every fluid particle (Jacobi, ping-pong on k's parity),
// with the positions carried as r-hat^k = r^{k+1/2} and the pressure as
// p-hat^k = p^{k+1/2}:
//   wall values at the moved fluid positions                       Sec. 3.2
//   rates at (r^{k+1/2}, V^k, p^{k+1/2}, V~^k):
//     dp/dtau = frozen terms + V~_i . sum_j m (p_i + p_j)/rho0^2 gradW_ij    Eq. (dp-dtau)
//     F       = frozen terms + sum_j m/rho0 (V_i + V_j) (V~_i . gradW_ij)   Eq. (discrete_ME)
//   dV/dtau = kappa (F - (3 V^k - 4 V^n + V^{n-1}) / (2 dt))      Eq. (dv_dtau_exact)
//   V^{k+1} = V^k + dtau dV/dtau                                   Eq. (vkp1)
//   V~^{k+1} = dt dV/dtau                                          Eq. (vtilde)
//   r^{k+1} = r^{k+1/2} + dtau/2 V~^{k+1}                          Eq. (rkp1)
//   r^{k+3/2} = r^{k+1} + dtau/2 V~^{k+1}                          Eq. (rkstar), next pass
//   p-hat^{k+1} = p-hat^k + dtau dp/dtau                           Eqs. (pkstar, pkp1)
// The walls stay where they are. The pair geometry changes every pass, so there
// is no pair cache: each pass walks the lists built at r^0 and recomputes r_ij,
// W and gradW from the current positions. With moving = 1 the lists are those
// of r^0 (neighbours not updated); with moving = 2 they are built with the
// cutoff 3h + skin, and a particle that moves farther than skin / 2 from r^0
// raises kErrSkin, so every pair within 3h of the moved positions is listed:
// the sums equal those over neighbours updated at every pass (the pairs beyond
// 3h add exact zeros).
#include "geometry.cuh"
#include "loop_rules.cuh"

namespace dtsph {

namespace {

inline int blocks(int n) { return (n + kBlock - 1) / kBlock; }

// r^{1/2} = r^0 (V~^0 = 0) in both position buffers, V~ = 0, and the loop state
// reset. Walls keep r^0 in both buffers for the whole loop.
template <bool F32>
__global__ void __launch_bounds__(kBlock) k_move_init(Buffers B)
{
    if (blockIdx.x == 0) {
        reset_loops(B);
    }
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.n || B.gid_a[s] == kNoParticle) return;
    for (int a = 0; a < B.dim; ++a) {
        const size_t q = (size_t)a * B.n + s;
        const double x0 = B.xp_a[q];
        B.xk[0][q] = x0;
        B.xk[1][q] = x0;
        B.vt[q] = 0.0;
    }
    if (F32) {
        B.offk[0][s] = B.off[s];
        B.offk[1][s] = B.off[s];
    }
}

// r_ij = r_i - r_j at the current positions of slots i and j (list entry code
// for the FP32C cell shift), in the working precision; returns |r_ij|^2.
template <int D, bool F32, typename T>
__device__ __forceinline__ T moved_sep(const Geom &G, const Buffers &B, int cur, const T *xi, float4 oi, int j,
                                       int code, T *d)
{
    if (F32) {
        int dx, dy, dz;
        decode_shift(code, dx, dy, dz);
        float f0, f1, f2;
        const float q2 = sep32<D>(shifted_offset<D>(oi, dx, dy, dz, G.s_f), B.offk[cur][j], f0, f1, f2);
        d[0] = (T)f0;
        d[1] = (T)f1;
        if (D == 3) d[2] = (T)f2;
        return (T)q2;
    } else {
        const double *xk = B.xk[cur];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double v = __dsub_rn((double)xi[a], xk[(size_t)a * B.n + j]);
            if (G.periodic[a]) {
                if (v > G.halfL[a]) v = __dsub_rn(v, G.L[a]);
                else if (v < -G.halfL[a]) v = __dadd_rn(v, G.L[a]);
            }
            d[a] = (T)v;
        }
        T r2 = Ar<T>::add(Ar<T>::mul(d[0], d[0]), Ar<T>::mul(d[1], d[1]));
        if (D == 3) r2 = Ar<T>::add(r2, Ar<T>::mul(d[2], d[2]));
        return r2;
    }
}

// Wall values of iteration k (iterate in buffer cur) at the moved fluid
// positions: p_w = (sum_f p_f W + rho0 g . sum_f r_wf W) / sum_f W and ghost
// velocity 2 v_w - sum_f V_f W / sum_f W (Adami et al., Sec. 3.2), zero when no
// fluid is in range; kept >= 0 in free-surface runs.
template <int D, bool F32>
__global__ void __launch_bounds__(kBlock) k_move_walls(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    __shared__ Geom G;
    __shared__ Phys P;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = block_instance(B, blockIdx.x * kBlock);
    const LoopState *ls = B.ls + inst;
    if (ls->done) return;                       // uniform over the block
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    if (s >= B.n) return;
    const uint32_t g = B.gid_a[s];
    if (g < (uint32_t)B.nf || g == kNoParticle) return;
    const int cur = ls->iter & 1;
    T xi[3] = {T(0), T(0), T(0)};
    float4 oi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (F32) {
        oi = B.offk[cur][s];
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) xi[a] = (T)B.xk[cur][(size_t)a * B.n + s];
    }
    const auto *nb = nb_ptr<T>(B, cur);
    const double sigma = P.sig_h * P.h;
    double sw = 0, sp = 0, sg = 0, sv[3] = {0, 0, 0};
    const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
    const int cnt = B.pcount[s];
    for (int k = 0; k < cnt; ++k) {
        const size_t e = base + (size_t)k * kWarp;
        const uint32_t jb = B.pj[e];
        if (jb & kWallBit) continue;            // fluid neighbours only
        const int j = entry_slot(jb);
        T d[3];
        const T r2 = moved_sep<D, F32, T>(G, B, cur, xi, oi, j, entry_code(jb), d);
        const double W = sigma * (double)quintic_w<T>(Ar<T>::mul(sqrt(r2), (T)P.inv_h));
        if (W == 0.0) continue;
        const auto q = nb[j];
        double gr = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) gr += P.g[a] * (double)d[a];
        sw += W;
        sp += (double)q.w * W;
        sg += P.rho0 * gr * W;
        sv[0] += (double)q.x * W;
        sv[1] += (double)q.y * W;
        sv[2] += (double)q.z * W;
    }
    double gv[3];
    for (int a = 0; a < 3; ++a) {
        const double vw = a < D ? B.vn_a[(size_t)a * B.n + s] : 0.0;
        gv[a] = 2.0 * vw - (sw > 0 ? sv[a] / sw : 0.0);
    }
    double pw = sw > 0 ? (sp + sg) / sw : 0.0;
    if (pw < 0.0 && P.free_surface) pw = 0.0;   // free-surface runs (Sec. 3.2)
    if (F32) B.nb32[cur][s] = make_float4((float)gv[0], (float)gv[1], (float)gv[2], (float)pw);
    else B.nb64[cur][s] = make_double4_32a(gv[0], gv[1], gv[2], pw);
}

// One moving iteration over all slots, L lanes per slot (lane l takes the list
// entries l, l + L, ...; the partial sums merge by warp shuffles and the first
// lane updates the particle) and one tile of kBlock / L slots per block; the last
// block of an instance applies its stop rules, the last block of all sets the
// while-node condition (as the frozen iterate kernel).
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_move_iter(Buffers B, unsigned long long cond, int use_cond)
{
    constexpr int PPB = kBlock / L;
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    using A = Ar<T>;
    __shared__ Geom G;
    __shared__ Phys P;
    __shared__ double red[2][kBlock / kWarp];
    __shared__ int last, tlo_sh;
    if (!use_cond && B.ctrl->active == 0) return;   // whole grid agrees: nothing to do
    const int n = B.n;
    const int inst = block_instance(B, blockIdx.x * PPB);
    LoopState *ls = B.ls + inst;
    int tlo, thi;
    instance_tiles(B.inst[inst], PPB, tlo, thi);
    const bool mine = (int)blockIdx.x < thi;        // false: a tile made of padding only
    const int it = ls->iter;
    const bool work = mine && !ls->done;
    if (work) {
        block_copy(G, B.geo[inst]);
        block_copy(P, B.phys[inst]);
        const int cur = it & 1, nxt = cur ^ 1;
        const int s = blockIdx.x * PPB + threadIdx.x / L, lane_in = threadIdx.x % L;
        const bool fl = s < n && B.gid_a[s] < (uint32_t)B.nf;
        double r_ap = 0.0, r_av = 0.0;
        Acc ap, Fa[3], gp[3];
        const PairConst<T> k = pair_const<T>(P);
        if (fl) {
            const auto *nb = nb_ptr<T>(B, cur);
            const auto qi = nb[s];
            const T vi[3] = {(T)qi.x, (T)qi.y, (T)qi.z};
            const T pi = (T)qi.w;
            double xh[3] = {0, 0, 0}, vt[3] = {0, 0, 0};
            T xi[3] = {T(0), T(0), T(0)}, ti[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const size_t q = (size_t)a * n + s;
                xh[a] = B.xk[cur][q];
                xi[a] = (T)xh[a];
                vt[a] = B.vt[q];
                ti[a] = (T)vt[a];
            }
            const float4 oi = F32 ? B.offk[cur][s] : make_float4(0.f, 0.f, 0.f, 0.f);
            const T rc2k = (T)(9.0 * P.h * P.h);
            const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
            const int cnt = B.pcount[s];
            // R entries per round: their indices, then their gathers, then the
            // pair terms, so that R loads are in flight per lane (the entries
            // stay in the order lane_in, lane_in + L, ...)
            constexpr int R = F32 ? 4 : 2;
            using Q = typename Packed<T>::type;
            for (int q0 = lane_in; q0 < cnt; q0 += L * R) {
                uint32_t jbv[R];
                int codev[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int q = q0 + r * L;
                    const size_t e = base + (size_t)min(q, cnt - 1) * kWarp;
                    jbv[r] = B.pj[e];
                    codev[r] = entry_code(jbv[r]);
                }
                Q qv[R];
                float4 ov[R];
                T xj[R][3];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int j = entry_slot(jbv[r]);
                    qv[r] = nb[j];
                    if (F32) {
                        ov[r] = B.offk[cur][j];
                    } else {
#pragma unroll
                        for (int a = 0; a < D; ++a) xj[r][a] = (T)B.xk[cur][(size_t)a * n + j];
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (q0 + r * L >= cnt) break;
                    const uint32_t jb = jbv[r];
                    const int j = entry_slot(jb);
                    T d[3], r2;
                    if (F32) {
                        int dx, dy, dz;
                        decode_shift(codev[r], dx, dy, dz);
                        float f0, f1, f2;
                        const float q2 = sep32<D>(shifted_offset<D>(oi, dx, dy, dz, G.s_f), ov[r], f0, f1, f2);
                        d[0] = (T)f0;
                        d[1] = (T)f1;
                        if (D == 3) d[2] = (T)f2;
                        r2 = (T)q2;
                    } else {
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            double v = __dsub_rn((double)xi[a], (double)xj[r][a]);
                            if (G.periodic[a]) {
                                if (v > G.halfL[a]) v = __dsub_rn(v, G.L[a]);
                                else if (v < -G.halfL[a]) v = __dadd_rn(v, G.L[a]);
                            }
                            d[a] = (T)v;
                        }
                        r2 = A::add(A::mul(d[0], d[0]), A::mul(d[1], d[1]));
                        if (D == 3) r2 = A::add(r2, A::mul(d[2], d[2]));
                    }
                    if (!(r2 < rc2k)) continue;          // outside the kernel support: adds nothing
                    T g[3], F;
                    grad_coef<D, T>(P, d, r2, g, F);
                    const Q qj = qv[r];
                    const T vv[3] = {(T)qj.x, (T)qj.y, (T)qj.z};
                    T vd[3] = {vv[0], vv[1], vv[2]};
                    if (jb & kWallBit) {
#pragma unroll
                        for (int a = 0; a < D; ++a) vd[a] = (T)B.vn_a[(size_t)a * n + j];
                    }
                    const T pj = (T)qj.w;
                    pair_accumulate<D, T, Acc>(k, g, F, vi, pi, vd, vv, pj, ap, Fa);
                    // advective terms of Eqs. (dp-dtau) and (discrete_ME)
                    T tg = T(0);
#pragma unroll
                    for (int a = 0; a < D; ++a) tg = A::fma(ti[a], g[a], tg);
                    const T pp = A::mul(k.c_p, A::add(pi, pj));
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        gp[a].add(A::mul(pp, g[a]));
                        Fa[a].add(A::mul(A::mul(k.vol, A::add(vi[a], vd[a])), tg));
                    }
                }
            }
        }
        // every lane takes part in the merges
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            ap.shfl_merge(o);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                Fa[a].shfl_merge(o);
                gp[a].shfl_merge(o);
            }
        }
        if (fl && lane_in == 0) {
            double xh[3] = {0, 0, 0}, vt[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const size_t q = (size_t)a * n + s;
                xh[a] = B.xk[cur][q];
                vt[a] = B.vt[q];
            }
            // update in FP64
            double apv = (double)(T)ap.value();
#pragma unroll
            for (int a = 0; a < D; ++a) apv = __fma_rn(vt[a], (double)(T)gp[a].value(), apv);
            double vnew[3] = {0, 0, 0}, xn[3] = {0, 0, 0};
            double av2 = 0.0;
            const double hdt = 0.5 * P.dtau;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const size_t q = (size_t)a * n + s;
                const double vk = B.vk[cur][q];
                const double Fv = (double)(T)Fa[a].value();
                const double av = __fma_rn(P.kappa, Fv, -__fma_rn(P.kc3, vk, B.s_a[q]));
                vnew[a] = __fma_rn(P.dtau, av, vk);
                B.vk[nxt][q] = vnew[a];
                const double vtn = __dmul_rn(P.dt, av);
                B.vt[q] = vtn;
                const double x1 = __dadd_rn(xh[a], __dmul_rn(hdt, vtn));
                double x2 = __dadd_rn(x1, __dmul_rn(hdt, vtn));
                if (G.periodic[a]) {
                    if (x2 >= G.hi[a]) x2 = __dsub_rn(x2, G.L[a]);
                    else if (x2 < G.lo[a]) x2 = __dadd_rn(x2, G.L[a]);
                }
                xn[a] = x2;
                B.xk[nxt][q] = x2;
                av2 = __fma_rn(av, av, av2);
            }
            if (F32) {
                // offsets from the slot's cell origin at r^0 (minimum image)
                const int lc = B.cell_a[s] - B.inst[inst].cell_off;
                const int c[3] = {lc % G.nc[0], (lc / G.nc[0]) % G.nc[1], lc / (G.nc[0] * G.nc[1])};
                float o[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    double v = xn[a] - (G.lo[a] + c[a] * G.s[a]);
                    if (G.periodic[a]) {
                        if (v > G.halfL[a]) v -= G.L[a];
                        else if (v < -G.halfL[a]) v += G.L[a];
                    }
                    o[a] = (float)v;
                }
                B.offk[nxt][s] = make_float4(o[0], o[1], o[2], 0.f);
                const float pnew = __fmaf_rn(P.dtau_f, (float)apv, B.nb32[cur][s].w);
                B.nb32[nxt][s] = make_float4((float)vnew[0], (float)vnew[1], (float)vnew[2], pnew);
            } else {
                const double pnew = __fma_rn(P.dtau, apv, B.nb64[cur][s].w);
                B.nb64[nxt][s] = make_double4_32a(vnew[0], vnew[1], vnew[2], pnew);
            }
            if (P.moving == 2) {
                // the lists cover displacements up to skin / 2 from r^0
                double d2 = 0.0;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    double v = xn[a] - B.xp_a[(size_t)a * n + s];
                    if (G.periodic[a]) {
                        if (v > G.halfL[a]) v -= G.L[a];
                        else if (v < -G.halfL[a]) v += G.L[a];
                    }
                    d2 += v * v;
                }
                if (!(d2 < P.disp2_max)) atomicOr(B.err, kErrSkin);
            }
            r_ap = fabs(apv);
            r_av = sqrt(av2);
        }
        // fixed-order block sum of the residual terms
        const double w_ap = warp_sum<double>(r_ap), w_av = warp_sum<double>(r_av);
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = w_ap;
            red[1][threadIdx.x >> 5] = w_av;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0;
            for (int w = 0; w < kBlock / kWarp; ++w) {
                a += red[0][w];
                b += red[1][w];
            }
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
            reduce_tiles(B.blk + 2 * tlo_sh, thi - tlo_sh, red, sa, sb);
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

}  // namespace

int launch_move_prepare(const Buffers &B, cudaStream_t st)
{
    launch_nlist(B, B.xp_a, B.cell_a, B.gid_a, st, true);   // walked every pass: sliced
    if (B.fp32c) k_move_init<true><<<blocks(B.n), kBlock, 0, st>>>(B);
    else k_move_init<false><<<blocks(B.n), kBlock, 0, st>>>(B);
    return 2;
}

int launch_move_iteration(const Buffers &B, unsigned long long cond, int use_cond, cudaStream_t st)
{
    int k = 0;
    if (B.nw > 0) {
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_move_walls<D, F32><<<blocks(B.n), kBlock, 0, st>>>(B)));
        ++k;
    }
    // n is a multiple of kSlotAlign, so the tiles of kBlock / L slots cover it exactly
    const int L = B.lanes, nb = (int)((long long)B.n * L / kBlock);
    if (L == 1) DTSPH_DISPATCH(B.dim, B.fp32c, (k_move_iter<D, F32, 1><<<nb, kBlock, 0, st>>>(B, cond, use_cond)));
    else if (L == 2) DTSPH_DISPATCH(B.dim, B.fp32c, (k_move_iter<D, F32, 2><<<nb, kBlock, 0, st>>>(B, cond, use_cond)));
    else if (L == 4) DTSPH_DISPATCH(B.dim, B.fp32c, (k_move_iter<D, F32, 4><<<nb, kBlock, 0, st>>>(B, cond, use_cond)));
    else DTSPH_DISPATCH(B.dim, B.fp32c, (k_move_iter<D, F32, 8><<<nb, kBlock, 0, st>>>(B, cond, use_cond)));
    return k + 1;
}

}  // namespace dtsph
