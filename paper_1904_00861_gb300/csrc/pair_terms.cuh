// Device functions of the pair summations, shared by the state-n pass (geometry
// computed on the fly) and the pseudo-time iteration (geometry from the pair
// cache).
//
// For a fluid particle i and a neighbour j, with gradW = dW/dr r_ij / r and
// F_ij = (r_ij . gradW) / (r^2 + eta h^2), the frozen EDAC rates of the paper
// (Eqs. dp-dtau-frozen-edac and mom-sph-frozen, rho_i = rho_j = rho0) are
//   dp_i/dtau += c_div (V_ij . gradW) + c_edac (p_i - p_j) F_ij
//   F_i       += -c_p (p_i + p_j) gradW - m Pi_ij gradW + c_visc F_ij V_ij
// where a wall neighbour j contributes its prescribed velocity to V_ij in the
// divergence term and its ghost velocity in the viscous and artificial-viscosity
// terms (Adami et al., cited in Sec. 3.2).
#pragma once

#include "dtsph_internal.cuh"

namespace dtsph {

// Rounded arithmetic with the rounding of every operation spelled out, so the
// pair terms give the same bits whichever kernel variant inlines them (the
// compiler may not fuse or reorder these).
template <typename T> struct Ar;
template <> struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// Quintic spline, dW/dq up to the factor sigma: -5(3-q)^4 + 30(2-q)^4 - 75(1-q)^4
// with each term present only inside its support (0 from q = 3 on, so a list
// built with a wider cutoff adds exact zeros).
template <typename T>
__device__ __forceinline__ T quintic_dwdq(T q)
{
    using A = Ar<T>;
    if (!(q < T(3))) return T(0);
    const T a = A::sub(T(3), q);
    const T a2 = A::mul(a, a);
    T s = A::mul(A::mul(T(-5), a2), a2);
    if (q < T(2)) {
        const T b = A::sub(T(2), q);
        const T b2 = A::mul(b, b);
        s = A::fma(A::mul(T(30), b2), b2, s);
    }
    if (q < T(1)) {
        const T c = A::sub(T(1), q);
        const T c2 = A::mul(c, c);
        s = A::fma(A::mul(T(-75), c2), c2, s);
    }
    return s;
}

// W(q) up to sigma: (3-q)^5 - 6(2-q)^5 + 15(1-q)^5 within the supports (0 from
// q = 3 on).
template <typename T>
__device__ __forceinline__ T quintic_w(T q)
{
    using A = Ar<T>;
    if (!(q < T(3))) return T(0);
    const T a = A::sub(T(3), q);
    const T a2 = A::mul(a, a);
    T s = A::mul(A::mul(a2, a2), a);
    if (q < T(2)) {
        const T b = A::sub(T(2), q);
        const T b2 = A::mul(b, b);
        s = A::fma(A::mul(T(-6), A::mul(b2, b2)), b, s);
    }
    if (q < T(1)) {
        const T c = A::sub(T(1), q);
        const T c2 = A::mul(c, c);
        s = A::fma(A::mul(T(15), A::mul(c2, c2)), c, s);
    }
    return s;
}

// Kahan-compensated accumulator (FP32C path).
struct Kahan {
    float s, c;
    __device__ __forceinline__ Kahan() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float v)
    {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s - c; }
    // merges the accumulator of another lane (the sum is s - c for both)
    __device__ __forceinline__ void merge(float os, float oc)
    {
        float t = s + os;
        float bp = t - s;
        float err = (s - (t - bp)) + (os - bp);   // t + err == s + os exactly
        c = c + oc - err;
        s = t;
    }
    __device__ __forceinline__ void shfl_merge(int lane_mask)
    {
        float os = __shfl_xor_sync(0xffffffffu, s, lane_mask);
        float oc = __shfl_xor_sync(0xffffffffu, c, lane_mask);
        merge(os, oc);
    }
};

struct Plain64 {
    double s;
    __device__ __forceinline__ Plain64() : s(0.0) {}
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ void shfl_merge(int lane_mask) { s += __shfl_xor_sync(0xffffffffu, s, lane_mask); }
};

template <typename T>
struct PairConst {
    T c_div, c_edac, c_p, c_visc, c_av_m;   // c_av_m = m * alpha h c / rho0
    T vol;                                   // m / rho0 (steady convection term)
    int edac, use_av, steady, rare;         // rare = use_av || steady
};

template <typename T>
__device__ __forceinline__ PairConst<T> pair_const(const Phys &P)
{
    PairConst<T> k;
    k.c_div = (T)P.c_div;
    k.c_edac = (T)P.c_edac;
    k.c_p = (T)P.c_p;
    k.c_visc = (T)P.c_visc;
    k.c_av_m = (T)(P.m * P.c_av);
    k.vol = (T)P.vol;
    k.edac = P.edac;
    k.use_av = P.use_av;
    k.steady = P.steady;
    k.rare = P.use_av || P.steady;
    return k;
}

// One pair's contribution. g: gradW_ij (D comps), F: F_ij. vi, pi: own velocity
// and pressure; vj_div, vj_vis: neighbour velocity seen by the divergence and by
// the viscous term (equal for fluid neighbours); pj: neighbour pressure. In the
// steady-state mode (k.steady) the convection term is added.
template <int D, typename T, typename Acc>
__device__ __forceinline__ void pair_accumulate(const PairConst<T> &k, const T *g, T F, const T *vi, T pi,
                                                const T *vj_div, const T *vj_vis, T pj, Acc &ap, Acc *Fi)
{
    using A = Ar<T>;
    T vdg = T(0);
    T vv[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        vdg = A::fma(A::sub(vi[a], vj_div[a]), g[a], vdg);
        vv[a] = A::sub(vi[a], vj_vis[a]);
    }
    T t_ap = A::mul(k.c_div, vdg);
    if (k.edac) t_ap = A::fma(A::mul(k.c_edac, A::sub(pi, pj)), F, t_ap);
    ap.add(t_ap);
    T pres = A::mul(k.c_p, A::add(pi, pj));
    const T cv = A::mul(k.c_visc, F);
    // the terms that most runs do without (artificial viscosity, the steady-mode
    // convection) sit behind one uniform test
    if (k.rare) {
        if (k.use_av) {
            // v_ij . r_ij < 0  <=>  v_ij . gradW > 0 (dW/dr < 0); phi_ij = (v_ij . gradW) F / |gradW|^2
            T vvg = T(0), g2 = T(0);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                vvg = A::fma(vv[a], g[a], vvg);
                g2 = A::fma(g[a], g[a], g2);
            }
            if (vvg > T(0) && g2 > T(0)) pres = A::sub(pres, A::mul(k.c_av_m, A::mul(vvg, F)) / g2);   // -m Pi_ij
        }
        if (k.steady) {
            // convection of Eq. (mom-steady): -(V_i m_i/rho_i + V_j m_j/rho_j) (V_i . gradW_ij),
            // V_j the divergence-side velocity (prescribed for a wall)
            T vg = T(0);
#pragma unroll
            for (int a = 0; a < D; ++a) vg = A::fma(vi[a], g[a], vg);
#pragma unroll
            for (int a = 0; a < D; ++a)
                Fi[a].add(A::sub(A::fma(cv, vv[a], A::mul(-pres, g[a])),
                                 A::mul(A::mul(k.vol, A::add(vi[a], vj_div[a])), vg)));
            return;
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) Fi[a].add(A::fma(cv, vv[a], A::mul(-pres, g[a])));
}

}  // namespace dtsph
