// Pair geometry shared by the kernels that walk neighbour lists: separations
// in FP64 (minimum image) and from FP32 cell offsets, the cell shift of a list
// entry, the kernel gradient and F_ij of a pair, and the packed neighbour
// records.
#pragma once

#include "pair_terms.cuh"

namespace dtsph {

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

// FP32 separation from cell offsets: the own offset is first moved by the cell
// shift (dx, dy, dz) s, then the neighbour's offset is subtracted; both the
// traversal test and the pair terms use this form, so they see the same bits.
template <int D>
__device__ __forceinline__ float4 shifted_offset(float4 oi, int dx, int dy, int dz, const float *sf)
{
    using A = Ar<float>;
    float4 p;
    p.x = A::fma(-(float)dx, sf[0], oi.x);
    p.y = A::fma(-(float)dy, sf[1], oi.y);
    p.z = D == 3 ? A::fma(-(float)dz, sf[2], oi.z) : 0.f;
    p.w = 0.f;
    return p;
}

template <int D>
__device__ __forceinline__ float sep32(float4 ps, float4 oj, float &f0, float &f1, float &f2)
{
    using A = Ar<float>;
    f0 = A::sub(ps.x, oj.x);
    f1 = A::sub(ps.y, oj.y);
    f2 = D == 3 ? A::sub(ps.z, oj.z) : 0.f;
    float q2 = A::fma(f1, f1, A::mul(f0, f0));
    if (D == 3) q2 = A::fma(f2, f2, q2);
    return q2;
}

// r_ij and |r_ij|^2 in the working precision T of a listed neighbour j (cell
// shift (dx, dy, dz)), with the arithmetic of the traversal test.
template <int D, bool F32, typename T>
__device__ __forceinline__ void listed_sep(const Geom &G, const double *__restrict__ x, const float4 *__restrict__ off,
                                           int n, int i, int j, float4 oi, int dx, int dy, int dz, T *d, T &r2)
{
    if (F32) {
        float f0, f1, f2;
        const float q2 = sep32<D>(shifted_offset<D>(oi, dx, dy, dz, G.s_f), off[j], f0, f1, f2);
        d[0] = (T)f0;
        d[1] = (T)f1;
        if (D == 3) d[2] = (T)f2;
        r2 = (T)q2;
    } else {
        double e[3];
        const double q2 = sep64<D>(G, x, n, i, j, e);
#pragma unroll
        for (int a = 0; a < D; ++a) d[a] = (T)e[a];
        r2 = (T)q2;
    }
}

// listed_sep's FP32C separation with the neighbour's offset oj already loaded
// (the same operations, so the same bits).
template <int D, typename T>
__device__ __forceinline__ void offset_sep(const Geom &G, float4 oi, float4 oj, int code, T *d, T &r2);

// Cell shift of a list entry.
__device__ __forceinline__ void decode_shift(int code, int &dx, int &dy, int &dz)
{
    dx = code % 3 - 1;
    dy = (code / 3) % 3 - 1;
    dz = code / 9 - 1;
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

template <int D, typename T>
__device__ __forceinline__ void offset_sep(const Geom &G, float4 oi, float4 oj, int code, T *d, T &r2)
{
    int dx, dy, dz;
    decode_shift(code, dx, dy, dz);
    float f0, f1, f2;
    const float q2 = sep32<D>(shifted_offset<D>(oi, dx, dy, dz, G.s_f), oj, f0, f1, f2);
    d[0] = (T)f0;
    d[1] = (T)f1;
    if (D == 3) d[2] = (T)f2;
    r2 = (T)q2;
}

}  // namespace dtsph
