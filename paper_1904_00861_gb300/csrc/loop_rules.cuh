// The stop rules of the pseudo-time loop and the fixed-order reductions of its
// residual partials, shared by every loop driver.
#pragma once

#include "dtsph_internal.cuh"

namespace dtsph {

// Stop rules of Sec. 3.4 on the residual history (ring of the last 16).
__device__ inline int stop_rule(const LoopState &L, int k1)
{
    double rp = L.hist_p[(k1 - 1) & 15], rv = L.hist_v[(k1 - 1) & 15];
    if (!isfinite(rp) || !isfinite(rv)) return 3;
    if (L.fixed_iters > 0) return k1 >= L.fixed_iters ? 4 : -1;
    if (rp < L.eps && rv < L.eps) return 0;
    int w = L.stag_window;
    if (w > 0 && k1 >= w) {
        bool stag = true;
        for (int which = 0; which < 2 && stag; ++which) {
            const double *h = which ? L.hist_v : L.hist_p;
            double lo = h[(k1 - 1) & 15], hi = lo;
            for (int t = k1 - w; t < k1; ++t) {
                double v = h[t & 15];
                lo = fmin(lo, v);
                hi = fmax(hi, v);
            }
            if (!(hi > 0.0 && (hi - lo) / hi < L.stag_tol)) stag = false;
        }
        if (stag) return 1;
    }
    if (k1 >= L.max_iter) return 2;
    return -1;
}

// stop_rule, or kPaused when no rule holds and the loop reached its pause count.
__device__ __forceinline__ int stop_or_pause(const LoopState &L, int k1)
{
    const int r = stop_rule(L, k1);
    return r < 0 && L.pause_at > 0 && k1 >= L.pause_at ? kPaused : r;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sum of (s + e) pairs with two-sum compensation: s accumulates the
// rounded sum, e the exact rounding errors of every addition.
__device__ __forceinline__ void warp_sum2(float &s, float &e)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, s, o);
        const float oe = __shfl_xor_sync(0xffffffffu, e, o);
        const float t = s + os;
        const float bp = t - s;
        const float err = (s - (t - bp)) + (os - bp);
        s = t;
        e = e + oe + err;
    }
}

// Fixed-order sum of the ntiles per-tile partials at blk (pairs of doubles), by
// the whole block; every caller gets the same bits. Result on thread 0.
__device__ __forceinline__ void reduce_tiles(const double *blk, int ntiles, double (&red)[2][kBlock / kWarp],
                                             double &sa, double &sb)
{
    double a = 0, b = 0;
    for (int q = threadIdx.x; q < ntiles; q += blockDim.x) {
        a += __ldcg(&blk[2 * q]);
        b += __ldcg(&blk[2 * q + 1]);
    }
    a = warp_sum<double>(a);
    b = warp_sum<double>(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sa = 0;
        sb = 0;
        for (int w = 0; w < kBlock / kWarp; ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
    }
}

// Resets the pseudo-time loop state of every instance for the loop of a new
// real step (one block: its threads loop over the instances), points each
// instance at the entry of the statistics ring that step will write and clears
// that entry's max|V|, which the outer step accumulates.
__device__ __forceinline__ void reset_loops(const Buffers &B)
{
    for (int i = threadIdx.x; i < B.ninst; i += blockDim.x) {
        LoopState *ls = B.ls + i;
        ls->iter = 0;
        ls->done = 0;
        ls->reason = -1;
        ls->ticket = 0;
        ls->rp = 0;
        ls->rv = 0;
        const int slot = (int)(ls->step % kStatRing);
        ls->stat_slot = slot;
        B.stats[(size_t)slot * B.ninst + i].vmax = 0.0;
        if (B.il) {
            B.il[i].claim = 0ull;
            B.il[i].done_tiles = 0u;
        }
    }
    if (threadIdx.x == 0) {
        B.ctrl->ticket = 0;
        B.ctrl->bar = 0;
        B.ctrl->active = B.ninst;
    }
}

// In a step graph that holds both pair-term forms (form = 0): true in a launch
// whose form_run is not the step's current form. Block-uniform, so a kernel
// may return before any barrier.
__device__ __forceinline__ bool skip_form(const Buffers &B)
{
    return B.form_sel && *(volatile const int *)B.form_sel != B.form_run;
}

// First tile and end tile of instance i for tiles of ppb slots.
__device__ __forceinline__ void instance_tiles(const Inst &I, int ppb, int &lo, int &hi)
{
    lo = I.slot_off / ppb;
    hi = (I.slot_off + I.nf + I.nw + ppb - 1) / ppb;
}

// Updates the loop state of one instance with the residual sums of iteration
// `it` and applies the stop rules; thread 0 only. Returns the stop reason (-1:
// continue; kPaused: the loop pauses, the instance leaves this launch).
__device__ __forceinline__ int finish_iteration(LoopState *ls, const Phys &P, int it, double sa, double sb)
{
    // work on a register copy: one batch of loads instead of a chain of
    // dependent global accesses
    LoopState st = *ls;
    const int k1 = it + 1;
    st.rp = sa * P.rp_scale;
    st.rv = sb * P.rv_scale;
    st.hist_p[it & 15] = st.rp;
    st.hist_v[it & 15] = st.rv;
    const int r = stop_or_pause(st, k1);
    ls->rp = st.rp;
    ls->rv = st.rv;
    ls->hist_p[it & 15] = st.rp;
    ls->hist_v[it & 15] = st.rv;
    ls->iter = k1;
    ls->reason = r;
    ls->done = r != -1;
    return r;
}

}  // namespace dtsph
