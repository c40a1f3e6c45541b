// The pseudo-time loop's host side: the launches of the per-iteration and
// persistent loop kernels (their device code is in loop_kernels.cuh), the outer
// step and the loop reset.
#include <algorithm>

#include "loop_kernels.cuh"

namespace dtsph {

int iterate_tiles(const Buffers &B) { return (B.n + kBlock / B.lanes - 1) / (kBlock / B.lanes); }

template <int D, bool F, bool W>
static void iterate_lanes(const Buffers &B, unsigned long long cond, int use_cond, cudaStream_t st)
{
    const int nb = iterate_tiles(B);
    switch (B.lanes) {
    case 1: k_iterate<D, F, W, 1><<<nb, kBlock, ring_bytes<D, F>(B.stages), st>>>(B, cond, use_cond); break;
    case 2: k_iterate<D, F, W, 2><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    case 4: k_iterate<D, F, W, 4><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    default: k_iterate<D, F, W, 8><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    }
}

int launch_walls_iter(const Buffers &B, cudaStream_t st)
{
    if (B.nw == 0) return 0;
    const int nb = (int)(((long long)B.nw * kWallLanes + kBlock - 1) / kBlock);
    if (B.dim == 2) {
        if (B.fp32c) k_walls_iter<2, true><<<nb, kBlock, 0, st>>>(B);
        else k_walls_iter<2, false><<<nb, kBlock, 0, st>>>(B);
    } else {
        if (B.fp32c) k_walls_iter<3, true><<<nb, kBlock, 0, st>>>(B);
        else k_walls_iter<3, false><<<nb, kBlock, 0, st>>>(B);
    }
    return 1;
}

int launch_iterate(const Buffers &B, unsigned long long cond, int use_cond, cudaStream_t st)
{
    if (B.form_a) {
        launch_iterate_fa(B, cond, use_cond, st);
        return 1;
    }
    const bool w = B.nw > 0;
    if (B.dim == 2) {
        if (B.fp32c) { if (w) iterate_lanes<2, true, true>(B, cond, use_cond, st); else iterate_lanes<2, true, false>(B, cond, use_cond, st); }
        else { if (w) iterate_lanes<2, false, true>(B, cond, use_cond, st); else iterate_lanes<2, false, false>(B, cond, use_cond, st); }
    } else {
        if (B.fp32c) { if (w) iterate_lanes<3, true, true>(B, cond, use_cond, st); else iterate_lanes<3, true, false>(B, cond, use_cond, st); }
        else { if (w) iterate_lanes<3, false, true>(B, cond, use_cond, st); else iterate_lanes<3, false, false>(B, cond, use_cond, st); }
    }
    return 1;
}

template <int D, bool F, bool W>
static const void *loop_lanes(int lanes)
{
    switch (lanes) {
    case 1: return loop_kernel<D, F, W, 1>();
    case 2: return loop_kernel<D, F, W, 2>();
    case 4: return loop_kernel<D, F, W, 4>();
    default: return loop_kernel<D, F, W, 8>();
    }
}

// Dynamic shared memory of the iterate and loop kernels of this shape.
static size_t iterate_smem(const Buffers &B)
{
    if (B.lanes != 1 || B.form_a) return 0;              // the ring holds cache rows only
    if (B.dim == 2) return B.fp32c ? ring_bytes<2, true>(B.stages) : ring_bytes<2, false>(B.stages);
    return B.fp32c ? ring_bytes<3, true>(B.stages) : ring_bytes<3, false>(B.stages);
}

template <int D, bool F, bool W>
static cudaError_t allow_ring_smem()
{
    const int bytes = (int)ring_bytes<D, F>(kMaxStages);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_iterate<D, F, W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)k_loop<D, F, W, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && !W)
        e = cudaFuncSetAttribute((const void *)k_loop_async<D, F, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    return e;
}

template <int D, bool F>
static const void *async_lanes(int lanes)
{
    switch (lanes) {
    case 1: return async_kernel<D, F, 1>();
    case 2: return async_kernel<D, F, 2>();
    case 4: return async_kernel<D, F, 4>();
    default: return async_kernel<D, F, 8>();
    }
}

static const void *loop_function(const Buffers &B)
{
    if (B.form_a) return loop_function_fa(B);
    if (B.async_loop) {
        if (B.dim == 2) return B.fp32c ? async_lanes<2, true>(B.lanes) : async_lanes<2, false>(B.lanes);
        return B.fp32c ? async_lanes<3, true>(B.lanes) : async_lanes<3, false>(B.lanes);
    }
    const bool w = B.nw > 0;
    if (B.dim == 2) {
        if (B.fp32c) return w ? loop_lanes<2, true, true>(B.lanes) : loop_lanes<2, true, false>(B.lanes);
        return w ? loop_lanes<2, false, true>(B.lanes) : loop_lanes<2, false, false>(B.lanes);
    }
    if (B.fp32c) return w ? loop_lanes<3, true, true>(B.lanes) : loop_lanes<3, true, false>(B.lanes);
    return w ? loop_lanes<3, false, true>(B.lanes) : loop_lanes<3, false, false>(B.lanes);
}

int loop_grid(const Buffers &B, int *grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, loop_function(B), kBlock, iterate_smem(B)) !=
            cudaSuccess ||
        per_sm < 1)
        return -1;
    *grid = std::min(iterate_tiles(B), per_sm * sms);
    return 0;
}

cudaError_t launch_loop(const Buffers &B, int grid, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = iterate_smem(B);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Buffers b = B;
    void *args[] = {(void *)&b};
    return cudaLaunchKernelExC(&cfg, loop_function(B), args);
}

int launch_outer(const Buffers &B, cudaStream_t st)
{
    if (B.dim == 2) {
        if (B.fp32c) k_outer<2, true><<<blocks(B.n), kBlock, 0, st>>>(B);
        else k_outer<2, false><<<blocks(B.n), kBlock, 0, st>>>(B);
    } else {
        if (B.fp32c) k_outer<3, true><<<blocks(B.n), kBlock, 0, st>>>(B);
        else k_outer<3, false><<<blocks(B.n), kBlock, 0, st>>>(B);
    }
    return 1;
}

int iterate_prepare()
{
    cudaError_t e = allow_ring_smem<2, true, false>();
    if (e == cudaSuccess) e = allow_ring_smem<2, true, true>();
    if (e == cudaSuccess) e = allow_ring_smem<2, false, false>();
    if (e == cudaSuccess) e = allow_ring_smem<2, false, true>();
    if (e == cudaSuccess) e = allow_ring_smem<3, true, false>();
    if (e == cudaSuccess) e = allow_ring_smem<3, true, true>();
    if (e == cudaSuccess) e = allow_ring_smem<3, false, false>();
    if (e == cudaSuccess) e = allow_ring_smem<3, false, true>();
    return e == cudaSuccess ? 0 : -1;
}

int launch_loop_reset(const Buffers &B, cudaStream_t st)
{
    k_loop_reset<<<1, kBlock, 0, st>>>(B);
    return 1;
}

int launch_restart_steps(const Buffers &B, cudaStream_t st)
{
    k_restart_steps<<<1, kBlock, 0, st>>>(B);
    return 1;
}

int launch_loop_resume(const Buffers &B, cudaStream_t st)
{
    k_loop_resume<<<1, kBlock, 0, st>>>(B);
    return 1;
}

}  // namespace dtsph

