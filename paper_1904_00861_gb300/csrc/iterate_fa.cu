// The pseudo-time loop kernels in the form without a pair cache ("Form A"):
// every pseudo-iteration recomputes the geometry of each pair from the
// neighbour lists at r^0 with the operations of the pair-cache pass, so the
// results are the bits of the cached form. It skips the pair-cache pass (a
// write of 16-36 bytes per pair per real step) and pays for it with the
// geometry of every pair in every iteration: the cheaper form when a step takes
// few iterations. Contexts without walls, particles frozen in pseudo-time.
// The kernels are those of loop_kernels.cuh, instantiated here for that form so
// that the two forms compile in parallel.
#include "loop_kernels.cuh"

namespace dtsph {

namespace {

template <int D, bool F>
void iterate_fa_lanes(const Buffers &B, unsigned long long cond, int use_cond, cudaStream_t st)
{
    const int nb = iterate_tiles(B);
    switch (B.lanes) {
    case 1: k_iterate<D, F, false, 1, true><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    case 2: k_iterate<D, F, false, 2, true><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    case 4: k_iterate<D, F, false, 4, true><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    default: k_iterate<D, F, false, 8, true><<<nb, kBlock, 0, st>>>(B, cond, use_cond); break;
    }
}

template <int D, bool F>
const void *loop_fa_lanes(const Buffers &B)
{
    if (B.async_loop) {
        switch (B.lanes) {
        case 1: return async_kernel<D, F, 1, true>();
        case 2: return async_kernel<D, F, 2, true>();
        case 4: return async_kernel<D, F, 4, true>();
        default: return async_kernel<D, F, 8, true>();
        }
    }
    switch (B.lanes) {
    case 1: return loop_kernel<D, F, false, 1, true>();
    case 2: return loop_kernel<D, F, false, 2, true>();
    case 4: return loop_kernel<D, F, false, 4, true>();
    default: return loop_kernel<D, F, false, 8, true>();
    }
}

}  // namespace

void launch_iterate_fa(const Buffers &B, unsigned long long cond, int use_cond, cudaStream_t st)
{
    if (B.dim == 2) {
        if (B.fp32c) iterate_fa_lanes<2, true>(B, cond, use_cond, st);
        else iterate_fa_lanes<2, false>(B, cond, use_cond, st);
    } else {
        if (B.fp32c) iterate_fa_lanes<3, true>(B, cond, use_cond, st);
        else iterate_fa_lanes<3, false>(B, cond, use_cond, st);
    }
}

const void *loop_function_fa(const Buffers &B)
{
    if (B.dim == 2) return B.fp32c ? loop_fa_lanes<2, true>(B) : loop_fa_lanes<2, false>(B);
    return B.fp32c ? loop_fa_lanes<3, true>(B) : loop_fa_lanes<3, false>(B);
}

}  // namespace dtsph
