// Allocation-free variant of the rate evaluation (dtsph_eval_rates_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the rates:
// code that runs while someone else's stream capture is open (a cudaMalloc there
// is not part of the capture and can invalidate it), solvers embedded in an
// application that reserved its whole device-memory budget up front, and code
// called from places where a synchronous allocation could stall or deadlock the
// host thread. This entry point serves them: it works entirely in one fixed
// scratch array that is part of the library image, and the caller passes device
// pointers for every input and output.
//
// The scratch array is a file-scope __device__ variable of kScratchBytes bytes;
// every GPU that loads the library holds it until the process exits. In host
// code its name is only a host-side stand-in, so its device address is fetched
// once per device with cudaGetSymbolAddress (on the first call made with that
// device current) and passed to the kernels. All calls share the array and it
// keeps the contents of the last call; the cell counters that must start at zero
// are cleared on every call. Two calls whose GPU work overlaps (on different
// streams, or from different host threads) race on the array and give wrong
// results; calls ordered on one stream are fine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "dtsph_internal.cuh"

namespace dtsph {
namespace {

// Limits of the fixed scratch: particles (fluid + wall), cells, and neighbour
// list entries (padded particles x neighbour capacity).
constexpr int kNoallocMaxParticles = 16384;
constexpr int kNoallocMaxCells = 32768;
constexpr size_t kNoallocMaxEntries = (size_t)kNoallocMaxParticles * 192;

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// The arrays carve() takes, in its order, for n slots, ncell cells and K list
// entries per slot: each size in bytes before its 256-byte rounding.
constexpr int kCarveArrays = 30;
struct Carve {
    size_t bytes[kCarveArrays];
    int count;
};
constexpr Carve carve_sizes(size_t n, size_t ncell, size_t K)
{
    const size_t nd = n * 3;
    Carve c{{4 * n, 8 * nd, 8 * nd, 8 * nd, 8 * n,               // gid_a, x_a, vn_a, vnm1_a, pn_a
             4 * n, 4 * n, 4 * n, 4 * n,                          // key, slot, unsorted, perm
             4 * n, 8 * nd, 8 * nd, 8 * nd, 8 * n, 4 * n,         // gid_b, x_b, vn_b, vnm1_b, pn_b, cell_b
             16 * n, 32 * n, 8 * n, 8 * nd, 4 * n,                // off, packed (V, p), ap_b, f_b, pcount
             4 * n * K, 4 * n * ((K + 7) / 8 * 8),                // pj, pjt (rows rounded up to 8)
             4 * (ncell + 1), 4 * (ncell + 1), 4 * (ncell / 4096 + 2),   // cell_count, cell_start, scan_tmp
             256, 2 * n, sizeof(Inst), sizeof(Geom), sizeof(Phys)},     // err, inst_of, tables
            kCarveArrays};
    return c;
}
constexpr size_t carve_total(size_t n, size_t ncell, size_t K)
{
    const Carve c = carve_sizes(n, ncell, K);
    size_t t = 0;
    for (int i = 0; i < c.count; ++i) t += round256(c.bytes[i]);
    return t;
}

// Scratch bytes: the carve of the largest accepted input (every limit at once),
// with room for the 256-byte rounding of each array and for the list staging
// rows, which are rounded up to 8 entries (at most 7 more per particle). Any
// input within the limits needs less: each array grows with n, the cells or n K
// only.
constexpr size_t kScratchBytes = carve_total(kNoallocMaxParticles, kNoallocMaxCells + 1, 192) +
                                 256 * kCarveArrays + 4 * 7 * (size_t)kNoallocMaxParticles;
static_assert(carve_total(kNoallocMaxParticles, kNoallocMaxCells + 1, 192) <= kScratchBytes,
              "the largest accepted input fits the scratch array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices];   // device address of the array, per device

// Device address of the scratch array on the current device (fetched once).
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return DTSPH_E_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DTSPH_E_CUDA;
        }
        g_scratch_ptr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_ptr[dev];
    return DTSPH_OK;
}

// Carves the arrays of a Buffers view out of the scratch array (256-byte
// aligned, the order and sizes of carve_sizes); returns the bytes used.
size_t carve(unsigned char *base, int n, int ncell, Buffers &B)
{
    const Carve sz = carve_sizes((size_t)n, (size_t)ncell, (size_t)B.K);
    size_t off = 0;
    int at = 0;
    auto take = [&]() {
        unsigned char *p = base + off;
        off += round256(sz.bytes[at++]);
        return (void *)p;
    };
    B.gid_a = (uint32_t *)take();
    B.x_a = (double *)take();
    B.vn_a = (double *)take();
    B.vnm1_a = (double *)take();
    B.pn_a = (double *)take();
    B.key = (int *)take();
    B.slot = (int *)take();
    B.unsorted = (int *)take();
    B.perm = (int *)take();
    B.gid_b = (uint32_t *)take();
    B.x_b = (double *)take();
    B.vn_b = (double *)take();
    B.vnm1_b = (double *)take();
    B.pn_b = (double *)take();
    B.cell_b = (int *)take();
    B.off = (float4 *)take();
    void *nb = take();
    if (B.fp32c) B.nb32[1] = (float4 *)nb;
    else B.nb64[1] = (double4_32a *)nb;
    B.ap_b = (double *)take();
    B.f_b = (double *)take();
    B.pcount = (int *)take();
    B.pj = (uint32_t *)take();
    B.pjt = (uint32_t *)take();
    B.cell_count = (int *)take();
    B.cell_start = (int *)take();
    B.scan_tmp = (int *)take();
    B.err = (uint32_t *)take();
    B.inst_of = (uint16_t *)take();
    B.inst = (Inst *)take();
    B.geo = (Geom *)take();
    B.phys = (Phys *)take();
    return at == sz.count ? off : (size_t)-1;
}

// The device-side error bits of the call as a status code for the caller.
__global__ void k_noalloc_status(const uint32_t *err, int32_t *status)
{
    const uint32_t e = *err;
    *status = (e & kErrCapacity) ? DTSPH_E_CAPACITY : (e & kErrDomain) ? DTSPH_E_DOMAIN : DTSPH_OK;
}

}  // namespace
}  // namespace dtsph

using namespace dtsph;

extern "C" int dtsph_eval_rates_noalloc(const dtsph_params *p, int64_t nf, const double *x, const double *v,
                                        const double *pr, int64_t nw, const double *xw, const double *vw, double *ap,
                                        double *F, int32_t *status, void *stream)
{
    if (!p || !x || !v || !pr || !ap || !F || nf <= 0 || nw < 0 || (nw > 0 && !xw)) return DTSPH_E_ARG;
    const int64_t nslots = (nf + nw + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
    if (nslots > kNoallocMaxParticles) return DTSPH_E_CAPACITY;   // beyond the fixed scratch
    // the same reading of the parameters as dtsph_create / dtsph_eval_rates
    int r = check_params(p, nullptr, 0);
    if (r) return r;
    Geom G;
    if ((r = make_geometry(*p, G, nullptr, 0))) return r;
    if (G.ncell + 1 > kNoallocMaxCells + 1) return DTSPH_E_CAPACITY;
    Phys P;
    make_phys(*p, P);

    // the kernels run on the caller's stream, so the scratch address must be the
    // one of that stream's device, which must be the current one
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return DTSPH_E_CUDA;
    }
    if (sdev != dev) return DTSPH_E_ARG;
    unsigned char *base = nullptr;
    if ((r = scratch_address(dev, &base))) return r;
    Buffers B;
    memset(&B, 0, sizeof B);
    B.n = (int)nslots;
    B.nf = (int)nf;
    B.nw = (int)nw;
    B.dim = p->dim;
    B.fp32c = p->precision == DTSPH_FP32C;
    B.ninst = 1;
    B.ncell = G.ncell + 1;           // the instance's cells and its empty sentinel cell
    B.nseg2 = (G.nc[0] + kSeg2 - 1) / kSeg2 * G.nc[1] * G.nc[2];   // the 2D FP32C builder's row segments
    B.K = neighbour_capacity(*p);
    if ((size_t)B.n * B.K > kNoallocMaxEntries) return DTSPH_E_CAPACITY;
    if (carve(base, B.n, B.ncell, B) > kScratchBytes) return DTSPH_E_CAPACITY;
    Inst I;
    memset(&I, 0, sizeof I);
    I.nf = (int)nf;
    I.nw = (int)nw;

    // the counting sort needs zeroed cell counters and -1 in the permutation
    // slots it never writes, and padding slots need empty neighbour lists; the
    // last call may have left any state there
    if (cudaMemsetAsync(B.cell_count, 0, sizeof(int) * (size_t)B.ncell, st) != cudaSuccess ||
        cudaMemsetAsync(B.err, 0, sizeof(uint32_t), st) != cudaSuccess ||
        cudaMemsetAsync(B.pcount, 0, sizeof(int) * (size_t)B.n, st) != cudaSuccess ||
        cudaMemsetAsync(B.unsorted, 0xff, sizeof(int) * (size_t)B.n, st) != cudaSuccess ||
        cudaMemsetAsync(B.perm, 0xff, sizeof(int) * (size_t)B.n, st) != cudaSuccess ||
        cudaMemsetAsync((void *)B.inst_of, 0, sizeof(uint16_t) * (size_t)B.n, st) != cudaSuccess) {
        cudaGetLastError();
        return DTSPH_E_CUDA;
    }
    launch_fill_instance((Inst *)B.inst, (Geom *)B.geo, (Phys *)B.phys, 0, I, G, P, st);
    launch_scatter_in(B, x, v, pr, nullptr, xw, vw, st);
    launch_binning(B, B.x_a, B.gid_a, st);
    launch_permute_a_to_b(B, st);
    launch_state_n(B, false, st);
    launch_unpermute(B, B.gid_b, B.ap_b, ap, 1, st);
    launch_unpermute(B, B.gid_b, B.f_b, F, B.dim, st);
    if (status) k_noalloc_status<<<1, 1, 0, st>>>(B.err, status);
    if (cudaGetLastError() != cudaSuccess) return DTSPH_E_CUDA;
    return DTSPH_OK;
}
