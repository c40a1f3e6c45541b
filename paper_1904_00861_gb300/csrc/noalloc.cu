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

#include "../../include/dtsph.h"
#include "dtsph_internal.cuh"

namespace dtsph {
namespace {

// Limits of the fixed scratch: particles (fluid + wall), cells, and neighbour
// list entries (padded particles x neighbour capacity).
constexpr int kNoallocMaxParticles = 16384;
constexpr int kNoallocMaxCells = 32768;
constexpr size_t kNoallocMaxEntries = (size_t)kNoallocMaxParticles * 192;

// Bytes per particle of the arrays the rate evaluation touches (see carve()).
constexpr size_t kPerParticle = 4 + 3 * 8 * 3 + 8 + 4 * 4 + 4 + 3 * 8 * 3 + 8 + 4 + 16 + 32 + 8 + 3 * 8 + 2;
constexpr size_t kScratchBytes =
    ((kPerParticle * kNoallocMaxParticles + 5 * kNoallocMaxEntries + 2 * 4 * (size_t)(kNoallocMaxCells + 1) +
      64 * 256) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices];   // device address of the array, per device

// Device address of the scratch array on the current device (fetched once).
int scratch_address(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DTSPH_E_CUDA;
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

// Carves the arrays of a Buffers view out of the scratch array (256-byte aligned);
// returns the bytes used.
size_t carve(unsigned char *base, int n, int ncell, Buffers &B)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base + off;
        off += (bytes + 255) / 256 * 256;
        return (void *)p;
    };
    const size_t nd = (size_t)n * 3;
    B.gid_a = (uint32_t *)take(4 * (size_t)n);
    B.x_a = (double *)take(8 * nd);
    B.vn_a = (double *)take(8 * nd);
    B.vnm1_a = (double *)take(8 * nd);
    B.pn_a = (double *)take(8 * (size_t)n);
    B.key = (int *)take(4 * (size_t)n);
    B.slot = (int *)take(4 * (size_t)n);
    B.unsorted = (int *)take(4 * (size_t)n);
    B.perm = (int *)take(4 * (size_t)n);
    B.gid_b = (uint32_t *)take(4 * (size_t)n);
    B.x_b = (double *)take(8 * nd);
    B.vn_b = (double *)take(8 * nd);
    B.vnm1_b = (double *)take(8 * nd);
    B.pn_b = (double *)take(8 * (size_t)n);
    B.cell_b = (int *)take(4 * (size_t)n);
    B.off = (float4 *)take(16 * (size_t)n);
    void *nb = take(32 * (size_t)n);
    if (B.fp32c) B.nb32[1] = (float4 *)nb;
    else B.nb64[1] = (double4_32a *)nb;
    B.ap_b = (double *)take(8 * (size_t)n);
    B.f_b = (double *)take(8 * nd);
    B.pcount = (int *)take(4 * (size_t)n);
    B.pj = (uint32_t *)take(4 * (size_t)n * B.K);
    B.pcode = (uint8_t *)take((size_t)n * B.K);
    B.cell_count = (int *)take(4 * (size_t)(ncell + 1));
    B.cell_start = (int *)take(4 * (size_t)(ncell + 1));
    B.scan_tmp = (int *)take(4 * (size_t)(ncell / 4096 + 2));
    B.err = (uint32_t *)take(256);
    B.inst_of = (uint16_t *)take(2 * (size_t)n);
    B.inst = (Inst *)take(sizeof(Inst));
    B.geo = (Geom *)take(sizeof(Geom));
    B.phys = (Phys *)take(sizeof(Phys));
    return off;
}

// Neighbour list entries per particle: max_neighbors, else 1.35 times the mean
// count of a uniform fill of the 3h sphere (disc) plus 8.
int neighbour_capacity_noalloc(const dtsph_params *p)
{
    if (p->max_neighbors > 0) return p->max_neighbors;
    const double pi = 3.14159265358979323846;
    const double vol = p->m / p->rho0, rc = 3.0 * p->h;
    const double expect = p->dim == 2 ? pi * rc * rc / vol : 4.0 / 3.0 * pi * rc * rc * rc / vol;
    const int k = (int)std::ceil(1.35 * expect) + 8;
    return std::min(std::max(k, 8), 4096);
}

double quintic_sigma_noalloc(int dim, double h)
{
    const double pi = 3.14159265358979323846;
    return dim == 2 ? 7.0 / (478.0 * pi * h * h) : 1.0 / (120.0 * pi * h * h * h);
}

}  // namespace
}  // namespace dtsph

using namespace dtsph;

extern "C" int dtsph_eval_rates_noalloc(const dtsph_params *p, int64_t nf, const double *x, const double *v,
                                        const double *pr, int64_t nw, const double *xw, const double *vw, double *ap,
                                        double *F, void *stream)
{
    if (!p || !x || !v || !pr || !ap || !F || nf <= 0 || nw < 0 || (nw > 0 && !xw)) return DTSPH_E_ARG;
    const int64_t nslots = (nf + nw + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
    if (nslots > kNoallocMaxParticles) return DTSPH_E_CAPACITY;   // beyond the fixed scratch
    if ((p->dim != 2 && p->dim != 3) || (p->precision != DTSPH_FP64 && p->precision != DTSPH_FP32C))
        return DTSPH_E_ARG;
    if (!(p->h > 0) || !(p->m > 0) || !(p->rho0 > 0) || !(p->beta > 0) || !(p->v_ref > 0) || !(p->dt > 0) ||
        !(p->eta > 0) || !(p->nu >= 0) || !(p->alpha >= 0))
        return DTSPH_E_ARG;
    if (p->edac_h2_literal) return DTSPH_E_UNSUPPORTED;

    // cell grid: cells wider than 3h, at least three per periodic axis
    Geom G;
    memset(&G, 0, sizeof G);
    G.dim = p->dim;
    const double rc = 3.0 * p->h;
    G.ncell = 1;
    for (int a = 0; a < 3; ++a) {
        G.periodic[a] = a < p->dim ? p->periodic[a] : 0;
        G.lo[a] = p->lo[a];
        G.hi[a] = p->hi[a];
        if (a >= p->dim) {
            G.nc[a] = 1;
            G.s[a] = G.inv_s[a] = G.L[a] = 1.0;
            G.s_f[a] = 1.f;
            G.halfL[a] = 0.5;
            continue;
        }
        const double L = p->hi[a] - p->lo[a];
        if (!(L > 0)) return DTSPH_E_ARG;
        long long k = (long long)std::floor(L / (rc * (1.0 + 1e-9)));
        if (k < 1) k = 1;
        if (G.periodic[a] && k < 3) return DTSPH_E_ARG;
        if (k >= kNoallocMaxCells || (long long)G.ncell * k >= kNoallocMaxCells) return DTSPH_E_CAPACITY;
        G.nc[a] = (int)k;
        G.s[a] = L / (double)k;
        G.inv_s[a] = 1.0 / G.s[a];
        G.s_f[a] = (float)G.s[a];
        G.L[a] = L;
        G.halfL[a] = 0.5 * L;
        G.ncell *= (int)k;
    }
    G.rc2 = rc * rc;
    G.rc2_lo = (float)(G.rc2 * (1.0 - 2e-5));
    G.rc2_hi = (float)(G.rc2 * (1.0 + 2e-5));

    // pair-term constants, rho_i = rho_j = rho0
    Phys P;
    memset(&P, 0, sizeof P);
    P.h = p->h;
    P.m = p->m;
    P.rho0 = p->rho0;
    P.c = p->beta * p->v_ref;
    P.nu = p->nu;
    P.nu_e = p->h * P.c / 16.0;
    P.dt = p->dt;
    P.dtau = p->dt / p->beta;
    P.dtau_f = (float)P.dtau;
    P.sig_h = quintic_sigma_noalloc(p->dim, p->h) / p->h;
    P.inv_h = 1.0 / p->h;
    P.eta_h2 = p->eta * p->h * p->h;
    P.edac_h2 = P.eta_h2;
    const double rho = p->rho0;
    P.c_div = p->m * (rho / rho) * P.c * P.c;
    P.c_edac = 4.0 * p->m / ((rho + rho) * rho) * P.nu_e;
    P.c_p = p->m / (rho * rho);
    P.c_visc = 4.0 * p->m * p->nu / (rho + rho);
    P.c_av = p->alpha * p->h * P.c / rho;
    for (int a = 0; a < 3; ++a) P.g[a] = a < p->dim ? p->g[a] : 0.0;
    P.edac = p->edac;
    P.use_av = p->alpha != 0.0;

    unsigned char *base = nullptr;
    int r = scratch_address(&base);
    if (r) return r;
    Buffers B;
    memset(&B, 0, sizeof B);
    B.n = (int)nslots;
    B.nf = (int)nf;
    B.nw = (int)nw;
    B.dim = p->dim;
    B.fp32c = p->precision == DTSPH_FP32C;
    B.ninst = 1;
    B.ncell = G.ncell + 1;           // the instance's cells and its empty sentinel cell
    B.K = neighbour_capacity_noalloc(p);
    if ((size_t)B.n * B.K > kNoallocMaxEntries) return DTSPH_E_CAPACITY;
    if (carve(base, B.n, B.ncell, B) > kScratchBytes) return DTSPH_E_CAPACITY;
    Inst I;
    memset(&I, 0, sizeof I);
    I.nf = (int)nf;
    I.nw = (int)nw;

    cudaStream_t st = (cudaStream_t)stream;
    // the counting sort needs zeroed cell counters and -1 in the permutation
    // slots it never writes; the last call may have left any state there
    if (cudaMemsetAsync(B.cell_count, 0, sizeof(int) * (size_t)B.ncell, st) != cudaSuccess ||
        cudaMemsetAsync(B.err, 0, sizeof(uint32_t), st) != cudaSuccess ||
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
    if (cudaGetLastError() != cudaSuccess) return DTSPH_E_CUDA;
    return DTSPH_OK;
}
