// Cell binning: cell keys, counting sort, per-cell ordering by caller index, and
// the gathers that move the particle state into the new order.
//
// The neighbour search of the paper (N(i) = all j with |r_ij| < 3h, Sec. 3) is
// built on cells of side >= 3h: a counting sort by cell gives every cell a
// contiguous slot range, and ordering each cell by caller index makes the
// result independent of the atomic order of the count pass.
#include "dtsph_internal.cuh"

namespace dtsph {

namespace {

__device__ __forceinline__ int cell_coord(double xa, double lo, double hi, double inv_s, int nc, int periodic,
                                          uint32_t *err)
{
    int k = (int)floor((xa - lo) * inv_s);
    if (k < 0) {
        if (!periodic && xa < lo) atomicOr(err, kErrDomain);
        k = 0;
    }
    if (k >= nc) {
        if (!periodic && xa > hi) atomicOr(err, kErrDomain);
        k = nc - 1;
    }
    return k;
}

__global__ void k_bin_keys(int n, Geom G, const double *__restrict__ x, int *__restrict__ key,
                           int *__restrict__ slot, int *__restrict__ count, uint32_t *err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0, mult = 1;
    for (int a = 0; a < G.dim; ++a) {
        int k = cell_coord(x[(size_t)a * n + i], G.lo[a], G.hi[a], G.inv_s[a], G.nc[a], G.periodic[a], err);
        c += k * mult;
        mult *= G.nc[a];
    }
    key[i] = c;
    slot[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan of the per-cell counts by one block; clears the counts for the
// next binning. Thread t owns a contiguous chunk of cells.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_counts(int ncell, int *__restrict__ count,
                                                              int *__restrict__ start)
{
    __shared__ int part[kScanThreads];
    int t = threadIdx.x;
    int chunk = (ncell + kScanThreads - 1) / kScanThreads;
    int b = t * chunk;
    int e = min(b + chunk, ncell);
    int sum = 0;
    for (int c = b; c < e; ++c) sum += count[c];
    part[t] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan of the chunk sums
    for (int off = 1; off < kScanThreads; off <<= 1) {
        int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - sum;
    for (int c = b; c < e; ++c) {
        int k = count[c];
        start[c] = run;
        run += k;
        count[c] = 0;
    }
    if (t == kScanThreads - 1) start[ncell] = part[t];
}

__global__ void k_scatter(int n, const int *__restrict__ key, const int *__restrict__ slot,
                          const int *__restrict__ start, int *__restrict__ perm)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[start[key[i]] + slot[i]] = i;
}

// Orders each cell by caller index: the particle in unsorted slot t moves to
// start[c] + (number of particles of its cell with a smaller caller index).
// One thread per particle; cells hold a few tens of particles.
__global__ void k_cell_rank(int n, const int *__restrict__ key, const int *__restrict__ start,
                            const int *__restrict__ unsorted, const uint32_t *__restrict__ gid, int *__restrict__ perm)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = unsorted[t];
    const int c = key[i];
    const uint32_t gi = gid[i];
    const int b = start[c], e = start[c + 1];
    int rank = 0;
    for (int u = b; u < e; ++u) rank += gid[unsorted[u]] < gi;
    perm[b + rank] = i;
}

__device__ __forceinline__ float4 cell_offset(const Geom &G, int cell, const double *x, int n, int s)
{
    int c0 = cell % G.nc[0];
    int c1 = (cell / G.nc[0]) % G.nc[1];
    int c2 = cell / (G.nc[0] * G.nc[1]);
    float4 o;
    o.x = (float)(x[s] - (G.lo[0] + c0 * G.s[0]));
    o.y = (float)(x[(size_t)n + s] - (G.lo[1] + c1 * G.s[1]));
    o.z = G.dim == 3 ? (float)(x[2 * (size_t)n + s] - (G.lo[2] + c2 * G.s[2])) : 0.f;
    o.w = 0.f;
    return o;
}

// A -> B at the start of a step: state n, and the packed (V^n, p^n) that the
// state-n pair pass gathers.
__global__ void k_permute_a_to_b(int n, int nf, int dim, int fp32c, Geom G, const int *__restrict__ perm,
                                 const int *__restrict__ key, const uint32_t *__restrict__ gid_a,
                                 const double *__restrict__ x_a, const double *__restrict__ vn_a,
                                 const double *__restrict__ vnm1_a, const double *__restrict__ pn_a,
                                 uint32_t *__restrict__ gid_b, double *__restrict__ x_b, double *__restrict__ vn_b,
                                 double *__restrict__ vnm1_b, double *__restrict__ pn_b, int *__restrict__ cell_b,
                                 float4 *__restrict__ off, double4_32a *__restrict__ nb64, float4 *__restrict__ nb32)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int o = perm[s];
    gid_b[s] = gid_a[o];
    int cell = key[o];
    cell_b[s] = cell;
    double v[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        size_t so = (size_t)a * n;
        x_b[so + s] = x_a[so + o];
        v[a] = vn_a[so + o];
        vn_b[so + s] = v[a];
        vnm1_b[so + s] = vnm1_a[so + o];
    }
    double p = pn_a[o];
    pn_b[s] = p;
    if (fp32c) {
        off[s] = cell_offset(G, cell, x_b, n, s);
        nb32[s] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)p);
    } else {
        nb64[s] = make_double4_32a(v[0], v[1], v[2], p);
    }
    (void)nf;
}

// B -> A after the predictor: the loop order. Carries r^n, r^0, V^n, the BDF2
// source, and seeds iterate 0 (V^0, p-hat^0).
__global__ void k_permute_b_to_a(int n, int dim, int fp32c, Geom G, const int *__restrict__ perm,
                                 const int *__restrict__ key, const uint32_t *__restrict__ gid_b,
                                 const double *__restrict__ x_b, const double *__restrict__ xp_b,
                                 const double *__restrict__ vn_b, const double *__restrict__ s_b,
                                 const double *__restrict__ v0_b, const double *__restrict__ ph0_b,
                                 uint32_t *__restrict__ gid_a, double *__restrict__ x_a, double *__restrict__ xp_a,
                                 double *__restrict__ vn_a, double *__restrict__ s_a, int *__restrict__ cell_a,
                                 float4 *__restrict__ off, double *__restrict__ vk0, double4_32a *__restrict__ nb64,
                                 float4 *__restrict__ nb32)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int o = perm[s];
    gid_a[s] = gid_b[o];
    int cell = key[o];
    cell_a[s] = cell;
    double v[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        size_t so = (size_t)a * n;
        x_a[so + s] = x_b[so + o];
        xp_a[so + s] = xp_b[so + o];
        vn_a[so + s] = vn_b[so + o];
        s_a[so + s] = s_b[so + o];
        v[a] = v0_b[so + o];
        vk0[so + s] = v[a];
    }
    double ph = ph0_b[o];
    if (fp32c) {
        off[s] = cell_offset(G, cell, xp_a, n, s);
        nb32[s] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)ph);
    } else {
        nb64[s] = make_double4_32a(v[0], v[1], v[2], ph);
    }
}

// Caller order -> order A (identity) from AoS inputs.
__global__ void k_scatter_in(int nf, int nw, int dim, const double *__restrict__ x, const double *__restrict__ v,
                             const double *__restrict__ p, const double *__restrict__ vprev,
                             const double *__restrict__ xw, const double *__restrict__ vw, uint32_t *__restrict__ gid,
                             double *__restrict__ x_a, double *__restrict__ vn_a, double *__restrict__ vnm1_a,
                             double *__restrict__ pn_a)
{
    int n = nf + nw;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    gid[s] = (uint32_t)s;
    if (s < nf) {
        for (int a = 0; a < dim; ++a) {
            size_t so = (size_t)a * n;
            x_a[so + s] = x[(size_t)s * dim + a];
            vn_a[so + s] = v[(size_t)s * dim + a];
            vnm1_a[so + s] = vprev ? vprev[(size_t)s * dim + a] : v[(size_t)s * dim + a];
        }
        pn_a[s] = p[s];
    } else {
        int w = s - nf;
        for (int a = 0; a < dim; ++a) {
            size_t so = (size_t)a * n;
            x_a[so + s] = xw[(size_t)w * dim + a];
            vn_a[so + s] = vw ? vw[(size_t)w * dim + a] : 0.0;
            vnm1_a[so + s] = vn_a[so + s];
        }
        pn_a[s] = 0.0;
    }
}

// Order A (SoA, comps components) -> caller order (AoS), fluid particles only.
__global__ void k_unpermute(int n, int nf, int comps, const uint32_t *__restrict__ gid, const double *__restrict__ src,
                            double *__restrict__ out)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint32_t g = gid[s];
    if (g >= (uint32_t)nf) return;
    for (int a = 0; a < comps; ++a) out[(size_t)g * comps + a] = src[(size_t)a * n + s];
}

inline int blocks(int n) { return (n + kBlock - 1) / kBlock; }

}  // namespace

int launch_binning(const Buffers &B, const Geom &G, const double *x_keys, const uint32_t *gid_src, cudaStream_t st)
{
    k_bin_keys<<<blocks(B.n), kBlock, 0, st>>>(B.n, G, x_keys, B.key, B.slot, B.cell_count, B.err);
    k_scan_counts<<<1, kScanThreads, 0, st>>>(G.ncell, B.cell_count, B.cell_start);
    k_scatter<<<blocks(B.n), kBlock, 0, st>>>(B.n, B.key, B.slot, B.cell_start, B.unsorted);
    k_cell_rank<<<blocks(B.n), kBlock, 0, st>>>(B.n, B.key, B.cell_start, B.unsorted, gid_src, B.perm);
    return 4;
}

int launch_permute_a_to_b(const Buffers &B, const Geom &G, cudaStream_t st)
{
    k_permute_a_to_b<<<blocks(B.n), kBlock, 0, st>>>(B.n, B.nf, B.dim, B.fp32c, G, B.perm, B.key, B.gid_a, B.x_a,
                                                     B.vn_a, B.vnm1_a, B.pn_a, B.gid_b, B.x_b, B.vn_b, B.vnm1_b,
                                                     B.pn_b, B.cell_b, B.off, B.nb64[1], B.nb32[1]);
    return 1;
}

int launch_permute_b_to_a(const Buffers &B, const Geom &G, cudaStream_t st)
{
    k_permute_b_to_a<<<blocks(B.n), kBlock, 0, st>>>(B.n, B.dim, B.fp32c, G, B.perm, B.key, B.gid_b, B.x_b, B.xp_b,
                                                     B.vn_b, B.s_b, B.v0_b, B.ph0_b, B.gid_a, B.x_a, B.xp_a, B.vn_a,
                                                     B.s_a, B.cell_a, B.off, B.vk[0], B.nb64[0], B.nb32[0]);
    return 1;
}

int launch_scatter_in(const Buffers &B, const double *x, const double *v, const double *p, const double *vprev,
                      const double *xw, const double *vw, cudaStream_t st)
{
    k_scatter_in<<<blocks(B.n), kBlock, 0, st>>>(B.nf, B.nw, B.dim, x, v, p, vprev, xw, vw, B.gid_a, B.x_a, B.vn_a,
                                                 B.vnm1_a, B.pn_a);
    return 1;
}

int launch_unpermute(const Buffers &B, const uint32_t *gid, const double *src, double *out, int comps, cudaStream_t st)
{
    k_unpermute<<<blocks(B.n), kBlock, 0, st>>>(B.n, B.nf, comps, gid, src, out);
    return 1;
}

}  // namespace dtsph
