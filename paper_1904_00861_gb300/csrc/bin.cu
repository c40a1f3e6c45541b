// Cell binning: cell keys, counting sort, per-cell ordering by caller index, and
// the gathers that move the particle state into the new order.
//
// The neighbour search of the paper (N(i) = all j with |r_ij| < 3h, Sec. 3) is
// built on cells of side > 3h: a counting sort by cell gives every cell a
// contiguous slot range, and ordering each cell by caller index makes the
// result independent of the atomic order of the count pass. All instances of a
// context are binned together: instance i's cells are numbered from its
// cell_off, and the scan places its particles at its own (tile-aligned) slot
// range.
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

// Cell (global index) of every particle of the source order; -1 for padding.
__global__ void __launch_bounds__(kBlock) k_bin_keys(Buffers B, const double *__restrict__ x,
                                                     const uint32_t *__restrict__ gid)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    if (gid[i] == kNoParticle) {
        B.key[i] = -1;
        return;
    }
    const int inst = B.inst_of[i];
    const Geom &G = B.geo[inst];
    int c = 0, mult = 1;
    for (int a = 0; a < G.dim; ++a) {
        int k = cell_coord(x[(size_t)a * B.n + i], G.lo[a], G.hi[a], G.inv_s[a], G.nc[a], G.periodic[a], B.err);
        c += k * mult;
        mult *= G.nc[a];
    }
    c += B.inst[inst].cell_off;
    B.key[i] = c;
    B.slot[i] = atomicAdd(&B.cell_count[c], 1);
}

// Exclusive scan of the per-cell counts, shifted so that each instance's
// particles start at its slot_off; clears the counts for the next binning.
// Three passes: per-block totals of kScanCells cells, a scan of those totals by
// one block, and the final per-cell scan of every block with its offset.
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;                              // cells per thread, several blocks
constexpr int kScanCells = kScanThreads * kScanPerThread;
constexpr int kScanPerThread1 = 16;                            // cells per thread, one block
constexpr int kScanCells1 = kScanThreads * kScanPerThread1;

// Exclusive prefix sum over the block (kScanThreads threads) of one value each.
__device__ __forceinline__ int block_exclusive_scan(int v)
{
    __shared__ int warp_tot[kScanThreads / kWarp];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        int z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        warp_tot[lane] = z - w;                 // exclusive prefix of the warp totals
    }
    __syncthreads();
    const int before = warp_tot[wid] + x - v;
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(Buffers B)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    const int base = blockIdx.x * kScanCells + threadIdx.x * kScanPerThread;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
        if (base + k < B.ncell) s += B.cell_count[base + k];
    // block sum
    __shared__ int red[kScanThreads / kWarp];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanThreads / kWarp; ++w) t += red[w];
        B.scan_tmp[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(Buffers B, int nblocks)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    // exclusive prefix of the block totals, in chunks of the block width
    int carry = 0;
    for (int base = 0; base < nblocks; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int v = i < nblocks ? B.scan_tmp[i] : 0;
        const int ex = block_exclusive_scan(v);
        if (i < nblocks) B.scan_tmp[i] = carry + ex;
        // block total: the inclusive value of the last thread
        __shared__ int last;
        if (threadIdx.x == kScanThreads - 1) last = ex + v;
        __syncthreads();
        carry += last;
        __syncthreads();
    }
}

// Instance owning cell c (instances are few; their cell ranges are ascending).
__device__ __forceinline__ int cell_instance(const Buffers &B, int c)
{
    int lo = 0, hi = B.ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.inst[mid].cell_off <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// PER cells per thread; MULTI: several blocks, each with the carry of the
// blocks before it (else one block scans every cell, with no carry)
template <int PER, bool MULTI>
__global__ void __launch_bounds__(kScanThreads) k_scan_final(Buffers B)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    const int base = blockIdx.x * kScanThreads * PER + threadIdx.x * PER;
    int v[PER];
    int s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = base + k < B.ncell ? B.cell_count[base + k] : 0;
        s += v[k];
    }
    int run = block_exclusive_scan(s) + (MULTI ? B.scan_tmp[blockIdx.x] : 0);
    if (base < B.ncell) {
        int inst = cell_instance(B, base);
        for (int k = 0; k < PER; ++k) {
            const int c = base + k;
            if (c >= B.ncell) break;
            while (inst + 1 < B.ninst && B.inst[inst + 1].cell_off <= c) ++inst;
            B.cell_start[c] = run + B.inst[inst].shift;
            run += v[k];
            B.cell_count[c] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) B.cell_start[B.ncell] = B.n;
}

__global__ void __launch_bounds__(kBlock) k_scatter(Buffers B)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.n) return;
    const int c = B.key[i];
    if (c < 0) return;
    B.unsorted[B.cell_start[c] + B.slot[i]] = i;
}

// Orders each cell by caller index: the particle in unsorted slot t moves to
// start[c] + (number of particles of its cell with a smaller caller index).
// One thread per slot; cells hold a few tens of particles; padding slots (never
// written by the scatter) stay -1.
__global__ void __launch_bounds__(kBlock) k_cell_rank(Buffers B, const uint32_t *__restrict__ gid)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.n) return;
    const int i = B.unsorted[t];
    if (i < 0) return;
    const int c = B.key[i];
    const uint32_t gi = gid[i];
    const int b = B.cell_start[c], e = B.cell_start[c + 1];
    int rank = 0;
    for (int u = b; u < e; ++u) rank += gid[B.unsorted[u]] < gi;
    B.perm[b + rank] = i;
}

// FP32 offset of slot s from the origin of its cell; .w is 1 for a wall particle.
__device__ __forceinline__ float4 cell_offset(const Geom &G, int local_cell, const double *x, int n, int s, bool wall)
{
    const int c0 = local_cell % G.nc[0];
    const int c1 = (local_cell / G.nc[0]) % G.nc[1];
    const int c2 = local_cell / (G.nc[0] * G.nc[1]);
    float4 o;
    o.x = (float)(x[s] - (G.lo[0] + c0 * G.s[0]));
    o.y = (float)(x[(size_t)n + s] - (G.lo[1] + c1 * G.s[1]));
    o.z = G.dim == 3 ? (float)(x[2 * (size_t)n + s] - (G.lo[2] + c2 * G.s[2])) : 0.f;
    o.w = wall ? 1.f : 0.f;
    return o;
}

// cell_offset of a particle that may have left its cell since the binning (the
// lists reused at r^n): on a periodic axis the nearest image of the position
// to the cell, so that a particle wrapped across the box edge keeps the offset
// that the lists' cell shifts assume.
__device__ __forceinline__ float4 cell_offset_near(const Geom &G, int local_cell, const double *x, int n, int s,
                                                   bool wall)
{
    const int c[3] = {local_cell % G.nc[0], (local_cell / G.nc[0]) % G.nc[1], local_cell / (G.nc[0] * G.nc[1])};
    float f[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < G.dim; ++a) {
        double d = x[(size_t)a * n + s] - (G.lo[a] + c[a] * G.s[a]);
        if (G.periodic[a]) {
            if (d > G.halfL[a]) d -= G.L[a];
            else if (d < -G.halfL[a]) d += G.L[a];
        }
        f[a] = (float)d;
    }
    return make_float4(f[0], f[1], f[2], wall ? 1.f : 0.f);
}

// A -> B at the start of a step: state n, and the packed (V^n, p^n) that the
// state-n pair pass gathers.
// The packed copy of a wall slot's prescribed velocity that the loop gathers
// with the neighbour states (contexts with walls only).
__device__ __forceinline__ void store_wall_velocity(const Buffers &B, int s, const double *u)
{
    if (B.wv32) B.wv32[s] = make_float4((float)u[0], (float)u[1], (float)u[2], 0.f);
    if (B.wv64) B.wv64[s] = make_double4_32a(u[0], u[1], u[2], 0.0);
}

// SAME: order B is order A (the r^0 lists of the previous step serve this
// step): every slot keeps its place and its cell of that binning, and the FP32
// offsets are taken at r^n from that cell's origin.
template <bool SAME>
__global__ void __launch_bounds__(kBlock) k_permute_a_to_b(Buffers B)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.n) return;
    const int o = SAME ? (B.gid_a[s] == kNoParticle ? -1 : s) : B.perm[s];
    if (o < 0) {
        B.gid_b[s] = kNoParticle;
        return;
    }
    const int n = B.n, dim = B.dim;
    const uint32_t g = B.gid_a[o];
    B.gid_b[s] = g;
    const int cell = SAME ? B.cell_a[s] : B.key[o];
    B.cell_b[s] = cell;
    double v[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        const size_t so = (size_t)a * n;
        B.x_b[so + s] = B.x_a[so + o];
        v[a] = B.vn_a[so + o];
        B.vn_b[so + s] = v[a];
        B.vnm1_b[so + s] = B.vnm1_a[so + o];
    }
    const double p = B.pn_a[o];
    B.pn_b[s] = p;
    if (B.fp32c) {
        const int inst = B.inst_of[s];
        B.off[s] = SAME ? cell_offset_near(B.geo[inst], cell - B.inst[inst].cell_off, B.x_b, n, s, g >= (uint32_t)B.nf)
                        : cell_offset(B.geo[inst], cell - B.inst[inst].cell_off, B.x_b, n, s, g >= (uint32_t)B.nf);
        B.nb32[1][s] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)p);
    } else {
        B.nb64[1][s] = make_double4_32a(v[0], v[1], v[2], p);
    }
}

// B -> A after the predictor: the loop order. Carries r^n, r^0, V^n, the BDF2
// source, and seeds iterate 0 (V^0, p-hat^0).
__global__ void __launch_bounds__(kBlock) k_permute_b_to_a(Buffers B)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (B.relist && s == 0) *B.relist = 0;   // the step's relisting, if any, is done
    if (s >= B.n) return;
    const int o = B.perm[s];
    if (o < 0) {
        B.gid_a[s] = kNoParticle;
        return;
    }
    const int n = B.n, dim = B.dim;
    const uint32_t g = B.gid_b[o];
    B.gid_a[s] = g;
    const bool wall = g >= (uint32_t)B.nf;
    if (B.slot_of && !wall) B.slot_of[g] = s;
    if (B.wslot_a && wall) B.wslot_a[g - (uint32_t)B.nf] = s;
    const int cell = B.key[o];
    B.cell_a[s] = cell;
    double v[3] = {0, 0, 0}, u[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        const size_t so = (size_t)a * n;
        B.x_a[so + s] = B.x_b[so + o];
        B.xp_a[so + s] = B.xp_b[so + o];
        u[a] = B.vn_b[so + o];
        B.vn_a[so + s] = u[a];
        B.s_a[so + s] = B.s_b[so + o];
        v[a] = B.v0_b[so + o];
        B.vk[0][so + s] = v[a];
    }
    if (wall) store_wall_velocity(B, s, u);
    const double ph = B.ph0_b[o];
    if (B.fp32c) {
        const int inst = B.inst_of[s];
        B.off[s] = cell_offset(B.geo[inst], cell - B.inst[inst].cell_off, B.xp_a, n, s, g >= (uint32_t)B.nf);
        B.nb32[0][s] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)ph);
    } else {
        B.nb64[0][s] = make_double4_32a(v[0], v[1], v[2], ph);
    }
}

// Caller order -> order A from AoS inputs: slot s of instance i holds its fluid
// particle s - slot_off (caller index foff + ...), then its walls, then padding.
// An input coordinate: flags a non-finite value; on a periodic axis brings a
// value outside [lo, hi) into it, x - floor((x - lo) / L) L, then once more by
// one L if rounding left it on the edge (every operation rounded as written).
__device__ __forceinline__ double input_coord(double xa, const Geom &G, int a, uint32_t *err)
{
    if (!isfinite(xa)) {
        atomicOr(err, kErrNonFinite);
        return G.lo[a];
    }
    if (!G.periodic[a] || (xa >= G.lo[a] && xa < G.hi[a])) return xa;
    const double q = floor(__ddiv_rn(__dsub_rn(xa, G.lo[a]), G.L[a]));
    double y = __dsub_rn(xa, __dmul_rn(q, G.L[a]));
    if (y >= G.hi[a]) y = __dsub_rn(y, G.L[a]);
    else if (y < G.lo[a]) y = __dadd_rn(y, G.L[a]);
    return y;
}

__global__ void __launch_bounds__(kBlock) k_scatter_in(Buffers B, const double *__restrict__ x,
                                                       const double *__restrict__ v, const double *__restrict__ p,
                                                       const double *__restrict__ vprev,
                                                       const double *__restrict__ xw, const double *__restrict__ vw)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.n) return;
    const int n = B.n, dim = B.dim;
    const Inst I = B.inst[B.inst_of[s]];
    const Geom &G = B.geo[B.inst_of[s]];
    const int local = s - I.slot_off;
    if (local < I.nf) {
        const size_t f = (size_t)I.foff + local;
        B.gid_a[s] = (uint32_t)f;
        for (int a = 0; a < dim; ++a) {
            const size_t so = (size_t)a * n;
            B.x_a[so + s] = input_coord(x[f * dim + a], G, a, B.err);
            B.vn_a[so + s] = v[f * dim + a];
            B.vnm1_a[so + s] = vprev ? vprev[f * dim + a] : v[f * dim + a];
        }
        B.pn_a[s] = p[f];
    } else if (local < I.nf + I.nw) {
        const size_t w = (size_t)I.woff + (local - I.nf);
        B.gid_a[s] = (uint32_t)(B.nf + w);
        if (B.wslot_a) B.wslot_a[w] = s;
        double u[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            const size_t so = (size_t)a * n;
            B.x_a[so + s] = input_coord(xw[w * dim + a], G, a, B.err);
            u[a] = vw ? vw[w * dim + a] : 0.0;
            B.vn_a[so + s] = u[a];
            B.vnm1_a[so + s] = u[a];
        }
        B.pn_a[s] = 0.0;
        store_wall_velocity(B, s, u);
    } else {
        B.gid_a[s] = kNoParticle;
    }
}

// Slot order -> caller order (AoS), fluid particles only.
__global__ void __launch_bounds__(kBlock) k_unpermute(int n, int nf, int comps, const uint32_t *__restrict__ gid,
                                                      const double *__restrict__ src, double *__restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t g = gid[s];
    if (g >= (uint32_t)nf) return;
    for (int a = 0; a < comps; ++a) out[(size_t)g * comps + a] = src[(size_t)a * n + s];
}

__global__ void k_fill_instance(Inst *inst, Geom *geo, Phys *phys, int i, Inst I, Geom G, Phys P)
{
    inst[i] = I;
    geo[i] = G;
    phys[i] = P;
}

inline int blocks(int n) { return (n + kBlock - 1) / kBlock; }

}  // namespace

int launch_binning(const Buffers &B, const double *x_keys, const uint32_t *gid_src, cudaStream_t st)
{
    k_bin_keys<<<blocks(B.n), kBlock, 0, st>>>(B, x_keys, gid_src);
    // up to kScanCells1 cells one block scans them all; more take the block
    // totals, their scan, and the block scans with their carries
    int k = 3;
    if (B.ncell <= kScanCells1) {
        k_scan_final<kScanPerThread1, false><<<1, kScanThreads, 0, st>>>(B);
    } else {
        const int nsb = (B.ncell + kScanCells - 1) / kScanCells;
        k_scan_partial<<<nsb, kScanThreads, 0, st>>>(B);
        k_scan_top<<<1, kScanThreads, 0, st>>>(B, nsb);
        k_scan_final<kScanPerThread, true><<<nsb, kScanThreads, 0, st>>>(B);
        k += 2;
    }
    k_scatter<<<blocks(B.n), kBlock, 0, st>>>(B);
    k_cell_rank<<<blocks(B.n), kBlock, 0, st>>>(B, gid_src);
    return k + 1;
}

int launch_permute_a_to_b(const Buffers &B, cudaStream_t st)
{
    k_permute_a_to_b<false><<<blocks(B.n), kBlock, 0, st>>>(B);
    return 1;
}

int launch_same_order_a_to_b(const Buffers &B, cudaStream_t st)
{
    k_permute_a_to_b<true><<<blocks(B.n), kBlock, 0, st>>>(B);
    return 1;
}

// Order B becomes order A as it is (the particles binned at r^n, before the
// first step that reuses the r^0 lists): slot, cell and the state that order A
// carries between steps.
__global__ void __launch_bounds__(kBlock) k_adopt_b(Buffers B)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.n) return;
    const uint32_t g = B.gid_b[s];
    B.gid_a[s] = g;
    if (g == kNoParticle) return;
    if (B.slot_of && g < (uint32_t)B.nf) B.slot_of[g] = s;
    B.cell_a[s] = B.cell_b[s];
    const int n = B.n;
    for (int a = 0; a < B.dim; ++a) {
        const size_t q = (size_t)a * n + s;
        B.x_a[q] = B.x_b[q];
        B.vn_a[q] = B.vn_b[q];
        B.vnm1_a[q] = B.vnm1_b[q];
    }
    B.pn_a[s] = B.pn_b[s];
}

int launch_adopt_b(const Buffers &B, cudaStream_t st)
{
    k_adopt_b<<<blocks(B.n), kBlock, 0, st>>>(B);
    return 1;
}

// One thread per fluid particle in caller order (contexts without walls): its
// new state into its slot of order A; the lists at r^0 stay valid while the
// position lies within list_skin / 2 of the slot's r^0 (nearest image).
__global__ void __launch_bounds__(kBlock) k_scatter_same(Buffers B, const double *__restrict__ x,
                                                         const double *__restrict__ v, const double *__restrict__ p,
                                                         const double *__restrict__ vprev)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= B.nf) return;
    const int s = B.slot_of[f];
    const int inst = B.inst_of[s];
    const Geom &G = B.geo[inst];
    const int n = B.n, dim = B.dim;
    double d2 = 0.0;
    for (int a = 0; a < dim; ++a) {
        const size_t so = (size_t)a * n;
        const double xa = input_coord(x[(size_t)f * dim + a], G, a, B.err);
        B.x_a[so + s] = xa;
        B.vn_a[so + s] = v[(size_t)f * dim + a];
        B.vnm1_a[so + s] = vprev ? vprev[(size_t)f * dim + a] : v[(size_t)f * dim + a];
        double d = xa - B.xp_a[so + s];
        if (G.periodic[a]) {
            if (d > G.halfL[a]) d -= G.L[a];
            else if (d < -G.halfL[a]) d += G.L[a];
        }
        d2 += d * d;
    }
    B.pn_a[s] = p[f];
    if (!(d2 < B.phys[inst].disp2_reuse)) *(volatile int *)B.relist = 1;
}

int launch_scatter_same(const Buffers &B, const double *x, const double *v, const double *p, const double *vprev,
                        cudaStream_t st)
{
    k_scatter_same<<<blocks(B.nf), kBlock, 0, st>>>(B, x, v, p, vprev);
    return 1;
}

int launch_permute_b_to_a(const Buffers &B, cudaStream_t st)
{
    k_permute_b_to_a<<<blocks(B.n), kBlock, 0, st>>>(B);
    return 1;
}

int launch_scatter_in(const Buffers &B, const double *x, const double *v, const double *p, const double *vprev,
                      const double *xw, const double *vw, cudaStream_t st)
{
    k_scatter_in<<<blocks(B.n), kBlock, 0, st>>>(B, x, v, p, vprev, xw, vw);
    return 1;
}

// Contiguous copy of count doubles between any two buffers the device can
// address (on devices with pageable-memory access: a caller's host array).
__global__ void __launch_bounds__(kBlock) k_copy(const double *__restrict__ src, double *__restrict__ dst,
                                                 size_t count)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) dst[i] = src[i];
}

int launch_copy(const double *src, double *dst, size_t count, cudaStream_t st)
{
    if (count == 0) return 0;
    const size_t want = (count + kBlock - 1) / kBlock;
    const int nb = (int)(want < 2048 ? want : 2048);
    k_copy<<<nb, kBlock, 0, st>>>(src, dst, count);
    return 1;
}

int launch_unpermute(const Buffers &B, const uint32_t *gid, const double *src, double *out, int comps, cudaStream_t st)
{
    k_unpermute<<<blocks(B.n), kBlock, 0, st>>>(B.n, B.nf, comps, gid, src, out);
    return 1;
}

int launch_fill_instance(Inst *inst, Geom *geo, Phys *phys, int i, const Inst &I, const Geom &G, const Phys &P,
                         cudaStream_t st)
{
    k_fill_instance<<<1, 1, 0, st>>>(inst, geo, phys, i, I, G, P);
    return 1;
}

}  // namespace dtsph
