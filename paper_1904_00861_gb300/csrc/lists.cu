// Neighbour lists N(i) = {j != i : |r_ij| < 3h} (Sec. 3; 3h + skin for moving
// particles with neighbour updates, 3h + list_skin for lists reused at the next
// r^n) of every slot, from the cell binning.
//
// One warp per home cell, the candidates in the lanes. The warp stages the
// particles of the 3^D surrounding cells in shared memory, in the order rows
// (dz, dy), then dx, then slot, each tagged with its list entry (slot, cell
// shift code, wall flag); then, for every chunk of 32 staged candidates (one per
// lane) and every home particle in turn, each lane tests its candidate against
// that home particle. A ballot ranks the hits, which join the home particle's
// list as one contiguous run, so a store of the warp touches one or two sectors
// instead of one per lane. The lists are written per slot (slot s at s Ks + k,
// Ks = K rounded up to 8); the state-n, pair-cache and uncached-loop passes read
// them there, and only the pass of particles moving in pseudo-time gets a copy
// sliced by warp (k_list_slice: entry k of slot s at ((s/32) K + k) 32 + s%32).
// Large 2D problems on the FP32C path take the row-segment builder
// (k_nlist_rows2_f32), 3D ones k_nlist_cells3_f32; every builder gives the same
// lists in the same order.
//
// The tests are those of the neighbour definition: FP64 positions, squares
// summed in axis order without FMA, minimum image on periodic axes; the FP32C
// path tests the FP32 separation from cell offsets, (o_i - shift s) - o_j as the
// pair kernels form it, and takes the FP64 test only inside a thin band around
// the cutoff, so both paths give the same sets, in the same order.
#include "geometry.cuh"

namespace dtsph {

namespace {

constexpr int kWarpsPerBlock = kBlock / kWarp;

// Global row segment g -> its instance (segments of instance i start at inst[i].seg_off).
__device__ __forceinline__ int segment_instance(const Buffers &B, int g)
{
    int lo = 0, hi = B.ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.inst[mid].seg_off <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Global cell c -> its instance (cells of instance i start at inst[i].cell_off).
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

// A staged candidate: FP32C its cell offset (.w = list entry bits), FP64 its
// position (.w = list entry bits).
template <bool F32> struct Staged;
template <> struct Staged<true> { using type = float4; };
template <> struct Staged<false> { using type = double4_32a; };

template <int D, bool F32>
__global__ void __launch_bounds__(kBlock) k_nlist_cells(Buffers B, const double *__restrict__ xpos,
                                                        const uint32_t *__restrict__ gid, uint32_t *__restrict__ lists,
                                                        int Ks)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    constexpr int NC = D == 3 ? 27 : 9;                 // surrounding cells
    constexpr int CH = F32 ? 256 : 128;                 // staged candidates per round
    using S = typename Staged<F32>::type;
    __shared__ S cand[kWarpsPerBlock][CH];
    __shared__ S home[kWarpsPerBlock][kWarp];
    __shared__ int tpre[kWarpsPerBlock][NC + 1];        // candidates before surrounding cell t
    __shared__ int tbeg[kWarpsPerBlock][NC];            // first slot of surrounding cell t
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int c = blockIdx.x * kWarpsPerBlock + w;      // global cell of this warp
    if (c >= B.ncell) return;                           // whole warp
    const int inst = cell_instance(B, c);
    const int cell_off = B.inst[inst].cell_off;
    const Geom &G = B.geo[inst];
    const int nx = G.nc[0], ny = G.nc[1], nz = G.nc[2];
    const int lc = c - cell_off;
    if (lc >= nx * ny * nz) return;                     // the instance's empty sentinel cell
    const int *start = B.cell_start + cell_off;
    const int hb = start[lc], he = start[lc + 1];
    if (hb == he) return;
    const int cx = lc % nx, cy = (lc / nx) % ny, cz = lc / (nx * ny);
    const float sf[3] = {G.s_f[0], G.s_f[1], G.s_f[2]};
    const float rc2_lo = G.rc2_lo, rc2_hi = G.rc2_hi;
    const double rc2 = G.rc2;
    // FP32C: squared distance from the home cell beyond which no home particle
    // can reach a candidate (the band's top, with a margin far above the
    // rounding of FP32 offsets, which lie in [0, s])
    const float box_cut2 = rc2_hi * 1.001f;
    const int n = B.n, K = B.K;
    // the surrounding cells side by side: lane t takes shift code
    // (dx + 1) + 3 (dy + 1) + 9 (dz + 1), dz = 0 in 2D (empty when off a closed edge)
    int m = 0;
    if (lane < NC) {
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = D == 3 ? lane / 9 - 1 : 0;
        int x = cx + dx, y = cy + dy, z = cz + dz;
        bool ok = true;
        if (x < 0 || x >= nx) { if (G.periodic[0]) x = x < 0 ? x + nx : x - nx; else ok = false; }
        if (y < 0 || y >= ny) { if (G.periodic[1]) y = y < 0 ? y + ny : y - ny; else ok = false; }
        if (D == 3 && (z < 0 || z >= nz)) { if (G.periodic[2]) z = z < 0 ? z + nz : z - nz; else ok = false; }
        if (ok) {
            const int nc = (z * ny + y) * nx + x;
            const int jb = start[nc];
            m = start[nc + 1] - jb;
            tbeg[w][lane] = jb;
        } else {
            tbeg[w][lane] = 0;
        }
    }
    int incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane < NC) tpre[w][lane] = incl - m;
    const int total = __shfl_sync(full, incl, NC - 1);
    if (lane == NC) tpre[w][NC] = total;
    __syncwarp();
    for (int h0 = hb; h0 < he; h0 += kWarp) {
        const int nh = min(kWarp, he - h0);
        // the home particles of this round, one per lane, into shared memory
        if (lane < nh) {
            const int s = h0 + lane;
            if constexpr (F32) {
                home[w][lane] = B.off[s];
            } else {
                S q;
                q.x = xpos[s];
                q.y = xpos[(size_t)n + s];
                q.z = D == 3 ? xpos[2 * (size_t)n + s] : 0.0;
                q.w = 0.0;
                home[w][lane] = q;
            }
        }
        int cnt = 0;                                    // list length of home particle h0 + lane
        int t = 0;                                      // surrounding cell of the next fill position
        for (int c0 = 0; c0 < total; c0 += CH) {
            const int span = min(total - c0, CH);
            // fill: stream position p is candidate p - tpre[t] of surrounding
            // cell t. FP32C drops, for the whole warp, a candidate farther than
            // the cutoff from every point of the home cell (the outer parts of
            // the edge and corner cells); the others keep their order
            int take = 0;
            for (int q0 = 0; q0 < span; q0 += kWarp) {
                const int q = q0 + lane;
                bool keep = false;
                S e;
                if (q < span) {
                    const int p = c0 + q;
                    while (tpre[w][t + 1] <= p) ++t;
                    const int j = tbeg[w][t] + (p - tpre[w][t]);
                    const int code = D == 3 ? t : t + 9;
                    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = D == 3 ? t / 9 - 1 : 0;
                    if constexpr (F32) {
                        const float4 oj = B.off[j];
                        e = oj;
                        e.w = __uint_as_float(list_entry((uint32_t)j, code, oj.w != 0.f));
                        const float ex = __fadd_rn(oj.x, (float)dx * sf[0]);
                        const float ey = __fadd_rn(oj.y, (float)dy * sf[1]);
                        const float ez = D == 3 ? __fadd_rn(oj.z, (float)dz * sf[2]) : 0.f;
                        const float bx = fmaxf(fmaxf(-ex, ex - sf[0]), 0.f);
                        const float by = fmaxf(fmaxf(-ey, ey - sf[1]), 0.f);
                        const float bz = D == 3 ? fmaxf(fmaxf(-ez, ez - sf[2]), 0.f) : 0.f;
                        keep = bx * bx + by * by + bz * bz < box_cut2;
                    } else {
                        e.x = xpos[j];
                        e.y = xpos[(size_t)n + j];
                        e.z = D == 3 ? xpos[2 * (size_t)n + j] : 0.0;
                        // entry bits in .w, the wall flag from the caller index
                        e.w = __longlong_as_double(
                            (long long)list_entry((uint32_t)j, code, gid[j] >= (uint32_t)B.nf));
                        keep = true;
                    }
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) cand[w][take + __popc(bal & lt)] = e;
                take += __popc(bal);
            }
            __syncwarp();
            for (int q0 = 0; q0 < take; q0 += kWarp) {
                const bool valid = q0 + lane < take;
                S e;
                if (valid) e = cand[w][q0 + lane];
                uint32_t ej = kNoParticle;
                if constexpr (F32) {
                    if (valid) ej = __float_as_uint(e.w);
                } else {
                    if (valid) ej = (uint32_t)__double_as_longlong(e.w);
                }
                const int j = entry_slot(ej);
                int dx, dy, dz;
                decode_shift(entry_code(ej), dx, dy, dz);
                for (int h = 0; h < nh; ++h) {
                    const int s = h0 + h;
                    bool in;
                    if constexpr (F32) {
                        const float4 oi = home[w][h];
                        float f0, f1, f2;
                        const float q2 = sep32<D>(shifted_offset<D>(oi, dx, dy, dz, sf), e, f0, f1, f2);
                        const bool cand_ok = valid && j != s;
                        in = cand_ok && q2 < rc2_lo;
                        const bool band = cand_ok && q2 >= rc2_lo && q2 < rc2_hi;
                        // the FP64 decision inside the band (rare)
                        if (__any_sync(full, band) && band) {
                            double d64[3];
                            in = sep64<D>(G, xpos, n, s, j, d64) < rc2;
                        }
                    } else {
                        const S xi = home[w][h];
                        const double xiv[3] = {xi.x, xi.y, xi.z}, xjv[3] = {e.x, e.y, e.z};
                        double d[3];
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            double v = __dsub_rn(xiv[a], xjv[a]);
                            if (G.periodic[a]) {
                                if (v > G.halfL[a]) v = __dsub_rn(v, G.L[a]);
                                else if (v < -G.halfL[a]) v = __dadd_rn(v, G.L[a]);
                            }
                            d[a] = v;
                        }
                        double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
                        if (D == 3) r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
                        in = valid && j != s && r2 < rc2;
                    }
                    const unsigned bal = __ballot_sync(full, in);
                    if (bal) {
                        const int base = __shfl_sync(full, cnt, h);
                        if (in) {
                            const int pos = base + __popc(bal & lt);
                            if (pos < K) lists[(size_t)s * Ks + pos] = ej;
                        }
                        if (lane == h) cnt += __popc(bal);
                    }
                }
            }
            __syncwarp();
        }
        if (lane < nh) {
            if (cnt > K) {
                atomicOr(B.err, kErrCapacity);
                cnt = K;
            }
            B.pcount[h0 + lane] = cnt;
        }
        __syncwarp();
    }
}

// 3D lists on the FP32C path, one warp per home cell with the home particles in
// the lanes (a 3D cell holds about 28, so the lanes stay busy): the staged
// candidates are moved into the home cell's frame (offset + shift s, tagged with
// the list entry), every lane tests them four at a time with broadcast reads,
// and appends its hits to an eight-entry buffer of its own in shared memory,
// which it writes out as one aligned 32-byte sector of its list (slot s at
// s Ks + k, Ks = K rounded up to 8) each time it fills. The FP32 separation here
// is o_i - (o_j + shift s); it decides outside the band around the cutoff
// exactly as the canonical form does, and the FP64 test decides inside it, so
// the sets and their order are those of k_nlist_cells.
constexpr int kBufEntries = 8;

__global__ void __launch_bounds__(kBlock) k_nlist_cells3_f32(Buffers B, const double *__restrict__ xpos,
                                                             uint32_t *__restrict__ lists, int Ks)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    constexpr int NC = 27;
    constexpr int CH = 256;
    __shared__ float4 cand[kWarpsPerBlock][CH];
    __shared__ __align__(16) uint32_t buf[kWarpsPerBlock][kWarp][kBufEntries];
    __shared__ int tpre[kWarpsPerBlock][NC + 1];
    __shared__ int tbeg[kWarpsPerBlock][NC];
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int c = blockIdx.x * kWarpsPerBlock + w;
    if (c >= B.ncell) return;
    const int inst = cell_instance(B, c);
    const int cell_off = B.inst[inst].cell_off;
    const Geom &G = B.geo[inst];
    const int nx = G.nc[0], ny = G.nc[1], nz = G.nc[2];
    const int lc = c - cell_off;
    if (lc >= nx * ny * nz) return;
    const int *start = B.cell_start + cell_off;
    const int hb = start[lc], he = start[lc + 1];
    if (hb == he) return;
    const int cx = lc % nx, cy = (lc / nx) % ny, cz = lc / (nx * ny);
    const float sf[3] = {G.s_f[0], G.s_f[1], G.s_f[2]};
    const float rc2_lo = G.rc2_lo, rc2_hi = G.rc2_hi;
    const double rc2 = G.rc2;
    const float box_cut2 = rc2_hi * 1.001f;
    const int n = B.n, K = B.K;
    int m = 0;
    if (lane < NC) {
        const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
        int x = cx + dx, y = cy + dy, z = cz + dz;
        bool ok = true;
        if (x < 0 || x >= nx) { if (G.periodic[0]) x = x < 0 ? x + nx : x - nx; else ok = false; }
        if (y < 0 || y >= ny) { if (G.periodic[1]) y = y < 0 ? y + ny : y - ny; else ok = false; }
        if (z < 0 || z >= nz) { if (G.periodic[2]) z = z < 0 ? z + nz : z - nz; else ok = false; }
        if (ok) {
            const int nc = (z * ny + y) * nx + x;
            const int jb = start[nc];
            m = start[nc + 1] - jb;
            tbeg[w][lane] = jb;
        } else {
            tbeg[w][lane] = 0;
        }
    }
    int incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane < NC) tpre[w][lane] = incl - m;
    const int total = __shfl_sync(full, incl, NC - 1);
    if (lane == NC) tpre[w][NC] = total;
    __syncwarp();
    uint32_t *my = buf[w][lane];
    for (int h0 = hb; h0 < he; h0 += kWarp) {
        const int s = h0 + lane;
        const bool act = s < he;
        // an idle lane tests from far away: it fails every distance test
        const float4 oi = act ? B.off[s] : make_float4(3e18f, 3e18f, 3e18f, 0.f);
        uint32_t *out = lists + (size_t)s * Ks;
        int cnt = 0;
        int t = 0;
        for (int c0 = 0; c0 < total; c0 += CH) {
            const int span = min(total - c0, CH);
            int take = 0;
            for (int q0 = 0; q0 < span; q0 += kWarp) {
                const int q = q0 + lane;
                bool keep = false;
                float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < span) {
                    const int p = c0 + q;
                    while (tpre[w][t + 1] <= p) ++t;
                    const int j = tbeg[w][t] + (p - tpre[w][t]);
                    const float4 oj = B.off[j];
                    const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
                    e.x = __fadd_rn(oj.x, (float)dx * sf[0]);
                    e.y = __fadd_rn(oj.y, (float)dy * sf[1]);
                    e.z = __fadd_rn(oj.z, (float)dz * sf[2]);
                    e.w = __uint_as_float(list_entry((uint32_t)j, t, oj.w != 0.f));
                    const float bx = fmaxf(fmaxf(-e.x, e.x - sf[0]), 0.f);
                    const float by = fmaxf(fmaxf(-e.y, e.y - sf[1]), 0.f);
                    const float bz = fmaxf(fmaxf(-e.z, e.z - sf[2]), 0.f);
                    keep = bx * bx + by * by + bz * bz < box_cut2;
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) cand[w][take + __popc(bal & lt)] = e;
                take += __popc(bal);
            }
            // pad to a multiple of four with entries that fail every test
            const int take4 = (take + 3) & ~3;
            if (take + lane < take4)
                cand[w][take + lane] = make_float4(-3e18f, -3e18f, -3e18f, __uint_as_float(kNoParticle));
            __syncwarp();
            for (int q = 0; q < take4; q += 4) {
                bool in[4], band[4];
                uint32_t ew[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 e = cand[w][q + u];
                    const float d0 = __fsub_rn(oi.x, e.x), d1 = __fsub_rn(oi.y, e.y), d2 = __fsub_rn(oi.z, e.z);
                    const float q2 = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
                    ew[u] = __float_as_uint(e.w);
                    const bool other = (ew[u] & kSlotMask) != (uint32_t)s;
                    in[u] = q2 < rc2_lo && other;
                    band[u] = q2 >= rc2_lo && q2 < rc2_hi && other;
                }
                // the FP64 decision inside the band (rare)
                if (__any_sync(full, band[0] || band[1] || band[2] || band[3])) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (band[u]) {
                            double d64[3];
                            in[u] = sep64<3>(G, xpos, n, s, entry_slot(ew[u]), d64) < rc2;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (in[u]) {
                        my[cnt & (kBufEntries - 1)] = ew[u];
                        ++cnt;
                        // a full buffer goes out as one aligned sector of the list
                        if ((cnt & (kBufEntries - 1)) == 0 && cnt <= K) {
                            const uint4 a = *reinterpret_cast<const uint4 *>(my);
                            const uint4 b = *reinterpret_cast<const uint4 *>(my + 4);
                            uint4 *dst = reinterpret_cast<uint4 *>(out + (cnt - kBufEntries));
                            dst[0] = a;
                            dst[1] = b;
                        }
                    }
                }
            }
            __syncwarp();
        }
        if (act) {
            // the entries since the last full buffer
            const int tail = cnt & (kBufEntries - 1);
            for (int k = 0; k < tail; ++k)
                if (cnt - tail + k < K) out[cnt - tail + k] = my[k];
            if (cnt > K) {
                atomicOr(B.err, kErrCapacity);
                cnt = K;
            }
            B.pcount[s] = cnt;
        }
        __syncwarp();
    }
}

// 2D lists on the FP32C path, one warp per row segment of up to kSeg2 cells along
// x (a 2D cell holds about 9 particles, so three cells fill most of the lanes) with
// the segment's particles in the lanes, as the 3D builder does for one cell. The
// warp stages the candidates of the 3 x (segment + 2) surrounding cells in the
// order rows (dy), then column, then slot, moved into the frame of the segment's
// first cell; each lane tests them four at a time against its particle, keeps
// those of the three columns around its own cell, and appends its hits through an
// eight-entry buffer as whole sectors of its list. For every particle the
// candidates of its own 3 x 3 cells come in the order rows, dx, slot, so its list
// holds the entries of k_nlist_cells in the same order; outside the band around
// the cutoff this FP32 separation decides as the canonical one does, and the FP64
// test decides inside it.
constexpr int kRowsMinSegments = 16384;

__global__ void __launch_bounds__(kBlock) k_nlist_rows2_f32(Buffers B, const double *__restrict__ xpos,
                                                            uint32_t *__restrict__ lists, int Ks)
{
    if (skip_relist(B)) return;   // (the step graph: relisting or not)
    constexpr int NCOL = kSeg2 + 2;                     // candidate columns
    constexpr int NT = 3 * NCOL;                        // candidate cells
    constexpr int CH = 256;
    __shared__ float4 cand[kWarpsPerBlock][CH];
    __shared__ __align__(16) uint32_t buf[kWarpsPerBlock][kWarp][kBufEntries];
    __shared__ int tpre[kWarpsPerBlock][NT + 1];
    __shared__ int tbeg[kWarpsPerBlock][NT];
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int g = blockIdx.x * kWarpsPerBlock + w;     // global row segment of this warp
    if (g >= B.nseg2) return;
    const int inst = segment_instance(B, g);
    const int cell_off = B.inst[inst].cell_off;
    const Geom &G = B.geo[inst];
    const int nx = G.nc[0], ny = G.nc[1];
    const int nsx = (nx + kSeg2 - 1) / kSeg2;           // segments per row
    const int ls = g - B.inst[inst].seg_off;
    const int cx = (ls % nsx) * kSeg2, cy = ls / nsx;
    const int lc = cy * nx + cx;
    const int ns = min(kSeg2, nx - cx);                 // cells of this segment
    const int *start = B.cell_start + cell_off;
    const int hb = start[lc], he = start[lc + ns];
    if (hb == he) return;
    // first slots of the segment's second and third cells
    const int b1 = ns > 1 ? start[lc + 1] : he, b2 = ns > 2 ? start[lc + 2] : he;
    const float sf[2] = {G.s_f[0], G.s_f[1]};
    const float rc2_lo = G.rc2_lo, rc2_hi = G.rc2_hi;
    const double rc2 = G.rc2;
    const float box_cut2 = rc2_hi * 1.001f;
    const float seg_w = (float)ns * sf[0];
    const int n = B.n, K = B.K;
    // the candidate cells side by side: lane t takes row t / NCOL (dy + 1) and
    // column t % NCOL (x = cx - 1 + column); empty when off a closed edge or past
    // the segment's last column
    int m = 0;
    if (lane < NT) {
        const int r = lane / NCOL, k = lane % NCOL;
        int x = cx - 1 + k, y = cy + r - 1;
        bool ok = k < ns + 2;
        if (ok && (x < 0 || x >= nx)) { if (G.periodic[0]) x = x < 0 ? x + nx : x - nx; else ok = false; }
        if (ok && (y < 0 || y >= ny)) { if (G.periodic[1]) y = y < 0 ? y + ny : y - ny; else ok = false; }
        if (ok) {
            const int nc = y * nx + x;
            const int jb = start[nc];
            m = start[nc + 1] - jb;
            tbeg[w][lane] = jb;
        } else {
            tbeg[w][lane] = 0;
        }
    }
    int incl = m;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane < NT) tpre[w][lane] = incl - m;
    const int total = __shfl_sync(full, incl, NT - 1);
    if (lane == NT) tpre[w][NT] = total;
    __syncwarp();
    uint32_t *my = buf[w][lane];
    for (int h0 = hb; h0 < he; h0 += kWarp) {
        const int s = h0 + lane;
        const bool act = s < he;
        const int kh = (s >= b1) + (s >= b2);           // the lane's cell in the segment
        // an idle lane tests from far away: it fails every distance test
        float4 oi = make_float4(3e18f, 3e18f, 0.f, 0.f);
        if (act) {
            oi = B.off[s];
            oi.x = __fadd_rn(oi.x, (float)kh * sf[0]);
        }
        uint32_t *out = lists + (size_t)s * Ks;
        int cnt = 0;
        int t = 0;
        for (int c0 = 0; c0 < total; c0 += CH) {
            const int span = min(total - c0, CH);
            int take = 0;
            for (int q0 = 0; q0 < span; q0 += kWarp) {
                const int q = q0 + lane;
                bool keep = false;
                float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < span) {
                    const int p = c0 + q;
                    while (tpre[w][t + 1] <= p) ++t;
                    const int j = tbeg[w][t] + (p - tpre[w][t]);
                    const float4 oj = B.off[j];
                    const int r = t / NCOL, k = t % NCOL;
                    e.x = __fadd_rn(oj.x, (float)(k - 1) * sf[0]);
                    e.y = __fadd_rn(oj.y, (float)(r - 1) * sf[1]);
                    // the column, and the list entry with the row's part of the shift
                    // code (dx + 1) + 3 (dy + 1) + 9: a lane adds its dx + 1
                    e.z = __int_as_float(k);
                    e.w = __uint_as_float(list_entry((uint32_t)j, 3 * r + 9, oj.w != 0.f));
                    const float bx = fmaxf(fmaxf(-e.x, e.x - seg_w), 0.f);
                    const float by = fmaxf(fmaxf(-e.y, e.y - sf[1]), 0.f);
                    keep = bx * bx + by * by < box_cut2;
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) cand[w][take + __popc(bal & lt)] = e;
                take += __popc(bal);
            }
            // pad to a multiple of four with entries that fail every test
            const int take4 = (take + 3) & ~3;
            if (take + lane < take4)
                cand[w][take + lane] = make_float4(-3e18f, -3e18f, __int_as_float(0x7f), __uint_as_float(kNoParticle));
            __syncwarp();
            // the tests set one bit (candidate q0 + b: bit b) per candidate of the
            // lane's three columns closer than the band's top, without branches;
            // each such candidate is then classified in candidate order: the lane's
            // own particle is skipped, below the band it is a neighbour, inside the
            // band (rare) the FP64 test decides
            for (int q0 = 0; q0 < take4; q0 += kWarp) {
                const int qn = min(kWarp, take4 - q0);
                uint32_t maybe = 0u;
                for (int q = 0; q < qn; q += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 e = cand[w][q0 + q + u];
                        const uint32_t dxp = (uint32_t)(__float_as_int(e.z) - kh);   // dx + 1 from the lane's cell
                        const float d0 = __fsub_rn(oi.x, e.x), d1 = __fsub_rn(oi.y, e.y);
                        const float q2 = __fmaf_rn(d1, d1, __fmul_rn(d0, d0));
                        if (q2 < rc2_hi && dxp <= 2u) maybe |= 1u << (q + u);
                    }
                }
                while (maybe) {
                    const int b = __ffs(maybe) - 1;
                    maybe &= maybe - 1u;
                    const float4 e = cand[w][q0 + b];
                    const uint32_t ej = __float_as_uint(e.w);
                    const int j = entry_slot(ej);
                    if (j == s) continue;
                    const float d0 = __fsub_rn(oi.x, e.x), d1 = __fsub_rn(oi.y, e.y);
                    const float q2 = __fmaf_rn(d1, d1, __fmul_rn(d0, d0));
                    bool in = q2 < rc2_lo;
                    if (!in) {
                        double d64[3];
                        in = sep64<2>(G, xpos, n, s, j, d64) < rc2;
                    }
                    if (!in) continue;
                    const uint32_t dxp = (uint32_t)(__float_as_int(e.z) - kh);
                    my[cnt & (kBufEntries - 1)] = ej + (dxp << kCodeShift);
                    ++cnt;
                    // a full buffer goes out as one aligned sector of the list
                    if ((cnt & (kBufEntries - 1)) == 0 && cnt <= K) {
                        const uint4 a = *reinterpret_cast<const uint4 *>(my);
                        const uint4 c4 = *reinterpret_cast<const uint4 *>(my + 4);
                        uint4 *dst = reinterpret_cast<uint4 *>(out + (cnt - kBufEntries));
                        dst[0] = a;
                        dst[1] = c4;
                    }
                }
            }
            __syncwarp();
        }
        if (act) {
            // the entries since the last full buffer
            const int tail = cnt & (kBufEntries - 1);
            for (int k = 0; k < tail; ++k)
                if (cnt - tail + k < K) out[cnt - tail + k] = my[k];
            if (cnt > K) {
                atomicOr(B.err, kErrCapacity);
                cnt = K;
            }
            B.pcount[s] = cnt;
        }
        __syncwarp();
    }
}

// The per-slot lists (slot s at s Ks + k) into the sliced layout, one warp per 32
// slots: 32-entry pieces of the 32 lists pass through a shared-memory tile, read
// as whole list segments and written as whole rows.
__global__ void __launch_bounds__(kBlock) k_list_slice(Buffers B, const uint32_t *__restrict__ lists, int Ks)
{
    __shared__ uint32_t tile[kWarpsPerBlock][kWarp][kWarp + 1];
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x >> 5;
    const int s0 = (blockIdx.x * kWarpsPerBlock + w) * kWarp;
    if (s0 >= B.n) return;                              // whole warp (n is a multiple of 32)
    const int K = B.K;
    // the builder writes the counts of the slots in cells; a padding slot's count
    // is whatever the array holds, so every count is clamped to [0, K] and the
    // accesses below stay inside the slot's own lists whatever memory held
    const int cnt = min(max(B.pcount[s0 + lane], 0), K);
    const int cmax = __reduce_max_sync(full, cnt);
    uint32_t *rows = B.pj + (size_t)(s0 >> 5) * K * kWarp;
    for (int k0 = 0; k0 < cmax; k0 += kWarp) {
        for (int r = 0; r < kWarp; ++r) {
            const int cr = __shfl_sync(full, cnt, r);
            if (k0 + lane < cr) tile[w][lane][r] = lists[(size_t)(s0 + r) * Ks + k0 + lane];
        }
        __syncwarp();
        const int kn = min(kWarp, cmax - k0);
        for (int kk = 0; kk < kn; ++kk)
            if (k0 + kk < cnt) rows[(size_t)(k0 + kk) * kWarp + lane] = tile[w][kk][lane];
        __syncwarp();
    }
}

}  // namespace

static_assert(list_stride(1) % kBufEntries == 0, "a list row holds whole buffers of the 3D builder");

// The lists of every slot at xpos into the per-slot layout (slot_list); with
// `sliced`, also copied into the sliced layout of pj for the kernels that walk
// them every pseudo-iteration (the moving pass). The passes that read a list
// once per step (state n, pair cache, shifting) read the per-slot layout.
void launch_nlist(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st,
                  bool sliced)
{
    (void)cell;
    const int nb = (B.ncell + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int Ks = list_stride(B.K);
    if (B.dim == 3 && B.fp32c) {
        k_nlist_cells3_f32<<<nb, kBlock, 0, st>>>(B, xpos, B.pjt, Ks);
    } else if (B.fp32c && B.nseg2 >= kRowsMinSegments) {
        // enough row segments to fill the GPU several times over; fewer, and a
        // warp per cell keeps more warps busy (both give the same lists)
        const int nb2 = (B.nseg2 + kWarpsPerBlock - 1) / kWarpsPerBlock;
        k_nlist_rows2_f32<<<nb2, kBlock, 0, st>>>(B, xpos, B.pjt, Ks);
    } else {
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_nlist_cells<D, F32><<<nb, kBlock, 0, st>>>(B, xpos, gid, B.pjt, Ks)));
    }
    if (sliced) k_list_slice<<<(B.n / kWarp + kWarpsPerBlock - 1) / kWarpsPerBlock, kBlock, 0, st>>>(B, B.pjt, Ks);
}

}  // namespace dtsph
