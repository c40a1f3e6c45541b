// Neighbour lists and the kernels that walk them: the wall extrapolation and the
// pair pass at the state n, and the pair-coefficient cache that the pseudo-time
// loop reads (geometry frozen for the whole loop, Sec. 2.2; caching kernel
// gradients across pseudo-iterations is the speed-up the paper points at in
// Sec. 4.7 but did not implement). The lists are built by a test-only kernel and
// walked densely by the others, so the pair arithmetic never runs under the
// distance test, which most candidates fail.
//
// Neighbour test: j != i and |r_ij|^2 < (3h)^2 in IEEE double, squares summed in
// axis order without FMA, minimum image on periodic axes. The FP32C path first
// tests an FP32 separation built from per-cell FP32 offsets and falls back to the
// FP64 test only inside a thin band around 3h, so both paths give the same sets.
#include "geometry.cuh"
#include "loop_rules.cuh"

namespace dtsph {

namespace {

// Candidate traversal by a warp, L lanes per slot (a group), called by every
// lane of the warp (active = false for a group without a particle to serve).
//
// The 32 / L slots of a warp are consecutive in cell order, so their home
// cells lie in one or two runs along x of a (y, z) row of cells. The groups of
// one row share a single candidate stream: for each of the 3^(D-1) neighbour
// rows, the cells from one left of the run to one right of it, each cell in
// slot order (the bounds of a row's cells are loaded by the lanes side by side).
// A round takes L U consecutive candidates of a cell, lane l of every group the
// candidates l, l + L, ...; a group tests them if the cell lies within one cell
// of its own along x. Per candidate slice of L, a group ballot ranks the
// neighbours found, so that each group sees the candidates of its 3^D cells in
// the order rows (dz, dy), then dx = -1, 0, 1, then slot, and emit(j, code,
// wall_j, rank) is called for each, with code = (dx + 1) + 3 (dy + 1) + 9 (dz +
// 1). Returns the group's neighbour count. The FP32C test takes the FP32
// separation from cell offsets (whose .w flags walls) and decides by the FP64
// test inside the band around 3h; the FP64 path takes the FP64 test. The loop
// has no divergent branch: out-of-range candidates are clamped and masked, and
// the band test runs only when some lane of the warp needs it.
template <int D, bool F32, int L, class Emit>
__device__ __forceinline__ int slice_candidates(const Geom &G, const int *__restrict__ start, int cell_off, int cell,
                                                bool active, int s, const double *__restrict__ x,
                                                const float4 *__restrict__ off, const uint32_t *__restrict__ gid,
                                                int n, int nf, Emit &&emit)
{
    constexpr unsigned full = 0xffffffffu;
    constexpr int U = L >= 4 ? 1 : 4 / L;  // candidates per lane and round
    const int lane = threadIdx.x & (kWarp - 1);
    const int sub = lane % L;
    const unsigned first = (unsigned)(lane - sub);
    const unsigned gbits = L == 32 ? full : ((1u << L) - 1u);
    const unsigned below = (1u << sub) - 1u;
    start += cell_off;            // the instance's cells, numbered from 0
    const int lcell = active ? cell - cell_off : 0;
    const int cx = lcell % G.nc[0];
    const int crow = lcell / G.nc[0];
    const float sf[3] = {G.s_f[0], G.s_f[1], G.s_f[2]};
    const float rc2_lo = G.rc2_lo, rc2_hi = G.rc2_hi;
    const double rc2 = G.rc2;
    const float4 oi = F32 && active ? off[s] : make_float4(0.f, 0.f, 0.f, 0.f);
    double xi[3] = {0, 0, 0};
    if (!F32 && active) {
#pragma unroll
        for (int a = 0; a < D; ++a) xi[a] = x[(size_t)a * n + s];
    }
    int cnt = 0;
    unsigned todo = __ballot_sync(full, active);
    while (todo) {
        // the groups whose home cell lies in the row of the first lane left
        const int srow = __shfl_sync(full, crow, __ffs(todo) - 1);
        const bool mine = ((todo >> lane) & 1u) && crow == srow;
        todo &= ~__ballot_sync(full, mine);
        const int xa = __reduce_min_sync(full, mine ? cx : 0x7fffffff);
        const int xb = __reduce_max_sync(full, mine ? cx : -1);
        const int ncx = xb - xa + 3;                 // cells of the stream in each row
        const int sy = srow % G.nc[1], sz = srow / G.nc[1];
        constexpr int zlo = D == 3 ? -1 : 0, zhi = D == 3 ? 1 : 0;
        for (int dz = zlo; dz <= zhi; ++dz) {
            int z = sz + dz;
            if (D == 3 && (z < 0 || z >= G.nc[2])) {
                if (!G.periodic[2]) continue;
                z = z < 0 ? z + G.nc[2] : z - G.nc[2];
            }
            for (int dy = -1; dy <= 1; ++dy) {
                int y = sy + dy;
                if (y < 0 || y >= G.nc[1]) {
                    if (!G.periodic[1]) continue;
                    y = y < 0 ? y + G.nc[1] : y - G.nc[1];
                }
                const int row = (z * G.nc[1] + y) * G.nc[0];
                for (int c0 = 0; c0 < ncx; c0 += kWarp) {
                    // lane k holds the slot range of stream cell c0 + k (empty if off the grid)
                    int kb = 0, ke = 0;
                    if (c0 + lane < ncx) {
                        int xc = xa - 1 + c0 + lane;
                        bool ok = true;
                        if (xc < 0 || xc >= G.nc[0]) {
                            if (G.periodic[0]) xc = xc < 0 ? xc + G.nc[0] : xc - G.nc[0];
                            else ok = false;
                        }
                        if (ok) {
                            kb = start[row + xc];
                            ke = start[row + xc + 1];
                        }
                    }
                    const int mc = min(kWarp, ncx - c0);
                    for (int t = 0; t < mc; ++t) {
                        const int jb = __shfl_sync(full, kb, t), je = __shfl_sync(full, ke, t);
                        if (jb == je) continue;
                        const int dx = xa - 1 + c0 + t - cx;
                        const bool part = mine && dx >= -1 && dx <= 1;
                        if (!__any_sync(full, part)) continue;
                        const int code = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                        const float4 ps = shifted_offset<D>(oi, dx, dy, dz, sf);
                        for (int j0 = jb; j0 < je; j0 += L * U) {
                            bool in[U], band[U], wl[U];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const int j = j0 + u * L + sub;
                                const bool cand = part && j < je && j != s;
                                const int jc = j < je ? j : je - 1;   // in range, result unused
                                if (F32) {
                                    const float4 oj = off[jc];
                                    float f0, f1, f2;
                                    const float q2 = sep32<D>(ps, oj, f0, f1, f2);
                                    in[u] = cand && q2 < rc2_lo;
                                    band[u] = cand && q2 >= rc2_lo && q2 < rc2_hi;
                                    wl[u] = oj.w != 0.f;
                                } else {
                                    double d[3];
#pragma unroll
                                    for (int a = 0; a < D; ++a) {
                                        double v = __dsub_rn(xi[a], x[(size_t)a * n + jc]);
                                        if (G.periodic[a]) {
                                            if (v > G.halfL[a]) v = __dsub_rn(v, G.L[a]);
                                            else if (v < -G.halfL[a]) v = __dadd_rn(v, G.L[a]);
                                        }
                                        d[a] = v;
                                    }
                                    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
                                    if (D == 3) r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
                                    in[u] = cand && r2 < rc2;
                                    band[u] = false;
                                    wl[u] = gid[jc] >= (uint32_t)nf;
                                }
                            }
                            if (F32) {
                                bool any_band = false;
#pragma unroll
                                for (int u = 0; u < U; ++u) any_band |= band[u];
                                // the FP64 decision inside the band (rare)
                                if (__any_sync(full, any_band)) {
#pragma unroll
                                    for (int u = 0; u < U; ++u) {
                                        if (band[u]) {
                                            double e[3];
                                            in[u] = sep64<D>(G, x, n, s, j0 + u * L + sub, e) < rc2;
                                        }
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                const unsigned bal = L == 1 ? (in[u] ? 1u : 0u)
                                                            : (__ballot_sync(full, in[u]) >> first) & gbits;
                                if (in[u]) emit(j0 + u * L + sub, code, wl[u], cnt + __popc(bal & below));
                                cnt += __popc(bal);
                            }
                        }
                    }
                }
            }
        }
    }
    return cnt;
}

// ------------------------------------------------------------- neighbour lists

// Neighbour list of every slot (order of the latest binning) at positions xpos:
// pj = j (| kWallBit when j is a wall) and pcode = the cell shift, in candidate
// order, sliced by warp (entry k of slot s at ((s/32) K + k) 32 + s%32), and
// pcount. One lane per slot (slice_candidates); the pair kernels then walk the
// lists densely.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_nlist(Buffers B, const double *__restrict__ xpos,
                                                  const int *__restrict__ cell, const uint32_t *__restrict__ gid)
{
    constexpr int SPB = kBlock / L;       // slots per block
    __shared__ Geom G;
    const int inst = block_instance(B, blockIdx.x * SPB);
    block_copy(G, B.geo[inst]);
    const int cell_off = B.inst[inst].cell_off;
    const int s = blockIdx.x * SPB + threadIdx.x / L;
    const int n = B.n, K = B.K;
    // every lane stays to the end: the traversal runs warp-synchronously
    const bool act = s < n && gid[s] != kNoParticle;
    const size_t base = (size_t)(s >> 5) * K * kWarp + (s & 31);
    int cnt = slice_candidates<D, F32, L>(G, B.cell_start, cell_off, act ? cell[s] : 0, act, s, xpos, B.off, gid, n,
                                          B.nf, [&](int j, int code, bool wall, int pos) {
                                              if (pos < K) {
                                                  const size_t e = base + (size_t)pos * kWarp;
                                                  B.pj[e] = (uint32_t)j | (wall ? kWallBit : 0u);
                                                  B.pcode[e] = (uint8_t)code;
                                              }
                                          });
    if (s >= n || threadIdx.x % L != 0) return;
    if (cnt > K) {
        atomicOr(B.err, kErrCapacity);
        cnt = K;
    }
    B.pcount[s] = cnt;
}

// Neighbour lists in 3D on the FP32C path, one warp per home cell. With cells
// of ~28 particles, a warp of 32 consecutive slots spans more than one cell and
// its shared candidate stream would hold four cells per row; here the warp
// serves exactly the particles of one cell (32 at a time), so every staged
// candidate is one of theirs. The warp stages the candidates of the 27
// surrounding cells in shared memory, in the order rows (dz, dy), then dx, then
// slot, each already moved into the home cell's frame (offset + shift s) and
// tagged with its slot and wall bit; then every lane tests them with broadcast
// reads. The FP32 test decides outside the band around 3h, the FP64 test inside
// it, as in slice_candidates, so the lists are the same.
constexpr int kCellChunk = 256;     // staged candidates per warp

__device__ __forceinline__ int instance_of_cell(const Buffers &B, int c)
{
    int lo = 0, hi = B.ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.inst[mid].cell_off <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kBlock) k_nlist_cells3(Buffers B, const double *__restrict__ xpos)
{
    __shared__ float4 cand[kBlock / kWarp][kCellChunk + 4];
    __shared__ uint8_t ccode[kBlock / kWarp][kCellChunk + 4];
    __shared__ int tpre[kBlock / kWarp][28];      // candidates before neighbour cell k (k = code)
    __shared__ int tbeg[kBlock / kWarp][27];      // first slot of neighbour cell k
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & (kWarp - 1), w = threadIdx.x >> 5;
    const int c = blockIdx.x * (kBlock / kWarp) + w;            // global cell of this warp
    if (c >= B.ncell) return;                                    // whole warp
    const int inst = instance_of_cell(B, c);
    const int cell_off = B.inst[inst].cell_off;
    const Geom &G = B.geo[inst];
    const int nx = G.nc[0], ny = G.nc[1], nz = G.nc[2];
    const int lc = c - cell_off;
    if (lc >= nx * ny * nz) return;                              // the instance's sentinel cell
    const int *start = B.cell_start + cell_off;
    const int hb = start[lc], he = start[lc + 1];
    if (hb == he) return;
    const int cx = lc % nx, cy = (lc / nx) % ny, cz = lc / (nx * ny);
    const float sf[3] = {G.s_f[0], G.s_f[1], G.s_f[2]};
    const float rc2_lo = G.rc2_lo, rc2_hi = G.rc2_hi;
    const double rc2 = G.rc2;
    // squared distance from the home cell beyond which no home particle can
    // reach a candidate: the band's top with a margin far above the rounding of
    // FP32 offsets (home offsets lie in [0, s] up to that rounding)
    const float box_cut2 = rc2_hi * 1.001f;
    const int n = B.n, K = B.K;
    float4 *buf = cand[w];
    uint8_t *cb = ccode[w];
    // the 27 neighbour cells, loaded side by side: lane k takes the cell with
    // code k = (dx + 1) + 3 (dy + 1) + 9 (dz + 1) (empty when off a closed edge)
    int m = 0;
    if (lane < 27) {
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
    if (lane < 27) tpre[w][lane] = incl - m;
    const int total = __shfl_sync(full, incl, 26);
    if (lane == 27) tpre[w][27] = total;
    __syncwarp();
    for (int h0 = hb; h0 < he; h0 += kWarp) {
        const int s = h0 + lane;
        const bool act = s < he;
        // an idle lane tests from far away: it fails every distance test
        const float4 oi = act ? B.off[s] : make_float4(3e18f, 3e18f, 3e18f, 0.f);
        const size_t base = (size_t)(s >> 5) * K * kWarp + (s & 31);
        uint32_t *pjw = B.pj + base;
        uint8_t *pcw = B.pcode + base;
        int cnt = 0;
        int k = 0;                                   // neighbour cell of this lane's next fill position
        for (int c0 = 0; c0 < total; c0 += kCellChunk) {
            const int span = min(total - c0, kCellChunk);
            // fill: position p of the stream is candidate p - tpre[k] of cell k.
            // A candidate farther than the cutoff from every point of the home
            // cell (the outer parts of the edge and corner cells, about a
            // quarter of the stream) is dropped here for the whole warp; the
            // others keep their order (ballot compaction), so the lists are
            // those of the full stream
            int take = 0;
            for (int q0 = 0; q0 < span; q0 += kWarp) {
                const int q = q0 + lane;
                bool keep = false;
                float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < span) {
                    const int p = c0 + q;
                    while (tpre[w][k + 1] <= p) ++k;
                    const int j = tbeg[w][k] + (p - tpre[w][k]);
                    const float4 oj = B.off[j];
                    const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
                    e.x = __fadd_rn(oj.x, (float)dx * sf[0]);
                    e.y = __fadd_rn(oj.y, (float)dy * sf[1]);
                    e.z = __fadd_rn(oj.z, (float)dz * sf[2]);
                    e.w = __uint_as_float((uint32_t)j | (oj.w != 0.f ? kWallBit : 0u));
                    const float bx = fmaxf(fmaxf(-e.x, e.x - sf[0]), 0.f);
                    const float by = fmaxf(fmaxf(-e.y, e.y - sf[1]), 0.f);
                    const float bz = fmaxf(fmaxf(-e.z, e.z - sf[2]), 0.f);
                    keep = bx * bx + by * by + bz * bz < box_cut2;
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) {
                    const int pos = take + __popc(bal & ((1u << lane) - 1u));
                    buf[pos] = e;
                    cb[pos] = (uint8_t)k;
                }
                take += __popc(bal);
            }
            // pad to a multiple of four with entries that fail every test
            const int take4 = (take + 3) & ~3;
            if (take + lane < take4) buf[take + lane] = make_float4(-3e18f, -3e18f, -3e18f, __uint_as_float(kNoParticle));
            __syncwarp();
            for (int q = 0; q < take4; q += 4) {
                bool in[4], band[4];
                uint32_t jw[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 e = buf[q + u];
                    const float d0 = __fsub_rn(oi.x, e.x), d1 = __fsub_rn(oi.y, e.y), d2 = __fsub_rn(oi.z, e.z);
                    const float q2 = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, __fmul_rn(d0, d0)));
                    jw[u] = __float_as_uint(e.w);
                    const bool other = (jw[u] & ~kWallBit) != (uint32_t)s;
                    in[u] = q2 < rc2_lo && other;
                    band[u] = q2 >= rc2_lo && q2 < rc2_hi && other;
                }
                // the FP64 decision inside the band (rare)
                if (__any_sync(full, band[0] || band[1] || band[2] || band[3])) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (band[u]) {
                            double ee[3];
                            in[u] = sep64<3>(G, xpos, n, s, (int)(jw[u] & ~kWallBit), ee) < rc2;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (in[u]) {
                        if (cnt < K) {
                            pjw[(size_t)cnt * kWarp] = jw[u];
                            pcw[(size_t)cnt * kWarp] = cb[q + u];
                        }
                        ++cnt;
                    }
                }
            }
            __syncwarp();
        }
        if (act) {
            if (cnt > K) {
                atomicOr(B.err, kErrCapacity);
                cnt = K;
            }
            B.pcount[s] = cnt;
        }
    }
}

// ---------------------------------------------------------------- walls, state n

// The list walkers below give each slot a group of L lanes; lane l of a group
// takes the list entries l, l + L, ... Summing kernels merge the lanes' partial
// sums by shuffles, so their summation order depends on L alone: they use the
// fixed kSumLanes, which keeps every context (solo or batched, any size) on
// the same order. One lane per slot measured fastest on large problems and
// costs little on small ones. Block b covers slots b * (kBlock / L) ...

constexpr int kSumLanes = 1;

// Adami et al. wall values at state n in order B: p_w = (sum_f p_f W + rho0 g .
// sum_f r_wf W) / sum_f W, ghost velocity 2 v_w - sum_f V_f W / sum_f W; written
// into the packed (V, p) of the wall slot, from its neighbour list at r^n.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_walls_state_n(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int SPB = kBlock / L;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * SPB);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int s = blockIdx.x * SPB + threadIdx.x / L, lane_in = threadIdx.x % L;
    // every lane stays to the end: the partial sums are merged by full-warp shuffles
    const uint32_t gs = s < B.n ? B.gid_b[s] : kNoParticle;
    const bool wall = gs != kNoParticle && gs >= (uint32_t)B.nf;
    const auto *nb = nb_ptr<T>(B, 1);
    const float4 oi = wall && F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    double acc[6] = {0, 0, 0, 0, 0, 0};   // sum W, sum p W, sum rho0 (g . r) W, sum V W
    const double sigma = P.sig_h * P.h;
    const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
    const int cnt = wall ? B.pcount[s] : 0;
    for (int k = lane_in; k < cnt; k += L) {
        const size_t e = base + (size_t)k * kWarp;
        const uint32_t jb = B.pj[e];
        if (jb & kWallBit) continue;                    // fluid neighbours only
        const int j = (int)jb;
        int dx, dy, dz;
        decode_shift(B.pcode[e], dx, dy, dz);
        T d[3], r2;
        listed_sep<D, F32, T>(G, B.x_b, B.off, B.n, s, j, oi, dx, dy, dz, d, r2);
        const double W = sigma * (double)quintic_w<T>(Ar<T>::mul(sqrt(r2), (T)P.inv_h));
        const auto q = nb[j];
        double gr = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) gr += P.g[a] * (double)d[a];
        acc[0] += W;
        acc[1] += (double)q.w * W;
        acc[2] += P.rho0 * gr * W;
        acc[3] += (double)q.x * W;
        acc[4] += (double)q.y * W;
        acc[5] += (double)q.z * W;
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1)
#pragma unroll
        for (int t = 0; t < 6; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    if (!wall || lane_in != 0) return;
    const double sw = acc[0];
    double gv[3];
    for (int a = 0; a < 3; ++a) {
        const double vw = a < D ? B.vn_b[(size_t)a * B.n + s] : 0.0;
        gv[a] = 2.0 * vw - (sw > 0 ? acc[3 + a] / sw : 0.0);
    }
    double pw = sw > 0 ? (acc[1] + acc[2]) / sw : 0.0;
    if (pw < 0.0 && P.free_surface) pw = 0.0;     // free-surface runs keep it >= 0 (Sec. 3.2)
    if (F32) B.nb32[1][s] = make_float4((float)gv[0], (float)gv[1], (float)gv[2], (float)pw);
    else B.nb64[1][s] = make_double4_32a(gv[0], gv[1], gv[2], pw);
}

// ------------------------------------------------------------------ state n pass

// Rates at (r^n, V^n, p^n) in order B over the neighbour lists at r^n. With
// PRED, also the predictor of Eqs. (v0, r0): V^0 = V^n + dt F^n, r^0 = r^n +
// dt V^n + dt^2/2 F^n; the first pressure half step p-hat^0 = p^n + dtau/2
// dp^n/dtau (Eq. pkstar_frozen with the state-n rate); and the BDF2 source
// (V^{n-1} - 4 V^n) / (2 dt) of Eq. (dv_dtau_exact), all in FP64.
template <int D, bool F32, bool PRED, bool WALLS, int L>
__global__ void __launch_bounds__(kBlock, F32 ? 3 : 1) k_state_n(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    constexpr int SPB = kBlock / L;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * SPB);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int n = B.n;
    const int s = blockIdx.x * SPB + threadIdx.x / L, lane_in = threadIdx.x % L;
    // every lane stays to the end: the partial sums are merged by full-warp shuffles
    const uint32_t gs = s < n ? B.gid_b[s] : kNoParticle;
    const bool fluid = gs < (uint32_t)B.nf;
    const auto *nb = nb_ptr<T>(B, 1);
    const PairConst<T> k = pair_const<T>(P);
    Acc ap, Fa[3];
    {
        const typename Packed<T>::type qi = fluid ? nb[s] : typename Packed<T>::type{};
        const T vi[3] = {(T)qi.x, (T)qi.y, (T)qi.z};
        const T pi = (T)qi.w;
        const float4 oi = F32 && fluid ? B.off[s] : make_float4(0, 0, 0, 0);
        const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
        const int cnt = fluid ? B.pcount[s] : 0;
        // R entries per round: their indices, then their gathers (neighbour
        // state and, FP32C, offset), then the pair terms, so that R loads are in
        // flight per lane; the entries keep their order
        constexpr int R = 4;
        using Q = typename Packed<T>::type;
        for (int q0 = lane_in; q0 < cnt; q0 += L * R) {
            uint32_t jbv[R];
            int cv[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const size_t e = base + (size_t)min(q0 + r * L, cnt - 1) * kWarp;
                jbv[r] = B.pj[e];
                cv[r] = B.pcode[e];
            }
            Q qv[R];
            float4 ov[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = (int)(jbv[r] & ~kWallBit);
                qv[r] = nb[j];
                ov[r] = F32 ? B.off[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (q0 + r * L >= cnt) break;
                const uint32_t jb = jbv[r];
                const int j = (int)(jb & ~kWallBit);
                T d[3], r2;
                if (F32) {
                    offset_sep<D, T>(G, oi, ov[r], cv[r], d, r2);
                } else {
                    int dx, dy, dz;
                    decode_shift(cv[r], dx, dy, dz);
                    listed_sep<D, F32, T>(G, B.x_b, B.off, n, s, j, oi, dx, dy, dz, d, r2);
                }
                T g[3], F;
                grad_coef<D, T>(P, d, r2, g, F);
                const auto qj = qv[r];
                const T vv[3] = {(T)qj.x, (T)qj.y, (T)qj.z};
                T vd[3] = {vv[0], vv[1], vv[2]};
                if (WALLS && (jb & kWallBit)) {
                    for (int a = 0; a < D; ++a) vd[a] = (T)B.vn_b[(size_t)a * n + j];
                }
                pair_accumulate<D, T, Acc>(k, g, F, vi, pi, vd, vv, (T)qj.w, ap, Fa);
            }
        }
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        ap.shfl_merge(o);
#pragma unroll
        for (int a = 0; a < D; ++a) Fa[a].shfl_merge(o);
    }
    if (gs == kNoParticle || lane_in != 0) return;
    if (!fluid) {
        if (PRED) {
            for (int a = 0; a < D; ++a) B.xp_b[(size_t)a * n + s] = B.x_b[(size_t)a * n + s];
        }
        return;
    }
    const double apv = (double)(T)ap.value();
    double Fv[3];
    for (int a = 0; a < D; ++a) Fv[a] = __dadd_rn((double)(T)Fa[a].value(), P.g[a]);
    B.ap_b[s] = apv;
    for (int a = 0; a < D; ++a) B.f_b[(size_t)a * n + s] = Fv[a];
    if (PRED && P.steady) {
        // steady mode: the iteration starts from the state itself, the particles
        // stay, and the source is -g (the loop forms F + g - 0)
        for (int a = 0; a < D; ++a) {
            const size_t q = (size_t)a * n + s;
            B.xp_b[q] = B.x_b[q];
            B.v0_b[q] = B.vn_b[q];
            B.s_b[q] = -P.g[a];
        }
        B.ph0_b[s] = __fma_rn(0.5 * P.dtau, apv, B.pn_b[s]);
    } else if (PRED) {
        for (int a = 0; a < D; ++a) {
            const size_t q = (size_t)a * n + s;
            // explicit roundings: the same bits in every kernel variant
            const double V = B.vn_b[q];
            double xp = __fma_rn(0.5 * P.dt * P.dt, Fv[a], __fma_rn(P.dt, V, B.x_b[q]));
            if (G.periodic[a]) {
                if (xp >= G.hi[a]) xp = __dsub_rn(xp, G.L[a]);
                else if (xp < G.lo[a]) xp = __dadd_rn(xp, G.L[a]);
            }
            B.xp_b[q] = xp;
            B.v0_b[q] = __fma_rn(P.dt, Fv[a], V);
            B.s_b[q] = __dmul_rn(P.kappa, __fma_rn(__fma_rn(-4.0, V, B.vnm1_b[q]), P.inv_2dt, -P.g[a]));
        }
        B.ph0_b[s] = __fma_rn(0.5 * P.dtau, apv, B.pn_b[s]);
    }
}

// --------------------------------------------------------------- pair cache

// The pair coefficients of every list entry (order of the latest binning):
// gradW_ij and F_ij for a fluid slot, W_wf and rho0 (g . r_wf) W_wf for a wall
// slot, at the entry's place in the sliced layout. Entries are independent, so
// L only sets the parallelism. Block 0 also resets the pseudo-time loop state.
template <int D, bool F32, int L>
__global__ void __launch_bounds__(kBlock) k_pair_cache(Buffers B, const double *__restrict__ xpos,
                                                       const uint32_t *__restrict__ gid)
{
    using T = typename std::conditional<F32, float, double>::type;
    constexpr int SPB = kBlock / L;
    __shared__ Geom G;
    __shared__ Phys P;
    if (blockIdx.x == 0) {
        reset_loops(B);
    }
    const int inst = block_instance(B, blockIdx.x * SPB);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int s = blockIdx.x * SPB + threadIdx.x / L, lane_in = threadIdx.x % L;
    const int n = B.n;
    if (s >= n || gid[s] == kNoParticle) return;
    const bool wall_s = gid[s] >= (uint32_t)B.nf;
    const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
    const float4 oi = F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    const T sigma = (T)(P.sig_h * P.h);
    const int cnt = B.pcount[s];
    // R entries per round, their offsets gathered together (as in k_state_n)
    constexpr int R = 4;
    for (int q0 = lane_in; q0 < cnt; q0 += L * R) {
        uint32_t jbv[R];
        int cv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const size_t e = base + (size_t)min(q0 + r * L, cnt - 1) * kWarp;
            jbv[r] = B.pj[e];
            cv[r] = B.pcode[e];
        }
        float4 ov[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            ov[r] = F32 ? B.off[(int)(jbv[r] & ~kWallBit)] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int q = q0 + r * L;
            if (q >= cnt) break;
            const size_t e = base + (size_t)q * kWarp;
            const uint32_t jb = jbv[r];
            const int j = (int)(jb & ~kWallBit);
            T d[3], r2;
            if (F32) {
                offset_sep<D, T>(G, oi, ov[r], cv[r], d, r2);
            } else {
                int dx, dy, dz;
                decode_shift(cv[r], dx, dy, dz);
                listed_sep<D, F32, T>(G, xpos, B.off, n, s, j, oi, dx, dy, dz, d, r2);
            }
            T c4[4] = {T(0), T(0), T(0), T(0)};
            if (wall_s) {
                const T W = Ar<T>::mul(sigma, quintic_w<T>(Ar<T>::mul(sqrt(r2), (T)P.inv_h)));
                T gr = T(0);
                for (int a = 0; a < D; ++a) gr += (T)P.g[a] * d[a];
                c4[0] = W;
                c4[1] = (T)P.rho0 * gr * W;
            } else {
                // layout (gradW, F_ij); FP32C in 2D packs (gx, gy, F_ij, index bits)
                T g[3], F;
                grad_coef<D, T>(P, d, r2, g, F);
                c4[0] = g[0];
                c4[1] = g[1];
                if (F32 && D == 2) {
                    c4[2] = F;
                } else {
                    c4[2] = D == 3 ? g[2] : T(0);
                    c4[3] = F;
                }
            }
            if (F32) {
                float4 v = make_float4((float)c4[0], (float)c4[1], (float)c4[2], (float)c4[3]);
                if (D == 2) v.w = __uint_as_float(jb);
                B.pc32[e] = v;
            } else {
                B.pc64[e] = make_double4_32a((double)c4[0], (double)c4[1], (double)c4[2], (double)c4[3]);
            }
        }
    }
}

// ---------------------------------------------------------------- shifting

// Particle shifting after the real step (Sec. 3.5), in order B at r^{n+1}, one
// lane per slot; the displacement over every neighbour (wall particles continue
// the particle distribution), the gradients of the correction over fluid
// neighbours (free-surface runs: particles with div r_i < dim - 1/2, fluid and
// wall neighbours counted, stay where they are):
//   dr_i = -(h^2/2) sum_j V_j (1 + W_ij / W(h)) gradW_ij          Eq. (shift-deltar)
//   f_i <- f_i + (grad f)_i . dr_i, (grad f)_i = sum_j V_j (f_j - f_i) gradW_ij
//                                                      for f = p, V   Eq. (shift-correct)
//   r_i <- r_i + dr_i (wrapped on periodic axes)
// with V_j = m / rho0 and W(h) the kernel at r = h. Every gradient uses the
// unshifted fields (reads order B); the shifted r, V, p go to the particle's
// slot in order A (perm), which the next step bins again.
template <int D, bool F32>
__global__ void __launch_bounds__(kBlock) k_shift(Buffers B)
{
    using T = typename std::conditional<F32, float, double>::type;
    using Acc = typename std::conditional<F32, Kahan, Plain64>::type;
    __shared__ Geom G;
    __shared__ Phys P;
    const int inst = block_instance(B, blockIdx.x * kBlock);
    block_copy(G, B.geo[inst]);
    block_copy(P, B.phys[inst]);
    const int n = B.n;
    const int s = blockIdx.x * kBlock + threadIdx.x;
    if (s >= n) return;
    if (B.gid_b[s] >= (uint32_t)B.nf) return;            // walls and padding stay
    const auto *nb = nb_ptr<T>(B, 1);                     // (V, p) at r^{n+1}, order B
    const auto qi = nb[s];
    const T vi[3] = {(T)qi.x, (T)qi.y, (T)qi.z};
    const T pi = (T)qi.w;
    const float4 oi = F32 ? B.off[s] : make_float4(0, 0, 0, 0);
    const T vol = (T)(P.m / P.rho0);
    const T sigma = (T)(P.sig_h * P.h);
    const T w_h = sigma * quintic_w<T>(T(1));
    Acc dr[3], gp[3], gv[3][3];
    double divr = 0.0;            // div r_i = -sum_j V_j r_ij . gradW_ij, walls included
    const size_t base = (size_t)(s >> 5) * B.K * kWarp + (s & 31);
    const int cnt = B.pcount[s];
    for (int k = 0; k < cnt; ++k) {
        const size_t e = base + (size_t)k * kWarp;
        const uint32_t jb = B.pj[e];
        const int j = (int)(jb & ~kWallBit);
        int dx, dy, dz;
        decode_shift(B.pcode[e], dx, dy, dz);
        T d[3], r2;
        listed_sep<D, F32, T>(G, B.x_b, B.off, n, s, j, oi, dx, dy, dz, d, r2);
        const T r = sqrt(r2);
        const T q = r * (T)P.inv_h;
        const T a = r > T(0) ? (T)P.sig_h * quintic_dwdq<T>(q) / r : T(0);
        divr -= (double)(vol * a * r2);                   // r_ij . gradW_ij = (dW/dr / r) r^2
        // the displacement counts every neighbour, wall particles included
        // (they continue the particle distribution)
        const T fdr = vol * (T(1) + sigma * quintic_w<T>(q) / w_h);
#pragma unroll
        for (int c = 0; c < D; ++c) dr[c].add(fdr * (a * d[c]));
        if (jb & kWallBit) continue;                      // the gradients: fluid neighbours only

        const auto qj = nb[j];
        const T vj[3] = {(T)qj.x, (T)qj.y, (T)qj.z};
        const T dp = vol * ((T)qj.w - pi);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const T gw = a * d[c];
            gp[c].add(dp * gw);
#pragma unroll
            for (int b2 = 0; b2 < D; ++b2) gv[b2][c].add(vol * (vj[b2] - vi[b2]) * gw);
        }
    }
    // a free-surface particle (Lind et al.'s test, Sec. 3.5) is not shifted
    const bool surface = P.free_surface && divr < (double)D - 0.5;
    const double dmul = surface ? 0.0 : -0.5 * P.h * P.h;
    double drv[3] = {0, 0, 0};
    for (int c = 0; c < D; ++c) drv[c] = dmul * (double)(T)dr[c].value();
    const int o = B.perm[s];
    double pnew = B.pn_b[s];
    for (int c = 0; c < D; ++c) pnew += (double)(T)gp[c].value() * drv[c];
    B.pn_a[o] = pnew;
    for (int b2 = 0; b2 < D; ++b2) {
        double v = B.vn_b[(size_t)b2 * n + s];
        for (int c = 0; c < D; ++c) v += (double)(T)gv[b2][c].value() * drv[c];
        B.vn_a[(size_t)b2 * n + o] = v;
        double x = B.x_b[(size_t)b2 * n + s] + drv[b2];
        if (G.periodic[b2]) {
            if (x >= G.hi[b2]) x -= G.L[b2];
            else if (x < G.lo[b2]) x += G.L[b2];
        }
        B.x_a[(size_t)b2 * n + o] = x;
    }
}

}  // namespace

// Lanes per slot of the list build: enough warps to fill the GPU on small
// problems (each group's candidate chain is latency-bound), one lane per slot
// on large ones.
int nlist_lanes(int n)
{
    int L = 1;
    while (L < 8 && (long long)n * L < 400000) L *= 2;
    return L;
}

void launch_nlist(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st)
{
    if (B.dim == 3 && B.fp32c) {
        k_nlist_cells3<<<(B.ncell + kBlock / kWarp - 1) / (kBlock / kWarp), kBlock, 0, st>>>(B, xpos);
        return;
    }
    const int L = nlist_lanes(B.n);
    const int nb = (int)(((long long)B.n * L + kBlock - 1) / kBlock);
    if (L == 1) DTSPH_DISPATCH(B.dim, B.fp32c, (k_nlist<D, F32, 1><<<nb, kBlock, 0, st>>>(B, xpos, cell, gid)));
    else if (L == 2) DTSPH_DISPATCH(B.dim, B.fp32c, (k_nlist<D, F32, 2><<<nb, kBlock, 0, st>>>(B, xpos, cell, gid)));
    else if (L == 4) DTSPH_DISPATCH(B.dim, B.fp32c, (k_nlist<D, F32, 4><<<nb, kBlock, 0, st>>>(B, xpos, cell, gid)));
    else DTSPH_DISPATCH(B.dim, B.fp32c, (k_nlist<D, F32, 8><<<nb, kBlock, 0, st>>>(B, xpos, cell, gid)));
}

// Neighbour lists at r^n (order B), then the wall values and the state-n pass.
int launch_state_n(const Buffers &B, bool predictor, cudaStream_t st)
{
    constexpr int L = kSumLanes;
    const int nb = (int)(((long long)B.n * L + kBlock - 1) / kBlock);
    launch_nlist(B, B.x_b, B.cell_b, B.gid_b, st);
    int k = 1;
    if (B.nw > 0) {
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_walls_state_n<D, F32, L><<<nb, kBlock, 0, st>>>(B)));
        ++k;
    }
    const bool w = B.nw > 0;
    if (predictor && w)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, true, true, L><<<nb, kBlock, 0, st>>>(B)));
    else if (predictor)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, true, false, L><<<nb, kBlock, 0, st>>>(B)));
    else if (w)
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, false, true, L><<<nb, kBlock, 0, st>>>(B)));
    else
        DTSPH_DISPATCH(B.dim, B.fp32c, (k_state_n<D, F32, false, false, L><<<nb, kBlock, 0, st>>>(B)));
    return k + 1;
}

// Neighbour lists at xpos, then the pair coefficients.
int launch_pair_cache(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st)
{
    launch_nlist(B, xpos, cell, gid, st);
    const int L = nlist_lanes(B.n);
    const int nb = (int)(((long long)B.n * L + kBlock - 1) / kBlock);
    if (L == 1) DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 1><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    else if (L == 2) DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 2><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    else if (L == 4) DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 4><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    else DTSPH_DISPATCH(B.dim, B.fp32c, (k_pair_cache<D, F32, 8><<<nb, kBlock, 0, st>>>(B, xpos, gid)));
    return 2;
}

int launch_shift(const Buffers &B, cudaStream_t st)
{
    int k = launch_binning(B, B.x_a, B.gid_a, st);            // cells at r^{n+1}
    k += launch_permute_a_to_b(B, st);
    launch_nlist(B, B.x_b, B.cell_b, B.gid_b, st);
    DTSPH_DISPATCH(B.dim, B.fp32c, (k_shift<D, F32><<<(B.n + kBlock - 1) / kBlock, kBlock, 0, st>>>(B)));
    return k + 2;
}

}  // namespace dtsph
