// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/dtsph.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/dtsph.h"

namespace dtsph {

constexpr int kBlock = 256;          // threads per block of every particle kernel
constexpr int kWarp = 32;
constexpr uint32_t kWallBit = 0x80000000u;   // set in a cached neighbour index when j is a wall

// A neighbour-list entry in one 32-bit word: the neighbour's slot (bits 0-25),
// the cell shift code (dx + 1) + 3 (dy + 1) + 9 (dz + 1) of its cell against the
// home cell (bits 26-30) and the wall flag (bit 31). The pair cache keeps the
// slot and the wall flag only (code bits clear).
constexpr int kCodeShift = 26;
constexpr uint32_t kSlotMask = (1u << kCodeShift) - 1u;
constexpr uint32_t kCodeMask = 31u << kCodeShift;
constexpr long long kMaxSlots = 1LL << kCodeShift;
__host__ __device__ __forceinline__ uint32_t list_entry(uint32_t j, int code, bool wall)
{
    return j | ((uint32_t)code << kCodeShift) | (wall ? kWallBit : 0u);
}
__host__ __device__ __forceinline__ int entry_slot(uint32_t e) { return (int)(e & kSlotMask); }
__host__ __device__ __forceinline__ int entry_code(uint32_t e) { return (int)((e >> kCodeShift) & 31u); }

// Error bits raised by kernels into Buffers::err (read by dtsph_sync).
enum : uint32_t { kErrCapacity = 1u, kErrDomain = 2u, kErrBarrier = 4u, kErrCopy = 8u, kErrSkin = 16u,
                  kErrNonFinite = 32u };

// A context advances one or more independent simulations ("instances") together.
// Instance i owns the slot range [slot_off, slot_off + nf + nw) of every particle
// array, with slot_off a multiple of kSlotAlign; the slots between ranges are
// padding (caller index kNoParticle). Every block of every particle kernel covers
// at most kSlotAlign consecutive slots from a multiple of its own width, so a
// block never straddles two instances.
constexpr int kSlotAlign = 256;
constexpr int kMaxStages = 8;        // deepest shared-memory ring of the one-lane iterate kernel
constexpr uint32_t kNoParticle = 0xFFFFFFFFu;
constexpr unsigned long long kBarrierWaitNs = 1000000000ull;   // grid-barrier give-up time (1 s)
// Batches of up to this many instances deal their active tiles to the blocks
// of the persistent loop (and may run the decoupled loop); larger batches take
// the tiles in the static order.
constexpr int kDealMaxInst = 1024;

constexpr int kPassWaveBlocksPerSm = 8;   // blocks per SM of a grid-stride pass that a graph may skip
constexpr int kSeg2 = 3;   // cells along x in one row segment of the 2D FP32C list builder

struct Inst {
    int slot_off;          // first slot
    int nf, nw;            // fluid and wall particles
    int foff, woff;        // first caller index of its fluid particles / of its walls
    int cell_off;          // first cell; the instance owns ncell + 1 cells, the last one
                           // always empty so that its start marks the end of the range
    int shift;             // slot_off minus the particles of the instances before it
    int seg_off;           // first row segment of the 2D FP32C list builder (kSeg2 cells along x)
};

// Cell grid and neighbour-test constants of one binning. Cells have side
// s[a] >= 3h, so every neighbour lies in the 3^dim surrounding cells.
struct Geom {
    int dim;
    int periodic[3];
    int nc[3];            // cells per axis
    int ncell;            // nc[0] * nc[1] * nc[2]
    double lo[3], hi[3];
    double L[3], halfL[3];
    double s[3], inv_s[3];
    float s_f[3];
    double rc2;           // (3h + skin)^2, the FP64 neighbour test (skin: moving = 2 only)
    float rc2_lo, rc2_hi; // FP32 pre-test band: below lo is in, above hi is out
};

// Physical constants of the pair terms, folded for rho_i = rho_j = rho0 and a
// uniform mass m (Sec. 3: density held fixed).
struct Phys {
    double h, m, rho0, c, nu, nu_e, dt, dtau;
    double sig_h;        // sigma / h: dW/dr = sig_h * dWdq(q)
    double eta_h2;       // eta h^2 (viscous and artificial-viscosity denominators)
    double edac_h2;      // eta h^2, or h^2 for the literal reading
    double c_div;        // m (rho_i / rho_j) c^2                       divergence term
    double c_edac;       // 4 m nu_e / ((rho_i + rho_j) rho_j)           EDAC term
    double c_p;          // m / rho0^2                                  pressure term
    double c_visc;       // 4 m nu / (rho_i + rho_j)                     viscous term
    double c_av;         // alpha h c / rho0                            artificial viscosity
    double g[3];
    double kappa;        // 2 dt / (2 dt + 3 dtau), Eq. (dv_dtau_exact)
    double c3;           // 3 / (2 dt)
    double kc3;          // kappa * 3 / (2 dt)
    double inv_h;        // 1 / h
    double inv_2dt;      // 1 / (2 dt)
    double rp_scale;     // dt / (rho0 c^2) / nf
    double rv_scale;     // dt / v_ref / nf
    float dtau_f;        // dtau rounded to FP32 (the FP32C p-hat update)
    int edac, use_av;
    int steady;          // steady-state mode: kappa = 1, no 3/(2dt) term, source -g,
                         // convection term, particles fixed
    int free_surface;    // wall pressure kept >= 0; free-surface particles not shifted
    double vol;          // m / rho0 (convection term)
    int moving;          // 0: particles fixed in pseudo-time; 1: moved (Algorithm 1),
                         // lists of r^0; 2: moved, lists with a skin
    int pad_m;
    double disp2_max;    // (skin / 2)^2: the largest squared pseudo-time displacement
                         // from r^0 that the lists with a skin cover (moving = 2)
    double disp2_reuse;  // (list_skin / 2)^2: the largest squared distance of r^{n+1}
                         // from r^0 that lets the r^0 lists serve the next step
};

// Stop reason of a loop without the pair cache that reached pause_at iterations
// without meeting a stop rule (the step goes on with the cache; never reported).
constexpr int kPaused = -2;

// Convergence control of one instance's pseudo-time loop, in device memory.
struct LoopState {
    int iter;              // iterations completed in this real step
    int done;              // 1 once a stop rule holds
    int reason;            // stop reason (dtsph_step_stats.reason), -1 while running
    unsigned int ticket;   // last-block election counter of the instance's tiles
    int last_iters;        // iterations of the latest finished real step (0: none since allocation)
    int pause_at;          // a loop without the pair cache pauses after this many iterations
                           // (0: never); the step then goes on with the cache
    double rp, rv;         // residuals of the last iteration
    double hist_p[16], hist_v[16];   // ring of the last residuals (stagnation test)
    int max_iter, fixed_iters, stag_window;
    int stat_slot;         // entry of the statistics ring this real step writes
    double eps, stag_tol;
    long long step;        // real steps completed (indexes the stats ring)
};

// Context-wide control words of the pseudo-time loop.
struct LoopCtrl {
    unsigned int ticket;   // last-block election over all tiles of the iterate kernel
    unsigned int bar;      // grid-barrier arrival counter of the persistent loop kernel
    int active;            // instances still iterating
    int pad;
};

// Work counters of one instance in the decoupled batch loop (k_loop_async):
// claim = (iteration << 32) | next tile of that iteration to hand out;
// done_tiles = tiles of the iteration finished so far.
struct InstLoop {
    unsigned long long claim;
    unsigned int done_tiles;
    int pad;
};

struct StatRec {
    int iters, reason;
    double rp, rv;
    double vmax;           // max |V^{n+1}| over the instance's fluid particles (before shifting)
    int form, pad;         // dtsph_step_stats.form of the step
};
constexpr int kStatRing = 65536;   // real steps kept per instance

// Device buffers of one context. Particle arrays hold all n = nf + nw particles
// in the order of the latest binning ("A" = the loop order kept between steps,
// "B" = the order of the binning at r^n inside a step). SoA per component.
struct Buffers {
    int n;                          // slots (all instances, padding included)
    int nf, nw;                     // fluid and wall particles of all instances
    int nseg2;                      // row segments of the 2D FP32C list builder, all instances
    int nsm;                        // streaming multiprocessors of the device
    int l2_stream;                  // 1: the pair cache exceeds half of L2 (its rows stream, evicting first)
    int reuse_lists;                // 1: the r^0 lists (with list_skin) serve the next step at r^n
    // with reused lists: *relist is 1 when a particle of the latest step ended
    // farther than list_skin / 2 from its r^0; the next step then bins and lists
    // at r^n. A launch with relist_run 0 or 1 runs only when *relist equals it
    // (-1: always); the pass to order A clears *relist
    int *relist;
    int relist_run;
    int *slot_of;                   // with reused lists: [nf] slot of each fluid particle (caller index)
    int dim, fp32c, K;              // K = neighbour capacity per particle
    int lanes;                      // lanes per particle in the iterate kernel (1, 2, 4 or 8)
    int stages;                     // pair-cache chunks in flight per warp (lanes = 1), 2..kMaxStages
    int ninst, ncell;               // instances; cells of all instances (sentinels included)
    unsigned long long barrier_ns;  // give-up time of the persistent loop's grid barrier
    const Inst *inst;               // [ninst]
    const Geom *geo;                // [ninst]
    const Phys *phys;               // [ninst]
    const uint16_t *inst_of;        // instance of each slot [n]
    // order A (persistent)
    uint32_t *gid_a;       // caller index of each slot (walls: nf + wall index; padding: kNoParticle)
    double *x_a;           // r^n           [dim][n]
    double *xp_a;          // r^0 (frozen)  [dim][n]
    double *vn_a;          // V^n (walls: prescribed velocity) [dim][n]
    double *vnm1_a;        // V^{n-1}       [dim][n]
    double *pn_a;          // p^n           [n]
    double *s_a;           // kappa ((V^{n-1} - 4 V^n) / (2 dt) - g): BDF2 source and body force [dim][n]
    int *cell_a;           // cell of each slot
    int *wslot_a;          // [nw] slot of each wall particle (by caller wall index), null where no loop runs
    float4 *wv32;          // FP32C: [n] V^n of each wall slot packed (prescribed velocity), null without walls
    double4_32a *wv64;     // FP64: the same in FP64
    // order B (scratch inside a step)
    uint32_t *gid_b;
    double *x_b, *vn_b, *vnm1_b, *pn_b, *xp_b, *v0_b, *ph0_b, *s_b;
    int *cell_b;
    // binning scratch
    int *key;              // cell of each particle in the pre-binning order
    int *slot;             // rank inside its cell (atomic order)
    int *unsorted;         // new slot -> old slot, cells in atomic order
    int *perm;             // new slot -> old slot, each cell ordered by caller index
    int *cell_count;       // [ncell], zero between binnings
    int *cell_start;       // [ncell + 1], slot of the first particle of each cell
    int *scan_tmp;         // [ncell / 4096 + 2] block totals of the cell-count scan
    // FP32 offsets of each particle from its cell origin (FP32C geometry);
    // .w is 1 for a wall particle
    float4 *off;           // [n]
    // pseudo-time iterates, ping-pong on the iteration parity
    double *vk[2];         // V^k FP64 [dim][n]
    double4_32a *nb64[2];      // FP64: (V, p-hat) packed for neighbour gathers
    float4 *nb32[2];       // FP32C: (V, p-hat) packed for neighbour gathers
    // pair cache, sliced by warp: entry k of slot i at ((i/32) K + k) 32 + i%32
    uint32_t *pj;          // list entries (list_entry); after the pair-cache pass slot | kWallBit
    uint32_t *pjt;         // neighbour lists, per slot: entry k of slot s at s Ks + k (Ks = list_stride(K))
    double4_32a *pc64;         // FP64: (gradW, F_ij)
    float4 *pc32;          // FP32C: (gradW, F_ij); in 2D .w holds the index bits
    int *pcount;           // neighbours of each slot
    // particles moving in pseudo-time (Algorithm 1; allocated only then), order A
    double *xk[2];         // r^{k+1/2} FP64 [dim][n], ping-pong
    float4 *offk[2];       // FP32C: FP32 offsets of r^{k+1/2} from the slot's cell origin at r^0
    double *vt;            // V~^k = dt (dV/dtau)^{k-1/2}, Eq. (vtilde) [dim][n] (own slot only)
    // state-n rates (test entry and predictor)
    double *ap_b;          // [n]
    double *f_b;           // [dim][n]
    // residual reduction
    double *blk;           // [2 x tiles], double-buffered: per-tile residual partial sums
    LoopState *ls;         // [ninst]
    LoopCtrl *ctrl;
    InstLoop *il;          // [ninst] work counters of the decoupled batch loop (null without it)
    const int *sched;      // [ninst] instances by ascending tile count (the decoupled loop's search order)
    int async_loop;        // 1: batches without walls run the decoupled loop kernel
    int form_a;            // 1: the loop recomputes the pair geometry from the lists (no pair cache)
    // the per-step choice of the pair-term form (form = 0), in the step graph
    // only (null elsewhere): k_loop_reset writes the step's form to *form_sel
    // (0 cache, 1 recomputed; k_loop_resume turns 1 into 2 when a paused loop
    // goes on with the cache) and counts it in form_count[form]; a launch of
    // the graph runs only when *form_sel equals its form_run
    int *form_sel;
    unsigned long long *form_count;   // [3]
    int form_run;
    double kstar;          // the uncached form runs when the latest step took at most kstar iterations
    StatRec *stats;        // [kStatRing][ninst]
    uint32_t *err;
};

// Runs the statement with D (2 or 3) and F32 (FP32C path) as constants.
#define DTSPH_DISPATCH(D_, F32_, ...)                                                                \
    do {                                                                                             \
        if ((D_) == 2 && !(F32_)) { constexpr int D = 2; constexpr bool F32 = false; __VA_ARGS__; } \
        else if ((D_) == 2) { constexpr int D = 2; constexpr bool F32 = true; __VA_ARGS__; }        \
        else if (!(F32_)) { constexpr int D = 3; constexpr bool F32 = false; __VA_ARGS__; }         \
        else { constexpr int D = 3; constexpr bool F32 = true; __VA_ARGS__; }                       \
    } while (0)

// Instance owning the block that covers slots [first, first + width): a block
// never straddles two instances.
__device__ __forceinline__ int block_instance(const Buffers &B, int first)
{
    return first < B.n ? (int)B.inst_of[first] : 0;
}

// ------------------------------------------------------------ launchers
// Every launcher enqueues on `st` and returns the number of kernels launched.

int launch_binning(const Buffers &B, const double *x_keys, const uint32_t *gid_src, cudaStream_t st);
int launch_permute_a_to_b(const Buffers &B, cudaStream_t st);
int launch_permute_b_to_a(const Buffers &B, cudaStream_t st);
#ifdef __CUDACC__
// True in a launch of the step graph guarded on relisting (see Buffers::relist)
// whose condition does not hold. Block-uniform.
__device__ __forceinline__ bool skip_relist(const Buffers &B)
{
    return B.relist && B.relist_run >= 0 && *(volatile const int *)B.relist != B.relist_run;
}
#endif
// Order B = order A with offsets at r^n from the slots' cells (lists reused).
int launch_same_order_a_to_b(const Buffers &B, cudaStream_t st);
// Order A = order B (after a binning at r^n that starts reusing lists).
int launch_adopt_b(const Buffers &B, cudaStream_t st);
// A new state (caller order) into the slots of order A as they are, the lists
// kept; a particle farther than list_skin / 2 from its r^0 sets *relist.
int launch_scatter_same(const Buffers &B, const double *x, const double *v, const double *p, const double *vprev,
                        cudaStream_t st);
// Neighbour lists of every slot at positions xpos (order of the latest binning);
// one launch.
void launch_nlist(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st,
                  bool sliced);
// The state-n pass at r^n in order B: its lists built first, or (build_lists
// false) the r^0 lists of the previous step, built with list_skin, as they are.
int launch_state_n(const Buffers &B, bool predictor, cudaStream_t st, bool build_lists = true);
int launch_loop_resume(const Buffers &B, cudaStream_t st);
int launch_restart_steps(const Buffers &B, cudaStream_t st);
int launch_pair_cache_pass(const Buffers &B, const double *xpos, const uint32_t *gid, cudaStream_t st);
int launch_pair_cache(const Buffers &B, const double *xpos, const int *cell, const uint32_t *gid, cudaStream_t st);
int launch_walls_iter(const Buffers &B, cudaStream_t st);
int launch_iterate(const Buffers &B, unsigned long long cond_handle, int use_cond, cudaStream_t st);
int launch_outer(const Buffers &B, cudaStream_t st);
// Particles moving in pseudo-time (Algorithm 1): the lists at r^0 (with the
// skin for moving = 2), the start iterate r^{1/2} = r^0, V~^0 = 0, and the loop
// state reset (replaces the pair cache of the frozen loop).
int launch_move_prepare(const Buffers &B, cudaStream_t st);
// One moving pseudo-iteration: the wall values at the moved positions, then the
// pair pass with the advective terms, the update of V, V~, r and p-hat, and the
// stop rules (sets the while-node condition when use_cond).
int launch_move_iteration(const Buffers &B, unsigned long long cond_handle, int use_cond, cudaStream_t st);
// Particle shifting of the fluid after the real step: bins at r^{n+1}, gathers
// the state into order B, builds the lists, and shifts (results written back to
// order A).
int launch_shift(const Buffers &B, cudaStream_t st);
// Persistent pseudo-time loop (one cooperative launch per real step): grid size
// (co-resident blocks, at most one per tile) and the launch itself.
int loop_grid(const Buffers &B, int *grid);
cudaError_t launch_loop(const Buffers &B, int grid, cudaStream_t st);
int launch_loop_reset(const Buffers &B, cudaStream_t st);
// Raises the dynamic shared-memory limit of the kernels that stage pair-cache
// rows (once per device, before any launch or capture); 0 on success.
int iterate_prepare();
int launch_unpermute(const Buffers &B, const uint32_t *gid, const double *src, double *out, int comps, cudaStream_t st);
// Contiguous copy of count doubles by a kernel (0 launches for count = 0).
int launch_copy(const double *src, double *dst, size_t count, cudaStream_t st);
int launch_scatter_in(const Buffers &B, const double *x, const double *v, const double *p, const double *vprev,
                      const double *xw, const double *vw, cudaStream_t st);
// Writes one instance's tables (inst/geo/phys entry i) from values, for callers
// whose tables live in device memory they cannot copy into from the host.
int launch_fill_instance(Inst *inst, Geom *geo, Phys *phys, int i, const Inst &I, const Geom &G, const Phys &P,
                         cudaStream_t st);

int iterate_tiles(const Buffers &B);   // tiles of the iterate kernel (one block each)
// The loop kernels without the pair cache (iterate_fa.cu; contexts without walls).
void launch_iterate_fa(const Buffers &B, unsigned long long cond, int use_cond, cudaStream_t st);
const void *loop_function_fa(const Buffers &B);
// Row length of the per-slot neighbour lists: K rounded up to 8 entries, so a
// row starts on a 32-byte boundary.
__host__ __device__ constexpr int list_stride(int K) { return (K + 7) / 8 * 8; }

// The neighbour list of slot s as the builders write it (entries in order,
// pcount[s] of them).
__device__ __forceinline__ const uint32_t *slot_list(const Buffers &B, int s)
{
    return B.pjt + (size_t)s * list_stride(B.K);
}

// ------------------------------------------------- one parameter set (api.cu)
// Shared by the context entry points and the allocation-free rate evaluation,
// so that both read dtsph_params the same way. The first two return DTSPH_OK or
// a DTSPH_E_* code with a one-line message in msg (capacity cap).
int check_params(const dtsph_params *p, char *msg, size_t cap);
int make_geometry(const dtsph_params &p, Geom &G, char *msg, size_t cap);
void make_phys(const dtsph_params &p, Phys &P);
int neighbour_capacity(const dtsph_params &p);

}  // namespace dtsph
