// C ABI of the library (include/dtsph.h): contexts of one or more independent
// instances, device memory, the per-step launch sequence, its CUDA-graph
// capture, the autotuner, and field read-back.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dtsph.h"
#include "dtsph_internal.cuh"

using namespace dtsph;

struct dtsph_ctx {
    int ninst = 1;
    std::vector<dtsph_params> prm;      // per instance; dim, precision, graph, lanes shared
    std::vector<Geom> G;
    std::vector<Phys> P;
    std::vector<Inst> I;
    Buffers B;
    cudaStream_t stream = nullptr;      // caller stream (may be the legacy default stream)
    cudaStream_t cap = nullptr;         // private stream used for graph capture
    int device = 0;
    bool have_particles = false;
    // the device reads and writes pageable host memory itself (Grace-based
    // systems over NVLink-C2C: cudaDevAttrPageableMemoryAccess), so the host
    // arrays of dtsph_set_particles and dtsph_read_field are accessed in place
    // by kernels instead of through cudaMemcpyAsync's pageable path
    bool host_direct = false;
    bool have_nbrs = false;             // dtsph_build_neighbors lists in order B
    std::vector<std::vector<double>> xw_host, vw_host;   // walls per instance
    std::vector<int64_t> nf_set;        // fluid particles per instance of the current allocation
    int64_t steps = 0;
    int64_t launches = 0;
    int per_step_fixed = 0;             // kernels per step outside the loop
    int per_iter = 0;                   // kernels per pseudo-iteration
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    std::string err;
    std::vector<void *> allocs;
    size_t alloc_bytes = 0;             // device bytes allocated by the context
    size_t alloc_limit = 0;             // 0, or a cap on alloc_bytes (DTSPH_TEST_ALLOC_LIMIT, tests only)
    double *sx = nullptr, *sv = nullptr, *sp = nullptr, *svp = nullptr, *sxw = nullptr, *svw = nullptr;
    double *rd = nullptr;                // dtsph_read_state: the fields in caller order (3 nf dim + nf)
    bool tuned = false;
    // events around the pseudo-time loop of each real step (pair step % kLoopEv),
    // recorded by event nodes of the step graph or on the stream
    static constexpr int kLoopEv = 256;
    std::vector<cudaEvent_t> ev_a, ev_b;
    cudaGraphNode_t node_a = nullptr, node_b = nullptr;
    // form = 0 with the persistent loop, no walls, frozen particles: the step
    // graph holds both pair-term forms and chooses one per step on the device
    // (without the cache when the latest finished step took at most kstar
    // iterations, the break-even count of the two forms' measured costs); both
    // give the same bits
    bool form_graph = false;            // the step graph chooses the form
    // reused lists (list_skin > 0): order A, its cells and the lists hold the
    // binning and the lists of the latest r^0 (or of r^n before the first step);
    // a call that bins or builds lists otherwise clears this, and the next step
    // first bins and lists at r^n
    bool lists_ready = false;
    int *form_sel = nullptr;            // device: the current step's form
    unsigned long long *form_count = nullptr;   // device: steps run in each form
    double kstar = -1.0;                // < 0: not measured
    float form_ms[3] = {-1.f, -1.f, -1.f};   // cache pass, cached loop and no-cache loop per iteration
    int64_t steps_cache = 0, steps_nocache = 0;   // steps of the other paths
    struct TuneRec { int lanes, stages; float ms; };
    std::vector<TuneRec> tune_log;      // candidates timed by the last tuning
};

namespace {

const char *kNoCtx = "null context";

// An NVTX range for the lifetime of the object (host-side spans that profilers
// such as Nsight Systems show beside the kernels).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

int fail(dtsph_ctx *c, int code, const char *fmt, ...)
{
    if (!c) return code;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return code;
}

// A non-negative integer from the environment, or dflt when unset or malformed.
unsigned long long env_u64(const char *name, unsigned long long dflt)
{
    const char *v = getenv(name);
    if (!v || !*v) return dflt;
    char *end = nullptr;
    const unsigned long long x = strtoull(v, &end, 10);
    return end && *end == 0 ? x : dflt;
}

// Formats a message into msg (capacity cap) and returns code.
int say(char *msg, size_t cap, int code, const char *fmt, ...)
{
    if (msg && cap) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(msg, cap, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(c, DTSPH_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

template <typename T>
int dalloc(dtsph_ctx *c, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (c->alloc_limit && c->alloc_bytes + count * sizeof(T) > c->alloc_limit)
        return fail(c, DTSPH_E_OOM, "allocation of %zu bytes would pass the cap of %zu bytes (DTSPH_TEST_ALLOC_LIMIT)",
                    count * sizeof(T), c->alloc_limit);
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DTSPH_E_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    c->alloc_bytes += count * sizeof(T);
    return DTSPH_OK;
}

void free_all(dtsph_ctx *c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->form_graph = false;
    c->lists_ready = false;
    c->form_sel = nullptr;
    c->form_count = nullptr;
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->alloc_bytes = 0;
    memset(&c->B, 0, sizeof(c->B));
    c->have_particles = false;
    c->have_nbrs = false;
}

double pi() { return 3.14159265358979323846; }

// Quintic spline normalisation: W integrates to 1 over R^dim.
double quintic_sigma(int dim, double h)
{
    return dim == 2 ? 7.0 / (478.0 * pi() * h * h) : 1.0 / (120.0 * pi() * h * h * h);
}

int setup_geometry(dtsph_ctx *c, const dtsph_params &p, Geom &G)
{
    char msg[256];
    const int r = dtsph::make_geometry(p, G, msg, sizeof msg);
    return r ? fail(c, r, "%s", msg) : DTSPH_OK;
}

}  // namespace

// Cell grid of one parameter set (cells of side > 3h, + skin for moving = 2).
int dtsph::make_geometry(const dtsph_params &p, Geom &G, char *msg, size_t cap)
{
    memset(&G, 0, sizeof G);
    G.dim = p.dim;
    // the lists cover 3h, plus the skin when the particles move in pseudo-time
    // with neighbour updates or when the r^0 lists serve the next step at r^n
    // (pairs beyond 3h add exact zeros)
    const double rc = 3.0 * p.h + (p.moving == 2 ? p.skin : 0.0) + p.list_skin;
    G.ncell = 1;
    for (int a = 0; a < 3; ++a) {
        G.periodic[a] = a < p.dim ? p.periodic[a] : 0;
        G.lo[a] = p.lo[a];
        G.hi[a] = p.hi[a];
        if (a >= p.dim) {
            G.nc[a] = 1;
            G.s[a] = 1.0;
            G.inv_s[a] = 1.0;
            G.s_f[a] = 1.f;
            G.L[a] = 1.0;
            G.halfL[a] = 0.5;
            continue;
        }
        double L = p.hi[a] - p.lo[a];
        if (!(L > 0)) return say(msg, cap, DTSPH_E_ARG, "axis %d: hi must exceed lo", a);
        // cells strictly wider than 3h so that rounding never separates neighbours
        // (cell_scale > 1: wider cells by that factor)
        const double side = rc * std::max(1.0, p.cell_scale);
        long long k = (long long)std::floor(L / (side * (1.0 + 1e-9)));
        if (k < 1) k = 1;
        if (G.periodic[a] && k < 3)
            return say(msg, cap, DTSPH_E_ARG, "periodic axis %d is shorter than three list cutoffs (%g < %g)", a,
                       L, 3 * rc);
        if (k > (1 << 20)) return say(msg, cap, DTSPH_E_ARG, "axis %d has too many cells", a);
        G.nc[a] = (int)k;
        G.s[a] = L / (double)k;
        G.inv_s[a] = 1.0 / G.s[a];
        G.s_f[a] = (float)G.s[a];
        G.L[a] = L;
        G.halfL[a] = 0.5 * L;
        G.ncell *= (int)k;
    }
    if ((long long)G.nc[0] * G.nc[1] * G.nc[2] > (1LL << 28)) return say(msg, cap, DTSPH_E_ARG, "too many cells");
    G.rc2 = rc * rc;
    // FP32 band around the cutoff: the FP32 separation from cell offsets is accurate
    // to a few 1e-7 h, so outside +-2e-5 relative the FP32 test decides
    G.rc2_lo = (float)(G.rc2 * (1.0 - 2e-5));
    G.rc2_hi = (float)(G.rc2 * (1.0 + 2e-5));
    return DTSPH_OK;
}

// Pair-term and update constants of one parameter set (rho_i = rho_j = rho0).
void dtsph::make_phys(const dtsph_params &p, Phys &P)
{
    memset(&P, 0, sizeof P);
    P.h = p.h;
    P.m = p.m;
    P.rho0 = p.rho0;
    P.c = p.beta * p.v_ref;
    P.nu = p.nu;
    P.nu_e = p.h * P.c / 16.0;
    P.dt = p.dt;
    P.dtau = p.dt / p.beta;
    P.dtau_f = (float)P.dtau;
    P.sig_h = quintic_sigma(p.dim, p.h) / p.h;
    P.eta_h2 = p.eta * p.h * p.h;
    P.edac_h2 = P.eta_h2;
    const double rho = p.rho0;
    P.c_div = p.m * (rho / rho) * P.c * P.c;
    P.c_edac = 4.0 * p.m / ((rho + rho) * rho) * P.nu_e;
    P.c_p = p.m / (rho * rho);
    P.c_visc = 4.0 * p.m * p.nu / (rho + rho);
    P.c_av = p.alpha * p.h * P.c / rho;
    for (int a = 0; a < 3; ++a) P.g[a] = a < p.dim ? p.g[a] : 0.0;
    P.kappa = 2.0 * p.dt / (2.0 * p.dt + 3.0 * P.dtau);
    P.c3 = 3.0 / (2.0 * p.dt);
    P.kc3 = P.kappa * P.c3;
    P.inv_h = 1.0 / p.h;
    P.inv_2dt = 1.0 / (2.0 * p.dt);
    P.edac = p.edac;
    P.use_av = p.alpha != 0.0;
    P.vol = p.m / p.rho0;
    P.steady = p.steady;
    P.free_surface = p.free_surface;
    P.moving = p.steady ? 0 : p.moving;
    P.disp2_max = p.moving == 2 ? 0.25 * p.skin * p.skin : 0.0;
    P.disp2_reuse = 0.25 * p.list_skin * p.list_skin;
    if (p.steady) {
        // Eq. (mom-steady): dV/dtau is the momentum rate itself (no BDF2 term);
        // the pressure rate has no EDAC term
        P.kappa = 1.0;
        P.kc3 = 0.0;
        P.edac = 0;
    }
}

// Range and consistency checks of one parameter set.
int dtsph::check_params(const dtsph_params *p, char *msg, size_t cap)
{
    if (p->dim != 2 && p->dim != 3) return say(msg, cap, DTSPH_E_ARG, "dim must be 2 or 3");
    if (p->precision != DTSPH_FP64 && p->precision != DTSPH_FP32C) return say(msg, cap, DTSPH_E_ARG, "bad precision");
    const double pos[] = {p->h, p->m, p->rho0, p->beta, p->v_ref, p->dt};
    const char *nm[] = {"h", "m", "rho0", "beta", "v_ref", "dt"};
    for (int i = 0; i < 6; ++i)
        if (!(pos[i] > 0) || !std::isfinite(pos[i])) return say(msg, cap, DTSPH_E_ARG, "%s must be positive and finite", nm[i]);
    if (!(p->nu >= 0) || !(p->eta > 0) || !(p->alpha >= 0) || !(p->eps >= 0) || !(p->stag_tol >= 0))
        return say(msg, cap, DTSPH_E_ARG, "nu, alpha, eps, stag_tol must be >= 0 and eta > 0");
    if (p->max_iter < 1 || p->max_iter > (1 << 24)) return say(msg, cap, DTSPH_E_ARG, "max_iter out of range");
    if (p->stag_window < 0 || p->stag_window > 16) return say(msg, cap, DTSPH_E_ARG, "stag_window must be in [0, 16]");
    if (p->fixed_iters < 0 || p->fixed_iters > (1 << 24)) return say(msg, cap, DTSPH_E_ARG, "fixed_iters out of range");
    if (p->edac_h2_literal) return say(msg, cap, DTSPH_E_UNSUPPORTED, "the literal r^2 + h^2 EDAC denominator is oracle-only");
    if (p->max_neighbors < 0 || p->max_neighbors > 4096) return say(msg, cap, DTSPH_E_ARG, "max_neighbors out of range");
    if (p->graph < 0 || p->graph > 2) return say(msg, cap, DTSPH_E_ARG, "graph must be 0, 1 or 2");
    if (p->lanes != 0 && p->lanes != 1 && p->lanes != 2 && p->lanes != 4 && p->lanes != 8)
        return say(msg, cap, DTSPH_E_ARG, "lanes must be 0, 1, 2, 4 or 8");
    if (p->stages != 0 && (p->stages < 2 || p->stages > kMaxStages))
        return say(msg, cap, DTSPH_E_ARG, "stages must be 0 or in [2, %d]", kMaxStages);
    if (p->shifting != 0 && p->shifting != 1) return say(msg, cap, DTSPH_E_ARG, "shifting must be 0 or 1");
    if (p->steady != 0 && p->steady != 1) return say(msg, cap, DTSPH_E_ARG, "steady must be 0 or 1");
    if (p->steady && p->shifting) return say(msg, cap, DTSPH_E_ARG, "the steady mode keeps the particles fixed: no shifting");
    if (p->free_surface != 0 && p->free_surface != 1) return say(msg, cap, DTSPH_E_ARG, "free_surface must be 0 or 1");
    if (p->moving < 0 || p->moving > 2) return say(msg, cap, DTSPH_E_ARG, "moving must be 0, 1 or 2");
    if (p->moving && p->steady) return say(msg, cap, DTSPH_E_ARG, "the steady mode keeps the particles fixed: moving must be 0");
    if (!(p->skin >= 0) || !std::isfinite(p->skin)) return say(msg, cap, DTSPH_E_ARG, "skin must be >= 0 and finite");
    if (!(p->cell_scale == 0.0 || (p->cell_scale >= 1.0 && p->cell_scale <= 4.0)))
        return say(msg, cap, DTSPH_E_ARG, "cell_scale must be 0 or in [1, 4]");
    if (p->moving == 2 && !(p->skin > 0)) return say(msg, cap, DTSPH_E_ARG, "moving = 2 needs a positive skin");
    if (p->form < 0 || p->form > 2) return say(msg, cap, DTSPH_E_ARG, "form must be 0, 1 or 2");
    if (p->form == 2 && p->moving)
        return say(msg, cap, DTSPH_E_UNSUPPORTED, "form 2 (no pair cache) needs particles fixed in pseudo-time");
    if (!(p->list_skin >= 0) || !std::isfinite(p->list_skin))
        return say(msg, cap, DTSPH_E_ARG, "list_skin must be >= 0 and finite");
    if (p->list_skin > 0 && (p->moving || p->steady || p->shifting || p->graph != 2))
        return say(msg, cap, DTSPH_E_UNSUPPORTED,
                   "list_skin needs graph = 2, particles fixed in pseudo-time, no shifting and no steady mode");
    return DTSPH_OK;
}

namespace {

int validate(dtsph_ctx *c, const dtsph_params *p)
{
    char msg[256];
    const int r = dtsph::check_params(p, msg, sizeof msg);
    return r ? fail(c, r, "%s", msg) : DTSPH_OK;
}

// Autotuner results: lanes per particle of the iterate kernel and, with one
// lane, its staging depth, keyed by (device, dim, precision, slots, instances,
// persistent loop or not), shared by every context of the process. With
// DTSPH_TUNE_CACHE set to a file name they also persist across processes: the
// file is read once per process, and every new choice is appended to it as one
// line "dtsph-tune-v1 <device> <dim> <precision> <slots> <instances> <loop>
// <lanes> <stages>" (the last line of a key wins).
struct TuneKey {
    std::string dev;   // device name and SM count, spaces replaced
    int dim, prec;
    int64_t n;
    int ninst, loop;
    bool operator<(const TuneKey &o) const
    {
        if (dev != o.dev) return dev < o.dev;
        if (dim != o.dim) return dim < o.dim;
        if (prec != o.prec) return prec < o.prec;
        if (n != o.n) return n < o.n;
        if (ninst != o.ninst) return ninst < o.ninst;
        return loop < o.loop;
    }
};
struct TuneChoice { int lanes, stages; };
std::map<TuneKey, TuneChoice> &tune_cache()
{
    static std::map<TuneKey, TuneChoice> m;
    return m;
}

constexpr int kDefaultStages = 3;
std::mutex tune_mu;
bool tune_file_read = false;

const char *tune_file() { return getenv("DTSPH_TUNE_CACHE"); }

// The costs the per-step choice of the pair-term form compares, per shape,
// lanes and staging depth: the break-even iteration count and the three times
// it comes from (cache pass; cached and uncached loop per pseudo-iteration, ms).
struct FormCosts { double kstar; float ms[3]; };
using FormKey = std::tuple<TuneKey, int, int>;
std::map<FormKey, FormCosts> &form_cache()
{
    static std::map<FormKey, FormCosts> m;
    return m;
}

// Reads the persisted choices once (tune_mu held): one record per line,
// "dtsph-tune-v1 <device> dim precision slots instances loop lanes stages" and
// "dtsph-form-v1 <device> dim precision slots instances loop lanes stages kstar
// cache_ms cached_ms uncached_ms"; other lines are skipped.
void load_tune_file()
{
    if (tune_file_read) return;
    tune_file_read = true;
    const char *path = tune_file();
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char tag[32], dev[160];
        TuneKey k;
        long long n = 0;
        TuneChoice ch;
        if (sscanf(line, "%31s %159s %d %d %lld %d %d %d %d", tag, dev, &k.dim, &k.prec, &n, &k.ninst, &k.loop,
                   &ch.lanes, &ch.stages) != 9)
            continue;
        const bool ok = (ch.lanes == 1 || ch.lanes == 2 || ch.lanes == 4 || ch.lanes == 8) && ch.stages >= 2 &&
                        ch.stages <= kMaxStages;
        if (!ok) continue;
        k.dev = dev;
        k.n = n;
        if (strcmp(tag, "dtsph-tune-v1") == 0) {
            tune_cache()[k] = ch;
        } else if (strcmp(tag, "dtsph-form-v1") == 0) {
            FormCosts fc;
            char t2[32], d2[160];
            int i0, i1, i2, i3, i4, i5;
            long long n2;
            if (sscanf(line, "%31s %159s %d %d %lld %d %d %d %d %lf %f %f %f", t2, d2, &i0, &i1, &n2, &i2, &i3, &i4,
                       &i5, &fc.kstar, &fc.ms[0], &fc.ms[1], &fc.ms[2]) == 13 &&
                std::isfinite(fc.kstar))
                form_cache()[FormKey{k, ch.lanes, ch.stages}] = fc;
        }
    }
    fclose(f);
}

// Appends one choice to the persisted file (tune_mu held).
void save_tune_choice(const TuneKey &k, const TuneChoice &ch)
{
    const char *path = tune_file();
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "dtsph-tune-v1 %s %d %d %lld %d %d %d %d\n", k.dev.c_str(), k.dim, k.prec, (long long)k.n, k.ninst,
            k.loop, ch.lanes, ch.stages);
    fclose(f);
}

// Appends the form costs of a shape to the persisted file (tune_mu held).
void save_form_costs(const TuneKey &k, int lanes, int stages, const FormCosts &fc)
{
    const char *path = tune_file();
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "dtsph-form-v1 %s %d %d %lld %d %d %d %d %.9g %.9g %.9g %.9g\n", k.dev.c_str(), k.dim, k.prec,
            (long long)k.n, k.ninst, k.loop, lanes, stages, fc.kstar, fc.ms[0], fc.ms[1], fc.ms[2]);
    fclose(f);
}

std::string device_tag(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    return name + "/" + std::to_string(prop.multiProcessorCount) + "sm";
}

TuneKey tune_key(const dtsph_ctx *c, int64_t n)
{
    return TuneKey{device_tag(c->device), c->prm[0].dim, c->prm[0].precision, n, c->ninst, c->prm[0].graph == 2};
}

// Lanes and stages for n slots: the parameters' when fixed, else the process
// cache's choice for the shape, else 4 lanes until the tuner runs.
TuneChoice kernel_choice(dtsph_ctx *c, int64_t n)
{
    const dtsph_params &p = c->prm[0];
    TuneChoice ch{p.lanes > 0 ? p.lanes : 4, p.stages > 0 ? p.stages : kDefaultStages};
    if (p.lanes == 0) {
        const TuneKey key = tune_key(c, n);
        std::lock_guard<std::mutex> g(tune_mu);
        load_tune_file();
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            ch = it->second;
            c->tuned = true;
        }
    }
    return ch;
}


}  // namespace

// Neighbour-list entries per particle: max_neighbors, else 1.35 times the mean
// count of a uniform fill of the list cutoff's disc (sphere) plus 8.
int dtsph::neighbour_capacity(const dtsph_params &p)
{
    if (p.max_neighbors > 0) return p.max_neighbors;
    const double vol = p.m / p.rho0;
    const double rc = 3.0 * p.h + (p.moving == 2 ? p.skin : 0.0) + p.list_skin;
    double expect = p.dim == 2 ? pi() * rc * rc / vol : 4.0 / 3.0 * pi() * rc * rc * rc / vol;
    int k = (int)std::ceil(1.35 * expect) + 8;
    return std::min(std::max(k, 8), 4096);
}

namespace {

// Device memory for nf[i] fluid particles per instance plus the walls set so far.
int allocate(dtsph_ctx *c, const int64_t *nf)
{
    free_all(c);
    c->kstar = -1.0;                  // the form costs belong to the particle set's shape
    // test hooks: a cap on the context's device memory (to exercise DTSPH_E_OOM)
    // and a shorter give-up time of the persistent loop's grid barrier (to
    // exercise DTSPH_E_TIMEOUT); both unset in normal use
    c->alloc_limit = (size_t)env_u64("DTSPH_TEST_ALLOC_LIMIT", 0);
    if (iterate_prepare() != 0) {
        cudaGetLastError();
        return fail(c, DTSPH_E_CUDA, "could not raise the shared-memory limit of the iterate kernels");
    }
    Buffers &B = c->B;
    const int ni = c->ninst;
    c->I.assign(ni, Inst{});
    int64_t slot = 0, fo = 0, wo = 0, co = 0, so = 0;
    int K = 0;
    for (int i = 0; i < ni; ++i) {
        if (nf[i] <= 0) return fail(c, DTSPH_E_ARG, "instance %d: nf must be positive", i);
        const int64_t nw = (int64_t)(c->xw_host[i].size() / c->prm[i].dim);
        Inst &I = c->I[i];
        slot = (slot + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
        I.slot_off = (int)slot;
        I.nf = (int)nf[i];
        I.nw = (int)nw;
        I.foff = (int)fo;
        I.woff = (int)wo;
        I.cell_off = (int)co;
        I.seg_off = (int)so;
        I.shift = (int)(slot - (fo + wo));
        slot += nf[i] + nw;
        fo += nf[i];
        wo += nw;
        co += c->G[i].ncell + 1;   // one empty sentinel cell per instance
        so += (int64_t)((c->G[i].nc[0] + kSeg2 - 1) / kSeg2) * c->G[i].nc[1] * c->G[i].nc[2];
        K = std::max(K, dtsph::neighbour_capacity(c->prm[i]));
        if (slot >= kMaxSlots - 4 * kSlotAlign || co >= (1LL << 31) - 2)
            return fail(c, DTSPH_E_ARG, "particle or cell count out of range (at most %lld slots in a context)",
                        kMaxSlots - 4 * kSlotAlign);
        c->P[i].rp_scale = c->P[i].dt / (c->P[i].rho0 * c->P[i].c * c->P[i].c) / (double)nf[i];
        c->P[i].rv_scale = c->P[i].dt / c->prm[i].v_ref / (double)nf[i];
    }
    const int n = (int)((slot + kSlotAlign - 1) / kSlotAlign * kSlotAlign);
    const int d = c->prm[0].dim;
    B.n = n;
    B.nf = (int)fo;
    B.nw = (int)wo;
    B.dim = d;
    B.fp32c = c->prm[0].precision == DTSPH_FP32C;
    B.K = K;
    B.ninst = ni;
    B.ncell = (int)co;
    B.nseg2 = (int)so;
    {
        // the pair cache's rows (sliced, K per slot) against half of L2
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess) {
            cudaGetLastError();
            l2 = 0;
        }
        const size_t row = B.fp32c ? (d == 2 ? 16 : 20) : (d == 2 ? 36 : 36);
        B.l2_stream = (size_t)n * (size_t)K * row > (size_t)l2 / 2 ? 1 : 0;
    }
    if (cudaDeviceGetAttribute(&B.nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        B.nsm = 1;
    }
    B.barrier_ns = env_u64("DTSPH_TEST_BARRIER_WAIT_NS", kBarrierWaitNs);
    {
        const TuneChoice ch = kernel_choice(c, n);
        B.lanes = ch.lanes;
        B.stages = ch.stages;
    }
    if (c->prm[0].moving && !c->prm[0].steady) {
        // the moving pass: the lanes asked for, else one lane per particle on
        // the FP32C path (measured fastest: more lanes add blocks beyond the
        // resident set and redundant per-lane state loads) and up to four on the
        // FP64 path (FP64-pipe-bound: more threads help while there are few)
        int L = c->prm[0].lanes;
        if (L == 0) {
            L = 1;
            if (!B.fp32c)
                while (L < 4 && (long long)n * L < 400000) L *= 2;
        }
        B.lanes = L;
    }
    const size_t nd = (size_t)n * d;
    const size_t nwarps = ((size_t)n + kWarp - 1) / kWarp;
    const size_t npair = nwarps * B.K * kWarp;
    Inst *d_inst;
    Geom *d_geo;
    Phys *d_phys;
    uint16_t *d_inst_of;
    int r;
#define A(p, cnt) { if ((r = dalloc(c, &(p), (cnt))) != DTSPH_OK) { free_all(c); return r; } }
    A(d_inst, ni) A(d_geo, ni) A(d_phys, ni) A(d_inst_of, n)
    A(B.gid_a, n) A(B.x_a, nd) A(B.xp_a, nd) A(B.vn_a, nd) A(B.vnm1_a, nd) A(B.pn_a, n) A(B.s_a, nd) A(B.cell_a, n)
    A(B.wslot_a, (size_t)wo)
    if (wo > 0) {
        // braces: A is an if statement, so a bare else would bind to it
        if (B.fp32c) {
            A(B.wv32, n)
        } else {
            A(B.wv64, n)
        }
    }
    A(B.gid_b, n) A(B.x_b, nd) A(B.vn_b, nd) A(B.vnm1_b, nd) A(B.pn_b, n) A(B.xp_b, nd) A(B.v0_b, nd)
    A(B.ph0_b, n) A(B.s_b, nd) A(B.cell_b, n)
    A(B.key, n) A(B.slot, n) A(B.unsorted, n) A(B.perm, n) A(B.cell_count, (size_t)B.ncell)
    A(B.cell_start, (size_t)B.ncell + 1) A(B.scan_tmp, (size_t)B.ncell / 4096 + 2)
    A(B.vk[0], nd) A(B.vk[1], nd)
    A(B.pcount, n) A(B.pj, npair) A(B.pjt, (size_t)n * list_stride(B.K))
    if (B.fp32c) {
        A(B.off, n) A(B.nb32[0], n) A(B.nb32[1], n) A(B.pc32, npair)
    } else {
        A(B.nb64[0], n) A(B.nb64[1], n) A(B.pc64, npair)
    }
    A(B.ap_b, n) A(B.f_b, nd)
    if (c->prm[0].moving && !c->prm[0].steady) {
        A(B.xk[0], nd) A(B.xk[1], nd) A(B.vt, nd)
        if (B.fp32c) {
            A(B.offk[0], n) A(B.offk[1], n)
        }
    }
    // two residual partials per tile (at most one tile per warp of slots),
    // double-buffered by the persistent loop
    A(B.blk, 4 * nwarps) A(B.ls, ni) A(B.ctrl, 1) A(B.stats, (size_t)kStatRing * ni) A(B.err, 1)
    // batches without walls (frozen particles) run the decoupled loop kernel,
    // unless DTSPH_LOCKSTEP_LOOP=1 asks for the lockstep one (comparisons)
    int *d_sched = nullptr;
    B.async_loop = ni > 1 && ni <= kDealMaxInst && wo == 0 && !(c->prm[0].moving && !c->prm[0].steady) &&
                   env_u64("DTSPH_LOCKSTEP_LOOP", 0) == 0;
    if (c->prm[0].form == 2 && wo > 0) {
        free_all(c);
        return fail(c, DTSPH_E_UNSUPPORTED, "form 2 (no pair cache) is for contexts without walls");
    }
    B.form_a = c->prm[0].form == 2;
    if (c->prm[0].list_skin > 0 && wo > 0) {
        free_all(c);
        return fail(c, DTSPH_E_UNSUPPORTED, "list_skin is for contexts without walls");
    }
    B.reuse_lists = c->prm[0].list_skin > 0;
    B.relist_run = -1;
    if (B.reuse_lists) {
        A(B.relist, 1) A(B.slot_of, (size_t)std::max(B.nf, 1))
    }
    if (B.async_loop) {
        A(B.il, ni) A(d_sched, ni)
    }
    A(c->form_sel, 1) A(c->form_count, 3)
#undef A
    if (wo > 0 && !(B.fp32c ? (const void *)B.wv32 : (const void *)B.wv64)) {
        free_all(c);
        return fail(c, DTSPH_E_STATE, "internal: the wall velocity array was not allocated");
    }
    B.inst = d_inst;
    B.geo = d_geo;
    B.phys = d_phys;
    B.inst_of = d_inst_of;
    std::vector<uint16_t> inst_of(n);
    for (int i = 0; i < ni; ++i) {
        const int lo = c->I[i].slot_off;
        const int hi = i + 1 < ni ? c->I[i + 1].slot_off : n;
        for (int s = lo; s < hi; ++s) inst_of[s] = (uint16_t)i;
    }
    std::vector<LoopState> ls(ni);
    for (int i = 0; i < ni; ++i) {
        LoopState &L = ls[i];
        memset(&L, 0, sizeof L);
        L.reason = -1;
        L.max_iter = c->prm[i].max_iter;
        L.fixed_iters = c->prm[i].fixed_iters;
        L.stag_window = c->prm[i].stag_window;
        L.eps = c->prm[i].eps;
        L.stag_tol = c->prm[i].stag_tol;
    }
    CK(cudaMemcpy(d_inst, c->I.data(), sizeof(Inst) * ni, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_geo, c->G.data(), sizeof(Geom) * ni, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_phys, c->P.data(), sizeof(Phys) * ni, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_inst_of, inst_of.data(), sizeof(uint16_t) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(B.ls, ls.data(), sizeof(LoopState) * ni, cudaMemcpyHostToDevice));
    if (B.async_loop) {
        // search order of the decoupled loop: the instances with the fewest
        // tiles first (they take the most iterations)
        std::vector<int> order(ni);
        for (int i = 0; i < ni; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return c->I[a].nf + c->I[a].nw < c->I[b].nf + c->I[b].nw;
        });
        CK(cudaMemcpy(d_sched, order.data(), sizeof(int) * ni, cudaMemcpyHostToDevice));
        CK(cudaMemset(B.il, 0, sizeof(InstLoop) * ni));
        B.sched = d_sched;
    }
    CK(cudaMemset(B.ctrl, 0, sizeof(LoopCtrl)));
    if (B.wv32) CK(cudaMemset(B.wv32, 0, sizeof(float4) * n));
    if (B.wv64) CK(cudaMemset(B.wv64, 0, sizeof(double4_32a) * n));
    CK(cudaMemset(B.cell_count, 0, sizeof(int) * B.ncell));
    CK(cudaMemset(B.err, 0, sizeof(uint32_t)));
    CK(cudaMemset(B.pcount, 0, sizeof(int) * n));
    // padding slots of the permutations are never written: -1 marks them
    CK(cudaMemset(B.unsorted, 0xff, sizeof(int) * n));
    CK(cudaMemset(B.perm, 0xff, sizeof(int) * n));
    CK(cudaDeviceSynchronize());
    c->nf_set.assign(nf, nf + ni);
    return DTSPH_OK;
}

// ---------------------------------------------------------------- step sequence

// Everything of a real step before the pseudo-time loop. Returns kernels launched.
int enqueue_pre_loop(dtsph_ctx *c, cudaStream_t st)
{
    const Buffers &B = c->B;
    int k = 0;
    if (B.reuse_lists) {
        // the lists at r^0 of the previous step (to 3h + list_skin) hold every
        // pair within 3h at r^n unless a particle ended the step farther than
        // list_skin / 2 from its r^0 (*relist): then this step bins and lists at
        // r^n as without reuse; either way the state-n pass runs on the lists
        Buffers Br = B;
        Br.relist_run = 1;
        k += launch_binning(Br, Br.x_a, Br.gid_a, st);
        k += launch_permute_a_to_b(Br, st);
        launch_nlist(Br, Br.x_b, Br.cell_b, Br.gid_b, st, false);
        Br.relist_run = 0;
        k += 1 + launch_same_order_a_to_b(Br, st);
        k += launch_state_n(B, true, st, false);
    } else {
        k += launch_binning(B, B.x_a, B.gid_a, st);      // cells at r^n
        k += launch_permute_a_to_b(B, st);
        k += launch_state_n(B, true, st);                 // walls, rates, predictor
    }
    k += launch_binning(B, B.xp_b, B.gid_b, st);         // cells at r^0
    k += launch_permute_b_to_a(B, st);
    if (B.xk[0]) {
        k += launch_move_prepare(B, st);                          // particles moving in pseudo-time
    } else if (B.form_sel) {
        // both forms in the graph: the reset kernel picks the step's form; the
        // pair-cache pass returns at once when the step recomputes the terms
        launch_nlist(B, B.xp_a, B.cell_a, B.gid_a, st, false);
        k += 1 + launch_loop_reset(B, st);
        k += launch_pair_cache_pass(B, B.xp_a, B.gid_a, st);
    } else if (B.form_a) {
        launch_nlist(B, B.xp_a, B.cell_a, B.gid_a, st, false);   // the loop recomputes the pair terms
        k += 1 + launch_loop_reset(B, st);
    } else {
        k += launch_pair_cache(B, B.xp_a, B.cell_a, B.gid_a, st);   // also resets the loop state
    }
    return k;
}

int enqueue_iteration(dtsph_ctx *c, cudaStream_t st, unsigned long long cond, int use_cond)
{
    if (c->B.xk[0]) return launch_move_iteration(c->B, cond, use_cond, st);
    int k = launch_walls_iter(c->B, st);
    k += launch_iterate(c->B, cond, use_cond, st);
    return k;
}

// After the loop: the position update and buffer rotation, then shifting if on.
int enqueue_post_loop(dtsph_ctx *c, cudaStream_t st)
{
    int k = launch_outer(c->B, st);
    if (c->prm[0].shifting) k += launch_shift(c->B, st);
    return k;
}

// The event-record nodes around the loop in a captured step graph.
int find_event_nodes(dtsph_ctx *c, cudaGraph_t g, cudaGraphNode_t *na, cudaGraphNode_t *nb)
{
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    *na = *nb = nullptr;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        if (ev == c->ev_a[0]) *na = nd;
        if (ev == c->ev_b[0]) *nb = nd;
    }
    if (!*na || !*nb) return fail(c, DTSPH_E_CUDA, "loop event nodes not found in the step graph");
    return DTSPH_OK;
}

// Graph of one real step with the persistent loop: pre-loop kernels -> one
// cooperative loop kernel -> outer. With the per-step choice of the pair-term
// form (form_sel) the graph holds the loop kernel of each form; the one of the
// form the step does not run returns at once.
int build_graph_persistent(dtsph_ctx *c, cudaGraph_t *g_out, cudaGraphExec_t *x_out, cudaGraphNode_t *na,
                           cudaGraphNode_t *nb)
{
    int grid = 0, grid_a = 0;
    if (loop_grid(c->B, &grid)) return fail(c, DTSPH_E_CUDA, "occupancy query for the loop kernel failed");
    const bool both = c->B.form_sel != nullptr;
    if (both) {
        Buffers Ba = c->B;
        Ba.form_a = 1;
        if (loop_grid(Ba, &grid_a)) return fail(c, DTSPH_E_CUDA, "occupancy query for the loop kernel failed");
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    *g_out = g;
    CK(cudaStreamBeginCaptureToGraph(c->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->per_step_fixed = enqueue_pre_loop(c, c->cap);
    cudaError_t e0 = cudaEventRecordWithFlags(c->ev_a[0], c->cap, cudaEventRecordExternal);
    cudaError_t e = launch_loop(c->B, grid, c->cap);
    if (both && e == cudaSuccess) {
        // without the cache (form_run 1), pausing after floor(kstar) iterations;
        // then, if it paused, the cache pass and the cached loop from there
        // (form_run 2)
        Buffers Ba = c->B;
        Ba.form_a = 1;
        Ba.form_run = 1;
        e = launch_loop(Ba, grid_a, c->cap);
        Ba.form_a = 0;
        c->per_step_fixed += 1 + launch_loop_resume(Ba, c->cap);
        Buffers Bc = c->B;
        Bc.form_run = 2;
        c->per_step_fixed += launch_pair_cache_pass(Bc, Bc.xp_a, Bc.gid_a, c->cap);
        if (e == cudaSuccess) e = launch_loop(Bc, grid, c->cap);
        c->per_step_fixed += 1;
    }
    cudaError_t e1 = cudaEventRecordWithFlags(c->ev_b[0], c->cap, cudaEventRecordExternal);
    c->per_step_fixed += 1 + enqueue_post_loop(c, c->cap);
    cudaGraph_t g2 = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g2);
    if (e != cudaSuccess) return fail(c, DTSPH_E_CUDA, "cooperative loop launch under capture: %s", cudaGetErrorString(e));
    CK(e0);
    CK(e1);
    CK(e2);
    c->per_iter = 0;
    int r = find_event_nodes(c, g, na, nb);
    if (r) return r;
    CK(cudaGraphInstantiate(x_out, g, 0));
    return DTSPH_OK;
}

// The per-step choice of the pair-term form applies: form = 0, the persistent
// loop (one instance, or the decoupled batch loop), no walls, particles frozen
// in pseudo-time.
bool auto_form(const dtsph_ctx *c)
{
    return c->prm[0].form == 0 && c->prm[0].graph == 2 && c->B.nw == 0 && !c->B.xk[0] &&
           (c->ninst == 1 || c->B.async_loop);
}

// Graph of one real step: pre-loop kernels -> while node (walls, iterate) -> outer.
int build_graph(dtsph_ctx *c)
{
    // the persistent loop kernel runs the frozen pass only; moving runs take the
    // while node
    if (c->prm[0].graph == 2 && !c->B.xk[0]) {
        // the kernels take Buffers by value: the words of the per-step form
        // choice are set in the graph's copies only
        c->form_graph = auto_form(c) && c->kstar >= 0.0;
        if (c->form_graph) {
            c->B.form_sel = c->form_sel;
            c->B.form_count = c->form_count;
            c->B.kstar = c->kstar;
        }
        const int r = build_graph_persistent(c, &c->graph, &c->exec, &c->node_a, &c->node_b);
        c->B.form_sel = nullptr;
        c->B.form_count = nullptr;
        if (r) c->form_graph = false;
        return r;
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    c->graph = g;
    CK(cudaStreamBeginCaptureToGraph(c->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->per_step_fixed = enqueue_pre_loop(c, c->cap);
    CK(cudaEventRecordWithFlags(c->ev_a[0], c->cap, cudaEventRecordExternal));
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(c->cap, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t wnode;
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    CK(cudaGraphAddNode(&wnode, g, dv.data(), nullptr, dv.size(), &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(c->cap, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaEventRecordWithFlags(c->ev_b[0], c->cap, cudaEventRecordExternal));
    c->per_step_fixed += enqueue_post_loop(c, c->cap);
    cudaGraph_t g2 = nullptr;
    CK(cudaStreamEndCapture(c->cap, &g2));
    CK(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c->per_iter = enqueue_iteration(c, c->cap, (unsigned long long)h, 1);
    cudaGraph_t b2 = nullptr;
    CK(cudaStreamEndCapture(c->cap, &b2));
    int r = find_event_nodes(c, g, &c->node_a, &c->node_b);
    if (r) return r;
    CK(cudaGraphInstantiate(&c->exec, g, 0));
    return DTSPH_OK;
}

// Plain launches: the loop runs in chunks of kernels that return at once when
// every instance has stopped; the host checks the device counter between chunks.
int step_plain(dtsph_ctx *c)
{
    const int k = (int)(c->steps % dtsph_ctx::kLoopEv);
    {
        Range r("dtsph pre-loop: binning, lists, state-n pass, pair cache");
        c->per_step_fixed = enqueue_pre_loop(c, c->stream);
    }
    c->launches += c->per_step_fixed;
    CK(cudaEventRecord(c->ev_a[k], c->stream));
    Range loop_range("dtsph pseudo-time loop");
    int cap = 1;
    for (const auto &p : c->prm) cap = std::max(cap, p.fixed_iters > 0 ? p.fixed_iters : p.max_iter);
    int issued = 0;
    LoopCtrl ctrl;
    while (true) {
        const int chunk = 8;
        for (int i = 0; i < chunk; ++i) {
            c->per_iter = enqueue_iteration(c, c->stream, 0ull, 0);
            c->launches += c->per_iter;
        }
        issued += chunk;
        CK(cudaMemcpyAsync(&ctrl, c->B.ctrl, sizeof ctrl, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (ctrl.active == 0) break;
        if (issued > cap + 16) return fail(c, DTSPH_E_STATE, "pseudo-time loop did not stop");
    }
    CK(cudaEventRecord(c->ev_b[k], c->stream));
    Range outer_range("dtsph outer step");
    c->launches += enqueue_post_loop(c, c->stream);
    CK(cudaGetLastError());
    return DTSPH_OK;
}

int device_error(dtsph_ctx *c)
{
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, c->B.err, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e & kErrNonFinite) return fail(c, DTSPH_E_ARG, "a particle position is not finite");
    if (e & kErrCapacity)
        return fail(c, DTSPH_E_CAPACITY, "a particle had more than %d neighbours (raise max_neighbors)", c->B.K);
    if (e & kErrDomain) return fail(c, DTSPH_E_DOMAIN, "a particle left the box of a non-periodic axis");
    if (e & kErrBarrier) return fail(c, DTSPH_E_TIMEOUT, "a grid barrier of the persistent loop timed out");
    if (e & kErrCopy) return fail(c, DTSPH_E_TIMEOUT, "a bulk copy of pair-cache rows did not complete");
    if (e & kErrSkin)
        return fail(c, DTSPH_E_SKIN, "a particle moved farther than skin / 2 from r^0 in pseudo-time (raise skin)");
    return DTSPH_OK;
}

// Mean duration of `launches` launches of the iterate kernel on the pair cache
// that B describes (each after a loop reset, bracketed by events).
int probe_ms(dtsph_ctx *c, const Buffers &B, int launches, float *out)
{
    std::vector<cudaEvent_t> ev(2 * launches);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    for (int i = 0; i < launches; ++i) {
        launch_loop_reset(B, c->stream);
        CK(cudaEventRecord(ev[2 * i], c->stream));
        // particles moving in pseudo-time: the whole pass (walls, then fluid)
        c->launches += B.xk[0] ? launch_move_iteration(B, 0ull, 0, c->stream) : launch_iterate(B, 0ull, 0, c->stream);
        CK(cudaEventRecord(ev[2 * i + 1], c->stream));
    }
    c->launches += launches;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    double tot = 0;
    for (int i = 0; i < launches; ++i) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        tot += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    *out = (float)(tot / launches);
    return DTSPH_OK;
}

// Mean device time per pseudo-iteration of the persistent loop kernel over
// `iters` iterations of every instance (fixed_iters forced on the loop state for
// the probe, then restored), `reps` launches after one untimed launch.
int probe_loop_ms(dtsph_ctx *c, int iters, int reps, float *out)
{
    const Buffers &B = c->B;
    int grid = 0;
    if (loop_grid(B, &grid)) return fail(c, DTSPH_E_CUDA, "occupancy query for the loop kernel failed");
    std::vector<LoopState> saved(c->ninst), probe;
    CK(cudaMemcpy(saved.data(), B.ls, sizeof(LoopState) * c->ninst, cudaMemcpyDeviceToHost));
    probe = saved;
    for (auto &l : probe) l.fixed_iters = iters;
    CK(cudaMemcpy(B.ls, probe.data(), sizeof(LoopState) * c->ninst, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float tot = 0;
    for (int i = 0; i <= reps; ++i) {
        launch_loop_reset(B, c->stream);
        CK(cudaEventRecord(e0, c->stream));
        CK(launch_loop(B, grid, c->stream));
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (i > 0) tot += ms;
    }
    c->launches += 2 * (reps + 1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemcpy(B.ls, saved.data(), sizeof(LoopState) * c->ninst, cudaMemcpyHostToDevice));
    *out = tot / (float)(reps * iters);
    return DTSPH_OK;
}

// Times the candidates of the iterate kernel (one lane per particle at
// staging depths 2, 3, 4 and 6 unless stages is fixed, then 2, 4 and 8 lanes)
// on a pair cache built at the initial positions and keeps the fastest: per
// iteration of the persistent loop kernel when the step runs it (graph = 2),
// else per launch of the per-iteration kernel. Runs
// once per shape in a process, before the first step, so that every step of
// every context of that shape uses the same kernel (and so the same summation
// order; the staging depth does not change the arithmetic). The loop buffers
// hold no state yet; they are zeroed for the timing runs.
int autotune(dtsph_ctx *c)
{
    Range range("dtsph autotune");
    const Buffers &B = c->B;
    const size_t nd = (size_t)B.n * B.dim;
    CK(cudaMemsetAsync(B.vk[0], 0, nd * sizeof(double), c->stream));
    CK(cudaMemsetAsync(B.s_a, 0, nd * sizeof(double), c->stream));
    if (B.fp32c) CK(cudaMemsetAsync(B.nb32[0], 0, (size_t)B.n * sizeof(float4), c->stream));
    else CK(cudaMemsetAsync(B.nb64[0], 0, (size_t)B.n * sizeof(double4_32a), c->stream));
    c->launches += launch_binning(B, B.x_a, B.gid_a, c->stream);
    c->launches += launch_permute_a_to_b(B, c->stream);
    c->launches += launch_pair_cache(B, B.x_b, B.cell_b, B.gid_b, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    std::vector<TuneChoice> cand;
    if (c->prm[0].stages > 0) cand.push_back({1, c->prm[0].stages});
    else
        for (int S : {2, 3, 4, 6}) cand.push_back({1, S});
    for (int L : {2, 4, 8}) cand.push_back({L, kDefaultStages});
    TuneChoice best{c->B.lanes, c->B.stages};
    float best_ms = 1e30f;
    c->tune_log.clear();
    for (const TuneChoice &ch : cand) {
        c->B.lanes = ch.lanes;
        c->B.stages = ch.stages;
        float ms = 0;
        int r;
        if (c->prm[0].graph == 2) {
            r = probe_loop_ms(c, 4, 5, &ms);
        } else {
            probe_ms(c, c->B, 3, &ms);         // warm-up
            r = probe_ms(c, c->B, 10, &ms);
        }
        if (r) return r;
        c->tune_log.push_back({ch.lanes, ch.lanes == 1 ? ch.stages : 0, ms});
        if (ms < best_ms) {
            best_ms = ms;
            best = ch;
        }
    }
    c->B.lanes = best.lanes;
    c->B.stages = best.stages;
    c->tuned = true;
    {
        const TuneKey key = tune_key(c, c->B.n);
        std::lock_guard<std::mutex> g(tune_mu);
        tune_cache()[key] = best;
        save_tune_choice(key, best);
    }
    return device_error(c);
}

// The per-step choice of the pair-term form (form = 0): on lists and a pair
// cache built at the current positions (binned as a step would; the next step
// rebuilds every array used here), times the pair-cache pass, which the
// uncached form leaves out (both build the lists), and one pseudo-iteration of
// the persistent loop in each form at the context's lanes and staging depth. A
// step of k iterations costs cache + k * cached against k * uncached, so the
// uncached form pays up to kstar = cache / (uncached - cached) iterations.
// Cached per shape in the process and in the persisted file.
int measure_form_costs(dtsph_ctx *c)
{
    Range range("dtsph form costs");
    Buffers &B = c->B;
    const TuneKey key = tune_key(c, B.n);
    {
        std::lock_guard<std::mutex> g(tune_mu);
        load_tune_file();
        auto it = form_cache().find(FormKey{key, B.lanes, B.stages});
        if (it != form_cache().end()) {
            c->kstar = it->second.kstar;
            for (int i = 0; i < 3; ++i) c->form_ms[i] = it->second.ms[i];
            return DTSPH_OK;
        }
    }
    const size_t nd = (size_t)B.n * B.dim;
    CK(cudaMemsetAsync(B.vk[0], 0, nd * sizeof(double), c->stream));
    CK(cudaMemsetAsync(B.s_a, 0, nd * sizeof(double), c->stream));
    if (B.fp32c) CK(cudaMemsetAsync(B.nb32[0], 0, (size_t)B.n * sizeof(float4), c->stream));
    else CK(cudaMemsetAsync(B.nb64[0], 0, (size_t)B.n * sizeof(double4_32a), c->stream));
    c->launches += launch_binning(B, B.x_a, B.gid_a, c->stream);
    c->launches += launch_permute_a_to_b(B, c->stream);
    constexpr int kReps = 5;
    cudaEvent_t e[2];
    for (auto &ev : e) CK(cudaEventCreate(&ev));
    float t_cache = 0;
    for (int rep = 0; rep <= kReps; ++rep) {          // the first is a warm-up
        launch_nlist(B, B.x_b, B.cell_b, B.gid_b, c->stream, false);
        CK(cudaEventRecord(e[0], c->stream));
        launch_pair_cache_pass(B, B.x_b, B.gid_b, c->stream);   // leaves lists and cache for the loops below
        CK(cudaEventRecord(e[1], c->stream));
        c->launches += 2;
        CK(cudaEventSynchronize(e[1]));
        float a = 0;
        CK(cudaEventElapsedTime(&a, e[0], e[1]));
        if (rep > 0) t_cache += a;
    }
    for (auto &ev : e) cudaEventDestroy(ev);
    const float ms_cache = t_cache / kReps;
    float ms_b = 0, ms_a = 0;
    B.form_a = 0;
    int r = probe_loop_ms(c, 4, 5, &ms_b);
    if (!r) {
        B.form_a = 1;
        r = probe_loop_ms(c, 4, 5, &ms_a);
        B.form_a = 0;
    }
    if (r) return r;
    FormCosts fc;
    fc.ms[0] = ms_cache;
    fc.ms[1] = ms_b;
    fc.ms[2] = ms_a;
    fc.kstar = ms_a > ms_b ? (double)ms_cache / (double)(ms_a - ms_b) : 1e9;
    c->kstar = fc.kstar;
    for (int i = 0; i < 3; ++i) c->form_ms[i] = fc.ms[i];
    {
        std::lock_guard<std::mutex> g(tune_mu);
        form_cache()[FormKey{key, B.lanes, B.stages}] = fc;
        save_form_costs(key, B.lanes, B.stages, fc);
    }
    return device_error(c);
}

int set_particles_impl(dtsph_ctx *c, const int64_t *nf, const double *x, const double *v, const double *p,
                       const double *vprev, bool device)
{
    Range range("dtsph_set_particles");
    if (!x || !v || !p || !nf) return fail(c, DTSPH_E_ARG, "x, v and p are required");
    CK(cudaSetDevice(c->device));
    int r;
    const int d = c->prm[0].dim;
    const int ni = c->ninst;
    int64_t NF = 0, NW = 0;
    for (int i = 0; i < ni; ++i) {
        if (nf[i] <= 0) return fail(c, DTSPH_E_ARG, "instance %d: nf must be positive", i);
        NF += nf[i];
        NW += (int64_t)(c->xw_host[i].size() / d);
    }
    const bool reuse = c->have_particles && c->nf_set.size() == (size_t)ni &&
                       std::equal(c->nf_set.begin(), c->nf_set.end(), nf) && c->B.nw == NW;
    if (!reuse) {
        if ((r = allocate(c, nf))) return r;
        // staging buffers for the AoS inputs, kept for later calls of the same size
        if ((r = dalloc(c, &c->sx, (size_t)NF * d)) || (r = dalloc(c, &c->sv, (size_t)NF * d)) ||
            (r = dalloc(c, &c->sp, NF)) || (r = dalloc(c, &c->svp, (size_t)NF * d)) ||
            (r = dalloc(c, &c->sxw, (size_t)std::max<int64_t>(NW, 1) * d)) ||
            (r = dalloc(c, &c->svw, (size_t)std::max<int64_t>(NW, 1) * d)) ||
            (r = dalloc(c, &c->rd, (size_t)NF * (3 * d + 1))))
            return r;
        if (NW > 0) {
            std::vector<double> xw, vw;
            for (int i = 0; i < ni; ++i) {
                xw.insert(xw.end(), c->xw_host[i].begin(), c->xw_host[i].end());
                vw.insert(vw.end(), c->vw_host[i].begin(), c->vw_host[i].end());
            }
            CK(cudaMemcpy(c->sxw, xw.data(), xw.size() * sizeof(double), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->svw, vw.data(), vw.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
    }
    const size_t bx = (size_t)NF * d * sizeof(double), bp = (size_t)NF * sizeof(double);
    double *svp = vprev ? c->svp : nullptr;
    // a new state restarts the step log and clears device-side error flags
    // (before the scatter, which flags a non-finite position)
    c->launches += launch_restart_steps(c->B, c->stream);
    CK(cudaMemsetAsync(c->B.err, 0, sizeof(uint32_t), c->stream));
    double *sxw = NW > 0 ? c->sxw : nullptr, *svw = NW > 0 ? c->svw : nullptr;
    // with reused lists and the same particles: the new state goes into the
    // slots of order A as they are and the lists stay; a particle beyond the
    // skin makes the next step bin and list at r^n (on the device)
    const bool same = reuse && c->B.reuse_lists && c->lists_ready;
    auto scatter = [&](const double *xs, const double *vs, const double *ps, const double *vps) {
        return same ? launch_scatter_same(c->B, xs, vs, ps, vps, c->stream)
                    : launch_scatter_in(c->B, xs, vs, ps, vps, sxw, svw, c->stream);
    };
    if (!device && c->host_direct) {
        // the scatter kernel reads the caller's arrays where they are
        c->launches += scatter(x, v, p, vprev);
    } else {
        const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(c->sx, x, bx, kind, c->stream));
        CK(cudaMemcpyAsync(c->sv, v, bx, kind, c->stream));
        CK(cudaMemcpyAsync(c->sp, p, bp, kind, c->stream));
        if (vprev) CK(cudaMemcpyAsync(svp, vprev, bx, kind, c->stream));
        c->launches += scatter(c->sx, c->sv, c->sp, svp);
    }
    CK(cudaGetLastError());
    if (!device) {
        CK(cudaStreamSynchronize(c->stream));   // host arrays may be reused once we return
        uint32_t e = 0;
        CK(cudaMemcpy(&e, c->B.err, sizeof e, cudaMemcpyDeviceToHost));
        if (e & kErrNonFinite) return fail(c, DTSPH_E_ARG, "a particle position is not finite");
    }
    c->have_particles = true;
    c->lists_ready = same;
    c->steps = 0;
    c->steps_cache = c->steps_nocache = 0;
    CK(cudaMemsetAsync(c->form_count, 0, 3 * sizeof(unsigned long long), c->stream));
    CK(cudaMemsetAsync(c->form_sel, 0, sizeof(int), c->stream));
    // the iteration counts of the latest finished step stay: a new state of the
    // same shape most often continues the same flow
    if (!c->tuned && c->prm[0].lanes == 0 && !c->B.xk[0]) {
        r = autotune(c);
        if (r) return r;
    }
    if (auto_form(c) && c->kstar < 0) {
        r = measure_form_costs(c);
        if (r) return r;
    }
    if (c->prm[0].graph && !c->exec) {
        r = build_graph(c);
        if (r) return r;
    }
    return DTSPH_OK;
}

int read_field_impl(dtsph_ctx *c, int32_t field, double *out, bool device)
{
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "no particles set");
    if (!out) return fail(c, DTSPH_E_ARG, "out is null");
    const Buffers &B = c->B;
    const double *src;
    int comps = B.dim;
    switch (field) {
    case DTSPH_FIELD_POS: src = B.x_a; break;
    case DTSPH_FIELD_VEL: src = B.vn_a; break;
    case DTSPH_FIELD_VEL_PREV: src = B.vnm1_a; break;
    case DTSPH_FIELD_P: src = B.pn_a; comps = 1; break;
    default: return fail(c, DTSPH_E_ARG, "unknown field %d", field);
    }
    const size_t bytes = (size_t)B.nf * comps * sizeof(double);
    double *dst = out;
    double *tmp = nullptr;
    if (!device) {
        CK(cudaMallocAsync((void **)&tmp, bytes, c->stream));
        dst = tmp;
    }
    c->launches += launch_unpermute(B, B.gid_a, src, dst, comps, c->stream);
    CK(cudaGetLastError());
    if (!device) {
        if (c->host_direct) c->launches += launch_copy(tmp, out, bytes / sizeof(double), c->stream);
        else CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaFreeAsync(tmp, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return DTSPH_OK;
}

// The fluid state in caller order into host arrays (any may be null): every
// field is unpermuted into the context's scratch, then copied out, with one
// wait for the stream at the end.
int read_state_impl(dtsph_ctx *c, double *x, double *v, double *p, double *vprev)
{
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "no particles set");
    const Buffers &B = c->B;
    const size_t nd = (size_t)B.nf * B.dim;
    struct Field { double *out; const double *src; int comps; size_t off; };
    const Field f[4] = {{x, B.x_a, B.dim, 0}, {v, B.vn_a, B.dim, nd}, {p, B.pn_a, 1, 2 * nd},
                        {vprev, B.vnm1_a, B.dim, 2 * nd + (size_t)B.nf}};
    for (const Field &q : f)
        if (q.out) c->launches += launch_unpermute(B, B.gid_a, q.src, c->rd + q.off, q.comps, c->stream);
    for (const Field &q : f) {
        if (!q.out) continue;
        const size_t cnt = (size_t)B.nf * q.comps;
        if (c->host_direct) c->launches += launch_copy(c->rd + q.off, q.out, cnt, c->stream);
        else CK(cudaMemcpyAsync(q.out, c->rd + q.off, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return DTSPH_OK;
}

int create_impl(int32_t ninst, const dtsph_params *params, void *stream, dtsph_ctx **out)
{
    if (!params || !out || ninst < 1 || ninst > 65535) return DTSPH_E_ARG;
    *out = nullptr;
    dtsph_ctx *c = new (std::nothrow) dtsph_ctx();
    if (!c) return DTSPH_E_OOM;
    c->ninst = ninst;
    c->prm.assign(params, params + ninst);
    c->G.resize(ninst);
    c->P.resize(ninst);
    c->xw_host.resize(ninst);
    c->vw_host.resize(ninst);
    for (int i = 0; i < ninst; ++i) {
        int r = validate(c, &params[i]);
        if (!r && (params[i].dim != params[0].dim || params[i].precision != params[0].precision ||
                   params[i].graph != params[0].graph || params[i].lanes != params[0].lanes ||
                   params[i].stages != params[0].stages || params[i].shifting != params[0].shifting ||
                   params[i].form != params[0].form ||
                   params[i].steady != params[0].steady || params[i].free_surface != params[0].free_surface ||
                   params[i].moving != params[0].moving || params[i].skin != params[0].skin ||
                   params[i].cell_scale != params[0].cell_scale ||
                   (params[i].list_skin > 0) != (params[0].list_skin > 0)))
            r = fail(c, DTSPH_E_ARG,
                     "instances must share dim, precision, graph, lanes, stages, shifting, form, steady, "
                     "free_surface, moving, skin and cell_scale, and list_skin > 0 or not");
        if (!r) r = setup_geometry(c, params[i], c->G[i]);
        if (r) {
            delete c;
            return r;
        }
        dtsph::make_phys(params[i], c->P[i]);
    }
    memset(&c->B, 0, sizeof c->B);
    c->stream = (cudaStream_t)stream;
    int pageable = 0;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return DTSPH_E_CUDA;
    }
    c->host_direct = pageable == 1;
    c->ev_a.assign(dtsph_ctx::kLoopEv, nullptr);
    c->ev_b.assign(dtsph_ctx::kLoopEv, nullptr);
    for (int k = 0; k < dtsph_ctx::kLoopEv; ++k) {
        if (cudaEventCreate(&c->ev_a[k]) != cudaSuccess || cudaEventCreate(&c->ev_b[k]) != cudaSuccess) {
            cudaGetLastError();
            dtsph_destroy(c);
            return DTSPH_E_CUDA;
        }
    }
    *out = c;
    return DTSPH_OK;
}

int set_boundary_impl(dtsph_ctx *c, int32_t inst, int64_t nw, const double *x, const double *v_wall)
{
    if (inst < 0 || inst >= c->ninst) return fail(c, DTSPH_E_ARG, "instance %d out of range", inst);
    if (nw < 0 || (nw > 0 && !x)) return fail(c, DTSPH_E_ARG, "bad wall arrays");
    const int d = c->prm[inst].dim;
    c->xw_host[inst].assign(x, x + (size_t)nw * d);
    if (v_wall) c->vw_host[inst].assign(v_wall, v_wall + (size_t)nw * d);
    else c->vw_host[inst].assign((size_t)nw * d, 0.0);
    free_all(c);   // walls change the particle set: particles must be set again
    return DTSPH_OK;
}

int read_stats_impl(dtsph_ctx *c, int32_t inst, int64_t first, int32_t count, dtsph_step_stats *out)
{
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "no particles set");
    if (inst < 0 || inst >= c->ninst) return fail(c, DTSPH_E_ARG, "instance %d out of range", inst);
    if (count < 0 || (count > 0 && !out) || first < 0 || first + count > c->steps)
        return fail(c, DTSPH_E_ARG, "steps [%lld, %lld) not taken (taken: %lld)", (long long)first,
                    (long long)(first + count), (long long)c->steps);
    if (c->steps - first > kStatRing) return fail(c, DTSPH_E_ARG, "step %lld no longer in the log", (long long)first);
    // the instance's records of the range, strided by the instance count in the
    // ring, in at most two strided copies (the ring wraps at most once), one wait
    std::vector<StatRec> recs((size_t)count);
    for (int32_t i = 0; i < count;) {
        const int64_t slot = (first + i) % kStatRing;
        const int32_t run = (int32_t)std::min<int64_t>(count - i, kStatRing - slot);
        CK(cudaMemcpy2DAsync(recs.data() + i, sizeof(StatRec), c->B.stats + (size_t)slot * c->ninst + inst,
                             sizeof(StatRec) * (size_t)c->ninst, sizeof(StatRec), (size_t)run, cudaMemcpyDeviceToHost,
                             c->stream));
        i += run;
    }
    if (count > 0) CK(cudaStreamSynchronize(c->stream));
    for (int32_t i = 0; i < count; ++i) {
        const StatRec &r = recs[(size_t)i];
        out[i].iters = r.iters;
        out[i].reason = r.reason;
        out[i].rp = r.rp;
        out[i].rv = r.rv;
        out[i].vmax = r.vmax;
        out[i].form = r.form;
        out[i].pad = 0;
    }
    return DTSPH_OK;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char *dtsph_version(void) { return DTSPH_VERSION; }

const char *dtsph_last_error(const dtsph_ctx *c) { return c ? c->err.c_str() : kNoCtx; }

int dtsph_create(const dtsph_params *params, void *stream, dtsph_ctx **out)
{
    return create_impl(1, params, stream, out);
}

int dtsph_batch_create(int32_t ninst, const dtsph_params *params, void *stream, dtsph_ctx **out)
{
    return create_impl(ninst, params, stream, out);
}

void dtsph_destroy(dtsph_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaEvent_t e : c->ev_a)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_b)
        if (e) cudaEventDestroy(e);
    delete c;
}

int dtsph_set_boundary(dtsph_ctx *c, int64_t nw, const double *x, const double *v_wall)
{
    if (!c) return DTSPH_E_ARG;
    return set_boundary_impl(c, 0, nw, x, v_wall);
}

int dtsph_batch_set_boundary(dtsph_ctx *c, int32_t inst, int64_t nw, const double *x, const double *v_wall)
{
    if (!c) return DTSPH_E_ARG;
    return set_boundary_impl(c, inst, nw, x, v_wall);
}

int dtsph_set_particles(dtsph_ctx *c, int64_t nf, const double *x, const double *v, const double *p,
                        const double *v_prev)
{
    if (!c) return DTSPH_E_ARG;
    if (c->ninst != 1) return fail(c, DTSPH_E_ARG, "a batch context takes dtsph_batch_set_particles");
    return set_particles_impl(c, &nf, x, v, p, v_prev, false);
}

int dtsph_set_particles_device(dtsph_ctx *c, int64_t nf, const double *x, const double *v, const double *p,
                               const double *v_prev)
{
    if (!c) return DTSPH_E_ARG;
    if (c->ninst != 1) return fail(c, DTSPH_E_ARG, "a batch context takes dtsph_batch_set_particles");
    return set_particles_impl(c, &nf, x, v, p, v_prev, true);
}

int dtsph_batch_set_particles(dtsph_ctx *c, const int64_t *nf, const double *x, const double *v, const double *p,
                              const double *v_prev)
{
    if (!c) return DTSPH_E_ARG;
    return set_particles_impl(c, nf, x, v, p, v_prev, false);
}

int dtsph_step(dtsph_ctx *c, int32_t nsteps)
{
    if (!c) return DTSPH_E_ARG;
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "dtsph_step before dtsph_set_particles");
    if (nsteps < 0) return fail(c, DTSPH_E_ARG, "nsteps must be >= 0");
    CK(cudaSetDevice(c->device));
    if (c->B.reuse_lists && !c->lists_ready && nsteps > 0) {
        // bin at r^n, make that order A, list to 3h + list_skin: what the
        // steps' state-n pass reads
        const Buffers &B = c->B;
        c->launches += launch_binning(B, B.x_a, B.gid_a, c->stream);
        c->launches += launch_permute_a_to_b(B, c->stream);
        c->launches += launch_adopt_b(B, c->stream);
        launch_nlist(B, B.x_a, B.cell_a, B.gid_a, c->stream, false);
        c->launches += 1;
        CK(cudaMemsetAsync(B.relist, 0, sizeof(int), c->stream));
        CK(cudaGetLastError());
        c->lists_ready = true;
    }
    Range range(c->exec ? "dtsph_step (step graphs)" : "dtsph_step");
    c->have_nbrs = false;
    for (int32_t s = 0; s < nsteps; ++s) {
        if (c->exec) {
            const int k = (int)(c->steps % dtsph_ctx::kLoopEv);
            // (the graph of the per-step form choice counts its steps on the device)
            if (!c->form_graph) ++(c->B.form_a ? c->steps_nocache : c->steps_cache);
            CK(cudaGraphExecEventRecordNodeSetEvent(c->exec, c->node_a, c->ev_a[k]));
            CK(cudaGraphExecEventRecordNodeSetEvent(c->exec, c->node_b, c->ev_b[k]));
            CK(cudaGraphLaunch(c->exec, c->stream));
        } else {
            int r = step_plain(c);
            if (r) return r;
            ++(c->B.form_a ? c->steps_nocache : c->steps_cache);
        }
        ++c->steps;
    }
    return DTSPH_OK;
}

int dtsph_sync(dtsph_ctx *c)
{
    if (!c) return DTSPH_E_ARG;
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "no particles set");
    CK(cudaStreamSynchronize(c->stream));
    return device_error(c);
}

int64_t dtsph_step_count(const dtsph_ctx *c) { return c ? c->steps : -1; }

int dtsph_loop_times(dtsph_ctx *c, int64_t first, int32_t count, float *ms)
{
    if (!c) return DTSPH_E_ARG;
    if (count < 0 || (count > 0 && !ms)) return fail(c, DTSPH_E_ARG, "bad output");
    if (first < 0 || first + count > c->steps || first < c->steps - dtsph_ctx::kLoopEv)
        return fail(c, DTSPH_E_ARG, "steps [%lld, %lld) are not among the last %d taken", (long long)first,
                    (long long)(first + count), dtsph_ctx::kLoopEv);
    CK(cudaSetDevice(c->device));
    for (int32_t i = 0; i < count; ++i) {
        const int k = (int)((first + i) % dtsph_ctx::kLoopEv);
        CK(cudaEventSynchronize(c->ev_b[k]));
        CK(cudaEventElapsedTime(&ms[i], c->ev_a[k], c->ev_b[k]));
    }
    return DTSPH_OK;
}

int dtsph_read_stats(dtsph_ctx *c, int64_t first, int32_t count, dtsph_step_stats *out)
{
    if (!c) return DTSPH_E_ARG;
    return read_stats_impl(c, 0, first, count, out);
}

int dtsph_batch_read_stats(dtsph_ctx *c, int32_t inst, int64_t first, int32_t count, dtsph_step_stats *out)
{
    if (!c) return DTSPH_E_ARG;
    return read_stats_impl(c, inst, first, count, out);
}

int dtsph_read_field(dtsph_ctx *c, int32_t field, double *out)
{
    if (!c) return DTSPH_E_ARG;
    CK(cudaSetDevice(c->device));
    return read_field_impl(c, field, out, false);
}

int dtsph_read_state(dtsph_ctx *c, double *x, double *v, double *p, double *v_prev)
{
    if (!c) return DTSPH_E_ARG;
    CK(cudaSetDevice(c->device));
    return read_state_impl(c, x, v, p, v_prev);
}

int dtsph_read_field_device(dtsph_ctx *c, int32_t field, double *out)
{
    if (!c) return DTSPH_E_ARG;
    CK(cudaSetDevice(c->device));
    return read_field_impl(c, field, out, true);
}

int dtsph_eval_rates(dtsph_ctx *c, double *ap, double *F)
{
    if (!c) return DTSPH_E_ARG;
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "no particles set");
    if (!ap || !F) return fail(c, DTSPH_E_ARG, "ap and F are required");
    CK(cudaSetDevice(c->device));
    const Buffers &B = c->B;
    c->lists_ready = false;                       // the lists are rebuilt at r^n in order B
    c->launches += launch_binning(B, B.x_a, B.gid_a, c->stream);
    c->launches += launch_permute_a_to_b(B, c->stream);
    c->launches += launch_state_n(B, false, c->stream);
    const size_t bf = (size_t)B.nf * B.dim * sizeof(double), bp = (size_t)B.nf * sizeof(double);
    double *tmp = nullptr;
    CK(cudaMallocAsync((void **)&tmp, bf + bp, c->stream));
    c->launches += launch_unpermute(B, B.gid_b, B.ap_b, tmp, 1, c->stream);
    c->launches += launch_unpermute(B, B.gid_b, B.f_b, tmp + B.nf, B.dim, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ap, tmp, bp, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(F, tmp + B.nf, bf, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaFreeAsync(tmp, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->have_nbrs = false;
    return device_error(c);
}

int dtsph_build_neighbors(dtsph_ctx *c)
{
    if (!c) return DTSPH_E_ARG;
    if (!c->have_particles) return fail(c, DTSPH_E_STATE, "no particles set");
    CK(cudaSetDevice(c->device));
    const Buffers &B = c->B;
    c->lists_ready = false;                       // the lists are rebuilt at r^n in order B
    c->launches += launch_binning(B, B.x_a, B.gid_a, c->stream);
    c->launches += launch_permute_a_to_b(B, c->stream);
    c->launches += launch_pair_cache(B, B.x_b, B.cell_b, B.gid_b, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    int r = device_error(c);
    c->have_nbrs = r == DTSPH_OK;
    return r;
}

int dtsph_get_neighbors(dtsph_ctx *c, int64_t i, int64_t *out, int64_t cap, int64_t *count)
{
    if (!c) return DTSPH_E_ARG;
    if (!c->have_nbrs) return fail(c, DTSPH_E_STATE, "call dtsph_build_neighbors first");
    const Buffers &B = c->B;
    if (i < 0 || i >= (int64_t)B.nf + B.nw || !count || (cap > 0 && !out))
        return fail(c, DTSPH_E_ARG, "bad index or output");
    std::vector<uint32_t> gid(B.n);
    CK(cudaMemcpy(gid.data(), B.gid_b, sizeof(uint32_t) * B.n, cudaMemcpyDeviceToHost));
    int s = -1;
    for (int q = 0; q < B.n; ++q)
        if (gid[q] == (uint32_t)i) { s = q; break; }
    if (s < 0) return fail(c, DTSPH_E_STATE, "particle %lld not found", (long long)i);
    int cnt = 0;
    CK(cudaMemcpy(&cnt, B.pcount + s, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<int64_t> got;
    std::vector<uint32_t> lst((size_t)std::max(cnt, 0));
    if (cnt > 0)
        CK(cudaMemcpy(lst.data(), B.pjt + (size_t)s * list_stride(B.K), sizeof(uint32_t) * cnt,
                      cudaMemcpyDeviceToHost));
    for (int k = 0; k < cnt; ++k) got.push_back((int64_t)gid[lst[k] & kSlotMask]);
    std::sort(got.begin(), got.end());
    *count = (int64_t)got.size();
    for (int64_t k = 0; k < cap && k < (int64_t)got.size(); ++k) out[k] = got[k];
    return DTSPH_OK;
}

int dtsph_probe_iterate(dtsph_ctx *c, int32_t launches, float *ms_per_launch, double *bytes_per_launch,
                        int64_t *pairs)
{
    if (!c) return DTSPH_E_ARG;
    if (!c->have_particles || c->steps == 0) return fail(c, DTSPH_E_STATE, "take a step before probing");
    if (launches < 1 || launches > 256 || !ms_per_launch) return fail(c, DTSPH_E_ARG, "launches must be in [1, 256]");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    // The shifting pass after the loop bins the particles again at r^{n+1} and
    // builds its neighbour lists over the index part of the step's pair cache.
    // With shifting on, the probe therefore builds a cache of its own for the
    // current positions, in that binned order (fluid flags and wall velocities
    // of the same order), from arrays that every step rebuilds before use.
    Buffers B = c->B;
    if (c->prm[0].shifting) {
        if (B.xk[0])
            return fail(c, DTSPH_E_STATE, "with particles moving in pseudo-time the probe needs a run without shifting");
        c->launches += launch_binning(B, B.x_a, B.gid_a, c->stream);
        c->launches += launch_permute_a_to_b(B, c->stream);
        c->launches += launch_pair_cache(B, B.x_b, B.cell_b, B.gid_b, c->stream);
        CK(cudaGetLastError());
        if (int r = device_error(c)) return r;
        B.gid_a = B.gid_b;
        B.vn_a = B.vn_b;
    }
    std::vector<int> cnt(B.n);
    std::vector<uint32_t> gid(B.n);
    CK(cudaMemcpy(cnt.data(), B.pcount, sizeof(int) * B.n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(gid.data(), B.gid_a, sizeof(uint32_t) * B.n, cudaMemcpyDeviceToHost));
    int64_t np = 0, npw = 0;
    for (int s = 0; s < B.n; ++s) {
        if (gid[s] < (uint32_t)B.nf) np += cnt[s];
        else if (gid[s] != kNoParticle) npw += cnt[s];
    }
    const int d = B.dim;
    const double packed = B.fp32c ? 16.0 : 32.0;
    double bytes;
    if (!B.xk[0]) {
        // per fluid particle: packed (V, p-hat) read and written, V^k (FP64) read
        // and written, BDF2 source read, neighbour count read; per pair: the cache entry
        const double per_particle = 2 * packed + 2 * 8.0 * d + 8.0 * d + 4.0;
        const double per_pair = B.fp32c ? (d == 2 ? 16.0 : 20.0) : 36.0;
        bytes = per_particle * B.nf + per_pair * (double)np;
    } else {
        // moving pass, per fluid particle: packed (V, p-hat), V^k, V~ and r^{k+1/2}
        // (FP64) read and written, BDF2 source read, slot id and neighbour count
        // read; FP32C: its FP32 offset read and written and its cell read; with
        // the skin: r^0 read. Per wall slot: slot id, count, prescribed velocity and
        // own position read, packed values written. Per list entry (fluid and wall
        // slots): neighbour index and cell shift.
        const double pos = B.fp32c ? 16.0 : 8.0 * d;
        double per_particle = 2 * packed + 3 * 2 * 8.0 * d + 8.0 * d + 8.0;
        if (B.fp32c) per_particle += 2 * 16.0 + 4.0;
        if (c->P[0].moving == 2) per_particle += 8.0 * d;
        const double per_wall = 8.0 + 8.0 * d + pos + packed;
        bytes = per_particle * B.nf + per_wall * B.nw + 5.0 * (double)(np + npw);
    }
    int r = probe_ms(c, B, launches, ms_per_launch);
    if (r) return r;
    if (bytes_per_launch) *bytes_per_launch = bytes;
    if (pairs) *pairs = np;
    return DTSPH_OK;
}

int dtsph_form_stats(const dtsph_ctx *c, double *kstar, float *ms, int64_t *steps_cache, int64_t *steps_nocache,
                     int64_t *steps_switched)
{
    if (!c) return DTSPH_E_ARG;
    if (kstar) *kstar = c->kstar;
    if (ms)
        for (int i = 0; i < 3; ++i) ms[i] = c->form_ms[i];
    int64_t a = c->steps_cache, b = c->steps_nocache, sw = 0;
    if (c->form_graph) {
        // the step graph counts its choices on the device
        unsigned long long n[3] = {0ull, 0ull, 0ull};
        if (cudaSetDevice(c->device) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess ||
            cudaMemcpy(n, c->form_count, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return DTSPH_E_CUDA;
        }
        a = (int64_t)n[0];
        b = (int64_t)n[1];
        sw = (int64_t)n[2];
    }
    if (steps_cache) *steps_cache = a;
    if (steps_nocache) *steps_nocache = b;
    if (steps_switched) *steps_switched = sw;
    return DTSPH_OK;
}

int dtsph_tuning(const dtsph_ctx *c, int32_t *lanes, float *ms_by_lanes)
{
    if (!c || !lanes) return DTSPH_E_ARG;
    *lanes = c->B.lanes;
    if (ms_by_lanes) {
        for (int i = 0; i < 4; ++i) ms_by_lanes[i] = -1.f;
        for (auto &e : c->tune_log) {
            int i = e.lanes == 1 ? 0 : e.lanes == 2 ? 1 : e.lanes == 4 ? 2 : 3;
            if (ms_by_lanes[i] < 0.f || e.ms < ms_by_lanes[i]) ms_by_lanes[i] = e.ms;
        }
    }
    return DTSPH_OK;
}

int dtsph_tuning_candidates(const dtsph_ctx *c, int32_t cap, int32_t *lanes, int32_t *stages, float *ms,
                            int32_t *count, int32_t *stages_in_use)
{
    if (!c || !count || cap < 0 || (cap > 0 && (!lanes || !stages || !ms))) return DTSPH_E_ARG;
    const int n = (int)c->tune_log.size();
    for (int i = 0; i < n && i < cap; ++i) {
        lanes[i] = c->tune_log[i].lanes;
        stages[i] = c->tune_log[i].stages;
        ms[i] = c->tune_log[i].ms;
    }
    *count = n;
    if (stages_in_use) *stages_in_use = c->B.lanes == 1 ? c->B.stages : 0;
    return DTSPH_OK;
}

int64_t dtsph_kernel_launches(const dtsph_ctx *c_)
{
    dtsph_ctx *c = const_cast<dtsph_ctx *>(c_);
    if (!c) return -1;
    if (!c->exec || c->steps == 0) return c->launches;
    // graph steps: fixed kernels per step plus, with the while node, the
    // per-iteration kernels of the longest instance of each step
    int64_t it = 0;
    if (c->per_iter > 0) {
        const int64_t first = std::max<int64_t>(0, c->steps - kStatRing);
        std::vector<StatRec> tmp((size_t)kStatRing * c->ninst);
        if (cudaMemcpyAsync(tmp.data(), c->B.stats, sizeof(StatRec) * tmp.size(), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return -1;
        for (int64_t s = first; s < c->steps; ++s) {
            int m = 0;
            for (int i = 0; i < c->ninst; ++i) m = std::max(m, tmp[(size_t)(s % kStatRing) * c->ninst + i].iters);
            it += m;
        }
    }
    return c->launches + c->steps * c->per_step_fixed + it * c->per_iter;
}

}  // extern "C"
