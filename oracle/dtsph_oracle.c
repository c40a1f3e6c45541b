/*
 * FP64 CPU oracle for the frozen-particle dual-time EDAC-SPH scheme (DTSPH,
 * Ramachandran, Muta & Ramakrishna, arXiv:1904.00861).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the CUDA library computes. Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant generator with the CUDA library, and the library
 * never calls it.
 *
 * Everything is IEEE double, compiled with -ffp-contract=off (no FMA), every
 * neighbour sum runs in ascending original particle index, and every loop over
 * particles is a gather, so results do not depend on the OpenMP thread count.
 *
 * What each function follows:
 *   orc_w / orc_dwdr     quintic spline of Morris et al. (cited in Sec. 3.1 for
 *                        the viscous term); the paper names the kernel only
 *                        (Sec. 4.1) and sets h = dx.
 *   orc_neighbors        N(i) of Sec. 3: all j != i with |r_ij| < 3h (the
 *                        quintic support), minimum image on periodic axes.
 *   orc_rates            frozen EDAC pressure rate, Eq. (dp-dtau-frozen-edac),
 *                        and frozen momentum rate, Eq. (mom-sph-frozen), with
 *                        Monaghan's artificial viscosity, Eqs. (mom-av, av-phiij),
 *                        and the Adami et al. wall treatment cited in Sec. 3.2.
 *   orc_step             Algorithm 2 (particles fixed in pseudo-time), one real
 *                        step: predictor Eqs. (v0, r0); pseudo iterations with
 *                        Eqs. (pkstar_frozen, vkp1_frozen, pkp1_frozen) and the
 *                        BDF2 pseudo-acceleration of Eq. (dv_dtau_exact), frozen
 *                        form of Sec. 2.2; convergence test Eq. (conv) with the
 *                        stagnation and iteration-cap rules of Sec. 3.4; position
 *                        update Eq. (r-update); optional shifting Eqs. (shift,
 *                        shift-deltar, shift-correct) of Sec. 3.5 (free-surface
 *                        particles not shifted in free-surface runs, where the
 *                        wall pressure is also kept >= 0, Sec. 3.2). Steady mode
 *                        (Sec. 2.3 "Steady state solutions", Eq. mom-steady):
 *                        particles fixed, no BDF2 term, no EDAC term, convection
 *                        term added, the pseudo-time loop as above.
 *                        Moving mode (Algorithm 1, Sec. 2.1 and 3.1 "Moving
 *                        particles in pseudo-time"): the pressure rate of
 *                        Eq. (dp-dtau) and the momentum rate of Eq.
 *                        (discrete_ME) with the pseudo-velocity V~; positions
 *                        staged by Eqs. (rkstar, rkp1), V~ by Eq. (vtilde);
 *                        neighbours either kept from r^0 or rebuilt at every
 *                        pass (the two advected variants of Sec. 4.1's table).
 *
 * Readings taken where the paper is silent or garbled (all listed in the design
 * notes): the EDAC diffusion denominator is r^2 + eta h^2 (edac_h2_literal = 1
 * gives the printed r^2 + h^2); one pair pass per pseudo iteration, whose first
 * pressure half step uses the rate of the previous pass (the state-n pass for
 * k = 0); Jacobi update; R_p = mean|dp/dtau| dt/(rho0 c^2), R_v = mean|dt dV/dtau|
 * / V_ref over fluid particles; stagnation = peak-to-peak/max below stag_tol for
 * both residuals over the last stag_window iterations; do-while loop capped at
 * max_iter iterations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* Parameters of one simulation. The oracle keeps its own copy of this layout;
 * the Python wrapper in this folder fills it. */
typedef struct {
    int32_t dim;              /* 2 or 3 */
    int32_t periodic[3];      /* 1 = periodic axis */
    double lo[3], hi[3];      /* domain box; periodic axes wrap to [lo, hi) */
    double h;                 /* smoothing length */
    double m;                 /* particle mass (uniform) */
    double rho0;              /* density, held fixed (Sec. 3) */
    double beta;              /* c = beta * v_ref (Sec. 3.4) */
    double v_ref;             /* reference speed */
    double nu;                /* kinematic viscosity */
    double dt;                /* real time step */
    double eta;               /* 0.01 (Sec. 3.1) */
    double alpha;             /* artificial viscosity coefficient */
    double g[3];              /* body force */
    double eps;               /* convergence tolerance, Eq. (conv) */
    double stag_tol;          /* 0.05 (Sec. 3.4) */
    int32_t stag_window;      /* 4 */
    int32_t max_iter;         /* 1000 (Sec. 3.4) */
    int32_t edac;             /* 1: pressure diffusion term on */
    int32_t edac_h2_literal;  /* 1: EDAC denominator r^2 + h^2 as printed */
    int32_t fixed_iters;      /* > 0: exactly this many iterations, no stop rules */
    int32_t use_bruteforce;   /* 1: O(N^2) neighbour search instead of cells */
    int32_t shifting;         /* 1: particle shifting after the real step */
    int32_t steady;           /* 1: steady-state mode (Sec. 2.3, Eq. mom-steady) */
    int32_t free_surface;     /* 1: free-surface run: wall pressure kept >= 0 (Sec. 3.2),
                                 free-surface particles not shifted (Sec. 3.5) */
    int32_t moving;           /* 0: particles fixed in pseudo-time (Algorithm 2); 1: moved
                                 in pseudo-time (Algorithm 1) over the neighbour lists of
                                 r^0; 2: moved, neighbours rebuilt at every pass */
} orc_params;

typedef struct {
    int32_t iters;
    int32_t reason;           /* 0 converged, 1 stagnated, 2 max_iter, 3 non-finite, 4 fixed */
    double rp, rv;            /* residuals of the last iteration */
} orc_stats;

/* ------------------------------------------------------------------ kernel */

static double sigma_of(int dim, double h)
{
    /* Normalisation of the quintic spline W = sigma * [(3-q)^5 - 6(2-q)^5 +
     * 15(1-q)^5], q = r/h, support 3h: integral of W over R^d equals 1. */
    if (dim == 2) return 7.0 / (478.0 * ORC_PI * h * h);
    if (dim == 3) return 1.0 / (120.0 * ORC_PI * h * h * h);
    return 1.0 / (120.0 * h);
}

static double pow5(double a) { return a * a * a * a * a; }
static double pow4(double a) { return a * a * a * a; }

double orc_w(double r, double h, int dim)
{
    double q = r / h;
    double s = 0.0;
    if (q < 3.0) s += pow5(3.0 - q);
    if (q < 2.0) s -= 6.0 * pow5(2.0 - q);
    if (q < 1.0) s += 15.0 * pow5(1.0 - q);
    return sigma_of(dim, h) * s;
}

/* dW/dr */
double orc_dwdr(double r, double h, int dim)
{
    double q = r / h;
    double s = 0.0;
    if (q < 3.0) s += -5.0 * pow4(3.0 - q);
    if (q < 2.0) s -= -30.0 * pow4(2.0 - q);
    if (q < 1.0) s += -75.0 * pow4(1.0 - q);
    return sigma_of(dim, h) * s / h;
}

/* --------------------------------------------------------------- geometry */

/* r_ij = r_i - r_j with the minimum image on periodic axes. */
static void separation(const orc_params *P, const double *ri, const double *rj, double *d)
{
    for (int a = 0; a < P->dim; ++a) {
        double dx = ri[a] - rj[a];
        if (P->periodic[a]) {
            double L = P->hi[a] - P->lo[a];
            double halfL = 0.5 * L;
            if (dx > halfL) dx = dx - L;
            else if (dx < -halfL) dx = dx + L;
        }
        d[a] = dx;
    }
}

static double norm2(const double *d, int dim)
{
    double r2 = d[0] * d[0] + d[1] * d[1];
    if (dim == 3) r2 = r2 + d[2] * d[2];
    return r2;
}

static void wrap(const orc_params *P, double *r)
{
    for (int a = 0; a < P->dim; ++a) {
        if (!P->periodic[a]) continue;
        double L = P->hi[a] - P->lo[a];
        if (r[a] >= P->hi[a]) r[a] = r[a] - L;
        else if (r[a] < P->lo[a]) r[a] = r[a] + L;
    }
}

/* Input positions: every coordinate must be finite; on a periodic axis a
 * coordinate outside [lo, hi) is brought into it, x - floor((x - lo) / L) L, then
 * once more by one L if rounding left it on the edge. The other axes are left as
 * given. x holds n particles. Returns 0, or -1 if a coordinate is not finite. */
int orc_prepare_positions(const orc_params *P, int64_t n, double *x)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < P->dim; ++a) {
            double *xa = x + i * P->dim + a;
            if (!isfinite(*xa)) return -1;
            if (!P->periodic[a] || (*xa >= P->lo[a] && *xa < P->hi[a])) continue;
            double L = P->hi[a] - P->lo[a];
            double q = floor((*xa - P->lo[a]) / L);
            *xa = *xa - q * L;
            if (*xa >= P->hi[a]) *xa = *xa - L;
            else if (*xa < P->lo[a]) *xa = *xa + L;
        }
    }
    return 0;
}

/* ------------------------------------------------------------- neighbours */

/* CSR neighbour lists: for particle i, idx[start[i] .. start[i+1]) holds every
 * j != i with r_ij^2 < (3h)^2, ascending. */
typedef struct {
    int64_t n;
    int64_t *start;
    int64_t *idx;
} nlist;

static void nlist_free(nlist *L)
{
    free(L->start);
    free(L->idx);
    L->start = L->idx = NULL;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int in_range(const orc_params *P, const double *x, int64_t i, int64_t j, double rc2)
{
    double d[3];
    separation(P, x + i * P->dim, x + j * P->dim, d);
    return norm2(d, P->dim) < rc2;
}

/* Brute force: the definition, O(N^2). Returns 0, or -1 on allocation failure. */
static int build_brute(const orc_params *P, int64_t n, const double *x, nlist *L)
{
    double rc = 3.0 * P->h;
    double rc2 = rc * rc;
    int64_t *cnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (j != i && in_range(P, x, i, j, rc2)) ++c;
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    L->n = n;
    L->start = cnt;
    L->idx = malloc((size_t)(cnt[n] > 0 ? cnt[n] : 1) * sizeof(int64_t));
    if (!L->idx) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cnt[i];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && in_range(P, x, i, j, rc2)) L->idx[c++] = j;
    }
    return 0;
}

/* Cell list: cells of side >= 3h, candidates from the 3^d surrounding cells,
 * the same distance test as the brute force, each list sorted ascending. */
static int build_cells(const orc_params *P, int64_t n, const double *x, nlist *L)
{
    int dim = P->dim;
    double rc = 3.0 * P->h;
    double rc2 = rc * rc;
    int64_t nc[3] = {1, 1, 1};
    double s[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        double len = P->hi[a] - P->lo[a];
        int64_t k = (int64_t)floor(len / rc);
        if (k < 1) k = 1;
        while (k > 1 && len / (double)k < rc) --k;
        /* a periodic axis with fewer than 3 cells would visit a cell twice */
        if (P->periodic[a] && k < 3) return build_brute(P, n, x, L);
        nc[a] = k;
        s[a] = len / (double)k;
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t *cell = malloc((size_t)n * sizeof(int64_t));
    int64_t *head = malloc((size_t)ncell * sizeof(int64_t));
    int64_t *next = malloc((size_t)n * sizeof(int64_t));
    if (!cell || !head || !next) { free(cell); free(head); free(next); return -1; }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t ci[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            int64_t k = (int64_t)floor((x[i * dim + a] - P->lo[a]) / s[a]);
            if (k < 0) k = 0;
            if (k >= nc[a]) k = nc[a] - 1;
            ci[a] = k;
        }
        int64_t c = (ci[2] * nc[1] + ci[1]) * nc[0] + ci[0];
        cell[i] = c;
        next[i] = head[c];
        head[c] = i;
    }
    int64_t *cnt = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t cap = 0;
    if (!cnt) { free(cell); free(head); free(next); return -1; }
    /* first pass counts, second pass fills */
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = cell[i];
            int64_t ci[3] = {c % nc[0], (c / nc[0]) % nc[1], c / (nc[0] * nc[1])};
            int64_t w = pass ? cnt[i] : 0;
            int dz0 = dim == 3 ? -1 : 0, dz1 = dim == 3 ? 1 : 0;
            for (int dz = dz0; dz <= dz1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int64_t cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                        int skip = 0;
                        for (int a = 0; a < 3; ++a) {
                            if (cc[a] < 0 || cc[a] >= nc[a]) {
                                if (a < dim && P->periodic[a]) cc[a] = (cc[a] + nc[a]) % nc[a];
                                else skip = 1;
                            }
                        }
                        if (skip) continue;
                        int64_t cn = (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
                        for (int64_t j = head[cn]; j >= 0; j = next[j]) {
                            if (j == i || !in_range(P, x, i, j, rc2)) continue;
                            if (pass) L->idx[w] = j;
                            ++w;
                        }
                    }
            if (!pass) cnt[i + 1] = w;
            else qsort(L->idx + cnt[i], (size_t)(w - cnt[i]), sizeof(int64_t), cmp_i64);
        }
        if (!pass) {
            for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
            cap = cnt[n] > 0 ? cnt[n] : 1;
            L->idx = malloc((size_t)cap * sizeof(int64_t));
            if (!L->idx) { free(cell); free(head); free(next); free(cnt); return -1; }
        }
    }
    L->n = n;
    L->start = cnt;
    free(cell);
    free(head);
    free(next);
    return 0;
}

static int build_neighbors(const orc_params *P, int64_t n, const double *x, nlist *L)
{
    memset(L, 0, sizeof(*L));
    return P->use_bruteforce ? build_brute(P, n, x, L) : build_cells(P, n, x, L);
}

/* Exported for the tests: neighbour lists of all n particles. start has n+1
 * entries; idx receives up to cap entries. Returns the total count (which may
 * exceed cap, in which case idx is truncated), or -1 on failure. */
int64_t orc_neighbors(const orc_params *P, int64_t n, const double *x,
                      int64_t *start, int64_t *idx, int64_t cap)
{
    nlist L;
    if (build_neighbors(P, n, x, &L)) return -1;
    int64_t tot = L.start[n];
    memcpy(start, L.start, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(idx, L.idx, (size_t)(tot < cap ? tot : cap) * sizeof(int64_t));
    nlist_free(&L);
    return tot;
}

/* ------------------------------------------------------------------ walls */

/* Adami et al. (2012), cited in Sec. 3.2 (static walls): for each wall particle
 * w, with fluid neighbours f,
 *   p_w      = (sum_f p_f W_wf + g . sum_f rho_f r_wf W_wf) / sum_f W_wf
 *   vtilde_w = sum_f V_f W_wf / sum_f W_wf,  ghost velocity 2 v_w - vtilde_w,
 * and p_w = 0, vtilde_w = 0 when no fluid particle is in range. */
static void wall_values(const orc_params *P, int64_t nf, int64_t nw, const double *x,
                        const double *v, const double *p, const double *vw, const nlist *L,
                        double *pw, double *vghost)
{
    int dim = P->dim;
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < nw; ++w) {
        int64_t iw = nf + w;
        double sw = 0.0, sp = 0.0, sg = 0.0, sv[3] = {0, 0, 0};
        for (int64_t e = L->start[iw]; e < L->start[iw + 1]; ++e) {
            int64_t f = L->idx[e];
            if (f >= nf) continue;
            double d[3];
            separation(P, x + iw * dim, x + f * dim, d);
            double r = sqrt(norm2(d, dim));
            double W = orc_w(r, P->h, dim);
            sw = sw + W;
            sp = sp + p[f] * W;
            double gr = 0.0;
            for (int a = 0; a < dim; ++a) gr = gr + P->g[a] * d[a];
            sg = sg + P->rho0 * gr * W;
            for (int a = 0; a < dim; ++a) sv[a] = sv[a] + v[f * dim + a] * W;
        }
        if (sw > 0.0) {
            pw[w] = (sp + sg) / sw;
            /* free-surface runs keep the wall pressure positive (Sec. 3.2) */
            if (P->free_surface && pw[w] < 0.0) pw[w] = 0.0;
            for (int a = 0; a < dim; ++a) vghost[w * dim + a] = 2.0 * vw[w * dim + a] - sv[a] / sw;
        } else {
            pw[w] = 0.0;
            for (int a = 0; a < dim; ++a) vghost[w * dim + a] = 2.0 * vw[w * dim + a];
        }
    }
}

/* ------------------------------------------------------------------ rates */

/* For every fluid particle i, with rho_i = rho_j = rho0:
 *  dp_i/dtau = sum_j m_j (rho_i/rho_j) c^2 V_ij . gradW_ij
 *            + sum_j 4 m_j / ((rho_i + rho_j) rho_j) nu_e p_ij (r_ij . gradW_ij) / (r_ij^2 + eta h^2)
 *  F_i       = -sum_j m_j (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) gradW_ij
 *            + sum_j m_j 4 nu (gradW_ij . r_ij) / ((rho_i + rho_j)(r_ij^2 + eta h^2)) V_ij + g
 * Wall neighbours supply p_w, their prescribed velocity in the divergence term,
 * and their ghost velocity in the viscous and artificial-viscosity terms.
 * With a pseudo-velocity vt (particles moving in pseudo-time), the advective
 * terms of Eqs. (dp-dtau) and (discrete_ME) are added:
 *  dp_i/dtau += V~_i . sum_j m_j (p_i/rho_i^2 + p_j/rho_j^2) gradW_ij
 *  F_i       += sum_j (V_i m_i/rho_i + V_j m_j/rho_j) (V~_i . gradW_ij)
 * (a wall neighbour supplying its prescribed velocity as V_j). */
static void rates(const orc_params *P, int64_t nf, const double *x, const double *v,
                  const double *p, const double *vw, const double *pw, const double *vghost,
                  const double *vt, const nlist *L, double *ap, double *F)
{
    int dim = P->dim;
    double h = P->h, m = P->m, rho = P->rho0;
    double c = P->beta * P->v_ref;
    double nu_e = h * c / 16.0;              /* Eq. (nu_edac) */
    double eh2 = P->edac_h2_literal ? h * h : P->eta * h * h;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nf; ++i) {
        double api = 0.0, Fi[3] = {0, 0, 0};
        double gp[3] = {0, 0, 0};    /* sum_j m_j (p_i/rho_i^2 + p_j/rho_j^2) gradW_ij */
        const double *vi = v + i * dim;
        const double *vti = vt ? vt + i * dim : NULL;
        for (int64_t e = L->start[i]; e < L->start[i + 1]; ++e) {
            int64_t j = L->idx[e];
            double d[3];
            separation(P, x + i * dim, x + j * dim, d);
            double r2 = norm2(d, dim);
            double r = sqrt(r2);
            double dwdr = orc_dwdr(r, h, dim);
            double gw[3] = {0, 0, 0};
            if (r > 0.0)
                for (int a = 0; a < dim; ++a) gw[a] = dwdr * d[a] / r;
            double rdotgw = 0.0;
            for (int a = 0; a < dim; ++a) rdotgw = rdotgw + d[a] * gw[a];

            double vdiv[3], vvis[3], pj;
            if (j < nf) {
                for (int a = 0; a < dim; ++a) vdiv[a] = vvis[a] = v[j * dim + a];
                pj = p[j];
            } else {
                int64_t w = j - nf;
                for (int a = 0; a < dim; ++a) {
                    vdiv[a] = vw[w * dim + a];
                    vvis[a] = vghost[w * dim + a];
                }
                pj = pw[w];
            }
            double vij_gw = 0.0;
            for (int a = 0; a < dim; ++a) vij_gw = vij_gw + (vi[a] - vdiv[a]) * gw[a];
            api = api + m * rho / rho * c * c * vij_gw;
            if (P->edac && !P->steady)   /* the steady pressure equation has no EDAC term */
                api = api + 4.0 * m / ((rho + rho) * rho) * nu_e * (p[i] - pj) * rdotgw / (r2 + eh2);

            double pi_ij = 0.0;
            if (P->alpha != 0.0) {
                double vr = 0.0;
                for (int a = 0; a < dim; ++a) vr = vr + (vi[a] - vvis[a]) * d[a];
                if (vr < 0.0) {
                    double phi = vr / (r2 + P->eta * h * h);   /* Eq. (av-phiij) */
                    pi_ij = -P->alpha * h * c * phi / rho;    /* Eq. (mom-av), h_ij = h, c_ij = c */
                }
            }
            double pres = p[i] / (rho * rho) + pj / (rho * rho) + pi_ij;
            double visc = m * 4.0 * P->nu * rdotgw / ((rho + rho) * (r2 + P->eta * h * h));
            for (int a = 0; a < dim; ++a)
                Fi[a] = Fi[a] - m * pres * gw[a] + visc * (vi[a] - vvis[a]);
            if (vti) {
                double tgw = 0.0;
                for (int a = 0; a < dim; ++a) tgw = tgw + vti[a] * gw[a];
                for (int a = 0; a < dim; ++a) {
                    gp[a] = gp[a] + m * (p[i] / (rho * rho) + pj / (rho * rho)) * gw[a];
                    Fi[a] = Fi[a] + (m / rho * vi[a] + m / rho * vdiv[a]) * tgw;
                }
            }
            if (P->steady) {
                /* convection of Eq. (mom-steady): V_i . sum_j (V_i m_i/rho_i + V_j m_j/rho_j)
                   gradW_ij, the wall's prescribed velocity for a wall neighbour */
                double vgw = 0.0;
                for (int a = 0; a < dim; ++a) vgw = vgw + vi[a] * gw[a];
                for (int a = 0; a < dim; ++a) Fi[a] = Fi[a] - (m / rho * vi[a] + m / rho * vdiv[a]) * vgw;
            }
        }
        if (vti)
            for (int a = 0; a < dim; ++a) api = api + vti[a] * gp[a];
        ap[i] = api;
        for (int a = 0; a < dim; ++a) F[i * dim + a] = Fi[a] + P->g[a];
    }
}

/* Exported for the tests: the two rates at a given state, with the advective
 * terms of a pseudo-velocity vt (nf*dim) if vt is not NULL. pw and vghost (nw
 * and nw*dim entries) receive the wall values, if there are walls. */
int orc_rates_vt(const orc_params *P, int64_t nf, int64_t nw, const double *x, const double *v,
                 const double *p, const double *vw, const double *vt, double *ap, double *F, double *pw,
                 double *vghost)
{
    nlist L;
    if (build_neighbors(P, nf + nw, x, &L)) return -1;
    if (nw > 0) wall_values(P, nf, nw, x, v, p, vw, &L, pw, vghost);
    rates(P, nf, x, v, p, vw, pw, vghost, vt, &L, ap, F);
    nlist_free(&L);
    return 0;
}

int orc_rates(const orc_params *P, int64_t nf, int64_t nw, const double *x, const double *v,
              const double *p, const double *vw, double *ap, double *F, double *pw, double *vghost)
{
    return orc_rates_vt(P, nf, nw, x, v, p, vw, NULL, ap, F, pw, vghost);
}

/* -------------------------------------------------------------- stop rules */

/* Sec. 3.4: stop when both residuals are below eps (Eq. conv); else when the
 * peak-to-peak change of each residual over the last `window` iterations,
 * relative to its largest value there, is below stag_tol; else at max_iter.
 * hist_p/hist_v hold the residuals of iterations 0..k (k+1 values).
 * Returns -1 to continue, otherwise the stop reason. */
int orc_stop_reason(const orc_params *P, int32_t k_plus_1, const double *hist_p, const double *hist_v)
{
    double rp = hist_p[k_plus_1 - 1], rv = hist_v[k_plus_1 - 1];
    if (!isfinite(rp) || !isfinite(rv)) return 3;
    if (P->fixed_iters > 0) return k_plus_1 >= P->fixed_iters ? 4 : -1;
    if (rp < P->eps && rv < P->eps) return 0;
    int wdw = P->stag_window;
    if (wdw > 0 && k_plus_1 >= wdw) {
        int stag = 1;
        for (int which = 0; which < 2; ++which) {
            const double *hh = which ? hist_v : hist_p;
            double lo = hh[k_plus_1 - 1], hi = lo;
            for (int t = k_plus_1 - wdw; t < k_plus_1; ++t) {
                if (hh[t] < lo) lo = hh[t];
                if (hh[t] > hi) hi = hh[t];
            }
            if (!(hi > 0.0 && (hi - lo) / hi < P->stag_tol)) stag = 0;
        }
        if (stag) return 1;
    }
    if (k_plus_1 >= P->max_iter) return 2;
    return -1;
}

/* --------------------------------------------------------------- shifting */

/* Sec. 3.5: dr_i = -(h^2/2) sum_j (m_j/rho_j)(1 + W_ij / W(dx, h)) gradW_ij with
 * dx = h over every neighbour j (wall particles included: they continue the
 * particle distribution, so a particle next to a wall is not pushed into it),
 * then phi_i' = phi_i + (grad phi)_i . dr_i for V and p, using
 * (grad phi)_i = sum_j (m_j/rho_j)(phi_j - phi_i) gradW_ij (fluid neighbours). */
static void shift(const orc_params *P, int64_t nf, double *x, double *v, double *p, const nlist *L)
{
    int dim = P->dim;
    double h = P->h, vol = P->m / P->rho0;
    double wdx = orc_w(h, h, dim);
    double *dr = calloc((size_t)nf * dim, sizeof(double));
    double *gv = calloc((size_t)nf * dim * dim, sizeof(double));
    double *gp = calloc((size_t)nf * dim, sizeof(double));
    if (!dr || !gv || !gp) { free(dr); free(gv); free(gp); return; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nf; ++i) {
        double divr = 0.0;    /* div r_i = -sum_j V_j r_ij . gradW_ij, walls included */
        for (int64_t e = L->start[i]; e < L->start[i + 1]; ++e) {
            int64_t j = L->idx[e];
            double d[3];
            separation(P, x + i * dim, x + j * dim, d);
            double r = sqrt(norm2(d, dim));
            double dwdr = orc_dwdr(r, h, dim);
            double W = orc_w(r, h, dim);
            if (r > 0.0) divr = divr - vol * dwdr * r;     /* r_ij . gradW_ij = dW/dr r */
            /* the displacement counts every neighbour, wall particles included
               (they continue the particle distribution); the gradients of the
               Taylor correction use fluid neighbours only */
            for (int a = 0; a < dim; ++a) {
                double gw = r > 0.0 ? dwdr * d[a] / r : 0.0;
                dr[i * dim + a] = dr[i * dim + a] + vol * (1.0 + W / wdx) * gw;
            }
            if (j >= nf) continue;
            for (int a = 0; a < dim; ++a) {
                double gw = r > 0.0 ? dwdr * d[a] / r : 0.0;
                gp[i * dim + a] = gp[i * dim + a] + vol * (p[j] - p[i]) * gw;
                for (int b = 0; b < dim; ++b)
                    gv[(i * dim + b) * dim + a] = gv[(i * dim + b) * dim + a] + vol * (v[j * dim + b] - v[i * dim + b]) * gw;
            }
        }
        /* Lind et al.'s free-surface test (Sec. 3.5): div r < d - 1/2 -> not shifted */
        const int surface = P->free_surface && divr < (double)dim - 0.5;
        for (int a = 0; a < dim; ++a) dr[i * dim + a] = surface ? 0.0 : -0.5 * h * h * dr[i * dim + a];
    }
    for (int64_t i = 0; i < nf; ++i) {
        double dp = 0.0;
        for (int a = 0; a < dim; ++a) dp = dp + gp[i * dim + a] * dr[i * dim + a];
        p[i] = p[i] + dp;
        for (int b = 0; b < dim; ++b) {
            double dvb = 0.0;
            for (int a = 0; a < dim; ++a) dvb = dvb + gv[(i * dim + b) * dim + a] * dr[i * dim + a];
            v[i * dim + b] = v[i * dim + b] + dvb;
        }
        for (int a = 0; a < dim; ++a) x[i * dim + a] = x[i * dim + a] + dr[i * dim + a];
        wrap(P, x + i * dim);
    }
    free(dr);
    free(gv);
    free(gp);
}

/* Exported for the tests: particle shifting alone (Sec. 3.5) on a given state,
 * with the neighbour lists built at x. x holds nf fluid then nw wall positions;
 * v (nf*dim) and p (nf) are corrected and the fluid positions shifted in place.
 * Returns 0, or -1 on allocation failure. */
int orc_shift(const orc_params *P, int64_t nf, int64_t nw, double *x, double *v, double *p)
{
    nlist L;
    if (build_neighbors(P, nf + nw, x, &L)) return -1;
    shift(P, nf, x, v, p, &L);
    nlist_free(&L);
    return 0;
}

/* ------------------------------------------------------------- real step */

/* One real step n -> n+1 of Algorithm 2.
 * x:      (nf+nw)*dim positions r^n (fluid first, then walls; walls never move)
 * v:      nf*dim V^n          (in: V^n, out: V^{n+1})
 * v_prev: nf*dim V^{n-1}      (in: V^{n-1}, out: V^n)
 * p:      nf     p^n          (in/out)
 * vw:     nw*dim prescribed wall velocities
 * hist:   optional per-iteration residual log, 2*cap doubles (R_p then R_v),
 *         cap = fixed_iters if set, else max_iter
 * x0_out: optional (nf+nw)*dim copy of the positions r^0 (after the predictor)
 * xk_out: optional (nf+nw)*dim copy of the pseudo-time positions r^K at the end
 *         of the loop (r^0 when the particles are fixed in pseudo-time)
 * Returns 0, or -1 on allocation failure. */
int orc_step(const orc_params *P, int64_t nf, int64_t nw, double *x, double *v, double *v_prev,
             double *p, const double *vw, orc_stats *st, double *hist, double *x0_out, double *xk_out)
{
    int dim = P->dim;
    int64_t n = nf + nw;
    double dt = P->dt;
    double c = P->beta * P->v_ref;
    double dtau = dt / P->beta;             /* Sec. 3.4 */
    size_t nfd = (size_t)nf * dim;
    int cap = P->fixed_iters > 0 ? P->fixed_iters : P->max_iter;
    if (cap < 1) cap = 1;

    double *x0 = malloc((size_t)n * dim * sizeof(double));
    double *vk = malloc(nfd * sizeof(double));
    double *vk1 = malloc(nfd * sizeof(double));
    double *pk = malloc((size_t)(nf ? nf : 1) * sizeof(double));
    double *phalf = malloc((size_t)(nf ? nf : 1) * sizeof(double));
    double *ap = malloc((size_t)(nf ? nf : 1) * sizeof(double));
    double *ap_prev = malloc((size_t)(nf ? nf : 1) * sizeof(double));
    double *F = malloc((nfd ? nfd : 1) * sizeof(double));
    double *pw = malloc((size_t)(nw ? nw : 1) * sizeof(double));
    double *vg = malloc((size_t)(nw ? nw : 1) * dim * sizeof(double));
    double *hp = malloc((size_t)cap * sizeof(double));
    double *hv = malloc((size_t)cap * sizeof(double));
    /* moving in pseudo-time: positions r^k and r^{k+1/2} of every particle, V~ */
    int moving = P->moving && !P->steady;
    double *xk = malloc((size_t)n * dim * sizeof(double));
    double *xh = malloc((size_t)n * dim * sizeof(double));
    double *vt = malloc((nfd ? nfd : 1) * sizeof(double));
    nlist L;
    int rc = -1;
    if (!x0 || !vk || !vk1 || !pk || !phalf || !ap || !ap_prev || !F || !pw || !vg || !hp || !hv || !xk || !xh ||
        !vt)
        goto out;

    /* rates at state n (Algorithms 1 and 2, before the predictor); with the
       particles moving, V~ starts at 0, so these are the frozen rates */
    if (build_neighbors(P, n, x, &L)) goto out;
    if (nw > 0) wall_values(P, nf, nw, x, v, p, vw, &L, pw, vg);
    rates(P, nf, x, v, p, vw, pw, vg, NULL, &L, ap_prev, F);
    nlist_free(&L);

    /* predictor, Eqs. (v0, r0); p^0 = p^n. Steady mode: the particles stay and
       the iteration starts from the state itself (Sec. 2.3) */
    memcpy(x0, x, (size_t)n * dim * sizeof(double));
    for (int64_t i = 0; i < nf; ++i) {
        for (int a = 0; a < dim; ++a) {
            size_t k = (size_t)i * dim + a;
            if (P->steady) {
                vk[k] = v[k];
            } else {
                vk[k] = v[k] + dt * F[k];
                x0[k] = x[k] + dt * v[k] + dt * dt / 2.0 * F[k];
            }
        }
        wrap(P, x0 + i * dim);
        pk[i] = p[i];
    }

    /* pseudo-time iterations: with the particles frozen at r^0 (Algorithm 2),
       or moving from r^0 with V~^0 = 0 (Algorithm 1; walls stay) */
    memcpy(xk, x0, (size_t)n * dim * sizeof(double));
    memcpy(xh, x0, (size_t)n * dim * sizeof(double));
    memset(vt, 0, (nfd ? nfd : 1) * sizeof(double));
    if (build_neighbors(P, n, x0, &L)) goto out;
    double kappa = 2.0 * dt / (2.0 * dt + 3.0 * dtau);
    int k = 0, reason = -1;
    while (reason < 0) {
        if (moving) {
            /* Eq. (rkstar): r^{k+1/2} = r^k + dtau/2 V~^k, wrapped onto the box */
            for (int64_t i = 0; i < nf; ++i) {
                for (int a = 0; a < dim; ++a) {
                    size_t q = (size_t)i * dim + a;
                    xh[q] = xk[q] + 0.5 * dtau * vt[q];
                }
                wrap(P, xh + i * dim);
            }
            if (P->moving == 2) {
                /* neighbours updated at the moved positions */
                nlist_free(&L);
                if (build_neighbors(P, n, xh, &L)) goto out;
            }
        }
        /* Eq. (pkstar_frozen) / (pkstar), with the rate of the previous pass */
        for (int64_t i = 0; i < nf; ++i) phalf[i] = pk[i] + 0.5 * dtau * ap_prev[i];
        if (nw > 0) wall_values(P, nf, nw, xh, vk, phalf, vw, &L, pw, vg);
        /* all rates before any update (Jacobi) */
        rates(P, nf, xh, vk, phalf, vw, pw, vg, moving ? vt : NULL, &L, ap, F);
        double sum_ap = 0.0, sum_av = 0.0;
        for (int64_t i = 0; i < nf; ++i) {
            double av2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                size_t q = (size_t)i * dim + a;
                /* Eq. (dv_dtau_exact), frozen form; steady mode: Eq. (mom-steady) as is */
                double av;
                if (P->steady) {
                    av = F[q];
                } else {
                    double bdf = (3.0 * vk[q] - 4.0 * v[q] + v_prev[q]) / (2.0 * dt);
                    av = (F[q] - bdf) * kappa;
                }
                vk1[q] = vk[q] + dtau * av;                   /* Eq. (vkp1_frozen) / (vkp1) */
                av2 = av2 + av * av;
                if (moving) {
                    vt[q] = dt * av;                          /* Eq. (vtilde) */
                    xk[q] = xh[q] + 0.5 * dtau * vt[q];       /* Eq. (rkp1) */
                }
            }
            double pnew = phalf[i] + 0.5 * dtau * ap[i];      /* Eq. (pkp1_frozen) */
            sum_ap = sum_ap + fabs(ap[i]);
            sum_av = sum_av + dt * sqrt(av2);                 /* |V~| = dt |dV/dtau| */
            pk[i] = pnew;
            ap_prev[i] = ap[i];
        }
        memcpy(vk, vk1, nfd * sizeof(double));
        double inv_n = nf > 0 ? 1.0 / (double)nf : 0.0;
        hp[k] = sum_ap * inv_n * dt / (P->rho0 * c * c);      /* Eq. (conv) */
        hv[k] = sum_av * inv_n / P->v_ref;
        if (hist) { hist[k] = hp[k]; hist[cap + k] = hv[k]; }
        ++k;
        reason = orc_stop_reason(P, k, hp, hv);
        if (reason < 0 && k >= cap) reason = 2;
    }
    nlist_free(&L);
    if (x0_out) memcpy(x0_out, x0, (size_t)n * dim * sizeof(double));
    if (xk_out) memcpy(xk_out, xk, (size_t)n * dim * sizeof(double));
    st->iters = k;
    st->reason = reason;
    st->rp = hp[k - 1];
    st->rv = hv[k - 1];

    /* Eq. (r-update), then V^{n-1} <- V^n, V^n <- V^{n+1}, p^n <- p^{n+1};
       steady mode: the particles stay */
    for (int64_t i = 0; i < nf; ++i) {
        for (int a = 0; a < dim; ++a) {
            size_t q = (size_t)i * dim + a;
            if (!P->steady) x[q] = x[q] + dt / 2.0 * (v[q] + vk[q]);
            v_prev[q] = v[q];
            v[q] = vk[q];
        }
        wrap(P, x + i * dim);
        p[i] = pk[i];
    }
    if (P->shifting && !P->steady) {
        if (build_neighbors(P, n, x, &L)) goto out;
        shift(P, nf, x, v, p, &L);
        nlist_free(&L);
    }
    rc = 0;
out:
    free(x0); free(vk); free(vk1); free(pk); free(phalf); free(ap); free(ap_prev);
    free(F); free(pw); free(vg); free(hp); free(hv); free(xk); free(xh); free(vt);
    return rc;
}

/* nsteps real steps; st receives nsteps entries. */
int orc_run(const orc_params *P, int64_t nf, int64_t nw, double *x, double *v, double *v_prev,
            double *p, const double *vw, int32_t nsteps, orc_stats *st)
{
    for (int32_t s = 0; s < nsteps; ++s)
        if (orc_step(P, nf, nw, x, v, v_prev, p, vw, st + s, NULL, NULL, NULL)) return -1;
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
