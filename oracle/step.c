/*
 * step.c -- the oracle's whole-grid 2D wave-propagation step.
 *
 * TEST INFRASTRUCTURE ONLY (see mcref.h).
 *
 * Structure follows the unfused, work-array form the paper describes for
 * Clawpack (§2: the Riemann kernel runs over every edge of a structured grid
 * and its results are kept in standard work arrays; Table 1: the Riemann
 * kernel maps cell centres to edge values, the limiter maps edge values back
 * to cell centres).  The arithmetic of the unsplit step is LeVeque (2002)
 * eq. 21.8 with the limited corrections of §6.13/§21.3 and the transverse
 * (corner-transport) terms of §21.2:
 *
 *   Q^{n+1}_ij = Q_ij - dt/dx (A+dQ_{i-1/2,j} + A-dQ_{i+1/2,j})
 *                     - dt/dy (B+dQ_{i,j-1/2} + B-dQ_{i,j+1/2})
 *                     - dt/dx (F_{i+1/2,j} - F_{i-1/2,j})
 *                     - dt/dy (G_{i,j+1/2} - G_{i,j-1/2})
 *
 * F, G hold the limited second-order corrections 1/2 |s|(1 - dt/dx|s|) W~
 * plus, for the transverse option, -dt/(2dx) times the transverse split of
 * the fluctuation that enters a neighbouring cell.
 *
 * Edge indexing: x-edge (i, j) lies between cells (i-1, j) and (i, j);
 * y-edge (i, j) lies between cells (i, j-1) and (i, j).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "mcref.h"

#define NXG(p) ((p)->mx + 2 * (p)->mbc)
#define NYG(p) ((p)->my + 2 * (p)->mbc)

static inline int64_t qidx(const mcref_problem* p, int m, int i, int j)
{
    return ((int64_t)m * NYG(p) + (j + p->mbc)) * NXG(p) + (i + p->mbc);
}

static void get_cell(const mcref_problem* p, const double* q, int i, int j, double* v)
{
    int meqn = mcref_nplane(p->solver);
    for (int m = 0; m < meqn; m++) v[m] = q[qidx(p, m, i, j)];
}

/* ghost value of a wall: mirror, with the momentum normal to the wall
 * (component 1 + dir) negated */
static void bc_copy(const mcref_problem* p, double* q, int i_dst, int j_dst, int i_src, int j_src,
                    int negate_comp)
{
    int meqn = mcref_nplane(p->solver);
    for (int m = 0; m < meqn; m++) {
        double v = q[qidx(p, m, i_src, j_src)];
        q[qidx(p, m, i_dst, j_dst)] = (m == negate_comp) ? -v : v;
    }
}

void mcref_bc_fill(const mcref_problem* p, double* q)
{
    const int mx = p->mx, my = p->my, mbc = p->mbc;
    /* x ghosts, interior rows */
    for (int j = 0; j < my; j++) {
        for (int k = 1; k <= mbc; k++) {
            switch (p->bc[0]) {
            case MCREF_BC_PERIODIC: bc_copy(p, q, -k, j, mx - k, j, -1); break;
            case MCREF_BC_EXTRAP:   bc_copy(p, q, -k, j, 0, j, -1); break;
            case MCREF_BC_GIVEN:    break;
            default:                bc_copy(p, q, -k, j, k - 1, j, 1); break;
            }
            switch (p->bc[1]) {
            case MCREF_BC_PERIODIC: bc_copy(p, q, mx - 1 + k, j, k - 1, j, -1); break;
            case MCREF_BC_EXTRAP:   bc_copy(p, q, mx - 1 + k, j, mx - 1, j, -1); break;
            case MCREF_BC_GIVEN:    break;
            default:                bc_copy(p, q, mx - 1 + k, j, mx - k, j, 1); break;
            }
        }
    }
    /* y ghosts across the full width, so corners take the x-filled values */
    for (int i = -mbc; i < mx + mbc; i++) {
        for (int k = 1; k <= mbc; k++) {
            switch (p->bc[2]) {
            case MCREF_BC_PERIODIC: bc_copy(p, q, i, -k, i, my - k, -1); break;
            case MCREF_BC_EXTRAP:   bc_copy(p, q, i, -k, i, 0, -1); break;
            case MCREF_BC_GIVEN:    break;
            default:                bc_copy(p, q, i, -k, i, k - 1, 2); break;
            }
            switch (p->bc[3]) {
            case MCREF_BC_PERIODIC: bc_copy(p, q, i, my - 1 + k, i, k - 1, -1); break;
            case MCREF_BC_EXTRAP:   bc_copy(p, q, i, my - 1 + k, i, my - 1, -1); break;
            case MCREF_BC_GIVEN:    break;
            default:                bc_copy(p, q, i, my - 1 + k, i, my - k, 2); break;
            }
        }
    }
}

/* Work arrays for the edges of one direction. */
typedef struct {
    int i0, i1, j0, j1;  /* inclusive edge-index ranges */
    int meqn, mw;
    double *wave, *s, *amdq, *apdq;
} edge_arrays;

static int64_t eidx(const edge_arrays* e, int i, int j)
{
    return (int64_t)(j - e->j0) * (e->i1 - e->i0 + 1) + (i - e->i0);
}

static int edges_alloc(edge_arrays* e, int i0, int i1, int j0, int j1, int meqn, int mw)
{
    e->i0 = i0; e->i1 = i1; e->j0 = j0; e->j1 = j1; e->meqn = meqn; e->mw = mw;
    int64_t n = (int64_t)(i1 - i0 + 1) * (j1 - j0 + 1);
    e->wave = malloc(sizeof(double) * n * mw * meqn);
    e->s = malloc(sizeof(double) * n * mw);
    e->amdq = malloc(sizeof(double) * n * meqn);
    e->apdq = malloc(sizeof(double) * n * meqn);
    return e->wave && e->s && e->amdq && e->apdq;
}

static void edges_free(edge_arrays* e)
{
    free(e->wave); free(e->s); free(e->amdq); free(e->apdq);
}

/* Normal solves at every edge of the range.  dir 0: edge (i, j) between
 * cells (i-1, j), (i, j); dir 1: between (i, j-1), (i, j). */
static int solve_edges(const mcref_problem* p, const double* q, int dir, edge_arrays* e, int nthreads)
{
    int flags = 0;
    const int meqn = e->meqn, mw = e->mw;
    (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : flags)
    for (int j = e->j0; j <= e->j1; j++) {
        double ql[MCREF_MAXEQN], qr[MCREF_MAXEQN];
        for (int i = e->i0; i <= e->i1; i++) {
            int64_t k = eidx(e, i, j);
            if (dir == 0) get_cell(p, q, i - 1, j, ql);
            else get_cell(p, q, i, j - 1, ql);
            get_cell(p, q, i, j, qr);
            flags |= mcref_rpn2(p, dir, ql, qr, e->wave + k * mw * meqn, e->s + k * mw,
                                e->amdq + k * meqn, e->apdq + k * meqn);
        }
    }
    return flags;
}

/* Limited correction 1/2 |s| (1 - dt/dx |s|) W~ summed over waves, for edge
 * (i, j) whose upwind neighbours are (i -+ 1, j) (dir 0) or (i, j -+ 1). */
static void limited_correction(const mcref_problem* p, const edge_arrays* e, int dir, int i, int j,
                               double dtdx, double* out)
{
    const int meqn = e->meqn, mw = e->mw;
    const double* W = e->wave + eidx(e, i, j) * mw * meqn;
    const double* S = e->s + eidx(e, i, j) * mw;
    for (int m = 0; m < meqn; m++) out[m] = 0.0;
    for (int w = 0; w < mw; w++) {
        const double* Ww = W + w * meqn;
        double dotr = 0.0;
        for (int m = 0; m < meqn; m++) dotr += Ww[m] * Ww[m];
        if (dotr == 0.0) continue;
        int iu = i, ju = j;
        if (dir == 0) iu = S[w] > 0.0 ? i - 1 : i + 1;
        else ju = S[w] > 0.0 ? j - 1 : j + 1;
        const double* Wu = e->wave + eidx(e, iu, ju) * mw * meqn + w * meqn;
        double dotl = 0.0;
        for (int m = 0; m < meqn; m++) dotl += Wu[m] * Ww[m];
        double phi = mcref_philim(p->limiter, dotl / dotr);
        double as = fabs(S[w]);
        double cf = 0.5 * as * (1.0 - dtdx * as) * phi;
        for (int m = 0; m < meqn; m++) out[m] += cf * Ww[m];
    }
}

/* The fluctuations an edge sends into its two cells, as the transverse split
 * sees them.  Option 1 splits A+dQ (into the high cell) and A-dQ (into the
 * low cell).  Option 2 splits the whole first- plus second-order
 * contribution of the edge to each cell: the update takes
 * -dt/dx (A+dQ - F) from the high cell and -dt/dx (A-dQ + F) from the low
 * cell, F the limited correction of the edge (LeVeque 2002, ch. 21:
 * transverse propagation of the correction waves; Clawpack's
 * transverse_waves = 2). */
static void effective_fluctuations(const mcref_problem* p, const edge_arrays* e, int dir, int i,
                                   int j, double dtdx, double* ap, double* am)
{
    const int meqn = e->meqn;
    const int64_t k = eidx(e, i, j);
    for (int m = 0; m < meqn; m++) {
        ap[m] = e->apdq[k * meqn + m];
        am[m] = e->amdq[k * meqn + m];
    }
    if (p->transverse == 2 && p->order >= 2) {
        double cq[MCREF_MAXEQN];
        limited_correction(p, e, dir, i, j, dtdx, cq);
        for (int m = 0; m < meqn; m++) {
            ap[m] -= cq[m];
            am[m] += cq[m];
        }
    }
}

int mcref_step(const mcref_problem* p, const double* qin, double* qout, double dt,
               double* smax_out, int nthreads)
{
    const int mx = p->mx, my = p->my;
    const int meqn = mcref_meqn(p->solver), mw = mcref_mwaves(p->solver);
    const double dtdx = dt / p->dx, dtdy = dt / p->dy;
    const int64_t nq = (int64_t)mcref_nplane(p->solver) * NXG(p) * NYG(p);
    const int var = p->solver == MCREF_ACOUSTICS_VAR;
    int flags = 0;
    if (nthreads < 1) nthreads = 1;

    double* q = malloc(sizeof(double) * nq);
    memcpy(q, qin, sizeof(double) * nq);
    mcref_bc_fill(p, q);

    /* x-edges: limiter neighbours need i in [-1, mx+1]; transverse terms
     * need rows [-1, my].  y-edges symmetric. */
    edge_arrays ex, ey;
    edges_alloc(&ex, -1, mx + 1, -1, my, meqn, mw);
    edges_alloc(&ey, -1, mx, -1, my + 1, meqn, mw);
    flags |= solve_edges(p, q, 0, &ex, nthreads);
    flags |= solve_edges(p, q, 1, &ey, nthreads);

    /* F on x-edges i in [0, mx], rows [0, my); G on y-edges j in [0, my],
     * columns [0, mx) */
    const int64_t nF = (int64_t)(mx + 1) * my, nG = (int64_t)mx * (my + 1);
    double* F = calloc((size_t)(nF * meqn), sizeof(double));
    double* G = calloc((size_t)(nG * meqn), sizeof(double));
#define FI(i, j) ((((int64_t)(j)) * (mx + 1) + (i)) * meqn)
#define GI(i, j) ((((int64_t)(j)) * mx + (i)) * meqn)

    if (p->order >= 2) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int j = 0; j < my; j++)
            for (int i = 0; i <= mx; i++) limited_correction(p, &ex, 0, i, j, dtdx, F + FI(i, j));
#pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int j = 0; j <= my; j++)
            for (int i = 0; i < mx; i++) limited_correction(p, &ey, 1, i, j, dtdy, G + GI(i, j));
    }

    if (p->transverse) {
        /* x-edge fluctuations split in y.  apdq of x-edge (i, j) enters cell
         * (i, j); amdq enters (i-1, j).  The split's down/up-going parts
         * cross the y-edges below/above the receiving cell. */
        const int nxe = mx + 1, nxr = my + 2;    /* x-edges i in [0,mx], rows [-1,my] */
        double* tx = malloc(sizeof(double) * (size_t)nxe * nxr * 4 * meqn);
#pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int j = -1; j <= my; j++) {
            double ql[MCREF_MAXEQN], qr[MCREF_MAXEQN];
            for (int i = 0; i <= mx; i++) {
                double* t = tx + (((int64_t)(j + 1)) * nxe + i) * 4 * meqn;
                get_cell(p, q, i - 1, j, ql);
                get_cell(p, q, i, j, qr);
                int64_t k = eidx(&ex, i, j);
                double ap[MCREF_MAXEQN], am[MCREF_MAXEQN];
                effective_fluctuations(p, &ex, 0, i, j, dtdx, ap, am);
                if (var) {
                    /* A+dQ enters cell (i, j), A-dQ cell (i-1, j); each is
                     * split between that cell's neighbours below and above */
                    double lo[MCREF_MAXEQN], hi[MCREF_MAXEQN];
                    get_cell(p, q, i, j - 1, lo);
                    get_cell(p, q, i, j + 1, hi);
                    mcref_rpt2_var(p, 0, lo, qr, hi, ap, t, t + meqn);
                    get_cell(p, q, i - 1, j - 1, lo);
                    get_cell(p, q, i - 1, j + 1, hi);
                    mcref_rpt2_var(p, 0, lo, ql, hi, am, t + 2 * meqn, t + 3 * meqn);
                } else {
                    mcref_rpt2(p, 0, ql, qr, ap, t, t + meqn);
                    mcref_rpt2(p, 0, ql, qr, am, t + 2 * meqn, t + 3 * meqn);
                }
                (void)k;
            }
        }
        for (int j = -1; j <= my; j++) {
            for (int i = 0; i <= mx; i++) {
                const double* t = tx + (((int64_t)(j + 1)) * nxe + i) * 4 * meqn;
                for (int m = 0; m < meqn; m++) {
                    if (i <= mx - 1) {  /* receiving cell (i, j) */
                        if (j >= 0 && j <= my) G[GI(i, j) + m] -= 0.5 * dtdx * t[m];
                        if (j + 1 >= 0 && j + 1 <= my) G[GI(i, j + 1) + m] -= 0.5 * dtdx * t[meqn + m];
                    }
                    if (i - 1 >= 0) {   /* receiving cell (i-1, j) */
                        if (j >= 0 && j <= my) G[GI(i - 1, j) + m] -= 0.5 * dtdx * t[2 * meqn + m];
                        if (j + 1 >= 0 && j + 1 <= my) G[GI(i - 1, j + 1) + m] -= 0.5 * dtdx * t[3 * meqn + m];
                    }
                }
            }
        }
        free(tx);

        /* y-edge fluctuations split in x.  bpdq of y-edge (i, j) enters cell
         * (i, j); bmdq enters (i, j-1). */
        const int nyc = mx + 2, nye = my + 1;    /* columns [-1,mx], y-edges j in [0,my] */
        double* ty = malloc(sizeof(double) * (size_t)nyc * nye * 4 * meqn);
#pragma omp parallel for schedule(static) num_threads(nthreads)
        for (int j = 0; j <= my; j++) {
            double ql[MCREF_MAXEQN], qr[MCREF_MAXEQN];
            for (int i = -1; i <= mx; i++) {
                double* t = ty + (((int64_t)j) * nyc + (i + 1)) * 4 * meqn;
                get_cell(p, q, i, j - 1, ql);
                get_cell(p, q, i, j, qr);
                double ap[MCREF_MAXEQN], am[MCREF_MAXEQN];
                effective_fluctuations(p, &ey, 1, i, j, dtdy, ap, am);
                if (var) {
                    /* B+dQ enters cell (i, j), B-dQ cell (i, j-1); each is
                     * split between that cell's neighbours left and right */
                    double lo[MCREF_MAXEQN], hi[MCREF_MAXEQN];
                    get_cell(p, q, i - 1, j, lo);
                    get_cell(p, q, i + 1, j, hi);
                    mcref_rpt2_var(p, 1, lo, qr, hi, ap, t, t + meqn);
                    get_cell(p, q, i - 1, j - 1, lo);
                    get_cell(p, q, i + 1, j - 1, hi);
                    mcref_rpt2_var(p, 1, lo, ql, hi, am, t + 2 * meqn, t + 3 * meqn);
                } else {
                    mcref_rpt2(p, 1, ql, qr, ap, t, t + meqn);
                    mcref_rpt2(p, 1, ql, qr, am, t + 2 * meqn, t + 3 * meqn);
                }
            }
        }
        for (int j = 0; j <= my; j++) {
            for (int i = -1; i <= mx; i++) {
                const double* t = ty + (((int64_t)j) * nyc + (i + 1)) * 4 * meqn;
                for (int m = 0; m < meqn; m++) {
                    if (j <= my - 1) {  /* receiving cell (i, j) */
                        if (i >= 0 && i <= mx) F[FI(i, j) + m] -= 0.5 * dtdy * t[m];
                        if (i + 1 >= 0 && i + 1 <= mx) F[FI(i + 1, j) + m] -= 0.5 * dtdy * t[meqn + m];
                    }
                    if (j - 1 >= 0) {   /* receiving cell (i, j-1) */
                        if (i >= 0 && i <= mx) F[FI(i, j - 1) + m] -= 0.5 * dtdy * t[2 * meqn + m];
                        if (i + 1 >= 0 && i + 1 <= mx) F[FI(i + 1, j - 1) + m] -= 0.5 * dtdy * t[3 * meqn + m];
                    }
                }
            }
        }
        free(ty);
    }

    /* update */
    memcpy(qout, q, sizeof(double) * nq);
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int j = 0; j < my; j++) {
        for (int i = 0; i < mx; i++) {
            const double* apl = ex.apdq + eidx(&ex, i, j) * meqn;
            const double* amr = ex.amdq + eidx(&ex, i + 1, j) * meqn;
            const double* bpb = ey.apdq + eidx(&ey, i, j) * meqn;
            const double* bmt = ey.amdq + eidx(&ey, i, j + 1) * meqn;
            for (int m = 0; m < meqn; m++) {
                double v = q[qidx(p, m, i, j)];
                v -= dtdx * (apl[m] + amr[m]);
                v -= dtdy * (bpb[m] + bmt[m]);
                v -= dtdx * (F[FI(i + 1, j) + m] - F[FI(i, j) + m]);
                v -= dtdy * (G[GI(i, j + 1) + m] - G[GI(i, j) + m]);
                qout[qidx(p, m, i, j)] = v;
            }
        }
    }
    mcref_bc_fill(p, qout);

    /* largest wave speed over the edges of the interior update */
    double smax = 0.0;
    for (int j = 0; j < my; j++)
        for (int i = 0; i <= mx; i++)
            for (int w = 0; w < mw; w++) {
                double v = fabs(ex.s[eidx(&ex, i, j) * mw + w]) / p->dx;
                if (v > smax) smax = v;
            }
    for (int j = 0; j <= my; j++)
        for (int i = 0; i < mx; i++)
            for (int w = 0; w < mw; w++) {
                double v = fabs(ey.s[eidx(&ey, i, j) * mw + w]) / p->dy;
                if (v > smax) smax = v;
            }
    if (smax_out) *smax_out = smax;

#undef FI
#undef GI
    free(F); free(G);
    edges_free(&ex); edges_free(&ey);
    free(q);
    return flags;
}

double mcref_max_cell_speed(const mcref_problem* p, const double* q)
{
    double smax = 0.0, v[MCREF_MAXEQN];
    for (int j = 0; j < p->my; j++) {
        for (int i = 0; i < p->mx; i++) {
            get_cell(p, q, i, j, v);
            double u = 0, w = 0, c;
            if (p->solver == MCREF_ACOUSTICS) {
                c = sqrt(p->param[1] / p->param[0]);
            } else if (p->solver == MCREF_ADVECTION) {
                u = p->param[0]; w = p->param[1];
                c = 0.0;
            } else if (p->solver == MCREF_ACOUSTICS_VAR) {
                c = v[4];
            } else if (p->solver == MCREF_SWE) {
                u = v[1] / v[0]; w = v[2] / v[0];
                c = sqrt(p->param[0] * v[0]);
            } else {
                u = v[1] / v[0]; w = v[2] / v[0];
                double pr = (p->param[0] - 1.0) * (v[3] - 0.5 * v[0] * (u * u + w * w));
                c = sqrt(p->param[0] * pr / v[0]);
            }
            double sx = (fabs(u) + c) / p->dx, sy = (fabs(w) + c) / p->dy;
            if (sx > smax) smax = sx;
            if (sy > smax) smax = sy;
        }
    }
    return smax;
}

/* Variable time step with rejection: the Courant number of an attempt is
 * dt * smax where smax comes from that attempt's edges.  An attempt above
 * cfl_max is discarded and retaken with dt = cfl_desired / smax; an accepted
 * one advances t and proposes dt = cfl_desired / smax for the next step. */
int mcref_advance(const mcref_problem* p, double* qa, double* qb, int nsteps,
                  double cfl_desired, double cfl_max, double* t, double* dt,
                  int* result_in_b, int* nrejected, int nthreads)
{
    int flags = 0, cur_b = 0, nrej = 0;
    int done = 0;
    while (done < nsteps) {
        double* qi = cur_b ? qb : qa;
        double* qo = cur_b ? qa : qb;
        double smax = 0.0;
        flags |= mcref_step(p, qi, qo, *dt, &smax, nthreads);
        double cfl = *dt * smax;
        if (cfl > cfl_max) {
            nrej++;
            *dt = cfl_desired / smax;
            if (nrej > 100 * (nsteps + 1)) break;
            continue;
        }
        *t += *dt;
        if (smax > 0.0) *dt = cfl_desired / smax;
        cur_b ^= 1;
        done++;
    }
    *result_in_b = cur_b;
    if (nrejected) *nrejected = nrej;
    return flags;
}
