/*
 * amr.c -- the oracle's coupling of refined patches to a coarse grid.
 *
 * TEST INFRASTRUCTURE ONLY (see mcref.h).
 *
 * The paper (§1.2, Table 1) lists "dynamic time stepping" among the kernels
 * of an explicit method: each refined grid takes its own time step, and the
 * values at refinement boundaries come from the adjacent grid by spatial and
 * temporal interpolation.  This file restates that for two levels in the
 * Berger-Oliger manner (Berger & Oliger 1984; Berger & LeVeque 1998):
 *
 *   one coarse step of dt, then r fine steps of dt/r on every patch, where
 *   before fine step s each patch's two ghost layers are filled, cell by
 *   cell, by a copy from the other patch that covers that fine cell, or else
 *   by interpolation of the coarse grid: in time linearly between the coarse
 *   states before and after its step (weight s/r), in space by the coarse
 *   cell's value plus MC-limited slopes (a conservative linear
 *   reconstruction: the r x r fine values of a coarse cell average to it);
 *   afterwards every coarse cell covered by a patch takes the average of its
 *   r x r fine cells.
 *
 * Optionally (reflux) the coupling is made conservative in the manner of
 * Berger & Colella (1989): the coarse step's flux through each coarse edge
 * on a patch boundary is replaced, for the coarse cell outside the patch, by
 * the mean of the fine fluxes through the same edge over the fine steps.  The
 * flux through an edge is the one the wave-propagation update implies,
 * f(Q_low) + A-dQ + F~ with F~ the limited correction and the transverse
 * terms (LeVeque 2002, §6.14 and ch. 21): the update of a cell is minus the
 * difference of these fluxes.  Edges on the domain boundary, and edges whose
 * outside cell is covered by another patch, are not corrected.
 *
 * Patches lie inside the coarse interior, do not overlap, and carry no
 * material planes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "mcref.h"

#define NXG(p) ((p)->mx + 2 * (p)->mbc)
#define NYG(p) ((p)->my + 2 * (p)->mbc)

static inline int64_t idx(const mcref_problem* p, int m, int i, int j)
{
    return ((int64_t)m * NYG(p) + (j + p->mbc)) * NXG(p) + (i + p->mbc);
}

static int floordiv(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

/* MC-limited slope from the one-sided differences a (left) and b (right):
 * minmod(2a, 2b, (a + b)/2) */
static double mc_slope(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    double c = 0.5 * (a + b), s = fabs(2.0 * a);
    if (fabs(2.0 * b) < s) s = fabs(2.0 * b);
    if (fabs(c) < s) s = fabs(c);
    return c > 0.0 ? s : -s;
}

/* ---- the flux through one edge, from the stencil around it ---------------- */

static void cell_of(const mcref_problem* p, const double* q, int i, int j, double* v)
{
    const int nplane = mcref_nplane(p->solver);
    for (int m = 0; m < nplane; m++) v[m] = q[idx(p, m, i, j)];
}

/* normal solve at the edge of direction dir with high cell (i, j) */
static void solve_at(const mcref_problem* p, const double* q, int dir, int i, int j, double* W,
                     double* s, double* am, double* ap)
{
    double ql[MCREF_MAXEQN], qr[MCREF_MAXEQN];
    cell_of(p, q, dir == 0 ? i - 1 : i, dir == 0 ? j : j - 1, ql);
    cell_of(p, q, i, j, qr);
    mcref_rpn2(p, dir, ql, qr, W, s, am, ap);
}

/* limited correction of that edge: sum over waves of 1/2 |s| (1 - dt/d |s|)
 * phi(theta) W, theta from the same wave of the upwind neighbour edge */
static void correction_at(const mcref_problem* p, const double* q, double dtd, int dir, int i, int j,
                          double* out)
{
    const int meqn = mcref_meqn(p->solver), mw = mcref_mwaves(p->solver);
    double W[MCREF_MAXEQN * 3], s[3], am[MCREF_MAXEQN], ap[MCREF_MAXEQN];
    double Wl[MCREF_MAXEQN * 3], sl[3], Wh[MCREF_MAXEQN * 3], sh[3];
    solve_at(p, q, dir, i, j, W, s, am, ap);
    solve_at(p, q, dir, dir == 0 ? i - 1 : i, dir == 0 ? j : j - 1, Wl, sl, am, ap);
    solve_at(p, q, dir, dir == 0 ? i + 1 : i, dir == 0 ? j : j + 1, Wh, sh, am, ap);
    for (int m = 0; m < meqn; m++) out[m] = 0.0;
    for (int w = 0; w < mw; w++) {
        double dotr = 0.0, dotl = 0.0;
        const double* Wu = s[w] > 0.0 ? Wl + w * meqn : Wh + w * meqn;
        for (int m = 0; m < meqn; m++) {
            dotr += W[w * meqn + m] * W[w * meqn + m];
            dotl += Wu[m] * W[w * meqn + m];
        }
        if (dotr == 0.0) continue;
        const double as = fabs(s[w]);
        const double cf = 0.5 * as * (1.0 - dtd * as) * mcref_philim(p->limiter, dotl / dotr);
        for (int m = 0; m < meqn; m++) out[m] += cf * W[w * meqn + m];
    }
}

/* the fluctuations of that edge as the transverse split takes them: A+dQ
 * (into the high cell) and A-dQ (into the low cell), with transverse option 2
 * at second order less / plus the limited correction */
static void fluct_at(const mcref_problem* p, const double* q, double dtd, int dir, int i, int j,
                     double* ap, double* am)
{
    const int meqn = mcref_meqn(p->solver);
    double W[MCREF_MAXEQN * 3], s[3];
    solve_at(p, q, dir, i, j, W, s, am, ap);
    if (p->transverse == 2 && p->order >= 2) {
        double c[MCREF_MAXEQN];
        correction_at(p, q, dtd, dir, i, j, c);
        for (int m = 0; m < meqn; m++) {
            ap[m] -= c[m];
            am[m] += c[m];
        }
    }
}

void mcref_edge_flux(const mcref_problem* p, const double* q, double dt, int dir, int i, int j,
                     double* F)
{
    const int meqn = mcref_meqn(p->solver);
    const double dtd = dt / (dir == 0 ? p->dx : p->dy), dto = dt / (dir == 0 ? p->dy : p->dx);
    double ql[MCREF_MAXEQN], W[MCREF_MAXEQN * 3], s[3], am[MCREF_MAXEQN], ap[MCREF_MAXEQN];
    /* f(Q_low) + A-dQ */
    cell_of(p, q, dir == 0 ? i - 1 : i, dir == 0 ? j : j - 1, ql);
    mcref_flux(p, dir, ql, F);
    solve_at(p, q, dir, i, j, W, s, am, ap);
    for (int m = 0; m < meqn; m++) F[m] += am[m];
    if (p->order >= 2) {
        double c[MCREF_MAXEQN];
        correction_at(p, q, dtd, dir, i, j, c);
        for (int m = 0; m < meqn; m++) F[m] += c[m];
    }
    if (!p->transverse) return;
    /* transverse terms: the fluctuations entering the edge's two cells across
     * the edges of the other direction, split along dir; the high cell gives
     * its part moving to lower indices, the low cell its part moving to
     * higher ones */
    const int o = 1 - dir;
    for (int side = 0; side < 2; side++) {          /* 0: low cell, 1: high cell */
        const int ci = dir == 0 ? i - 1 + side : i, cj = dir == 0 ? j : j - 1 + side;
        for (int e = 0; e < 2; e++) {               /* 0: the cell's low edge, 1: high edge */
            const int ei = o == 0 ? ci + e : ci, ej = o == 0 ? cj : cj + e;
            double eap[MCREF_MAXEQN], eam[MCREF_MAXEQN], lo[MCREF_MAXEQN], hi[MCREF_MAXEQN];
            double bm[MCREF_MAXEQN], bp[MCREF_MAXEQN];
            fluct_at(p, q, dto, o, ei, ej, eap, eam);
            cell_of(p, q, o == 0 ? ei - 1 : ei, o == 0 ? ej : ej - 1, lo);
            cell_of(p, q, ei, ej, hi);
            /* the low edge's A+dQ and the high edge's A-dQ enter the cell */
            mcref_rpt2(p, o, lo, hi, e == 0 ? eap : eam, bm, bp);
            for (int m = 0; m < meqn; m++) F[m] -= 0.5 * dto * (side == 1 ? bm[m] : bp[m]);
        }
    }
}

void mcref_fine_problem(const mcref_problem* coarse, int ratio, const mcref_amr_patch* pt,
                        mcref_problem* fine)
{
    *fine = *coarse;
    fine->mx = ratio * pt->cw;
    fine->my = ratio * pt->ch;
    fine->dx = coarse->dx / ratio;
    fine->dy = coarse->dy / ratio;
    for (int k = 0; k < 4; k++) fine->bc[k] = MCREF_BC_GIVEN;
}

/* value of field m at fine cell (gx, gy) (global fine indices) by the
 * coarse reconstruction of the time-interpolated coarse state */
static double coarse_interp(const mcref_problem* pc, const double* qc0, const double* qc1,
                            double alpha, int ratio, int m, int gx, int gy)
{
    const int cx = floordiv(gx, ratio), cy = floordiv(gy, ratio);
#define QT(i, j) ((1.0 - alpha) * qc0[idx(pc, m, (i), (j))] + alpha * qc1[idx(pc, m, (i), (j))])
    const double q = QT(cx, cy);
    const double sx = mc_slope(q - QT(cx - 1, cy), QT(cx + 1, cy) - q);
    const double sy = mc_slope(q - QT(cx, cy - 1), QT(cx, cy + 1) - q);
#undef QT
    /* fine cell centre relative to the coarse cell centre, in coarse cells */
    const double ox = ((gx - ratio * cx) + 0.5) / ratio - 0.5;
    const double oy = ((gy - ratio * cy) + 0.5) / ratio - 0.5;
    return q + ox * sx + oy * sy;
}

void mcref_amr_fill_ghosts(const mcref_problem* pc, int ratio, const double* qc0, const double* qc1,
                           double alpha, const mcref_amr_patch* pts, int npatch, double** qf)
{
    const int nplane = mcref_nplane(pc->solver);
    for (int p = 0; p < npatch; p++) {
        mcref_problem pf;
        mcref_fine_problem(pc, ratio, &pts[p], &pf);
        for (int fj = -pf.mbc; fj < pf.my + pf.mbc; fj++) {
            for (int fi = -pf.mbc; fi < pf.mx + pf.mbc; fi++) {
                if (fi >= 0 && fi < pf.mx && fj >= 0 && fj < pf.my) continue;   /* interior */
                const int gx = ratio * pts[p].ci0 + fi, gy = ratio * pts[p].cj0 + fj;
                /* another patch covering this fine cell? */
                int src = -1, si = 0, sj = 0;
                for (int q = 0; q < npatch && src < 0; q++) {
                    if (q == p) continue;
                    const int qi = gx - ratio * pts[q].ci0, qj = gy - ratio * pts[q].cj0;
                    if (qi >= 0 && qi < ratio * pts[q].cw && qj >= 0 && qj < ratio * pts[q].ch) {
                        src = q;
                        si = qi;
                        sj = qj;
                    }
                }
                for (int m = 0; m < nplane; m++) {
                    double v;
                    if (src >= 0) {
                        mcref_problem pq;
                        mcref_fine_problem(pc, ratio, &pts[src], &pq);
                        v = qf[src][idx(&pq, m, si, sj)];
                    } else {
                        v = coarse_interp(pc, qc0, qc1, alpha, ratio, m, gx, gy);
                    }
                    qf[p][idx(&pf, m, fi, fj)] = v;
                }
            }
        }
    }
}

void mcref_amr_average_down(const mcref_problem* pc, int ratio, const mcref_amr_patch* pts,
                            int npatch, double* const* qf, double* qc)
{
    const int nplane = mcref_nplane(pc->solver);
    for (int p = 0; p < npatch; p++) {
        mcref_problem pf;
        mcref_fine_problem(pc, ratio, &pts[p], &pf);
        for (int cj = 0; cj < pts[p].ch; cj++)
            for (int ci = 0; ci < pts[p].cw; ci++)
                for (int m = 0; m < nplane; m++) {
                    double s = 0.0;
                    for (int b = 0; b < ratio; b++)
                        for (int a = 0; a < ratio; a++) s += qf[p][idx(&pf, m, ratio * ci + a, ratio * cj + b)];
                    qc[idx(pc, m, pts[p].ci0 + ci, pts[p].cj0 + cj)] = s / (ratio * ratio);
                }
    }
}

/* the coarse edges on the patches' boundaries that get a flux correction:
 * the edge (dir, ci, cj) with high cell (ci, cj), the outside coarse cell
 * (oi, oj), the sign of the outside cell's update from this edge (+1 if the
 * edge is its high edge), the patch, and the fine edge (high cell) of the
 * first of its ratio fine edges in the patch's local indices */
typedef struct {
    int dir, ci, cj, oi, oj, sgn, patch, fi, fj;
} reflux_edge;

static int covered(const mcref_amr_patch* pts, int npatch, int i, int j)
{
    for (int q = 0; q < npatch; q++)
        if (i >= pts[q].ci0 && i < pts[q].ci0 + pts[q].cw && j >= pts[q].cj0 && j < pts[q].cj0 + pts[q].ch)
            return 1;
    return 0;
}

static int reflux_edges(const mcref_problem* pc, int ratio, const mcref_amr_patch* pts, int npatch,
                        reflux_edge* out)
{
    int n = 0;
    for (int p = 0; p < npatch; p++) {
        const mcref_amr_patch* a = &pts[p];
        for (int side = 0; side < 4; side++) {
            const int len = side < 2 ? a->ch : a->cw;
            for (int k = 0; k < len; k++) {
                reflux_edge e;
                e.patch = p;
                if (side < 2) {
                    e.dir = 0;
                    e.cj = a->cj0 + k;
                    e.ci = side == 0 ? a->ci0 : a->ci0 + a->cw;
                    e.oi = side == 0 ? a->ci0 - 1 : a->ci0 + a->cw;
                    e.oj = e.cj;
                    e.sgn = side == 0 ? 1 : -1;
                    e.fi = side == 0 ? 0 : ratio * a->cw;
                    e.fj = ratio * k;
                } else {
                    e.dir = 1;
                    e.ci = a->ci0 + k;
                    e.cj = side == 2 ? a->cj0 : a->cj0 + a->ch;
                    e.oi = e.ci;
                    e.oj = side == 2 ? a->cj0 - 1 : a->cj0 + a->ch;
                    e.sgn = side == 2 ? 1 : -1;
                    e.fi = ratio * k;
                    e.fj = side == 2 ? 0 : ratio * a->ch;
                }
                if (e.oi < 0 || e.oi >= pc->mx || e.oj < 0 || e.oj >= pc->my) continue;
                if (covered(pts, npatch, e.oi, e.oj)) continue;
                if (out) out[n] = e;
                n++;
            }
        }
    }
    return n;
}

int mcref_amr_step(const mcref_problem* pc, int ratio, const mcref_amr_patch* pts, int npatch,
                   const double* qc_in, double* qc_out, double** qf, double dt, int reflux,
                   int nthreads)
{
    int flags = 0;
    double smax;
    const int meqn = mcref_meqn(pc->solver);
    /* the coarse grid's step; its filled input is the time-interpolation base */
    const int64_t nc = (int64_t)mcref_nplane(pc->solver) * NXG(pc) * NYG(pc);
    double* qc0 = malloc(sizeof(double) * nc);
    memcpy(qc0, qc_in, sizeof(double) * nc);
    mcref_bc_fill(pc, qc0);
    /* refluxing: D = coarse flux - mean fine flux per corrected edge */
    const int ne = reflux ? reflux_edges(pc, ratio, pts, npatch, NULL) : 0;
    reflux_edge* edges = malloc(sizeof(reflux_edge) * (ne > 0 ? ne : 1));
    double* D = calloc((size_t)(ne > 0 ? ne : 1) * meqn, sizeof(double));
    if (ne > 0) reflux_edges(pc, ratio, pts, npatch, edges);
    for (int k = 0; k < ne; k++) mcref_edge_flux(pc, qc0, dt, edges[k].dir, edges[k].ci, edges[k].cj, D + k * meqn);
    flags |= mcref_step(pc, qc0, qc_out, dt, &smax, nthreads);
    /* r fine steps of every patch */
    double** tmp = malloc(sizeof(double*) * (npatch > 0 ? npatch : 1));
    for (int p = 0; p < npatch; p++) {
        mcref_problem pf;
        mcref_fine_problem(pc, ratio, &pts[p], &pf);
        tmp[p] = malloc(sizeof(double) * (int64_t)mcref_nplane(pf.solver) * NXG(&pf) * NYG(&pf));
    }
    for (int s = 0; s < ratio; s++) {
        mcref_amr_fill_ghosts(pc, ratio, qc0, qc_out, (double)s / ratio, pts, npatch, qf);
        for (int k = 0; k < ne; k++) {
            /* the ratio fine edges along coarse edge k, each weighted by
             * (dt/r)(d/r) / (dt d) */
            mcref_problem pf;
            mcref_fine_problem(pc, ratio, &pts[edges[k].patch], &pf);
            for (int t = 0; t < ratio; t++) {
                double Ff[MCREF_MAXEQN];
                const int fi = edges[k].fi + (edges[k].dir == 1 ? t : 0);
                const int fj = edges[k].fj + (edges[k].dir == 0 ? t : 0);
                mcref_edge_flux(&pf, qf[edges[k].patch], dt / ratio, edges[k].dir, fi, fj, Ff);
                for (int m = 0; m < meqn; m++) D[k * meqn + m] -= Ff[m] / ((double)ratio * ratio);
            }
        }
        for (int p = 0; p < npatch; p++) {
            mcref_problem pf;
            mcref_fine_problem(pc, ratio, &pts[p], &pf);
            flags |= mcref_step(&pf, qf[p], tmp[p], dt / ratio, &smax, nthreads);
        }
        for (int p = 0; p < npatch; p++) {
            mcref_problem pf;
            mcref_fine_problem(pc, ratio, &pts[p], &pf);
            memcpy(qf[p], tmp[p], sizeof(double) * (int64_t)mcref_nplane(pf.solver) * NXG(&pf) * NYG(&pf));
        }
    }
    mcref_amr_average_down(pc, ratio, pts, npatch, qf, qc_out);
    /* the outside cells: their update used the coarse flux through the edge */
    for (int k = 0; k < ne; k++) {
        const double dtd = dt / (edges[k].dir == 0 ? pc->dx : pc->dy);
        for (int m = 0; m < meqn; m++)
            qc_out[idx(pc, m, edges[k].oi, edges[k].oj)] += edges[k].sgn * dtd * D[k * meqn + m];
    }
    mcref_bc_fill(pc, qc_out);
    free(edges);
    free(D);
    for (int p = 0; p < npatch; p++) free(tmp[p]);
    free(tmp);
    free(qc0);
    return flags;
}
