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
 * Coarse-fine flux correction (refluxing) is not part of this coupling.
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

int mcref_amr_step(const mcref_problem* pc, int ratio, const mcref_amr_patch* pts, int npatch,
                   const double* qc_in, double* qc_out, double** qf, double dt, int nthreads)
{
    int flags = 0;
    double smax;
    /* the coarse grid's step; its filled input is the time-interpolation base */
    const int64_t nc = (int64_t)mcref_nplane(pc->solver) * NXG(pc) * NYG(pc);
    double* qc0 = malloc(sizeof(double) * nc);
    memcpy(qc0, qc_in, sizeof(double) * nc);
    mcref_bc_fill(pc, qc0);
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
    mcref_bc_fill(pc, qc_out);
    for (int p = 0; p < npatch; p++) free(tmp[p]);
    free(tmp);
    free(qc0);
    return flags;
}
