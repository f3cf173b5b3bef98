/*
 * exact.c -- the oracle's exact Riemann solver for the 1D Euler equations.
 *
 * TEST INFRASTRUCTURE ONLY (see mcref.h).
 *
 * The paper names Euler among its Riemann kernels (§3, Table 2, Table 3) but
 * gives no solver formulas.  The exact solver is restated from Toro,
 * "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4: the
 * star pressure p* is the root of
 *     f(p) = f_L(p) + f_R(p) + (u_R - u_L),
 * with f_K the shock branch (Rankine-Hugoniot) for p > p_K and the
 * rarefaction branch (isentropic) otherwise, found by Newton's method from a
 * pressure guess; u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.  The guesses
 * are Toro's primitive-variable (PVRS), two-rarefaction (TR) and two-shock
 * (TS) approximations and his adaptive choice between them (§9.5).
 *
 * Convergence test: |p_{k+1} - p_k| / p_{k+1} < tol.  An iteration is one
 * Newton update.
 */
#include <math.h>
#include <stdlib.h>
#include "mcref.h"

static double sound(double gamma, double rho, double p)
{
    return sqrt(gamma * p / rho);
}

/* one side's branch of the pressure function and its derivative */
static void fK(double gamma, double p, double rK, double pK, double cK, double* f, double* fd)
{
    if (p > pK) {
        double A = 2.0 / ((gamma + 1.0) * rK);
        double B = (gamma - 1.0) / (gamma + 1.0) * pK;
        double q = sqrt(A / (B + p));
        *f = (p - pK) * q;
        *fd = q * (1.0 - 0.5 * (p - pK) / (B + p));
    } else {
        double pr = p / pK;
        *f = 2.0 * cK / (gamma - 1.0) * (pow(pr, 0.5 * (gamma - 1.0) / gamma) - 1.0);
        *fd = 1.0 / (rK * cK) * pow(pr, -0.5 * (gamma + 1.0) / gamma);
    }
}

void mcref_pressure_function(double gamma, double rl, double ul, double pl,
                             double rr, double ur, double pr, double p,
                             double* f, double* fd)
{
    double fl, fdl, fr, fdr;
    fK(gamma, p, rl, pl, sound(gamma, rl, pl), &fl, &fdl);
    fK(gamma, p, rr, pr, sound(gamma, rr, pr), &fr, &fdr);
    *f = fl + fr + (ur - ul);
    *fd = fdl + fdr;
}

static const double PFLOOR = 1e-12;

double mcref_seed(int mode, double gamma, double rl, double ul, double pl,
                  double rr, double ur, double pr)
{
    const double cl = sound(gamma, rl, pl), cr = sound(gamma, rr, pr);
    const double du = ur - ul;
    const double z = 0.5 * (gamma - 1.0) / gamma;
    double ppv = 0.5 * (pl + pr) - 0.125 * du * (rl + rr) * (cl + cr);
    if (ppv < PFLOOR) ppv = PFLOOR;
    double ptr = pow((cl + cr - 0.5 * (gamma - 1.0) * du) / (cl / pow(pl, z) + cr / pow(pr, z)), 1.0 / z);
    double gl = sqrt(2.0 / ((gamma + 1.0) * rl) / ((gamma - 1.0) / (gamma + 1.0) * pl + ppv));
    double gr = sqrt(2.0 / ((gamma + 1.0) * rr) / ((gamma - 1.0) / (gamma + 1.0) * pr + ppv));
    double pts = (gl * pl + gr * pr - du) / (gl + gr);
    if (pts < PFLOOR) pts = PFLOOR;
    const double pmin = pl < pr ? pl : pr, pmax = pl < pr ? pr : pl;
    switch (mode) {
    case MCREF_SEED_PV: return ppv;
    case MCREF_SEED_TR: return ptr;
    case MCREF_SEED_TS: return pts;
    case MCREF_SEED_PVTR:
        return (pmax / pmin < 2.0 && ppv >= pmin && ppv <= pmax) ? ppv : ptr;
    default:
        if (pmax / pmin < 2.0 && ppv >= pmin && ppv <= pmax) return ppv;
        if (ppv < pmin) return ptr;
        return pts;
    }
}

static int is_vacuum(double gamma, double rl, double ul, double pl, double rr, double ur, double pr)
{
    double cl = sound(gamma, rl, pl), cr = sound(gamma, rr, pr);
    return 2.0 / (gamma - 1.0) * (cl + cr) <= ur - ul;
}

/* Newton from p0; returns 1 on convergence.  *iters is incremented per
 * update. */
static int newton(double gamma, double rl, double ul, double pl, double rr, double ur, double pr,
                  double p0, double tol, int max_iter, double* pstar, int* iters)
{
    double p = p0;
    for (int k = 0; k < max_iter; k++) {
        double f, fd;
        mcref_pressure_function(gamma, rl, ul, pl, rr, ur, pr, p, &f, &fd);
        double pn = p - f / fd;
        if (pn < PFLOOR) pn = PFLOOR;
        (*iters)++;
        if (!isfinite(pn)) return 0;
        if (fabs(pn - p) / pn < tol) {
            *pstar = pn;
            return 1;
        }
        p = pn;
    }
    *pstar = p;
    return 0;
}

static double star_velocity(double gamma, double rl, double ul, double pl, double rr, double ur,
                            double pr, double ps)
{
    double fl, fdl, fr, fdr;
    fK(gamma, ps, rl, pl, sound(gamma, rl, pl), &fl, &fdl);
    fK(gamma, ps, rr, pr, sound(gamma, rr, pr), &fr, &fdr);
    return 0.5 * (ul + ur) + 0.5 * (fr - fl);
}

int mcref_exact_riemann(double gamma, double rl, double ul, double pl,
                        double rr, double ur, double pr, int seed_mode, double p_given,
                        double tol, int max_iter, double* pstar, double* ustar, int* iters)
{
    *iters = 0;
    if (is_vacuum(gamma, rl, ul, pl, rr, ur, pr)) {
        *pstar = 0.0;
        *ustar = NAN;
        return MCREF_RS_VACUUM;
    }
    int flag = MCREF_RS_OK;
    double ps = 0.0;
    if (seed_mode == MCREF_SEED_GIVEN) {
        const double pmin = pl < pr ? pl : pr, pmax = pl < pr ? pr : pl;
        int physical = isfinite(p_given) && p_given >= 1e-6 * pmin && p_given <= 1e6 * pmax;
        if (physical && newton(gamma, rl, ul, pl, rr, ur, pr, p_given, tol, max_iter, &ps, iters)) {
            *pstar = ps;
            *ustar = star_velocity(gamma, rl, ul, pl, rr, ur, pr, ps);
            return flag;
        }
        flag |= MCREF_RS_FALLBACK;
        seed_mode = MCREF_SEED_ADAPTIVE;
    }
    double p0 = mcref_seed(seed_mode, gamma, rl, ul, pl, rr, ur, pr);
    if (!newton(gamma, rl, ul, pl, rr, ur, pr, p0, tol, max_iter, &ps, iters)) flag |= MCREF_RS_NOCONV;
    *pstar = ps;
    *ustar = star_velocity(gamma, rl, ul, pl, rr, ur, pr, ps);
    return flag;
}

/* Bisection on the monotone pressure function, for pinning Newton. */
int mcref_exact_bisect(double gamma, double rl, double ul, double pl,
                       double rr, double ur, double pr, double* pstar, double* ustar)
{
    if (is_vacuum(gamma, rl, ul, pl, rr, ur, pr)) {
        *pstar = 0.0;
        *ustar = NAN;
        return MCREF_RS_VACUUM;
    }
    double lo = 0.0, hi = pl > pr ? pl : pr, f, fd;
    for (;;) {
        mcref_pressure_function(gamma, rl, ul, pl, rr, ur, pr, hi, &f, &fd);
        if (f > 0.0) break;
        lo = hi;
        hi *= 2.0;
    }
    for (int k = 0; k < 400; k++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        mcref_pressure_function(gamma, rl, ul, pl, rr, ur, pr, mid, &f, &fd);
        if (f > 0.0) hi = mid;
        else lo = mid;
    }
    *pstar = 0.5 * (lo + hi);
    *ustar = star_velocity(gamma, rl, ul, pl, rr, ur, pr, *pstar);
    return MCREF_RS_OK;
}

void mcref_exact_batch(int64_t n, double gamma, const double* rl, const double* ul,
                       const double* pl, const double* rr, const double* ur, const double* pr,
                       int seed_mode, const double* p_given, double tol, int max_iter,
                       double* pstar, double* ustar, int32_t* iters, int32_t* flags,
                       int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t k = 0; k < n; k++) {
        int it = 0;
        flags[k] = mcref_exact_riemann(gamma, rl[k], ul[k], pl[k], rr[k], ur[k], pr[k], seed_mode,
                                       p_given ? p_given[k] : 0.0, tol, max_iter, &pstar[k],
                                       &ustar[k], &it);
        iters[k] = it;
    }
}


/* ------------------------------------------------------------------ */
/* Godunov normal solve with the exact solution (Toro ch. 4)           */
/* ------------------------------------------------------------------ */

/* Star-region density behind the wave facing side K: Rankine-Hugoniot for a
 * shock (p* > p_K, Toro eq. 4.50), isentropic for a rarefaction (eq. 4.53). */
static double star_density(double gamma, double rK, double pK, double ps)
{
    const double r = ps / pK;
    if (ps > pK) {
        const double g6 = (gamma - 1.0) / (gamma + 1.0);
        return rK * (r + g6) / (g6 * r + 1.0);
    }
    return rK * pow(r, 1.0 / gamma);
}

/* Speed of the shock facing side K (sgn = -1 left, +1 right; Toro eq. 4.52). */
static double shock_speed(double gamma, double uK, double pK, double cK, double ps, double sgn)
{
    return uK + sgn * cK * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pK + (gamma - 1.0) / (2.0 * gamma));
}

void mcref_exact_sample(double gamma, double rl, double ul, double pl, double rr, double ur,
                        double pr, double pstar, double ustar, double* rho0, double* u0, double* p0)
{
    /* Toro §4.5 at x/t = 0.  The side of the contact that contains the
     * interface is the left one if u* >= 0; the mirror image handles the
     * right side (sgn = +1 flips velocities of the left-side formulas). */
    const int left = ustar >= 0.0;
    const double rK = left ? rl : rr, pK = left ? pl : pr;
    const double sgn = left ? -1.0 : 1.0;          /* wave facing side K travels in direction sgn */
    const double uK = left ? ul : ur;
    const double cK = sound(gamma, rK, pK);
    if (pstar > pK) {
        const double S = shock_speed(gamma, uK, pK, cK, pstar, sgn);
        if ((left && S >= 0.0) || (!left && S <= 0.0)) {
            *rho0 = rK; *u0 = uK; *p0 = pK;
        } else {
            *rho0 = star_density(gamma, rK, pK, pstar); *u0 = ustar; *p0 = pstar;
        }
        return;
    }
    const double head = uK + sgn * cK;
    const double cs = cK * pow(pstar / pK, 0.5 * (gamma - 1.0) / gamma);
    const double tail = ustar + sgn * cs;
    if ((left && head >= 0.0) || (!left && head <= 0.0)) {
        *rho0 = rK; *u0 = uK; *p0 = pK;
    } else if ((left && tail <= 0.0) || (!left && tail >= 0.0)) {
        *rho0 = star_density(gamma, rK, pK, pstar); *u0 = ustar; *p0 = pstar;
    } else {
        /* inside the fan, at x/t = 0 (Toro eq. 4.56 / 4.63 with S = 0) */
        const double c = 2.0 / (gamma + 1.0) * (cK - sgn * 0.5 * (gamma - 1.0) * uK);
        *u0 = -sgn * c;
        *rho0 = rK * pow(c / cK, 2.0 / (gamma - 1.0));
        *p0 = pK * pow(c / cK, 2.0 * gamma / (gamma - 1.0));
    }
}

/* conserved vector of (rho, u_n, u_t, p) on the edge of normal dir */
static void conserved(double gamma, int dir, double rho, double un, double ut, double pr, double* q)
{
    const int mu = 1 + dir, mv = 2 - dir;
    q[0] = rho;
    q[mu] = rho * un;
    q[mv] = rho * ut;
    q[3] = pr / (gamma - 1.0) + 0.5 * rho * (un * un + ut * ut);
}

int mcref_godunov_rpn2(const mcref_problem* p, int dir, const double* ql, const double* qr,
                       double* wave, double* s, double* amdq, double* apdq)
{
    const int mu = 1 + dir, mv = 2 - dir;
    const double gamma = p->param[0];
    for (int k = 0; k < 12; k++) wave[k] = 0.0;
    for (int k = 0; k < 3; k++) s[k] = 0.0;
    for (int m = 0; m < 4; m++) amdq[m] = apdq[m] = 0.0;
    if (!(ql[0] > 0.0 && qr[0] > 0.0)) return MCREF_F_NONPHYS;
    const double rl = ql[0], ul = ql[mu] / rl, vl = ql[mv] / rl;
    const double rr = qr[0], ur = qr[mu] / rr, vr = qr[mv] / rr;
    const double pl = (gamma - 1.0) * (ql[3] - 0.5 * rl * (ul * ul + vl * vl));
    const double pr = (gamma - 1.0) * (qr[3] - 0.5 * rr * (ur * ur + vr * vr));
    if (!(pl > 0.0 && pr > 0.0)) return MCREF_F_NONPHYS;
    double ps, us;
    int it;
    int fl = mcref_exact_riemann(gamma, rl, ul, pl, rr, ur, pr, MCREF_SEED_ADAPTIVE, 0.0, 1e-14, 100,
                                 &ps, &us, &it);
    if (fl & MCREF_RS_VACUUM) return MCREF_F_NONPHYS;
    if (fl & MCREF_RS_NOCONV) mcref_exact_bisect(gamma, rl, ul, pl, rr, ur, pr, &ps, &us);
    const double cl = sound(gamma, rl, pl), cr = sound(gamma, rr, pr);
    /* states on either side of the contact, and the jumps across the waves */
    double qsl[4], qsr[4];
    conserved(gamma, dir, star_density(gamma, rl, pl, ps), us, vl, ps, qsl);
    conserved(gamma, dir, star_density(gamma, rr, pr, ps), us, vr, ps, qsr);
    for (int m = 0; m < 4; m++) {
        wave[m] = qsl[m] - ql[m];
        wave[4 + m] = qsr[m] - qsl[m];
        wave[8 + m] = qr[m] - qsr[m];
    }
    /* wave speeds: the shock speed, or a rarefaction's head (its fastest
     * signal), the contact at u* */
    s[0] = ps > pl ? shock_speed(gamma, ul, pl, cl, ps, -1.0) : ul - cl;
    s[1] = us;
    s[2] = ps > pr ? shock_speed(gamma, ur, pr, cr, ps, 1.0) : ur + cr;
    /* fluctuations: flux differences to the interface state */
    double r0, u0, p0, q0[4], f0[4], fl_[4], fr_[4];
    mcref_exact_sample(gamma, rl, ul, pl, rr, ur, pr, ps, us, &r0, &u0, &p0);
    conserved(gamma, dir, r0, u0, us >= 0.0 ? vl : vr, p0, q0);
    mcref_flux(p, dir, q0, f0);
    mcref_flux(p, dir, ql, fl_);
    mcref_flux(p, dir, qr, fr_);
    for (int m = 0; m < 4; m++) {
        amdq[m] = f0[m] - fl_[m];
        apdq[m] = fr_[m] - f0[m];
    }
    return 0;
}
