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
