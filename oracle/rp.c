/*
 * rp.c -- pointwise Riemann solvers and limiter functions of the oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see mcref.h).
 *
 * The paper (§1.1, §2) treats the Riemann problem as a pointwise kernel that
 * maps the states of two adjacent cells to waves, speeds and fluctuations at
 * their common edge, and defers the formulas to Clawpack.  The formulas here
 * are restated from LeVeque (2002): acoustics eigenstructure (§3.9, §18.9),
 * Roe linearisations for shallow water (§15.3.3) and Euler (§15.3.4),
 * Harten-Hyman entropy fix (§15.3.5), wave limiters (§6.9-6.12) and the
 * transverse split used by the 2D unsplit method (§21.2).
 *
 * Index convention: for an edge whose normal is direction dir (0 = x,
 * 1 = y) the normal momentum/velocity component is mu = 1 + dir and the
 * tangential one is mv = 2 - dir.
 */
#include <math.h>
#include <string.h>
#include "mcref.h"

int mcref_meqn(int solver)
{
    if (solver == MCREF_EULER || solver == MCREF_EULER_GODUNOV) return 4;
    return solver == MCREF_ADVECTION ? 1 : 3;
}

int mcref_nplane(int solver)
{
    return mcref_meqn(solver) + (solver == MCREF_ACOUSTICS_VAR ? 2 : 0);
}

int mcref_mwaves(int solver)
{
    /* acoustics: the zero-speed wave carrying the tangential velocity jump
     * produces no fluctuation and no correction, so it is not carried.
     * Euler: entropy and shear waves travel at the same speed and are
     * carried as one wave. */
    if (solver == MCREF_ADVECTION) return 1;
    return (solver == MCREF_ACOUSTICS || solver == MCREF_ACOUSTICS_VAR) ? 2 : 3;
}

/* ------------------------------------------------------------------ */
/* Linearised state of an edge and its eigen-decomposition             */
/* ------------------------------------------------------------------ */

typedef struct {
    double un, ut;  /* Roe-averaged normal / tangential velocity */
    double c;       /* Roe-averaged sound (or gravity-wave) speed */
    double H;       /* Roe-averaged total enthalpy (Euler only) */
    int ok;
} roe_state;

static roe_state roe_average(const mcref_problem* p, int dir, const double* ql, const double* qr)
{
    const int mu = 1 + dir, mv = 2 - dir;
    roe_state r = {0, 0, 0, 0, 1};
    if (p->solver == MCREF_ACOUSTICS) {
        r.c = sqrt(p->param[1] / p->param[0]);
        return r;
    }
    if (ql[0] <= 0.0 || qr[0] <= 0.0) {
        r.ok = 0;
        return r;
    }
    double sl = sqrt(ql[0]), sr = sqrt(qr[0]);
    double ul = ql[mu] / ql[0], ur = qr[mu] / qr[0];
    double vl = ql[mv] / ql[0], vr = qr[mv] / qr[0];
    r.un = (sl * ul + sr * ur) / (sl + sr);
    r.ut = (sl * vl + sr * vr) / (sl + sr);
    if (p->solver == MCREF_SWE) {
        double g = p->param[0];
        r.c = sqrt(g * 0.5 * (ql[0] + qr[0]));
    } else {
        double gam = p->param[0];
        double pl = (gam - 1.0) * (ql[3] - 0.5 * ql[0] * (ul * ul + vl * vl));
        double pr = (gam - 1.0) * (qr[3] - 0.5 * qr[0] * (ur * ur + vr * vr));
        double Hl = (ql[3] + pl) / ql[0], Hr = (qr[3] + pr) / qr[0];
        r.H = (sl * Hl + sr * Hr) / (sl + sr);
        double c2 = (gam - 1.0) * (r.H - 0.5 * (r.un * r.un + r.ut * r.ut));
        if (!(c2 > 0.0)) {
            r.ok = 0;
            return r;
        }
        r.c = sqrt(c2);
    }
    return r;
}

/*
 * Eigen-decomposition of a vector d in direction dir at the linearised
 * state st, where st.un is the velocity NORMAL to dir and st.ut the one
 * tangential to dir.  Produces nw eigen-pieces vec[k] (meqn each) with
 * speeds lam[k]; sum_k vec[k] == d.  For Euler the last two pieces share a
 * speed (entropy and shear) and are returned separately here (nw = 4); the
 * normal solver merges them.
 */
static int eig_split(const mcref_problem* p, int dir, const roe_state* st, const double* d,
                     double vec[4][MCREF_MAXEQN], double* lam)
{
    const int mu = 1 + dir, mv = 2 - dir;
    const double u = st->un, v = st->ut, c = st->c;
    memset(vec, 0, sizeof(double) * 4 * MCREF_MAXEQN);
    if (p->solver == MCREF_ACOUSTICS) {
        const double Z = p->param[0] * c;
        /* eigenvectors (p, u_n) = (-Z, 1) for speed -c and (Z, 1) for +c */
        double a1 = (-d[0] + Z * d[mu]) / (2.0 * Z);
        double a2 = (d[0] + Z * d[mu]) / (2.0 * Z);
        vec[0][0] = -Z * a1; vec[0][mu] = a1; lam[0] = -c;
        vec[1][0] = Z * a2;  vec[1][mu] = a2; lam[1] = c;
        return 2;
    }
    if (p->solver == MCREF_SWE) {
        /* r1 = (1, u-c, v), r2 = (0, 0, 1), r3 = (1, u+c, v) in (h, m_n, m_t) */
        double a1 = ((u + c) * d[0] - d[mu]) / (2.0 * c);
        double a2 = d[mv] - v * d[0];
        double a3 = (d[mu] - (u - c) * d[0]) / (2.0 * c);
        vec[0][0] = a1; vec[0][mu] = a1 * (u - c); vec[0][mv] = a1 * v; lam[0] = u - c;
        vec[1][mv] = a2;                                                lam[1] = u;
        vec[2][0] = a3; vec[2][mu] = a3 * (u + c); vec[2][mv] = a3 * v; lam[2] = u + c;
        return 3;
    }
    /* Euler: r1 = (1, u-c, v, H-uc), r_ent = (1, u, v, (u^2+v^2)/2),
     * r_shear = (0, 0, 1, v), r4 = (1, u+c, v, H+uc) in (rho, m_n, m_t, E). */
    {
        const double gm1 = p->param[0] - 1.0, H = st->H;
        double a_sh = d[mv] - v * d[0];
        double a_en = gm1 / (c * c) * ((H - u * u - v * v) * d[0] + u * d[mu] + v * d[mv] - d[3]);
        double a4 = 0.5 * (d[0] - a_en + (d[mu] - u * d[0]) / c);
        double a1 = 0.5 * (d[0] - a_en - (d[mu] - u * d[0]) / c);
        vec[0][0] = a1; vec[0][mu] = a1 * (u - c); vec[0][mv] = a1 * v; vec[0][3] = a1 * (H - u * c);
        lam[0] = u - c;
        vec[1][0] = a_en; vec[1][mu] = a_en * u; vec[1][mv] = a_en * v;
        vec[1][3] = a_en * 0.5 * (u * u + v * v);
        lam[1] = u;
        vec[2][mv] = a_sh; vec[2][3] = a_sh * v;
        lam[2] = u;
        vec[3][0] = a4; vec[3][mu] = a4 * (u + c); vec[3][mv] = a4 * v; vec[3][3] = a4 * (H + u * c);
        lam[3] = u + c;
        return 4;
    }
}

/* Characteristic speed u_n - c (sgn = -1) or u_n + c (sgn = +1) of a cell
 * state; returns 0 if the state is not physical. */
static int char_speed(const mcref_problem* p, int dir, const double* q, int sgn, double* lam)
{
    const int mu = 1 + dir, mv = 2 - dir;
    if (!(q[0] > 0.0)) return 0;
    double un = q[mu] / q[0];
    double c;
    if (p->solver == MCREF_SWE) {
        c = sqrt(p->param[0] * q[0]);
    } else {
        double ut = q[mv] / q[0];
        double pr = (p->param[0] - 1.0) * (q[3] - 0.5 * q[0] * (un * un + ut * ut));
        if (!(pr > 0.0)) return 0;
        c = sqrt(p->param[0] * pr / q[0]);
    }
    *lam = un + sgn * c;
    return 1;
}

int mcref_rpn2(const mcref_problem* p, int dir, const double* ql, const double* qr,
               double* wave, double* s, double* amdq, double* apdq)
{
    const int meqn = mcref_meqn(p->solver), mw = mcref_mwaves(p->solver);
    double d[MCREF_MAXEQN], vec[4][MCREF_MAXEQN], lam[4];
    int flags = 0;
    if (p->solver == MCREF_EULER_GODUNOV) return mcref_godunov_rpn2(p, dir, ql, qr, wave, s, amdq, apdq);
    for (int m = 0; m < meqn; m++) d[m] = qr[m] - ql[m];
    if (p->solver == MCREF_ADVECTION) {
        /* one wave, the jump, moving at the velocity normal to the edge
         * (LeVeque 2002, §4.8 and §20.1) */
        const double sn = p->param[dir];
        wave[0] = d[0];
        s[0] = sn;
        amdq[0] = (sn < 0.0 ? sn : 0.0) * d[0];
        apdq[0] = (sn > 0.0 ? sn : 0.0) * d[0];
        return 0;
    }
    if (p->solver == MCREF_ACOUSTICS_VAR) {
        /* LeVeque (2002) §9.6: the left-going wave lies along the left
         * medium's eigenvector (-Z_l, 1, 0) at speed -c_l, the right-going one
         * along the right medium's (Z_r, 1, 0) at speed +c_r; the two
         * strengths follow from the jump in p and the normal velocity. */
        const int un = 1 + dir, ut = 2 - dir;
        const double zl = ql[3] * ql[4], zr = qr[3] * qr[4];
        const double a1 = (-d[0] + zr * d[un]) / (zl + zr);
        const double a2 = (d[0] + zl * d[un]) / (zl + zr);
        double* w1 = wave;
        double* w2 = wave + meqn;
        w1[0] = -zl * a1; w1[un] = a1; w1[ut] = 0.0;
        w2[0] = zr * a2;  w2[un] = a2; w2[ut] = 0.0;
        s[0] = -ql[4];
        s[1] = qr[4];
        for (int m = 0; m < meqn; m++) {
            amdq[m] = s[0] * w1[m];
            apdq[m] = s[1] * w2[m];
        }
        return 0;
    }
    roe_state st = roe_average(p, dir, ql, qr);
    if (!st.ok) {
        /* Non-physical input: report it and return zero waves. */
        memset(wave, 0, sizeof(double) * mw * meqn);
        memset(s, 0, sizeof(double) * mw);
        memset(amdq, 0, sizeof(double) * meqn);
        memset(apdq, 0, sizeof(double) * meqn);
        return MCREF_F_NONPHYS;
    }
    int nv = eig_split(p, dir, &st, d, vec, lam);
    if (p->solver == MCREF_EULER) {
        /* merge entropy and shear pieces into the middle wave */
        for (int m = 0; m < meqn; m++) vec[1][m] += vec[2][m];
        for (int m = 0; m < meqn; m++) vec[2][m] = vec[3][m];
        lam[2] = lam[3];
        nv = 3;
    }
    for (int w = 0; w < nv; w++) {
        s[w] = lam[w];
        for (int m = 0; m < meqn; m++) wave[w * meqn + m] = vec[w][m];
    }

    /* fluctuations: left-going part of every wave */
    for (int m = 0; m < meqn; m++) amdq[m] = 0.0;
    for (int w = 0; w < mw; w++) {
        double coef = s[w] < 0.0 ? s[w] : 0.0;
        if (p->efix && p->solver != MCREF_ACOUSTICS && (w == 0 || w == mw - 1)) {
            /* Harten-Hyman: speeds on either side of a nonlinear wave */
            double qm[MCREF_MAXEQN], lam_l, lam_r;
            int okl, okr;
            if (w == 0) {
                for (int m = 0; m < meqn; m++) qm[m] = ql[m] + wave[m];
                okl = char_speed(p, dir, ql, -1, &lam_l);
                okr = char_speed(p, dir, qm, -1, &lam_r);
            } else {
                for (int m = 0; m < meqn; m++) qm[m] = qr[m] - wave[w * meqn + m];
                okl = char_speed(p, dir, qm, +1, &lam_l);
                okr = char_speed(p, dir, qr, +1, &lam_r);
            }
            if (!(okl && okr)) {
                flags |= MCREF_F_NONPHYS;
            } else if (lam_l < 0.0 && lam_r > 0.0) {
                double beta = (lam_r - s[w]) / (lam_r - lam_l);
                coef = beta * lam_l;
            }
        }
        for (int m = 0; m < meqn; m++) amdq[m] += coef * wave[w * meqn + m];
    }
    /* right-going part: the rest of sum_p s^p W^p, so amdq + apdq equals the
     * linearised flux difference whether or not the fix changed amdq */
    for (int m = 0; m < meqn; m++) {
        double tot = 0.0;
        for (int w = 0; w < mw; w++) tot += s[w] * wave[w * meqn + m];
        apdq[m] = tot - amdq[m];
    }
    return flags;
}

int mcref_rpt2(const mcref_problem* p, int dir, const double* ql, const double* qr,
               const double* asdq, double* bmasdq, double* bpasdq)
{
    const int meqn = mcref_meqn(p->solver);
    double vec[4][MCREF_MAXEQN], lam[4];
    if (p->solver == MCREF_ACOUSTICS_VAR) {
        /* needs the receiving cell and its neighbours: mcref_rpt2_var */
        for (int m = 0; m < meqn; m++) bmasdq[m] = bpasdq[m] = 0.0;
        return MCREF_F_NONPHYS;
    }
    if (p->solver == MCREF_ADVECTION) {
        /* the transverse velocity carries the whole fluctuation (§20.2) */
        const double st = p->param[1 - dir];
        bmasdq[0] = (st < 0.0 ? st : 0.0) * asdq[0];
        bpasdq[0] = (st > 0.0 ? st : 0.0) * asdq[0];
        return 0;
    }
    roe_state st = roe_average(p, dir, ql, qr);
    for (int m = 0; m < meqn; m++) bmasdq[m] = bpasdq[m] = 0.0;
    if (!st.ok) return MCREF_F_NONPHYS;
    /* decompose in the transverse direction: the roles of the normal and
     * tangential velocities swap */
    roe_state tr = st;
    tr.un = st.ut;
    tr.ut = st.un;
    int nv = eig_split(p, 1 - dir, &tr, asdq, vec, lam);
    for (int w = 0; w < nv; w++) {
        double lm = lam[w] < 0.0 ? lam[w] : 0.0;
        double lp = lam[w] > 0.0 ? lam[w] : 0.0;
        for (int m = 0; m < meqn; m++) {
            bmasdq[m] += lm * vec[w][m];
            bpasdq[m] += lp * vec[w][m];
        }
    }
    return 0;
}

int mcref_rpt2_var(const mcref_problem* p, int dir, const double* qlo, const double* qc,
                   const double* qhi, const double* asdq, double* bmasdq, double* bpasdq)
{
    /* LeVeque (2002) §21.x for heterogeneous acoustics: the part of asdq
     * that moves toward qlo is its component along qlo's medium eigenvector
     * (-Z_lo, 1) (velocity along the split direction) in the decomposition
     * at the interface between qlo and qc, times -c_lo; the part moving
     * toward qhi is its component along (Z_hi, 1) at the interface between
     * qc and qhi, times +c_hi.  Reflections at the two interfaces are why
     * the parts do not add up to B asdq. */
    (void)p;
    const int vn = 2 - dir, vt = 1 + dir;   /* velocity along / across the split direction */
    const double zlo = qlo[3] * qlo[4], z = qc[3] * qc[4], zhi = qhi[3] * qhi[4];
    const double bdown = (-asdq[0] + z * asdq[vn]) / (zlo + z);
    const double bup = (asdq[0] + z * asdq[vn]) / (z + zhi);
    bmasdq[0] = qlo[4] * zlo * bdown;
    bmasdq[vn] = -qlo[4] * bdown;
    bmasdq[vt] = 0.0;
    bpasdq[0] = qhi[4] * zhi * bup;
    bpasdq[vn] = qhi[4] * bup;
    bpasdq[vt] = 0.0;
    return 0;
}

void mcref_flux(const mcref_problem* p, int dir, const double* q, double* f)
{
    const int mu = 1 + dir, mv = 2 - dir;
    if (p->solver == MCREF_ACOUSTICS_VAR) {
        /* p_t + K div u = 0, u_t + grad p / rho = 0 with the cell's own
         * material, K = rho c^2 */
        const double rho = q[3], K = q[3] * q[4] * q[4];
        f[0] = K * q[mu];
        f[mu] = q[0] / rho;
        f[mv] = 0.0;
        return;
    }
    if (p->solver == MCREF_ADVECTION) {
        f[0] = p->param[dir] * q[0];
        return;
    }
    if (p->solver == MCREF_ACOUSTICS) {
        double rho = p->param[0], K = p->param[1];
        f[0] = K * q[mu];
        f[mu] = q[0] / rho;
        f[mv] = 0.0;
        return;
    }
    double un = q[mu] / q[0];
    if (p->solver == MCREF_SWE) {
        double g = p->param[0];
        f[0] = q[mu];
        f[mu] = q[mu] * un + 0.5 * g * q[0] * q[0];
        f[mv] = q[mv] * un;
        return;
    }
    double ut = q[mv] / q[0];
    double pr = (p->param[0] - 1.0) * (q[3] - 0.5 * q[0] * (un * un + ut * ut));
    f[0] = q[mu];
    f[mu] = q[mu] * un + pr;
    f[mv] = q[mv] * un;
    f[3] = (q[3] + pr) * un;
}

double mcref_philim(int limiter, double theta)
{
    switch (limiter) {
    case MCREF_LIM_MINMOD: {
        double a = theta < 1.0 ? theta : 1.0;
        return a > 0.0 ? a : 0.0;
    }
    case MCREF_LIM_SUPERBEE: {
        /* max(0, min(1, 2 theta), min(2, theta)) */
        double a = 2.0 * theta < 1.0 ? 2.0 * theta : 1.0;
        double b = theta < 2.0 ? theta : 2.0;
        double c = a > b ? a : b;
        return c > 0.0 ? c : 0.0;
    }
    case MCREF_LIM_VANLEER: {
        /* (theta + |theta|) / (1 + |theta|) */
        double at = fabs(theta);
        return (theta + at) / (1.0 + at);
    }
    case MCREF_LIM_MC: {
        double a = 0.5 * (1.0 + theta);
        if (2.0 < a) a = 2.0;
        if (2.0 * theta < a) a = 2.0 * theta;
        return a > 0.0 ? a : 0.0;
    }
    default:
        return 1.0;
    }
}
