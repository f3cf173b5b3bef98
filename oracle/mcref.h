/*
 * mcref.h -- declarations of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, deliberately unfused
 * restatement of the wave-propagation method in double precision.  It is used
 * by the test-suite (parity and pins), by the smoke check and by the CPU
 * baseline leg of the benchmark.  The product library never includes, links
 * or calls anything in this directory, and this directory includes nothing
 * from the product library.
 *
 * Sources of the arithmetic (the paper describes the method in words only,
 * §1.1 and §1.2 with Table 1, and defers the formulas to Clawpack):
 *   - wave propagation, limiters, corner-transport (CTU) transverse terms:
 *     R. J. LeVeque, Finite Volume Methods for Hyperbolic Problems (2002),
 *     ch. 6 (limiters), ch. 15 (Roe solvers, Harten-Hyman entropy fix),
 *     ch. 19-21 (2D unsplit wave propagation with transverse splitting);
 *   - exact Euler Riemann solver, PVRS/TR/TS pressure guesses:
 *     E. F. Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics,
 *     ch. 4 (exact solver) and ch. 9 (approximate-state solvers).
 */
#ifndef MCREF_H
#define MCREF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* MCREF_ADVECTION: scalar q_t + u q_x + v q_y = 0 with constant (u, v) =
 * (param[0], param[1]) (the paper's advection solver, §3) */
/* MCREF_ACOUSTICS_VAR: acoustics with a density rho and sound speed c per
 * cell (the paper's variable-coefficient acoustics, §3, Table 2); the state
 * carries them as two extra planes after (p, u, v), which the step copies
 * unchanged. */
/* MCREF_EULER_GODUNOV: the Euler equations with the exact Riemann solution
 * (Toro ch. 4) in the normal solve instead of Roe's linearisation: the
 * fluctuations are flux differences to the state sampled at x/t = 0, the
 * waves are the jumps across the two nonlinear waves and the contact; the
 * transverse split stays Roe's. */
enum { MCREF_ACOUSTICS = 1, MCREF_SWE = 2, MCREF_EULER = 3, MCREF_ADVECTION = 4,
       MCREF_ACOUSTICS_VAR = 5, MCREF_EULER_GODUNOV = 6 };
/* Clawpack numbering: 1 minmod, 2 superbee, 3 van Leer, 4 monotonized central */
enum { MCREF_LIM_NONE = 0, MCREF_LIM_MINMOD = 1, MCREF_LIM_SUPERBEE = 2, MCREF_LIM_VANLEER = 3,
       MCREF_LIM_MC = 4 };
/* MCREF_BC_GIVEN leaves that side's ghost layers as the caller set them: the
 * step of a window cut out of a larger grid then uses the true neighbours. */
enum { MCREF_BC_PERIODIC = 0, MCREF_BC_EXTRAP = 1, MCREF_BC_WALL = 2, MCREF_BC_GIVEN = 3 };

/* Flags raised by the oracle (bitmask). */
enum { MCREF_F_NONPHYS = 1 };

#define MCREF_MAXEQN 5   /* planes of a cell vector: conserved fields + material */
#define MCREF_MAXWAVE 3

typedef struct {
    int solver;      /* MCREF_ACOUSTICS | MCREF_SWE | MCREF_EULER | MCREF_ADVECTION */
    int mx, my;      /* interior cells */
    int mbc;         /* ghost layers, 2 */
    double dx, dy;
    int limiter;     /* MCREF_LIM_* */
    int order;       /* 1: no second-order corrections, 2: limited corrections */
    int transverse;  /* 0: none, 1: transverse split of the fluctuations,
                      * 2: also of the limited corrections */
    int efix;        /* Harten-Hyman entropy fix on the nonlinear fields */
    int bc[4];       /* xlo, xhi, ylo, yhi */
    double param[4]; /* acoustics: rho, K | swe: g | euler: gamma | advection: u, v */
} mcref_problem;

int mcref_meqn(int solver);
/* planes of a state array: mcref_meqn conserved fields, then material planes */
int mcref_nplane(int solver);
int mcref_mwaves(int solver);

/* Pointwise normal Riemann solve across an edge whose normal is direction
 * dir (0 = x, 1 = y); ql is the cell on the low side.  Outputs waves
 * (mwaves x meqn, row-major), speeds, and the fluctuations.  Returns a
 * MCREF_F_* mask. */
int mcref_rpn2(const mcref_problem* p, int dir, const double* ql, const double* qr,
               double* wave, double* s, double* amdq, double* apdq);

/* Transverse split of a fluctuation asdq produced at an edge of normal dir:
 * asdq is decomposed in the eigenvectors of the other direction, taken at
 * the same linearised state as the normal solve of (ql, qr). */
int mcref_rpt2(const mcref_problem* p, int dir, const double* ql, const double* qr,
               const double* asdq, double* bmasdq, double* bpasdq);

/* Transverse split for variable-coefficient acoustics: asdq enters the cell
 * qc (an edge of normal dir), and qlo / qhi are that cell's neighbours on
 * either side in the other direction; the down- (left-) going part moves
 * into qlo's medium, the up- (right-) going part into qhi's.  Cell vectors
 * carry (p, u, v, rho, c). */
int mcref_rpt2_var(const mcref_problem* p, int dir, const double* qlo, const double* qc,
                   const double* qhi, const double* asdq, double* bmasdq, double* bpasdq);

/* Godunov normal solve of MCREF_EULER_GODUNOV (called by mcref_rpn2). */
int mcref_godunov_rpn2(const mcref_problem* p, int dir, const double* ql, const double* qr,
                       double* wave, double* s, double* amdq, double* apdq);

/* The state of the exact 1D Euler Riemann solution at x/t = 0 (primitive
 * rho, u, p of the normal problem; Toro §4.5), for the pins. */
void mcref_exact_sample(double gamma, double rl, double ul, double pl, double rr, double ur,
                        double pr, double pstar, double ustar, double* rho0, double* u0, double* p0);

/* Physical flux in direction dir (used by the pins). */
void mcref_flux(const mcref_problem* p, int dir, const double* q, double* f);

double mcref_philim(int limiter, double theta);

/* Arrays q are planar: q[m][j][i] with j in [0, my+2mbc), i in [0, mx+2mbc),
 * ghost layers included, contiguous. */
void mcref_bc_fill(const mcref_problem* p, double* q);

/* One CTU step: copies qin, fills its ghosts, computes every edge and writes
 * the updated interior of qout, then fills qout's ghosts.  cfl_out gets
 * dt * max_edge |s|/dx.  Returns a MCREF_F_* mask. */
int mcref_step(const mcref_problem* p, const double* qin, double* qout, double dt,
               double* smax_out, int nthreads);

/* max over interior cells of max((|u|+c)/dx, (|v|+c)/dy). */
double mcref_max_cell_speed(const mcref_problem* p, const double* q);

/* Variable-dt driver with the accept/reject rule.  qa holds the initial
 * state; the result ends in qa or qb (*result_in_b).  t/dt are in-out. */
int mcref_advance(const mcref_problem* p, double* qa, double* qb, int nsteps,
                  double cfl_desired, double cfl_max, double* t, double* dt,
                  int* result_in_b, int* nrejected, int nthreads);

/* ---- exact Euler Riemann solver (1D) ---- */
enum { MCREF_SEED_ADAPTIVE = 0, MCREF_SEED_PV = 1, MCREF_SEED_TR = 2, MCREF_SEED_TS = 3,
       MCREF_SEED_PVTR = 4, MCREF_SEED_GIVEN = 5 };
enum { MCREF_RS_OK = 0, MCREF_RS_VACUUM = 1, MCREF_RS_NOCONV = 2, MCREF_RS_FALLBACK = 4 };

double mcref_seed(int mode, double gamma, double rl, double ul, double pl,
                  double rr, double ur, double pr);
/* f(p) = f_L(p) + f_R(p) + (u_R - u_L) and its derivative. */
void mcref_pressure_function(double gamma, double rl, double ul, double pl,
                             double rr, double ur, double pr, double p,
                             double* f, double* fd);
/* Newton from a seed.  seed_mode selects the guess; for MCREF_SEED_GIVEN
 * p_given is the proposal, and a non-physical proposal or a non-converged
 * run restarts from the adaptive seed (flag MCREF_RS_FALLBACK).  iters counts
 * every Newton update performed, including wasted ones. */
int mcref_exact_riemann(double gamma, double rl, double ul, double pl,
                        double rr, double ur, double pr, int seed_mode, double p_given,
                        double tol, int max_iter, double* pstar, double* ustar, int* iters);
int mcref_exact_bisect(double gamma, double rl, double ul, double pl,
                       double rr, double ur, double pr, double* pstar, double* ustar);
void mcref_exact_batch(int64_t n, double gamma, const double* rl, const double* ul,
                       const double* pl, const double* rr, const double* ur, const double* pr,
                       int seed_mode, const double* p_given, double tol, int max_iter,
                       double* pstar, double* ustar, int32_t* iters, int32_t* flags,
                       int nthreads);

/* ---- seed network (10 -> 64 -> 64 -> 1, ReLU) ---- */
#define MCREF_NIN 10
#define MCREF_KIN 16
#define MCREF_NH 64
/* Raw (unstandardised) features of one interface, MCREF_NIN values. */
void mcref_mlp_features(double gamma, double rl, double ul, double pl,
                        double rr, double ur, double pr, double* feat);
/* Forward pass over B rows of X (B x 16, already standardised and padded).
 * W1: 16x64, W2: 64x64 (both [in][out]), W3: 64, b1, b2: 64, b3: 1.
 * bf16 != 0 rounds every GEMM operand to bfloat16 (round to nearest even)
 * before it is multiplied; sums are exact-ish double.  H1, H2 (B x 64,
 * post-activation, after the bf16 rounding if any) may be NULL. */
void mcref_mlp_forward(int64_t B, const double* X, const double* W1, const double* b1,
                       const double* W2, const double* b2, const double* W3, const double* b3,
                       int bf16, double* out, double* H1, double* H2);
/* Gradients of L = (1/B) sum_b (out_b - y_b)^2. */
double mcref_mlp_backward(int64_t B, const double* X, const double* y,
                          const double* W1, const double* b1, const double* W2, const double* b2,
                          const double* W3, const double* b3, int bf16,
                          double* gW1, double* gb1, double* gW2, double* gb2,
                          double* gW3, double* gb3);
double mcref_round_bf16(double x);

/* ------------------------------------------------------------------ */
/* Refined patches on a coarse grid (amr.c)                            */
/* ------------------------------------------------------------------ */

/* A fine patch over the coarse cells [ci0, ci0+cw) x [cj0, cj0+ch): its grid
 * has ratio*cw x ratio*ch cells of size dx/ratio, dy/ratio. */
typedef struct {
    int ci0, cj0, cw, ch;
} mcref_amr_patch;

/* the fine patch's problem: coarse one with the fine sizes and given ghosts */
void mcref_fine_problem(const mcref_problem* coarse, int ratio, const mcref_amr_patch* pt,
                        mcref_problem* fine);
/* Ghost layers of every patch: copy from another patch covering the fine
 * cell, else conservative MC-limited linear interpolation of the coarse state
 * (1 - alpha) qc0 + alpha qc1 (both with filled ghosts).  qf[p] are the
 * patches' state arrays. */
void mcref_amr_fill_ghosts(const mcref_problem* pc, int ratio, const double* qc0, const double* qc1,
                           double alpha, const mcref_amr_patch* pts, int npatch, double** qf);
/* Covered coarse cells take the mean of their ratio x ratio fine cells. */
void mcref_amr_average_down(const mcref_problem* pc, int ratio, const mcref_amr_patch* pts,
                            int npatch, double* const* qf, double* qc);
/* One coarse step of dt with ratio fine steps of dt/ratio on every patch
 * (Berger-Oliger); qf[p] are updated in place, qc_out gets filled ghosts.
 * reflux != 0: the coarse cells outside the patches get the flux correction
 * of Berger & Colella (coarse flux replaced by the mean fine flux). */
int mcref_amr_step(const mcref_problem* pc, int ratio, const mcref_amr_patch* pts, int npatch,
                   const double* qc_in, double* qc_out, double** qf, double dt, int reflux,
                   int nthreads);
/* The flux through one edge implied by the step of q (filled ghosts) with dt:
 * f(Q_low) + A-dQ + limited correction + transverse terms, so that a cell's
 * update is minus the difference of its edges' fluxes.  dir 0: x-edge with
 * high cell (i, j); dir 1: y-edge with high cell (i, j).  F: meqn values. */
void mcref_edge_flux(const mcref_problem* p, const double* q, double dt, int dir, int i, int j,
                     double* F);

#ifdef __cplusplus
}
#endif
#endif
