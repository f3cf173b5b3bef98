/*
 * manyclaw.h -- C ABI of the GB300 wave-propagation library.
 *
 * What it computes.  arXiv 1308.1464 (ManyClaw) decomposes an explicit
 * finite-volume step for hyperbolic PDEs into kernels by arithmetic intensity
 * (§1.2, Table 1): a Riemann kernel that maps the states of adjacent cell
 * centres to values at their common edge, and a limiter kernel that maps edge
 * values back to cell centres; the Riemann kernel is pointwise and unaware of
 * the parallelism around it (§1.1, §2).  This library runs both kernels, for
 * every x- and y-edge of a 2D uniform grid, fused in one pass per tile on an
 * sm_103a GPU: the 2D unsplit wave-propagation step with limited second-order
 * corrections and transverse (corner-transport) splits.  Solvers: constant-
 * coefficient acoustics (§3, Table 2), shallow water and Euler with Roe's
 * linearisation and the Harten-Hyman entropy fix.
 *
 * Conventions, for every entry point:
 *  - Plain pointers and sizes only.  A "device" pointer is CUDA global memory
 *    of the current device; a "host" pointer is ordinary (pageable or pinned)
 *    host memory.  Streams are cudaStream_t passed as void* (NULL = legacy
 *    default stream).
 *  - The caller owns every state, aux and I/O buffer.  The library owns only
 *    what its *_create calls allocate (contexts, small device scratch, CUDA
 *    graphs, tensor maps) and frees it in the matching *_destroy.
 *  - Every call returns an mc_status (0 = MC_OK).  Nothing throws.  Calls that
 *    take a stream enqueue work asynchronously unless they say they
 *    synchronise; errors raised by device code (non-physical states, bounded
 *    waits that gave up) are latched in a device status word and reported by
 *    the next call that synchronises.  mc_last_error() gives a message for the
 *    last failing call on the calling host thread.
 *  - The library holds no global mutable state except the per-thread error
 *    message; contexts are not thread-safe (one host thread per context).
 *
 * State layout (device).  q is planar: field m, cell (i, j), with
 * i in [-mbc, mx + mbc) and j in [-mbc, my + mbc) (ghost cells included), is
 * element   m * ld_field + (j + mbc) * ld_x + x_offset + i   of an array of
 * float (MC_F32) or double (MC_F64).  mc_layout_of() gives x_offset, ld_x,
 * ld_field: the interior of every row starts 16-byte aligned and rows are
 * padded to 128 bytes, so tiles can be moved by the tensor-memory accelerator.
 * The base pointer must be 16-byte aligned.
 */
#ifndef MANYCLAW_H
#define MANYCLAW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MC_OK = 0,
    MC_EINVAL = -1,     /* invalid argument (size, pointer, alignment, enum) */
    MC_ECUDA = -2,      /* a CUDA runtime/driver call failed */
    MC_ENOMEM = -3,     /* allocation failed */
    MC_ECFL = -4,       /* a step was rejected (Courant number above the limit) */
    MC_ENONPHYS = -5,   /* non-physical state met (depth/density/pressure <= 0, NaN) */
    MC_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
    MC_ENOTSUP = -7     /* combination not supported */
} mc_status;

/* MC_ADVECTION: scalar q_t + u q_x + v q_y = 0 with constant (u, v) =
 * (param[0], param[1]), the paper's advection solver (§3).
 * MC_ACOUSTICS_VAR: acoustics with a density rho and sound speed c per cell,
 * the paper's variable-coefficient acoustics (§3, Table 2); the state array
 * holds (p, u, v, rho, c): the two material planes follow the three fields
 * and every step copies them unchanged into its output, ghost layers filled
 * like the fields (never negated).  Not available for batched patches. */
/* MC_EULER_GODUNOV: the Euler equations with the exact Riemann solution in
 * the normal solve (Toro ch. 4: p* by Newton from Toro's adaptive guess,
 * the state at x/t = 0 per Toro §4.5): fluctuations are flux differences to
 * that state, waves the jumps across the two nonlinear waves and the contact
 * (at the shock speeds or rarefaction heads and u*), and the transverse split
 * is Roe's.  param[0] = gamma; efix is ignored.  Newton stops at a relative
 * change of 1e-6 (FP32) or 1e-14 (FP64), at most 40 updates. */
enum { MC_ACOUSTICS = 1, MC_SWE_ROE = 2, MC_EULER_ROE = 3, MC_ADVECTION = 4, MC_ACOUSTICS_VAR = 5,
       MC_EULER_GODUNOV = 6 };
/* limiter numbering as in Clawpack: 0 none (Lax-Wendroff), 1 minmod,
 * 2 superbee, 3 van Leer, 4 MC (LeVeque 2002, eq. 6.39) */
enum { MC_LIM_NONE = 0, MC_LIM_MINMOD = 1, MC_LIM_SUPERBEE = 2, MC_LIM_VANLEER = 3, MC_LIM_MC = 4 };
/* boundary kinds; MC_BC_GIVEN: the caller writes that side's two ghost
 * layers before every step (a neighbouring block's halo, mc_halo_unpack) and
 * the ghost fills leave them as they are.  A grid with a GIVEN side needs at
 * least 2 x 2 cells; mc_advance, mc_advance_host, the batch and the refined
 * patches reject it. */
enum { MC_BC_PERIODIC = 0, MC_BC_EXTRAP = 1, MC_BC_WALL = 2, MC_BC_GIVEN = 3 };
enum { MC_F32 = 0, MC_F64 = 1 };

/* A 2D problem.  The planes of a state array follow from the solver
 * (acoustics (p, u, v): 3; shallow water (h, hu, hv): 3; Euler (rho, rho u,
 * rho v, E): 4; advection (q): 1; variable-coefficient acoustics
 * (p, u, v, rho, c): 5; Euler with either normal solve: 4). */
typedef struct mc_problem {
    int32_t solver;      /* MC_ACOUSTICS | MC_SWE_ROE | MC_EULER_ROE | MC_ADVECTION |
                          * MC_ACOUSTICS_VAR | MC_EULER_GODUNOV */
    int32_t dtype;       /* MC_F32 | MC_F64: storage and arithmetic precision */
    int32_t mx, my;      /* interior cells, each >= 1 */
    int32_t mbc;         /* ghost layers; must be 2 */
    int32_t limiter;     /* MC_LIM_* */
    int32_t order;       /* 1: first order, 2: limited second-order corrections */
    int32_t transverse;  /* 0: none, 1: transverse split of the fluctuations,
                          * 2: also of the limited corrections (LeVeque 2002,
                          * ch. 21; each edge's whole contribution to a cell,
                          * A+dQ - F or A-dQ + F, is split) */
    int32_t efix;        /* 1: Harten-Hyman entropy fix (shallow water, Euler) */
    int32_t bc[4];       /* boundary kinds at xlo, xhi, ylo, yhi (MC_BC_*) */
    double dx, dy;       /* cell sizes, > 0 */
    double param[4];     /* acoustics: rho, K | shallow water: g | Euler: gamma |
                          * advection: u, v.  Shallow water and Euler, FP32
                          * only: param[3] = tau of the FP64 guard (0: the
                          * default 1e-3; negative: guard off).  A guarded
                          * edge -- across a near-dry or near-vacuum front
                          * (smaller depth or density below tau times the
                          * larger) or, for Euler, with Roe sound speed
                          * c^2 < tau (gamma - 1) H (cold, high-Mach flow) --
                          * has its normal solve and transverse splits
                          * computed in FP64; with the guard on, the speeds
                          * and split of a transonic entropy fix are formed
                          * in FP64 too (mc_guard_stats counts the edges). */
} mc_problem;

typedef struct mc_layout {
    int64_t x_offset;    /* element offset of cell i = 0 within a row */
    int64_t ld_x;        /* row pitch, elements */
    int64_t ld_field;    /* field-plane pitch, elements */
    int64_t elem_bytes;  /* 4 or 8 */
    int64_t meqn;        /* planes of a state array (fields, then material planes) */
    int64_t bytes;       /* bytes of one state array */
} mc_layout;

typedef struct mc_ctx mc_ctx;

/* Human-readable name of a status code (static string). */
const char* mc_status_string(int status);

/* Copies the message of the last failing call on this host thread into buf
 * (NUL-terminated, truncated to n bytes).  Returns the status of that call. */
int mc_last_error(char* buf, size_t n);

/* Validates p and fills *out with the state layout.  Host only; no GPU. */
mc_status mc_layout_of(const mc_problem* p, mc_layout* out);

/* Creates a context for problem p on the current device: validates p,
 * allocates a few hundred bytes of device scratch (time-step scalars, the
 * device status word) and picks the tile shape.  *out is owned by the
 * caller and released with mc_destroy. */
mc_status mc_create(const mc_problem* p, mc_ctx** out);
mc_status mc_destroy(mc_ctx* ctx);

/* Rows of cells each warp sweeps per task (the tile height); 0 restores the
 * default.  Used by the autotuner; results do not depend on it. */
mc_status mc_set_tile_rows(mc_ctx* ctx, int rows);

/* Refined patches with their own time steps (the paper's "dynamic time
 * stepping" kernel, §1.2 Table 1: each refined grid manages its own time step
 * and takes the values at its boundary from the adjacent grid by spatial and
 * temporal interpolation).  Two levels, Berger-Oliger: one coarse step of dt
 * on the whole coarse grid, then `ratio` steps of dt/ratio on every patch;
 * before each, the patches' two ghost layers are filled cell by cell from the
 * other patch covering the cell, or else from the coarse state interpolated
 * linearly in time and by a conservative MC-limited linear reconstruction in
 * space; afterwards every covered coarse cell takes the mean of its fine
 * cells.  There is no flux correction at coarse-fine boundaries (refluxing).
 *
 * A patch covers the coarse cells [ci0, ci0+cw) x [cj0, cj0+ch) inside the
 * coarse interior; patches do not overlap.  Its grid has ratio*cw x ratio*ch
 * cells of size dx/ratio x dy/ratio (mc_amr_fine_problem gives the problem,
 * and mc_layout_of of it the layout of its two buffers qa, qb, caller-owned).
 * The initial fine state goes into qa (interior).  Not for variable-
 * coefficient acoustics (MC_ENOTSUP). */
typedef struct mc_amr_patch {
    int32_t ci0, cj0, cw, ch;
    void* qa;
    void* qb;
} mc_amr_patch;
typedef struct mc_amr mc_amr;
mc_status mc_amr_fine_problem(const mc_problem* coarse, int32_t ratio, const mc_amr_patch* patch,
                              mc_problem* out);
mc_status mc_amr_create(const mc_problem* coarse, int32_t ratio, const mc_amr_patch* patches,
                        int32_t npatch, mc_amr** out);
/* Conservative coupling (off by default): after each coarse step the coarse
 * cells outside the patches take dt/d times the difference between the flux
 * the coarse step put through their patch-boundary edge and the mean of the
 * fine fluxes through it over the fine steps (Berger & Colella 1989; the flux
 * of an edge is f(Q_low) + A-dQ plus the limited correction and transverse
 * terms).  Edges on the domain boundary and edges between two patches are not
 * corrected.  on: 0 or 1. */
mc_status mc_amr_set_reflux(mc_amr* amr, int32_t on);
mc_status mc_amr_destroy(mc_amr* amr);
/* nsteps coarse steps of dt.  The coarse state alternates between qc_a and
 * qc_b (coarse_in_b: which holds the result); every patch's state is in its
 * qb after the call when *fine_in_b is 1, else in its qa (the same for all
 * patches, and carried over to the next call).  Asynchronous on stream except
 * for the final status check (MC_ENONPHYS, MC_ETIMEOUT from any grid). */
mc_status mc_amr_advance(mc_amr* amr, void* qc_a, void* qc_b, int32_t nsteps, double dt,
                         int32_t* coarse_in_b, int32_t* fine_in_b, void* stream);

/* Pressure seeds for the exact-solution Euler solver (MC_EULER_GODUNOV): with
 * a trained seed network attached (see mc_mlp_* below), a normal solve of the
 * fused step across a strong jump (pressure ratio 2 or more, where Toro's
 * adaptive rule leaves the PV guess) starts Newton from the network's
 * proposal p_TR exp(net(x)),
 * evaluated per warp on the tensor cores when any lane of the warp needs it;
 * it restarts from Toro's adaptive guess when the proposal is implausible or
 * does not converge (the Riemann kernel stays pointwise, as the paper keeps
 * it, §2; only its starting guess changes).  net = NULL detaches.  The network is
 * borrowed: it must outlive every step that uses it.  Changing it drops the
 * context's captured step graphs.  MC_ENOTSUP for other solvers. */
typedef struct mc_mlp mc_mlp;
mc_status mc_set_seed_net(mc_ctx* ctx, const mc_mlp* net);
/* Newton updates and normal solves the exact-solution solver counted in this
 * context's fused steps since the last reset (synchronises the stream;
 * reset != 0 zeroes the counters afterwards). */
mc_status mc_newton_stats(mc_ctx* ctx, int64_t* updates, int64_t* solves, int32_t reset, void* stream);

/* Interior edges whose normal solve the FP64 guard of an FP32 shallow-water
 * or Euler step recomputed (see mc_problem.param[3]; paper §1.2, "local
 * precision": precision spent only where the state needs it), counted over
 * this context's fused steps since the last reset.  Synchronises the stream;
 * reset != 0 zeroes the counter afterwards. */
mc_status mc_guard_stats(mc_ctx* ctx, int64_t* edges, int32_t reset, void* stream);

/* Host <-> device copies between a dense interior array (meqn x my x mx,
 * x fastest, the problem's dtype) and a device state in the library layout.
 * Asynchronous on stream. */
mc_status mc_upload(mc_ctx* ctx, const void* host_dense, void* q_dev, void* stream);
mc_status mc_download(mc_ctx* ctx, const void* q_dev, void* host_dense, void* stream);

/* Device-side repacking of a whole interior between the dense order of
 * mc_upload (meqn x my x mx, x fastest) and the library layout: to_layout
 * != 0 reads dense src and writes the interior of the state dst (ghosts and
 * padding untouched), 0 the reverse.  Both are device pointers to buffers of
 * the caller that must not overlap (a dense copy needs meqn*my*mx elements;
 * a spare state buffer holds one).  With it a host transfer moves one
 * contiguous block instead of one row at a time.  Asynchronous on stream;
 * MC_EINVAL for NULL or equal pointers. */
mc_status mc_repack(mc_ctx* ctx, const void* src, void* dst, int32_t to_layout, void* stream);

/* Fills the ghost layers of the device state q from its interior: periodic
 * wrap, zero-order extrapolation, or a reflecting wall (mirror with the
 * wall-normal momentum negated), per side (LeVeque 2002, ch. 7 and §21.8).
 * Corners take the values of filling x ghosts of the interior rows first and
 * then y ghosts over the full width.  Sides of kind MC_BC_GIVEN are left as
 * they are. */
mc_status mc_bc_fill(mc_ctx* ctx, void* q, void* stream);

/* ---- Blocks of a decomposed grid ------------------------------------------
 * A grid split into blocks (one per device or rank) steps each block alone;
 * a cell's update reads cells up to two away, diagonal ones included through
 * the transverse terms (LeVeque 2002, §21.8), so before every step the two
 * ghost layers on a side shared with another block must hold that block's
 * two interior layers next to the side, while sides on the global boundary
 * keep their kind.  Corners come out as in mc_bc_fill when the fill runs in
 * two phases: (x) exchange the x strips and mc_bc_fill_dir(.., 0, ..), then
 * (y) exchange the y strips, which span the ghost columns, and
 * mc_bc_fill_dir(.., 1, ..).  Sides: 0 xlo, 1 xhi, 2 ylo, 3 yhi.
 *
 * Strip layout (dense, the state's element type): x sides [meqn][my][2],
 * the two interior columns next to the side (pack) or its two ghost columns
 * (unpack), in increasing i, interior rows only; y sides [meqn][2][mx + 4],
 * the two interior rows next to the side or its two ghost rows, in
 * increasing j, columns -2 .. mx + 1.  The strip packed at side s of one
 * block is unpacked at side s ^ 1 of its neighbour.  Buffers are device
 * memory owned by the caller; the calls are asynchronous on `stream`. */

/* Elements of the strip of `side` for problem p (grids of at least 2 x 2). */
mc_status mc_halo_elems(const mc_problem* p, int32_t side, int64_t* elems);
/* Copies the two interior layers of q next to `side` into buf. */
mc_status mc_halo_pack(mc_ctx* ctx, const void* q, int32_t side, void* buf, void* stream);
/* Copies a strip from buf into the two ghost layers of q on `side`. */
mc_status mc_halo_unpack(mc_ctx* ctx, const void* buf, int32_t side, void* q, void* stream);
/* One phase of mc_bc_fill: dir 0 fills the x ghost columns of the interior
 * rows, dir 1 the y ghost rows across the full padded width, each on the
 * sides whose kind is not MC_BC_GIVEN.  dir 0 then dir 1 equals mc_bc_fill. */
mc_status mc_bc_fill_dir(mc_ctx* ctx, void* q, int32_t dir, void* stream);

/* A block stepped with its time-step state on the device (§1.2, Table 1,
 * "dynamic time stepping", over a decomposed grid): between mc_block_begin
 * and mc_block_end the context's device state holds dt, t, the buffer index
 * cur (the state is qa when cur = 0, qb when 1) and the counters, so a rank
 * enqueues attempt after attempt without reading anything back:
 *   for direction x then y: mc_block_pack of the shared sides, exchange the
 *     strips, mc_block_unpack, mc_block_fill_dir;
 *   mc_block_sweep (q[cur] -> q[cur ^ 1] with the device dt; the speed
 *     maximum of the step accumulates into *smax_dev, a uint64 holding the
 *     bits of a non-negative double, so an integer max-reduction over ranks
 *     is the maximum of the speeds);
 *   the max-reduction of *smax_dev over the ranks, in place;
 *   mc_block_dt_rule: the accept/reject rule of mc_advance on the reduced
 *     maximum (reject above cfl_max and retake with cfl_desired / smax,
 *     otherwise advance t, flip cur and propose cfl_desired / smax); it
 *     zeroes *smax_dev for the next attempt.
 * Every rank takes the same decisions.  mc_block_end synchronises and
 * returns t, dt, cur and the accepted and rejected attempts; it reports
 * MC_ENONPHYS / MC_ETIMEOUT / MC_EINVAL from the device status word.  All
 * calls are asynchronous on `stream` except begin and end. */
mc_status mc_block_begin(mc_ctx* ctx, double t, double dt, void* stream);
mc_status mc_block_pack(mc_ctx* ctx, const void* qa, const void* qb, int32_t side, void* buf,
                        void* stream);
mc_status mc_block_unpack(mc_ctx* ctx, const void* buf, int32_t side, void* qa, void* qb,
                          void* stream);
mc_status mc_block_fill_dir(mc_ctx* ctx, void* qa, void* qb, int32_t dir, void* stream);
mc_status mc_block_sweep(mc_ctx* ctx, void* qa, void* qb, uint64_t* smax_dev, void* stream);
mc_status mc_block_dt_rule(mc_ctx* ctx, uint64_t* smax_dev, double cfl_desired, double cfl_max,
                           void* stream);
mc_status mc_block_end(mc_ctx* ctx, double* t, double* dt, int32_t* cur, int32_t* naccepted,
                       int32_t* nrejected, void* stream);

/* One unsplit step with explicit dt: fills q_in's ghosts, then writes the
 * updated interior of q_out (q_out's ghosts are left untouched; q_in and
 * q_out must not overlap).  The fused kernel performs, per tile, the normal
 * Riemann solves at every x- and y-edge (paper Table 1, Riemann row), the
 * limited corrections and transverse splits (Table 1, limiter row) and the
 * flux-difference update.  If smax_out is not NULL the call synchronises the
 * stream and stores max over the interior edges of |s|/dx (x-edges) and
 * |s|/dy (y-edges), so the Courant number of the step is dt * smax; it then
 * also reports MC_ENONPHYS if the device flagged a non-physical state. */
mc_status mc_step(mc_ctx* ctx, void* q_in, void* q_out, double dt, double* smax_out, void* stream);

/* The fused step alone: like mc_step but q_in's ghost layers must already be
 * filled (mc_bc_fill) and nothing is synchronised; smax is accumulated
 * (running maximum) into the context's device scalar, which mc_step resets. */
mc_status mc_sweep(mc_ctx* ctx, const void* q_in, void* q_out, double dt, void* stream);

/* mc_step without a context and without allocating device memory.  The paper
 * has no counterpart; this exists for callers that cannot call cudaMalloc --
 * plug-ins whose host hands them a fixed device-memory budget and owns every
 * allocation, and loops that must not risk the device-wide synchronisation
 * that allocating or freeing can cause.  It performs the same ghost fill and
 * fused step as mc_step (same results) and keeps its scratch -- speed
 * maximum, status word and the tensor map of q_in, 192 bytes -- in a 256-byte
 * static device array that every device loading the library holds until the
 * process exits.  Problems are validated as by mc_layout_of and rejected with
 * MC_EINVAL and a message; the scratch does not grow with the grid, so every
 * grid mc_layout_of accepts fits.  The first call on a device (with that
 * device current) looks up the array's device address and raises the dynamic
 * shared-memory limits of every solver's kernels; if that set-up fails the
 * call returns MC_ECUDA and the next call retries it.  The array is shared by
 * all calls and keeps the previous call's contents (each call clears what
 * must start at zero): calls that overlap on the GPU, from other streams or
 * host threads, race on it.  smax_out and the status report behave as in
 * mc_step (the call synchronises the stream when smax_out != NULL). */
mc_status mc_step_noalloc(const mc_problem* p, void* q_in, void* q_out, double dt,
                          double* smax_out, void* stream);

/* ---- Throughput microbenchmarks (no counterpart in the paper) -----------
 * The step kernels are bound by instruction issue and by their arithmetic
 * pipes, not by HBM alone; these launches measure the denominators of those
 * rooflines on the device at hand.  mc_peak_run launches one kernel of `kind`
 * with blocks_per_sm blocks of 256 threads on every SM of the current device
 * (the SM count the device reports); every thread runs `iters` loop
 * iterations of 16 steps of 8 independent dependency chains.  *ops_out (host)
 * receives the operations of the launch: flops for MC_PEAK_FFMA, _FFMA2
 * (packed FP32 pairs) and _DFMA (2 per fused multiply-add), results for
 * MC_PEAK_RSQRT and _RCP (the FP32 hardware approximations), and thread
 * instructions for MC_PEAK_IADD (integer multiply-adds) and MC_PEAK_ISSUE
 * (independent FP32 multiply-adds, which issue at the full rate of one warp
 * instruction per scheduler and cycle: the issue ceiling).  The caller times
 * the launch (events on `stream`).  sink: a device float the kernel writes
 * only for impossible results (keeps the chains from being optimised away).
 * Asynchronous; MC_EINVAL for a bad kind or size. */
enum { MC_PEAK_FFMA = 0, MC_PEAK_FFMA2 = 1, MC_PEAK_DFMA = 2, MC_PEAK_RSQRT = 3, MC_PEAK_RCP = 4,
       MC_PEAK_IADD = 5, MC_PEAK_ISSUE = 6, MC_PEAK_NKINDS = 7 };
mc_status mc_peak_run(int32_t kind, int32_t blocks_per_sm, int64_t iters, float* sink,
                      double* ops_out, void* stream);

/* max over interior cells of max((|u|+c)/dx, (|v|+c)/dy), synchronising. */
mc_status mc_max_cell_speed(mc_ctx* ctx, const void* q, double* smax_out, void* stream);

/* Advances nsteps accepted steps with the variable time step rule of
 * dynamic time stepping (paper §1.2, Table 1, "dynamic time stepping"): the
 * Courant number of an attempt is dt * smax over its edges; an attempt above
 * cfl_max is rejected and retaken with dt = cfl_desired / smax; an accepted
 * one advances *t_inout and proposes dt = cfl_desired / smax.  The state
 * starts in qa; the result ends in qa (*result_in_b = 0) or qb (= 1).  The
 * whole attempt sequence runs as one CUDA graph with dt, t and the buffer
 * index kept on the device; the call synchronises once at the end.
 * nrejected (nullable) receives the number of rejected attempts. */
mc_status mc_advance(mc_ctx* ctx, void* qa, void* qb, int nsteps, double cfl_desired,
                     double cfl_max, double* t_inout, double* dt_inout, int* result_in_b,
                     int* nrejected, void* stream);

/* End-to-end form with host buffers: uploads host_q0 (dense interior) into
 * qa, runs mc_advance, downloads the result into host_q (dense interior),
 * synchronising.  Each transfer moves one contiguous block: the upload lands
 * densely in qb and a kernel repacks it into qa's layout; the result is
 * repacked densely into the buffer that does not hold it and copied out.
 * Both buffers' previous contents are overwritten; qa and qb must differ
 * (MC_EINVAL).  host buffers in pinned memory give the full transfer rate. */
mc_status mc_advance_host(mc_ctx* ctx, const void* host_q0, void* host_q, void* qa, void* qb,
                          int nsteps, double cfl_desired, double cfl_max, double* t_inout,
                          double* dt_inout, int* nrejected, void* stream);

/* ------------------------------------------------------------------------
 * Batched uneven patches.
 *
 * The paper's execution model lets larger threads schedule pieces of work to
 * finer-grained ones, and lets each refined grid manage its own time step
 * ("local precision with minimal effects to global time stepping", §1.2,
 * Table 1 "dynamic time stepping").  A batch is a set of independent patches
 * of one problem kind (proto: solver, dtype, limiter, order, transverse, efix,
 * param; all four boundaries must be MC_BC_WALL), each with its own size and
 * spacing and two caller-owned device buffers in the layout mc_layout_of
 * gives for that size.  Each patch advances with its own dt = cfl / smax,
 * smax taken from the patch's previous step (from its initial cell speeds for
 * the first step); there is no reject/retake in this form.
 * ------------------------------------------------------------------------ */
typedef struct mc_patch {
    int32_t mx, my;      /* interior cells, each >= 4 */
    double dx, dy;
    void* qa;            /* device state holding the initial data (interior) */
    void* qb;            /* device state, scratch of the ping-pong */
} mc_patch;
typedef struct mc_batch mc_batch;

/* Validates the patches, builds their tensor maps and work tables (device
 * memory owned by the batch).  Synchronous. */
mc_status mc_batch_create(const mc_problem* proto, const mc_patch* patches, int32_t npatch,
                          mc_batch** out);
mc_status mc_batch_destroy(mc_batch* b);
/* Rows per warp task for every patch (the per-patch work split); results do
 * not depend on it.  The autotuner sets it. */
mc_status mc_batch_set_tile_rows(mc_batch* b, const int32_t* rows);
/* Advances every patch nsteps steps in ONE persistent launch captured in a
 * CUDA graph (with the initial ghost fill and cell-speed pass before it): a
 * global counter hands out (step, patch, task) items in step order; a task
 * waits (bounded, MC_ETIMEOUT) for the previous step of its patch; tasks write
 * the ghost cells of the next step themselves.  Result in qa if nsteps is even
 * (*result_in_b = 0), else qb.  t_out (host, npatch, nullable) gets each
 * patch's elapsed time.  Synchronous. */
mc_status mc_batch_advance(mc_batch* b, int32_t nsteps, double cfl, double* t_out,
                           int* result_in_b, void* stream);
/* The same computation as one launch per patch per step (dt, ghost fill and
 * fused step per patch), for comparison; bitwise equal interiors. */
mc_status mc_batch_advance_plain(mc_batch* b, int32_t nsteps, double cfl, double* t_out,
                                 int* result_in_b, void* stream);
/* The same computation as one launch per step over all patches (the
 * persistent kernel restricted to one step per launch, all nsteps launches
 * captured in one CUDA graph, after the same ghost fill and cell-speed pass):
 * the launch boundary orders the steps instead of per-patch completion
 * counters.  Bitwise equal interiors; for comparison with mc_batch_advance.
 * Synchronous. */
mc_status mc_batch_advance_steps(mc_batch* b, int32_t nsteps, double cfl, double* t_out,
                                 int* result_in_b, void* stream);
/* Failure-detection hook for tests (no counterpart in the paper): during the
 * next mc_batch_advance only, the tasks of `patch` wait for one more finished
 * task of their previous step than will ever exist.  Their bounded waits give
 * up after about a second, the kernel ends, the call returns MC_ETIMEOUT, and
 * the batch stays usable (that patch's state is left part-advanced). */
mc_status mc_batch_inject_stall(mc_batch* b, int32_t patch);

/* ------------------------------------------------------------------------
 * Exact Euler Riemann solver with a learned pressure seed.
 *
 * The paper lists Euler among its Riemann kernels (§3, Tables 2-3) and keeps
 * each solve pointwise (§2).  mc_riemann_exact solves n independent 1D Euler
 * Riemann problems exactly (Toro, ch. 4): the star pressure p* is the root of
 * f(p) = f_L(p) + f_R(p) + u_R - u_L, found by Newton's method in FP64 from a
 * seed, stopping when |p_{k+1} - p_k| / p_{k+1} < tol; u* follows from p*.
 * Inputs and outputs are FP32 structure-of-arrays device buffers of length n.
 * Seeds: Toro's adaptive choice between the primitive-variable (PV),
 * two-rarefaction (TR) and two-shock (TS) guesses, each of them alone, PV/TR
 * only, or the seed network (MC_SEED_MLP), whose proposal is used only if it
 * is finite and within [1e-6 min(pL,pR), 1e6 max(pL,pR)] and Newton from it
 * converges within max_iter; otherwise Newton restarts from the adaptive
 * seed (flag MC_RS_FALLBACK) and iters counts the wasted updates too.
 * Interfaces that generate vacuum (2 (cL + cR) / (gamma - 1) <= uR - uL) get
 * p* = 0, u* = NaN, flag MC_RS_VACUUM and no iterations.
 * ------------------------------------------------------------------------ */
enum { MC_SEED_ADAPTIVE = 0, MC_SEED_PV = 1, MC_SEED_TR = 2, MC_SEED_TS = 3, MC_SEED_PVTR = 4,
       MC_SEED_MLP = 5 };
/* Added to a seed mode: Newton first iterates in FP32 from the seed (the
 * network's proposal included) until |dp|/p < 1e-5 (at most 12 updates; a
 * stalled or failed FP32 stage hands over its last finite iterate, else the
 * FP64 adaptive guess), then FP64 updates finish with the same stopping test
 * |p_{k+1} - p_k| / p_{k+1} < tol, usually two of them.  iters counts the
 * updates of both stages; stats then needs 8 entries, [6] the FP32 and [7]
 * the FP64 updates.  (GB300's FP64 rate is 1/73 of its FP32 rate.) */
enum { MC_NEWTON_MIXED = 16 };
enum { MC_RS_OK = 0, MC_RS_VACUUM = 1, MC_RS_NOCONV = 2, MC_RS_FALLBACK = 4 };

/* Seed network: 10 features -> 64 -> 64 -> 1 (ReLU), BF16 weights and FP32
 * accumulation on the tensor cores.  Parameters travel as one FP32 vector
 * ("master" copy) in the order W1[16][64] (input-major; rows 10..15 are
 * padding and must be zero), b1[64], W2[64][64], b2[64], W3[64], b3[1],
 * followed by the feature standardisation mu[10], sigma[10]:
 * MC_MLP_NPARAM values.  Features of an interface, before standardisation:
 * ln rhoL, ln rhoR, ln pL, ln pR, ln cL, ln cR, uR - uL, (uR - uL)/(cL + cR),
 * ln p_TR, ln max(p_PV, 1e-6); the output is ln p* - ln p_TR. */
#define MC_MLP_NWEIGHT (16 * 64 + 64 + 64 * 64 + 64 + 64 + 1)
#define MC_MLP_NPARAM (MC_MLP_NWEIGHT + 20)
/* (mc_mlp is declared above, with mc_set_seed_net) */

/* Allocates the network's device storage (zero weights) on the current device. */
mc_status mc_mlp_create(mc_mlp** out);
mc_status mc_mlp_destroy(mc_mlp* net);
/* Host FP32 parameter vector of MC_MLP_NPARAM values in / out; set_params
 * also rounds the weights to the BF16 copy the kernels use.  Synchronous. */
mc_status mc_mlp_set_params(mc_mlp* net, const float* host_params);
mc_status mc_mlp_get_params(const mc_mlp* net, float* host_params);

/* Raw features (n x 10, row-major, FP32) of n interfaces given as device
 * SoA states; rows of vacuum-generating interfaces are NaN.  If p_star is
 * not NULL, target[i] = ln p_star[i] - ln p_TR[i] (the network's training
 * target), NaN where p_star is not positive.  Asynchronous. */
mc_status mc_mlp_features(int64_t n, double gamma, const float* rho_l, const float* u_l,
                          const float* p_l, const float* rho_r, const float* u_r,
                          const float* p_r, const float* p_star, float* features, float* target,
                          void* stream);

/* Network forward over n raw feature rows (device, n x 10): standardised by
 * the network's mu/sigma, BF16 tensor-core layers, out[n] on the device. */
mc_status mc_mlp_forward(const mc_mlp* net, int64_t n, const float* features, float* out,
                         void* stream);

/* Gradient of L = (1/n) sum (out_i - y_i)^2 over n rows (device features n x
 * 10, targets n) with the precision model of training: BF16 operands of
 * every product of activations, weights and back-propagated activation
 * gradients, FP32 accumulation.  grads: device, MC_MLP_NWEIGHT floats in the
 * parameter order, overwritten; loss: device float, overwritten.  Rows with a
 * non-finite target contribute nothing.  Asynchronous. */
mc_status mc_mlp_grad(mc_mlp* net, int64_t n, const float* features, const float* target,
                      float* grads, float* loss, void* stream);

typedef struct mc_train_cfg {
    int64_t batch;          /* rows per Adam step */
    int32_t epochs;
    float lr, beta1, beta2, eps;   /* Adam (Kingma & Ba 2015) */
    uint64_t seed;          /* per-epoch row order */
    int32_t fit_norm;       /* 1: set mu/sigma from the features first */
    float clip;             /* >= 1: a step's gradient is scaled down to at most clip
                             * times the running mean of the (clipped) gradient
                             * norms; 0: no clipping */
    float lr_final;         /* learning rate of the last step: cosine decay from lr
                             * over the call's steps (lr_final = lr: constant) */
} mc_train_cfg;

/* Trains the network on n rows (device features n x 10, targets n) with
 * minibatch Adam on the GPU (the same kernels as mc_mlp_grad), optionally
 * clipping each step's gradient norm and decaying the learning rate (see
 * mc_train_cfg).  Rows with a non-finite feature or target are skipped.  Each epoch visits the rows in
 * the order i -> (a i + b) mod n with a coprime to n drawn from seed.
 * loss_per_epoch (host, nullable): mean loss of each epoch.  Synchronous. */
mc_status mc_mlp_train(mc_mlp* net, int64_t n, const float* features, const float* target,
                       const mc_train_cfg* cfg, float* loss_per_epoch, void* stream);

/* stats (nullable): device int64[6], accumulated (the caller zeroes it):
 * interfaces, vacuum, fallback, not converged, total Newton updates,
 * largest per-interface count; with MC_NEWTON_MIXED 8 entries, [6] FP32 and
 * [7] FP64 updates. */
mc_status mc_riemann_exact(int64_t n, double gamma, const float* rho_l, const float* u_l,
                           const float* p_l, const float* rho_r, const float* u_r,
                           const float* p_r, float* p_star, float* u_star, uint8_t* iters,
                           uint8_t* flags, int seed_mode, const mc_mlp* net, double tol,
                           int max_iter, int64_t* stats, void* stream);

#ifdef __cplusplus
}
#endif
#endif
