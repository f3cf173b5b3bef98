// mc_sweep.cuh -- the fused wave-propagation step and its companions
// (ghost fill, time-step rule, cell-speed reduction), templated on the
// Riemann solver.
//
// Paper mapping.  Table 1 (§1.2) splits an explicit step into a Riemann
// kernel (cell centres -> edge values) and a limiter kernel (edge values ->
// cell centres); §2 keeps edge results in work arrays "that in practice
// will cause bandwidth bottlenecks" and finds that computing both directions
// per cell ("cell-wise") with tiling is fastest on CPUs.  Here both kernels
// are fused: edge results live only in registers and are exchanged between
// neighbouring columns with warp shuffles, so HBM sees one read and one
// write of the state per step.
//
// The arithmetic is the 2D unsplit wave-propagation step (LeVeque 2002,
// eq. 21.8 with §6.13 limited corrections and §21.2 transverse splits):
//   Q' = Q - nu_x (A+dQ_{i-1/2} + A-dQ_{i+1/2}) - nu_y (B+dQ_{j-1/2} + B-dQ_{j+1/2})
//          - nu_x (F_{i+1/2} - F_{i-1/2}) - nu_y (G_{j+1/2} - G_{j-1/2}),
// F = 1/2 sum_p |s^p| (1 - nu_x |s^p|) phi(theta^p) W^p
//     - nu_y/2 (transverse splits of the y-fluctuations entering the two
//       cells of the edge), G likewise with x and y exchanged.
//
// Work decomposition.  A warp owns a band of 32 columns c = i0-1 .. i0+30
// (lane l <-> column i0-1+l) and marches up the rows j0 .. j0+TY-1 of a
// task.  At iteration k lane l:
//   1. takes row k+2 of its column (and of column c-1) from a shared-memory
//      ring filled by TMA (one 3D box = all fields of RS rows per stage);
//   2. solves the y-edge between rows k+1 and k+2 and splits both of its
//      fluctuations in x;
//   3. solves the x-edge c-1/2 of row k+1 and splits both fluctuations in y;
//   4. completes F at x-edge (c-1/2, k+1): the limiter reads the upwind
//      neighbour edge's waves from lane l-1 or l+1, the transverse part the
//      A+ pieces of column c-1 from lane l-1;
//   5. completes G at y-edge (c, k+1/2): limiter from the three y-edges it
//      holds in registers, transverse pieces of x-edge c+1/2 from lane l+1;
//   6. writes cell (c, k).
// Lanes 1..29 see every neighbour they need; lanes 0, 30, 31 only feed them.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "mc_device.cuh"
#include "mc_riemann.cuh"
#include "mc_seednet.cuh"
#include "mc_tile.h"

namespace mc {

// Tasks of one fused step that met a guarded or transonic edge: the step
// kernel counts (and lists) them, the guard kernel recomputes them and its
// last block resets the queue for the next step.
struct GuardQueue {
    unsigned count, done;
};

// ------------------------------------------------------------------ time step

struct DevState {
    unsigned long long smax_bits;
    double dt, t, cfl_last, cfl_maxseen;
    int cur, nacc, nrej, status;
    unsigned long long newton[2];   // Newton updates and normal solves (exact-solution solver)
    unsigned long long guard;       // interior edges of FP32 steps recomputed in FP64
    GuardQueue gq;                  // tasks queued for the FP64 guard's recompute
};

// The time-step rule of one attempt (paper §1.2, "dynamic time stepping"),
// applied by one thread once the attempt's speed maximum *sm is complete:
// Courant number = dt * smax; above cfl_max the attempt is rejected and
// retaken with dt = cfl_desired / smax, otherwise it is accepted (t advances,
// the buffer index flips) and proposes dt = cfl_desired / smax.  Resets *sm
// for the next attempt.
__device__ __forceinline__ void dt_rule_apply(DevState* st, double cfl_desired, double cfl_max,
                                              unsigned long long* sm)
{
    // a volatile read: other blocks' atomics may have completed it in this kernel
    const double smax = __longlong_as_double((long long)*reinterpret_cast<volatile unsigned long long*>(sm));
    const double dt = st->dt, cfl = dt * smax;
    st->cfl_last = cfl;
    if (cfl > cfl_max) {
        st->nrej++;
        if (smax > 0.0) st->dt = cfl_desired / smax;
    } else {
        st->t += dt;
        st->cur ^= 1;
        st->nacc++;
        if (cfl > st->cfl_maxseen) st->cfl_maxseen = cfl;
        if (smax > 0.0) st->dt = cfl_desired / smax;
    }
    *sm = 0ull;
}

template <class RP>
struct SweepArgs {
    using T = typename RP::real;
    RP rp;
    T* qa;
    T* qb;
    const int* cur;          // device buffer index (0: a -> b, 1: b -> a), or null: a -> b
    const double* dt_dev;    // device time step, or null: use dt
    double dt;
    double dx, dy;
    int mx, my;
    long long ld_x, ld_field, x_offset;
    int limiter, order, transverse;
    int nbands, ntasks, tile_rows;
    int split, nbig;                 // rows [0, split) in the first nbig tasks, TALL_TILES tiles each
    unsigned long long* smax_bits;
    int* status;
    const MlpDev* net;                    // pressure-seed network, or null (solvers with SEEDED)
    unsigned long long* newton_updates;   // [0] Newton updates, [1] normal solves, or null
    unsigned long long* guard_edges;      // edges recomputed in FP64 (FP32 pair solvers), or null
    GuardQueue* gq;                       // tasks the FP64 guard recomputes, or null (no guard)
    int* gq_tasks;                        // their indices (capacity ntasks), or null: all tasks
    // the attempt's time-step rule, applied by the guard kernel once the
    // speed maximum is complete (a loop of attempts that folds it there), or
    // null: the caller applies it
    DevState* dt_state;
    double cfl_desired, cfl_max;
};

// Solvers that take each state's 1/sqrt(h) from the caller (RS_CACHE):
// the scalar sweep forms it once per cell and carries it down the march,
// instead of twice per edge.
template <class RP, class = void>
struct rs_cache : std::false_type {};
template <class RP>
struct rs_cache<RP, std::void_t<decltype(RP::RS_CACHE)>> : std::bool_constant<RP::RS_CACHE> {};

// The FP64 guard of FP32 pair solvers inside a task: none (the batched and
// multi-grid forms), detect (mark a task that meets a guarded or transonic
// edge), redo (recompute those edges in FP64).
constexpr int GUARD_NONE = 0, GUARD_DETECT = 1, GUARD_REDO = 2;

// Resident CTAs per SM the fused kernels are compiled for (a register cap):
// a solver's MIN_CTAS, else 1.  The FP64 guard's rare path would otherwise
// set the register count of the whole kernel.
template <class RP, class = void>
struct min_ctas : std::integral_constant<int, 1> {};
template <class RP>
struct min_ctas<RP, std::void_t<decltype(RP::MIN_CTAS)>> : std::integral_constant<int, RP::MIN_CTAS> {};

// theta = dl / dr of K waves.  FP32: one hardware reciprocal each.  FP64:
// one correctly rounded reciprocal for all K (simultaneous inversion: prefix
// products of the dr, the reciprocal of their product, then each 1/dr_k as
// that reciprocal times the other factors), where a division costs about as
// much as eight multiplications.  A zero wave (dr = 0, so dl = 0) takes
// dr = 1 and theta = 0; a product outside [1e-290, 1e290] falls back to K
// reciprocals.  Results differ from dl / dr by a few ulp.
template <int K, typename T>
__device__ __forceinline__ void ratios(const T (&dl)[K], const T (&dr)[K], T (&th)[K])
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < K; k++) th[k] = dl[k] * rcp_(dr[k]);
    } else {
        T d[K], pre[K];
#pragma unroll
        for (int k = 0; k < K; k++) d[k] = dr[k] > T(0) ? dr[k] : T(1);
        pre[0] = d[0];
#pragma unroll
        for (int k = 1; k < K; k++) pre[k] = pre[k - 1] * d[k];
        const T P = pre[K - 1];
        if (P > T(1e-290) && P < T(1e290)) {
            T r = rcp_(P);
#pragma unroll
            for (int k = K - 1; k >= 1; k--) {
                th[k] = dl[k] * (r * pre[k - 1]);
                r *= d[k];
            }
            th[0] = dl[0] * r;
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) th[k] = dl[k] * rcp_(d[k]);
        }
    }
}

// phi(theta) of K ratios theta = dl / dr at once (LeVeque 2002, eq. 6.39):
// minmod (1), superbee (2), van Leer (3), MC (4) or none (0: phi = 1).  The
// limiter is warp-uniform, so one branch selects the formula for all K
// ratios; with a compile-time limiter the selection folds away.  A zero wave
// (dr = 0) needs no test: theta is then NaN or infinite, min/max return their
// other operand, so phi stays in [0, 2] and multiplies a wave whose
// components are all zero.  Van Leer's (theta + |theta|)/(1 + |theta|) is
// written as 2 - 2/(1 + t) with t = max(theta, 0), which keeps that property.
template <int K, typename T>
__device__ __forceinline__ void limiter_phis(int lim, const T (&th)[K], T (&phi)[K])
{
    if (lim == 4) {
#pragma unroll
        for (int k = 0; k < K; k++)
            phi[k] = fmax(T(0), fmin(fmin(T(0.5) * (T(1) + th[k]), T(2)), T(2) * th[k]));
    } else if (lim == 1) {
#pragma unroll
        for (int k = 0; k < K; k++) phi[k] = fmax(T(0), fmin(T(1), th[k]));
    } else if (lim == 2) {
#pragma unroll
        for (int k = 0; k < K; k++)
            phi[k] = fmax(T(0), fmax(fmin(T(1), T(2) * th[k]), fmin(T(2), th[k])));
    } else if (lim == 3) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            const T t = fmax(th[k], T(0));
            phi[k] = T(2) - T(2) * rcp_(T(1) + t);
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; k++) phi[k] = T(1);
    }
}

// Per-warp TMA ring: NSTAGE stages of one box each, one mbarrier per stage;
// with a seed network also the CTA's shared copy of it and the warp's scratch
// tiles for its inference, and the Newton counters.
struct WarpRing {
    uint64_t* bars;
    unsigned char* ring;
    uint32_t phase;   // per-stage completion parity
    const MlpShared* net = nullptr;
    __nv_bfloat16* xs = nullptr;
    float* outs = nullptr;
    unsigned long long* newton = nullptr;
    unsigned long long* guard = nullptr;   // count of edges recomputed in FP64, or null
};

// One warp task: the rows [j0, jend) of the band of columns starting at i0
// of one grid, read from the state behind `map`, written to qout.  Returns
// false if a bounded wait gave up.  With WALL_GHOSTS each written cell also
// writes the ghost cells it is the mirror source of (reflecting walls on all
// sides: x ghosts negate component 1, y ghosts component 2, corners both), so
// the next step needs no separate ghost fill.
//
// MODE_FAST compiles the common scheme (MC limiter, second order, transverse
// splits of the fluctuations) with those choices fixed; MODE_TRANS2 fixes
// second order with transverse option 2 and MODE_GENERAL transverse option
// 0 or 1 (option 2 at first order is option 1); the other choices are read
// at run time.
//
// Transverse option 2 splits each edge's whole contribution to a cell
// (A+dQ - F into the high cell, A-dQ + F into the low one, F the limited
// correction).  An x-edge's F is known in the iteration that solves it, so
// its splits only move behind the limiter.  A y-edge's limiter needs the edge
// above it, so the y splits of edge (c, k+1/2) run one iteration late, at k:
// the part entering row k+1 joins F of row k+1 as before, and the part
// entering row k is added to row k's carried x-edge terms just before row k
// is updated.
template <class RP, bool WALL_GHOSTS, int MODE, int GUARD = GUARD_NONE>
__device__ __forceinline__ bool sweep_task(const RP& rp, const CUtensorMap* map,
                                           typename RP::real* __restrict__ qout, int mx, int my,
                                           long long ld_x, long long ld_field, long long x_offset,
                                           int i0, int j0, int jend, typename RP::real nux,
                                           typename RP::real nuy, int limiter_rt, bool second_rt,
                                           int transverse_rt, WarpRing& W, bool& bad,
                                           typename RP::real& smx, typename RP::real& smy,
                                           int* status, bool* flagged = nullptr)
{
    constexpr bool FAST = MODE == MODE_FAST;
    constexpr bool trans2 = MODE == MODE_TRANS2;
    const int limiter = FAST ? 4 : limiter_rt;
    const bool second = MODE != MODE_GENERAL ? true : second_rt;
    const bool trans = MODE != MODE_GENERAL ? true : transverse_rt != 0;
    using T = typename RP::real;
    // N conserved fields; NP state planes (with material planes after them)
    constexpr int N = RP::NEQ, NW = RP::NW, NP = RP::NPLANE;
    constexpr int ES = sizeof(T);
    constexpr int AL = align_elems(ES);
    constexpr int BW = box_w(ES);
    constexpr int RS = stage_rows(ES);
    constexpr int SB = stage_bytes(ES, NP);
    constexpr int TB = box_bytes(ES, NP);
    const int lane = threadIdx.x & 31;
    const T hnux = T(0.5) * nux, hnuy = T(0.5) * nuy;

    const int c = i0 - 1 + lane;
    const bool out_lane = lane >= 1 && lane <= BAND_W && c < mx;
    const bool xe_lane = c >= 0 && c <= mx;      // x-edge c-1/2 is an interior edge
    const bool ye_lane = c >= 0 && c < mx;       // y-edges of column c are interior
    const long long gx = x_offset + i0 - 2;
    const int box_x = int(gx - ((gx % AL) + AL) % AL);
    const int sx = lane + 1 + int(gx - box_x);   // smem column of c; c-1 is sx-1
    const int rbase = j0 - 2;
    const int nfill = (jend + 1 - rbase + RS) / RS;
    // TMA precondition, checked instead of trusted: a 16-byte aligned box start
    if ((box_x * ES) % 16 != 0 || box_x < 0) {
        if (lane == 0) atomicOr(status, ST_BADARG);
        return true;
    }

    // start the ring
    if (lane == 0) {
        for (int f = 0; f < NSTAGE && f < nfill; f++) {
            mbar_arrive_expect_tx(&W.bars[f], TB);
            tma_load_3d(W.ring + f * SB, map, &W.bars[f], box_x, rbase + f * RS + 2, 0);
        }
    }

    // fetch row r of columns c and c-1 into registers; a stage goes back to
    // the TMA once its last row has been read
    // Rows are fetched strictly in order (rbase, rbase + 1, ...), so the ring
    // position is kept as counters: fr the row within the stage, fs the
    // stage, ff the stage's fill index, frow the lane's element of the row.
    int fr = 0, fs = 0, ff = 0;
    const T* frow = reinterpret_cast<const T*>(W.ring) + sx;
    auto fetch = [&](int, T* qc, T* ql) -> bool {
        if (fr == 0) {
            const bool ok = mbar_wait_bounded(&W.bars[fs], (W.phase >> fs) & 1u);
            if (!__all_sync(0xffffffffu, ok)) return false;
            W.phase ^= 1u << fs;
        }
#pragma unroll
        for (int m = 0; m < NP; m++) {
            qc[m] = frow[m * RS * BW];
            ql[m] = frow[m * RS * BW - 1];
        }
        if (fr == RS - 1) {
            __syncwarp();
            const int fn = ff + NSTAGE;
            if (lane == 0 && fn < nfill) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&W.bars[fs], TB);
                tma_load_3d(W.ring + fs * SB, map, &W.bars[fs], box_x, rbase + fn * RS + 2, 0);
            }
            ff++;
            fs = fs == NSTAGE - 1 ? 0 : fs + 1;
            fr = 0;
            frow = reinterpret_cast<const T*>(W.ring + fs * SB) + sx;
        } else {
            fr++;
            frow += BW;
        }
        return true;
    };

    // carried state (see the header comment for the schedule).  The y-limiter
    // of edge (c, k+1/2) needs, when s^p > 0, the dot product of its wave p
    // with that of the edge below: a solver with CARRY_DOT keeps that product
    // (dlo, formed one row earlier), otherwise the waves themselves (Wy0) are
    // kept -- whichever the solver's register budget favours.
    constexpr bool CD = RP::CARRY_DOT;
    T qc0[NP], qc1[NP], ql1[NP];
    T Wy0[CD ? 1 : NW][N], Wy1[NW][N], sy1[NW], dlo[NW];
    // XP = A+dQ(c-1/2) - F(c-1/2) and XM = A-dQ(c-1/2) + F(c-1/2) of row k (XM
    // goes to lane l-1, whose right edge this is); Z = B+dQ(k-1/2) + B-dQ(k+1/2)
    // - G(k-1/2) of row k: what the update of cell (c, k) needs from earlier
    // iterations
    T bp_pend[N], tyP_m[N], tyP_p[N];
    T XP0[N], XM0[N], Z0[N], BpAp0[N], BpAm0[N];
    // transverse option 2: B-dQ of y-edge (c, k+1/2) and that edge's
    // linearised state, split one iteration late
    T bm_prev[N];
    typename RP::Lin Lx_cur{}, Ly_cur{}, Ly_prev{};
#pragma unroll
    for (int m = 0; m < NP; m++) qc0[m] = T(0);
#pragma unroll
    for (int m = 0; m < N; m++) {
        bp_pend[m] = tyP_m[m] = tyP_p[m] = bm_prev[m] = T(0);
        XP0[m] = XM0[m] = Z0[m] = BpAp0[m] = BpAm0[m] = T(0);
    }
#pragma unroll
    for (int p = 0; p < NW; p++) {
        sy1[p] = dlo[p] = T(0);
#pragma unroll
        for (int m = 0; m < N; m++) {
            Wy1[p][m] = T(0);
            if constexpr (!CD) Wy0[p][m] = T(0);
        }
    }
    if (!fetch(rbase, qc1, ql1)) return false;
    // 1/sqrt(h) of qc1 and ql1 for RS_CACHE solvers
    constexpr bool RSC = rs_cache<RP>::value && !RP::PAIRED;
    T rs_c1 = T(0), rs_l1 = T(0);
    if constexpr (RSC) {
        rs_c1 = rp.rs_of(qc1);
        rs_l1 = rp.rs_of(ql1);
    }

    // transverse splits.  A y-edge fluctuation entering the cell of column c
    // whose plane vector is `cell`; with material planes the split needs that
    // cell's left and right neighbours, held by lanes l-1 and l+1.
    auto tsplit_y = [&](const typename RP::Lin& L, const T* cell, const T* a, T* bm, T* bp) {
        if constexpr (RP::NAUX > 0) {
            T lo[RP::NAUX > 0 ? RP::NAUX : 1], hi[RP::NAUX > 0 ? RP::NAUX : 1];
#pragma unroll
            for (int q = 0; q < RP::NAUX; q++) {
                lo[q] = shfl_up1(cell[N + q]);
                hi[q] = shfl_down1(cell[N + q]);
            }
            rp.template transverse_cells<1>(lo, cell + N, hi, a, bm, bp);
        } else {
            rp.template transverse<1>(L, a, bm, bp);
        }
    };
    // An x-edge fluctuation entering a cell whose neighbours below and above
    // have plane vectors lo and hi.
    auto tsplit_x = [&](const typename RP::Lin& L, const T* lo, const T* mid, const T* hi, const T* a,
                        T* bm, T* bp) {
        if constexpr (RP::NAUX > 0) rp.template transverse_cells<0>(lo + N, mid + N, hi + N, a, bm, bp);
        else rp.template transverse<0>(L, a, bm, bp);
    };

    int newton_n = 0, newton_s = 0;   // Newton updates and solves of this lane (SEEDED solvers)
    int guard_n = 0;                  // interior edges this lane recomputed in FP64
    int hh = 0;                       // halves of this lane's edges with a near-sonic transonic
                                      // speed, accumulated over the march (GUARD_DETECT)
    float g_lo = 3.0e38f, g_hi = 0.0f;   // range of the first field (GUARD_DETECT)
    // this lane's output cell of row k (from k = j0 on), advanced one row at a time
    T* orow = qout + (long long)(j0 + 2) * ld_x + x_offset + c;
    for (int k = j0 - 3; k < jend; k++) {
        T qc2[NP], ql2[NP];
        // material of cell (c-1, k), the neighbour below where A-dQ of x-edge
        // (c-1/2, k+1) enters
        T ql0[NP];
        if constexpr (RP::NAUX > 0) {
#pragma unroll
            for (int q = 0; q < RP::NAUX; q++) ql0[N + q] = shfl_up1(qc0[N + q]);
        }
        if (!fetch(k + 2, qc2, ql2)) return false;
        if constexpr (GUARD == GUARD_DETECT) {
            // the range of the first field (depth, density) over the cells
            // this lane reads: the guard's near-dry test is a ratio of two
            // of them, so a task whose range stays within 1/tau has no
            // near-dry edge
            g_lo = fminf(g_lo, fminf(float(qc2[0]), float(ql2[0])));
            g_hi = fmaxf(g_hi, fmaxf(float(qc2[0]), float(ql2[0])));
        }
        T rs_c2 = T(0), rs_l2 = T(0);
        if constexpr (RSC) {
            rs_c2 = rp.rs_of(qc2);
            rs_l2 = rp.rs_of(ql2);
        }

        // ---- y-edge between rows k+1 and k+2 of column c, x-edge c-1/2 of row k+1
        T Wy2[NW][N], sy2[NW], bm2[N], bp2[N];
        T t1[N], t2[N];     // x-splits of the y-fluctuations entering row k+1
        T nPm[N], nPp[N];   // ... entering row k+2
        T Wx[NW][N], sxw[NW], amdq1[N], apdq1[N];
        T BmAp1[N], BpAp1[N], BmAm1[N], BpAm1[N];
        T TAm[N], TAp[N], dqy_n[N], dhi[NW];
        // what the y-edge's results feed: the transverse sums entering row
        // k+1, B+dQ(k+1/2) + B-dQ(k+3/2) waiting for row k+1's update, and,
        // with CARRY_DOT, the dot products of the waves of y-edge (c, k+1/2)
        // with those of the edge above (the next row's dlo)
        auto y_tail = [&]() {
            if (trans && !trans2) {
#pragma unroll
                for (int m = 0; m < N; m++) {
                    TAm[m] = tyP_m[m] + t1[m];
                    TAp[m] = tyP_p[m] + t2[m];
                }
            }
#pragma unroll
            for (int m = 0; m < N; m++) dqy_n[m] = bp_pend[m] + bm2[m];
#pragma unroll
            for (int p = 0; p < NW; p++) {
                dhi[p] = T(0);
#pragma unroll
                for (int m = 0; m < N; m++)
                    if (CD && second && RP::template wave_nz<1>(p, m)) dhi[p] += Wy2[p][m] * Wy1[p][m];
            }
        };
        if constexpr (RP::PAIRED) {
            // both edges at once in the edge-normal frame: half .x the
            // x-edge (ql1 | qc1), half .y the y-edge (qc1 | qc2); the x-edge
            // of the first march row is solved too (its row is resident) and
            // left unused
            f2 QL[N], QR[N];
#pragma unroll
            for (int m = 0; m < N; m++) {
                QL[m] = make_float2(ql1[m], qc1[frame_comp(m, 1)]);
                QR[m] = make_float2(qc1[m], qc2[frame_comp(m, 1)]);
            }
            f2 W2[NW][N], s2[NW], am2[N], ap2[N];
            typename RP::LinP L2;
            bool badx = false, bady = false;
            rp.template normal_pair<GUARD == GUARD_REDO>(QL, QR, W2, s2, am2, ap2, L2, badx, bady, hh);
            const bool trans1 = trans && !trans2;
            f2 Tm[N], Tp[N], Um[N], Up[N];
            if (trans1) {
                // the wall-ghost form (the batched kernel) keeps the general
                // split: the subsonic one's code would push it past its
                // register cap into spills
                rp.template transverse_pair<!WALL_GHOSTS>(L2, am2, Tm, Tp);
                rp.template transverse_pair<!WALL_GHOSTS>(L2, ap2, Um, Up);
            }
            const bool yin = ye_lane && k + 2 >= 0 && k + 2 <= my;
            const bool xin = xe_lane && k + 1 >= 0 && k + 1 < my;
            // FP32 runs with the FP64 guard: in the step kernel a task with a
            // guarded or transonic edge is only marked (its speeds and flags
            // are left out, and the guard kernel recomputes it); the guard
            // kernel recomputes those edges in FP64
            // (GUARD_DETECT: near-sonic edges accumulate in hh, near-dry
            // ones show in the task's depth range; both are read at the end)
            if constexpr (GUARD == GUARD_REDO) {
                // only edges between cells of the ghosted grid: lanes of the
                // last band past column mx + 1 hold no state (zeros), and
                // would look near-dry
                const bool gvalid = c >= -1 && c <= mx + 1;
                const int gm = gvalid ? rp.guard_mask(QL, QR, L2) : 0;
                if (gm) {
                    rp.guard_redo(QL, QR, gm, trans1, W2, s2, am2, ap2, L2, Tm, Tp, Um, Up, badx, bady);
                    // count each interior edge once: the x-edge c-1/2 of row
                    // k+1 and the y-edge below row k+2 belong to the task
                    // whose output lanes and rows hold column c and that row
                    // (the grid's last edges to its last band and tile)
                    const bool own_c = lane >= 1 && lane <= BAND_W;
                    const bool xown =
                        ((own_c && c <= mx) || (lane == BAND_W + 1 && c == mx && i0 + BAND_W == mx)) &&
                        k + 1 >= j0 && k + 1 < jend;
                    const bool yown = own_c && c < mx && k + 2 >= j0 && (k + 2 < jend || k + 2 == my);
                    guard_n += int((gm & 1) && xown) + int((gm & 2) && yown);
                }
            }
#pragma unroll
            for (int p = 0; p < NW; p++) {
                sxw[p] = s2[p].x;
                sy2[p] = s2[p].y;
#pragma unroll
                for (int m = 0; m < N; m++) {
                    Wx[p][m] = W2[p][m].x;
                    Wy2[p][frame_comp(m, 1)] = W2[p][m].y;
                }
            }
#pragma unroll
            for (int m = 0; m < N; m++) {
                amdq1[m] = am2[m].x;
                apdq1[m] = ap2[m].x;
                bm2[frame_comp(m, 1)] = am2[m].y;
                bp2[frame_comp(m, 1)] = ap2[m].y;
            }
            if (trans2) {
                Lx_cur = rp.lin_half(L2, 0);
                Ly_cur = rp.lin_half(L2, 1);
            } else if (trans) {
#pragma unroll
                for (int m = 0; m < N; m++) {
                    BmAm1[m] = Tm[m].x; BpAm1[m] = Tp[m].x;
                    BmAp1[m] = Um[m].x; BpAp1[m] = Up[m].x;
                    t1[frame_comp(m, 1)] = Tm[m].y; t2[frame_comp(m, 1)] = Tp[m].y;
                    nPm[frame_comp(m, 1)] = Um[m].y; nPp[frame_comp(m, 1)] = Up[m].y;
                }
            }
            bad |= yin && bady;
            smy = fmax(smy, yin ? rp.max_speed(L2, 1) : T(0));
            bad |= xin && badx;
            smx = fmax(smx, xin ? rp.max_speed(L2, 0) : T(0));
            y_tail();
        } else {
            typename RP::Lin Ly;
            bool bady = false;
            // pressure seeds of the two normal problems from the network, for
            // edges with a strong jump (pressure ratio 2 or more); the whole
            // warp evaluates it for its x-edges when one of its lanes has
            // such an x-edge, and likewise for the y-edges
            T seed_x = T(0), seed_y = T(0);
            if constexpr (RP::SEEDED) {
                if (W.net) {
                    const bool okx = rp.seed_mild(ql1, qc1), oky = rp.seed_mild(qc1, qc2);
                    if (__any_sync(0xffffffffu, !okx)) {
                        float f[10], tr;
                        rp.template seed_features<0>(ql1, qc1, f, tr);
#pragma unroll
                        for (int m = 0; m < 10; m++) f[m] = (f[m] - W.net->mu[m]) / W.net->sig[m];
                        const float o = mlp_infer_warp(*W.net, f, W.xs, W.outs);
                        if (!okx) seed_x = T(tr * __expf(o));
                    }
                    if (__any_sync(0xffffffffu, !oky)) {
                        float f[10], tr;
                        rp.template seed_features<1>(qc1, qc2, f, tr);
#pragma unroll
                        for (int m = 0; m < 10; m++) f[m] = (f[m] - W.net->mu[m]) / W.net->sig[m];
                        const float o = mlp_infer_warp(*W.net, f, W.xs, W.outs);
                        if (!oky) seed_y = T(tr * __expf(o));
                    }
                }
                newton_n += rp.template normal_seeded<1>(qc1, qc2, seed_y, Wy2, sy2, bm2, bp2, Ly, bady);
                newton_s += 1;
            } else if constexpr (RSC) {
                rp.template normal_rs<1>(qc1, qc2, rs_c1, rs_c2, Wy2, sy2, bm2, bp2, Ly, bady);
            } else {
                rp.template normal<1>(qc1, qc2, Wy2, sy2, bm2, bp2, Ly, bady);
            }
            if (trans2) {
                Ly_cur = Ly;
            } else if (trans) {
                tsplit_y(Ly, qc1, bm2, t1, t2);
                tsplit_y(Ly, qc2, bp2, nPm, nPp);
            }
            y_tail();
            {
                const bool in = ye_lane && k + 2 >= 0 && k + 2 <= my;
                bad |= in && bady;
                smy = fmax(smy, in ? rp.max_speed(Ly) : T(0));
            }
            if (k >= j0 - 2) {
                typename RP::Lin Lx;
                bool badx = false;
                if constexpr (RP::SEEDED) {
                    newton_n += rp.template normal_seeded<0>(ql1, qc1, seed_x, Wx, sxw, amdq1, apdq1, Lx, badx);
                    newton_s += 1;
                } else if constexpr (RSC) {
                    rp.template normal_rs<0>(ql1, qc1, rs_l1, rs_c1, Wx, sxw, amdq1, apdq1, Lx, badx);
                } else {
                    rp.template normal<0>(ql1, qc1, Wx, sxw, amdq1, apdq1, Lx, badx);
                }
                if (trans2) {
                    Lx_cur = Lx;
                } else if (trans) {
                    tsplit_x(Lx, qc0, qc1, qc2, apdq1, BmAp1, BpAp1);
                    tsplit_x(Lx, ql0, ql1, ql2, amdq1, BmAm1, BpAm1);
                }
                const bool in = xe_lane && k + 1 >= 0 && k + 1 < my;
                bad |= in && badx;
                smx = fmax(smx, in ? rp.max_speed(Lx) : T(0));
            }
        }

        T Fn[N], Gn[N];
        // with option 2 the x-edge splits live in this block, and those of
        // row j0-1 feed G at y-edge (c, j0-1/2): start one row earlier (the
        // extra row's other results are not used)
        if (k >= j0 - (trans2 ? 2 : 1)) {
            // ---- limited corrections: F at x-edge (c-1/2, k+1), G at y-edge (c, k+1/2)
#pragma unroll
            for (int m = 0; m < N; m++) Fn[m] = Gn[m] = T(0);
            if (second) {
                // ratios of all waves of both edges (x: 0..NW-1, y:
                // NW..2NW-1), then one branch on the limiter
                T dl[2 * NW], dr[2 * NW], th[2 * NW], phi[2 * NW];
#pragma unroll
                for (int p = 0; p < NW; p++) {
                    const int src = (sxw[p] > T(0) ? lane - 1 : lane + 1) & 31;
                    dl[p] = dr[p] = T(0);
#pragma unroll
                    for (int m = 0; m < N; m++) {
                        if (!RP::template wave_nz<0>(p, m)) continue;
                        const T wu = shfl(Wx[p][m], src);
                        dl[p] += wu * Wx[p][m];
                        dr[p] += Wx[p][m] * Wx[p][m];
                    }
                }
#pragma unroll
                for (int p = 0; p < NW; p++) {
                    const bool upl = sy1[p] > T(0);
                    T dly = T(0), dry = T(0);
#pragma unroll
                    for (int m = 0; m < N; m++) {
                        if (!RP::template wave_nz<1>(p, m)) continue;
                        if constexpr (!CD) dly += (upl ? Wy0[p][m] : Wy2[p][m]) * Wy1[p][m];
                        dry += Wy1[p][m] * Wy1[p][m];
                    }
                    if constexpr (CD) dly = upl ? dlo[p] : dhi[p];
                    dl[NW + p] = dly;
                    dr[NW + p] = dry;
                }
                ratios<2 * NW>(dl, dr, th);
                limiter_phis<2 * NW>(limiter, th, phi);
#pragma unroll
                for (int p = 0; p < NW; p++) {
                    const T as = fabs(sxw[p]);
                    const T cf = T(0.5) * as * (T(1) - nux * as) * phi[p];
#pragma unroll
                    for (int m = 0; m < N; m++)
                        if (RP::template wave_nz<0>(p, m)) Fn[m] += cf * Wx[p][m];
                }
#pragma unroll
                for (int p = 0; p < NW; p++) {
                    const T as = fabs(sy1[p]);
                    const T cf = T(0.5) * as * (T(1) - nuy * as) * phi[NW + p];
#pragma unroll
                    for (int m = 0; m < N; m++)
                        if (RP::template wave_nz<1>(p, m)) Gn[m] += cf * Wy1[p][m];
                }
            }
            if (trans2) {
                // option 2: split the x-edge fluctuations of row k+1 together
                // with its limited correction (Fn holds only that so far) ...
                T apx[N], amx[N];
#pragma unroll
                for (int m = 0; m < N; m++) {
                    apx[m] = apdq1[m] - Fn[m];
                    amx[m] = amdq1[m] + Fn[m];
                }
                tsplit_x(Lx_cur, qc0, qc1, qc2, apx, BmAp1, BpAp1);
                tsplit_x(Lx_cur, ql0, ql1, ql2, amx, BmAm1, BpAm1);
                // ... and those of y-edge (c, k+1/2), now that its limited
                // correction (Gn so far) is known: the part entering row k+1
                // feeds F of row k+1 below, the part entering row k completes
                // row k's x-edge terms
                T bmL[N], bpL[N], sm_[N], sp_[N];
#pragma unroll
                for (int m = 0; m < N; m++) {
                    bmL[m] = bm_prev[m] + Gn[m];
                    bpL[m] = bp_pend[m] - Gn[m];
                }
                tsplit_y(Ly_prev, qc0, bmL, sm_, sp_);
                tsplit_y(Ly_prev, qc1, bpL, TAm, TAp);
#pragma unroll
                for (int m = 0; m < N; m++) {
                    const T dF = -hnuy * (sm_[m] + shfl_up1(sp_[m]));
                    XP0[m] -= dF;
                    XM0[m] += dF;
                }
            }
            // ---- transverse parts of F and G
            if (trans) {
#pragma unroll
                for (int m = 0; m < N; m++) {
                    Fn[m] -= hnuy * (TAm[m] + shfl_up1(TAp[m]));
                    Gn[m] -= hnux * (BpAp0[m] + BmAp1[m] + shfl_down1(BpAm0[m] + BmAm1[m]));
                }
            }
        }

        // ---- cell (c, k)
        if (k >= j0) {
            T xr[N];
#pragma unroll
            for (int m = 0; m < N; m++) xr[m] = shfl_down1(XM0[m]);
            T qn[N];
#pragma unroll
            for (int m = 0; m < N; m++)
                qn[m] = qc0[m] - nux * (XP0[m] + xr[m]) - nuy * (Z0[m] + Gn[m]);
            if (RP::POSITIVE) bad |= out_lane && !(qn[0] > T(0));
            else bad |= out_lane && qn[0] != qn[0];
            if (out_lane) {
                T* o = orow;
#pragma unroll
                for (int m = 0; m < N; m++) o[m * ld_field] = qn[m];
#pragma unroll
                for (int m = N; m < NP; m++) o[m * ld_field] = qc0[m];   // material, unchanged
                if (WALL_GHOSTS) {
                    const bool hx = c < 2 || c >= mx - 2, hy = k < 2 || k >= my - 2;
                    if (hx || hy) {
                        // mirrors of this cell, addressed from its own slot o
                        const int gi = c < 2 ? -1 - c : 2 * mx - 1 - c;
                        const int gj = k < 2 ? -1 - k : 2 * my - 1 - k;
                        T* ox = o + (gi - c);
                        T* oy = o + (long long)(gj - k) * ld_x;
                        T* oxy = oy + (gi - c);
#pragma unroll
                        for (int m = 0; m < N; m++) {
                            if (hx) ox[m * ld_field] = m == 1 ? -qn[m] : qn[m];
                            if (hy) oy[m * ld_field] = m == 2 ? -qn[m] : qn[m];
                            if (hx && hy) oxy[m * ld_field] = (m == 1 || m == 2) ? -qn[m] : qn[m];
                        }
                    }
                }
            }
        }

        if (k >= j0) orow += ld_x;
        // ---- rotate
#pragma unroll
        for (int m = 0; m < NP; m++) {
            qc0[m] = qc1[m]; qc1[m] = qc2[m]; ql1[m] = ql2[m];
        }
        rs_c1 = rs_c2;
        rs_l1 = rs_l2;
#pragma unroll
        for (int m = 0; m < N; m++) {
            Z0[m] = dqy_n[m] - Gn[m];
            bp_pend[m] = bp2[m];
            if (trans && !trans2) { tyP_m[m] = nPm[m]; tyP_p[m] = nPp[m]; }
            if (trans2) bm_prev[m] = bm2[m];
            XP0[m] = apdq1[m] - Fn[m];
            XM0[m] = amdq1[m] + Fn[m];
            if (trans) { BpAp0[m] = BpAp1[m]; BpAm0[m] = BpAm1[m]; }
        }
        if (trans2) Ly_prev = Ly_cur;
#pragma unroll
        for (int p = 0; p < NW; p++) {
            sy1[p] = sy2[p];
            if constexpr (CD) dlo[p] = dhi[p];
#pragma unroll
            for (int m = 0; m < N; m++) {
                if constexpr (!CD) Wy0[p][m] = Wy1[p][m];
                Wy1[p][m] = Wy2[p][m];
            }
        }
    }
    if constexpr (GUARD == GUARD_DETECT) {
        if (flagged) {
            if (c > mx + 1) {   // no state in these lanes
                g_lo = 3.0e38f;
                g_hi = 0.0f;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                g_lo = fminf(g_lo, __shfl_xor_sync(0xffffffffu, g_lo, o));
                g_hi = fmaxf(g_hi, __shfl_xor_sync(0xffffffffu, g_hi, o));
            }
            const bool dry = rp.guard_on() && !(g_lo >= rp.gtau * g_hi);
            const bool sonic = hh != 0 && c >= -1 && c <= mx + 1 && rp.guard_on();
            *flagged = dry || __any_sync(0xffffffffu, sonic);
        }
    }
    if constexpr (GUARD == GUARD_REDO) {
        if (W.guard && __any_sync(0xffffffffu, guard_n != 0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) guard_n += __shfl_xor_sync(0xffffffffu, guard_n, o);
            if (lane == 0) atomicAdd(W.guard, (unsigned long long)guard_n);
        }
    }
    if constexpr (RP::SEEDED) {
        if (W.newton) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                newton_n += __shfl_xor_sync(0xffffffffu, newton_n, o);
                newton_s += __shfl_xor_sync(0xffffffffu, newton_s, o);
            }
            if (lane == 0) {
                atomicAdd(&W.newton[0], (unsigned long long)newton_n);
                atomicAdd(&W.newton[1], (unsigned long long)newton_s);
            }
        }
    }
    __syncwarp();
    return true;
}

// Bounded drain of the copies still in flight after a failed wait.
__device__ __forceinline__ void drain_ring(WarpRing& W)
{
    for (int s = 0; s < NSTAGE; s++) (void)mbar_wait_bounded(&W.bars[s], (W.phase >> s) & 1u);
}

__device__ __forceinline__ WarpRing warp_ring(unsigned char* smem, int es, int neq)
{
    const int warp = threadIdx.x >> 5;
    WarpRing W;
    W.bars = reinterpret_cast<uint64_t*>(smem) + warp * NSTAGE;
    W.ring = smem + 128 + warp * NSTAGE * stage_bytes(es, neq);
    W.phase = 0;
    if ((threadIdx.x & 31) == 0) {
        for (int s = 0; s < NSTAGE; s++) mbar_init(&W.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    return W;
}

// The fused step over one grid.  The tensor maps of the two state buffers
// live in device global memory (64-byte aligned, written by the host before
// the launch); the kernel takes plain pointers to them.
// The band and rows of a warp task: the first nbig tasks cut rows
// [0, split) in tiles of TALL_TILES * tile_rows, the others the rows from
// split on in tiles of tile_rows; bands vary fastest.
template <class A>
__device__ __forceinline__ void task_extent(const A& a, int task, int& i0, int& j0, int& jend)
{
    if (task < a.nbig) {
        i0 = (task % a.nbands) * BAND_W;
        j0 = (task / a.nbands) * (TALL_TILES * a.tile_rows);
        jend = j0 + TALL_TILES * a.tile_rows;
    } else {
        const int t = task - a.nbig;
        i0 = (t % a.nbands) * BAND_W;
        j0 = a.split + (t / a.nbands) * a.tile_rows;
        jend = min(j0 + a.tile_rows, a.my);
    }
}

template <class RP, int MODE>
__global__ void __launch_bounds__(SWEEP_WARPS * 32, min_ctas<RP>::value)
    ctu_sweep_kernel(const CUtensorMap* map_a, const CUtensorMap* map_b, const SweepArgs<RP> a)
{
    using T = typename RP::real;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpRing W = warp_ring(smem, sizeof(T), RP::NPLANE);
    if constexpr (RP::SEEDED) {
        // the seed network after the rings: weights, then per-warp scratch
        W.newton = a.newton_updates;
        if (a.net) {
            unsigned char* base = smem + sweep_smem_bytes(sizeof(T), RP::NPLANE);
            MlpShared* ns = reinterpret_cast<MlpShared*>(base);
            mlp_load_shared(a.net, ns);
            W.net = ns;
            W.xs = reinterpret_cast<__nv_bfloat16*>(base + sizeof(MlpShared)) + warp * 32 * XP;
            W.outs = reinterpret_cast<float*>(base + sizeof(MlpShared) + SWEEP_WARPS * 32 * XP * 2) + warp * 32;
            __syncthreads();
        }
    }

    W.guard = a.guard_edges;
    const int cur = a.cur ? *a.cur : 0;
    const CUtensorMap* map = cur ? map_b : map_a;
    T* __restrict__ qout = cur ? a.qa : a.qb;
    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    const T nux = T(dt / a.dx), nuy = T(dt / a.dy);
    const bool second = a.order >= 2;

    // TMA precondition, checked instead of trusted: a 64-byte aligned map
    const bool map_ok = (reinterpret_cast<uintptr_t>(map) & 63) == 0;
    if (!map_ok && lane == 0) atomicOr(a.status, ST_BADARG);
    if (lane == 0 && map_ok) {
        acquire_tensormap(map);
        prefetch_tensormap(map);
    }
    __syncwarp();

    // warps per CTA: SWEEP_WARPS, or fewer to spread a small grid's tasks
    // over more SMs
    const int nw = blockDim.x >> 5;
    bool failed = false, bad = false;
    T smx = T(0), smy = T(0);
    // FP32 pair solvers detect the edges of the FP64 guard: a task that
    // meets one is queued for the guard kernel and contributes neither its
    // speeds nor its flags here (the guard kernel's recompute does)
    constexpr int GD = RP::PAIRED ? GUARD_DETECT : GUARD_NONE;
    for (int task = blockIdx.x * nw + warp; task < a.ntasks && !failed && map_ok;
         task += gridDim.x * nw) {
        int i0, j0, jend;
        task_extent(a, task, i0, j0, jend);
        bool fl = false, tb = false;
        T tx = T(0), ty = T(0);
        failed = !sweep_task<RP, false, MODE, GD>(a.rp, map, qout, a.mx, a.my, a.ld_x, a.ld_field,
                                             a.x_offset, i0, j0, jend, nux, nuy, a.limiter, second,
                                             a.transverse, W, tb, tx, ty, a.status, &fl);
        if (fl && a.gq) {
            if (lane == 0) {
                const unsigned slot = atomicAdd(&a.gq->count, 1u);
                if (a.gq_tasks) a.gq_tasks[slot] = task;
            }
        } else {
            bad |= tb;
            smx = fmax(smx, tx);
            smy = fmax(smy, ty);
        }
    }

    if (failed) {
        drain_ring(W);
        if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, ST_NONPHYS);
    double v = fmax(double(smx) / a.dx, double(smy) / a.dy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomic_max_nonneg(a.smax_bits, v);
}

// The guard kernel of an FP32 pair solver's step: recomputes the queued
// tasks (all tasks when the queue keeps no list) with the guarded and
// transonic edges in FP64, contributes their speeds and flags, and resets the
// queue.  Launched after the step kernel on the same stream; with an empty
// queue every block returns at once.
template <class RP, int MODE>
__global__ void __launch_bounds__(SWEEP_WARPS * 32)
    ctu_guard_kernel(const CUtensorMap* map_a, const CUtensorMap* map_b, const SweepArgs<RP> a)
{
    using T = typename RP::real;
    const unsigned n = a.gq->count;
    if (n == 0) {
        // nothing queued: the step kernel's speed maximum is complete
        if (a.dt_state && blockIdx.x == 0 && threadIdx.x == 0)
            dt_rule_apply(a.dt_state, a.cfl_desired, a.cfl_max, a.smax_bits);
        return;
    }
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpRing W = warp_ring(smem, sizeof(T), RP::NPLANE);
    W.guard = a.guard_edges;
    const int cur = a.cur ? *a.cur : 0;
    const CUtensorMap* map = cur ? map_b : map_a;
    T* __restrict__ qout = cur ? a.qa : a.qb;
    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    const T nux = T(dt / a.dx), nuy = T(dt / a.dy);
    const bool second = a.order >= 2;
    const bool map_ok = (reinterpret_cast<uintptr_t>(map) & 63) == 0;
    if (!map_ok && lane == 0) atomicOr(a.status, ST_BADARG);
    if (lane == 0 && map_ok) acquire_tensormap(map);
    __syncwarp();
    const int nw = blockDim.x >> 5;
    const int total = a.gq_tasks ? int(n) : a.ntasks;
    bool failed = false, bad = false;
    T smx = T(0), smy = T(0);
    for (int idx = blockIdx.x * nw + warp; idx < total && !failed && map_ok; idx += gridDim.x * nw) {
        const int task = a.gq_tasks ? a.gq_tasks[idx] : idx;
        int i0, j0, jend;
        task_extent(a, task, i0, j0, jend);
        failed = !sweep_task<RP, false, MODE, GUARD_REDO>(a.rp, map, qout, a.mx, a.my, a.ld_x,
                                                          a.ld_field, a.x_offset, i0, j0, jend, nux,
                                                          nuy, a.limiter, second, a.transverse, W,
                                                          bad, smx, smy, a.status);
    }
    if (failed) {
        drain_ring(W);
        if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, ST_NONPHYS);
    double v = fmax(double(smx) / a.dx, double(smy) / a.dy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomic_max_nonneg(a.smax_bits, v);
    // the last block to finish empties the queue for the next step and, when
    // asked, applies the time-step rule to the now complete speed maximum
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.gq->done, 1u) == gridDim.x - 1) {
            __threadfence();
            a.gq->count = 0;
            a.gq->done = 0;
            if (a.dt_state) dt_rule_apply(a.dt_state, a.cfl_desired, a.cfl_max, a.smax_bits);
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------ ghosts

template <typename T>
struct BcArgs {
    T* qa;
    T* qb;
    const int* cur;   // fill qa (cur == 0 or null) or qb (cur == 1)
    int mx, my, meqn;
    long long ld_x, ld_field, x_offset;
    int bc[4];
};

__device__ __forceinline__ int bc_map(int i, int n, int lo_kind, int hi_kind, bool& flip)
{
    for (int it = 0; it < 4 && (i < 0 || i >= n); it++) {
        const int kind = i < 0 ? lo_kind : hi_kind;
        if (kind == 0) {
            i = ((i % n) + n) % n;
        } else if (kind == 1) {
            i = i < 0 ? 0 : n - 1;
        } else {
            i = i < 0 ? -i - 1 : 2 * n - 1 - i;
            flip = !flip;
        }
    }
    return i;
}

template <typename T>
__global__ void bc_fill_kernel(const BcArgs<T> a)
{
    const int W = a.mx + 4;
    const long long total = 4LL * W + 4LL * a.my;
    T* q = (a.cur && *a.cur) ? a.qb : a.qa;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (t < 4LL * W) {
            const int jr = int(t / W);
            j = jr < 2 ? jr - 2 : a.my + jr - 2;
            i = int(t % W) - 2;
        } else {
            const long long u = t - 4LL * W;
            j = int(u / 4);
            const int ir = int(u % 4);
            i = ir < 2 ? ir - 2 : a.mx + ir - 2;
        }
        bool fx = false, fy = false;
        const int si = bc_map(i, a.mx, a.bc[0], a.bc[1], fx);
        const int sj = bc_map(j, a.my, a.bc[2], a.bc[3], fy);
        const long long dst = (long long)(j + 2) * a.ld_x + a.x_offset + i;
        const long long src = (long long)(sj + 2) * a.ld_x + a.x_offset + si;
        // all planes' loads first (at most BC_MAX_PLANES), so their latencies
        // overlap, then the stores
        T v[BC_MAX_PLANES];
#pragma unroll
        for (int m = 0; m < BC_MAX_PLANES; m++)
            if (m < a.meqn) v[m] = q[m * a.ld_field + src];
#pragma unroll
        for (int m = 0; m < BC_MAX_PLANES; m++)
            if (m < a.meqn) q[m * a.ld_field + dst] = ((m == 1 && fx) || (m == 2 && fy)) ? -v[m] : v[m];
    }
}

// ------------------------------------------------------------------ cell speeds

template <class RP>
__global__ void max_cell_speed_kernel(const RP rp, const typename RP::real* q, int mx, int my,
                                      long long ld_x, long long ld_field, long long x_offset,
                                      double dx, double dy, unsigned long long* out)
{
    // warps take rows, lanes columns.  The maxima of the x and y speeds are
    // kept in the state's precision and divided by dx, dy once: division by
    // a positive number preserves order, so the result equals the maximum of
    // the per-cell quotients.
    using T = typename RP::real;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T msx = T(0), msy = T(0);
    for (int j = blockIdx.x * nw + (threadIdx.x >> 5); j < my; j += gridDim.x * nw) {
        const T* row = q + (long long)(j + 2) * ld_x + x_offset;
        for (int i = lane; i < mx; i += 32) {
            T qq[RP::NPLANE];
            for (int m = 0; m < RP::NPLANE; m++) qq[m] = row[m * ld_field + i];
            T sx, sy;
            rp.cell_speeds(qq, sx, sy);
            msx = fmax(msx, sx);
            msy = fmax(msy, sy);
        }
    }
    double v = fmax(double(msx) / dx, double(msy) / dy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomic_max_nonneg(out, v);
}

}  // namespace mc
