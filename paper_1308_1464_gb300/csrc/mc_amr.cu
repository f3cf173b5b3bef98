// mc_amr.cu -- refined patches on a coarse grid with their own time steps.
//
// The paper's "dynamic time stepping" kernel (§1.2, Table 1): each refined
// grid manages its own time step, and the values at refinement boundaries
// come from the adjacent grid by spatial and temporal interpolation.  Two
// levels in the Berger-Oliger manner: one coarse step of dt (the fused step
// on the whole coarse grid), then `ratio` fused steps of dt/ratio on every
// patch; before each, one kernel fills all patches' ghost layers, cell by
// cell: a copy from the other patch that covers that fine cell, or else the
// coarse state interpolated linearly in time (weight s/ratio between the
// coarse states before and after its step) and in space by the coarse
// cell's value plus MC-limited slopes, a conservative reconstruction.
// The patches' steps are one launch of the fused step over all of them
// (mc_multi.cuh).  Afterwards one kernel replaces every covered coarse cell by
// the mean of its fine cells.  With refluxing on (mc_amr_set_reflux), the
// coarse cells outside the patches get the flux correction of Berger &
// Colella: the flux the coarse step put through each patch-boundary edge is
// recorded (mc_edge_flux.cuh), the fine fluxes through the same edge are
// subtracted over the fine steps with weight 1/ratio^2 each, and the outside
// cell receives dt/d times the difference.  Edges on the domain boundary and
// edges whose outside cell lies in another patch are not corrected.
// Everything is enqueued on the caller's stream; the only synchronisation is
// the status check at the end.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mc_edge_flux.cuh"
#include "mc_internal.h"
#include "mc_multi.cuh"

namespace mc {

struct AmrPatchDev {
    int ci0, cj0, cw, ch;        // coarse cells covered
    int fw, fh;                  // fine interior size (ratio cw x ratio ch)
    long long ld_x, ld_field;    // fine layout
    void* q[2];                  // the patch's two state buffers
    int nb_begin, nb_count;      // the patches that reach into its ghost layers (AmrArgs::nb)
};

struct AmrArgs {
    const AmrPatchDev* P;
    const int* nb;               // neighbour lists, ascending patch index
    int npatch, ratio, nplane, cur;
    long long x_offset;          // element offset of cell 0 within a row (same for all layouts)
    const void* qc0;             // coarse state before its step (ghosts filled)
    const void* qc1;             // ... after its step (ghosts filled); average-down target
    long long c_ldx, c_ldf;
    double alpha;
};

// A coarse edge on a patch boundary that gets the flux correction: normal
// dir, high cell (ci, cj), the outside coarse cell (oi, oj) and the sign of
// its update from this edge (+1: the edge is the cell's high edge), the
// patch, and the high cell (fi, fj) of the first of the ratio fine edges
// along it in the patch's local indices.
struct RefluxEdge {
    int dir, ci, cj, oi, oj, sgn, patch, fi, fj;
};

template <class RP>
__global__ void amr_coarse_flux_kernel(const RP rp, const StateView<typename RP::real> V,
                                       const RefluxEdge* E, int n, typename RP::real dtdx,
                                       typename RP::real dtdy, const EdgeScheme S, double* D)
{
    using T = typename RP::real;
    constexpr int N = RP::NEQ;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        T F[N];
        if (E[e].dir == 0) edge_flux<RP, 0>(rp, V, E[e].ci, E[e].cj, dtdx, dtdy, S, F);
        else edge_flux<RP, 1>(rp, V, E[e].ci, E[e].cj, dtdy, dtdx, S, F);
#pragma unroll
        for (int m = 0; m < N; m++) D[(long long)e * N + m] = double(F[m]);
    }
}

template <class RP>
__global__ void amr_fine_flux_kernel(const RP rp, const AmrPatchDev* P, int cur, long long x_offset,
                                     const RefluxEdge* E, int n, int ratio, typename RP::real dtdx,
                                     typename RP::real dtdy, const EdgeScheme S, double* D)
{
    using T = typename RP::real;
    constexpr int N = RP::NEQ;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const AmrPatchDev& d = P[E[e].patch];
        const StateView<T> V{static_cast<const T*>(d.q[cur]), d.ld_x, d.ld_field, x_offset};
        double acc[N];
#pragma unroll
        for (int m = 0; m < N; m++) acc[m] = 0.0;
        for (int t = 0; t < ratio; t++) {
            T F[N];
            if (E[e].dir == 0) edge_flux<RP, 0>(rp, V, E[e].fi, E[e].fj + t, dtdx, dtdy, S, F);
            else edge_flux<RP, 1>(rp, V, E[e].fi + t, E[e].fj, dtdy, dtdx, S, F);
#pragma unroll
            for (int m = 0; m < N; m++) acc[m] += double(F[m]);
        }
        const double w = 1.0 / (double(ratio) * ratio);
#pragma unroll
        for (int m = 0; m < N; m++) D[(long long)e * N + m] -= w * acc[m];
    }
}

// the correction of the outside cells of edges [begin, end), whose outside
// cells are distinct (one normal and sign class)
template <typename T>
__global__ void amr_reflux_kernel(T* qc, long long ldx, long long ldf, long long x_offset,
                                  const RefluxEdge* E, int begin, int end, int meqn, double dtdx,
                                  double dtdy, const double* D)
{
    for (int e = begin + blockIdx.x * blockDim.x + threadIdx.x; e < end; e += gridDim.x * blockDim.x) {
        T* c = qc + (long long)(E[e].oj + 2) * ldx + x_offset + E[e].oi;
        const double f = E[e].sgn * (E[e].dir == 0 ? dtdx : dtdy);
        for (int m = 0; m < meqn; m++) c[m * ldf] += T(f * D[(long long)e * meqn + m]);
    }
}

__device__ __forceinline__ int floordiv_(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

template <typename T>
__device__ __forceinline__ T mc_slope(T a, T b)
{
    // minmod(2a, 2b, (a + b)/2)
    if (a * b <= T(0)) return T(0);
    const T c = T(0.5) * (a + b);
    T s = fmin(fabs(T(2) * a), fabs(T(2) * b));
    s = fmin(s, fabs(c));
    return c > T(0) ? s : -s;
}

template <typename T>
__global__ void amr_ghost_kernel(const AmrArgs a)
{
    const T* qc0 = static_cast<const T*>(a.qc0);
    const T* qc1 = static_cast<const T*>(a.qc1);
    const T alpha = T(a.alpha);
    // patches along y of the grid, each patch's ghost cells along x
    for (int p = blockIdx.y; p < a.npatch; p += gridDim.y) {
        const AmrPatchDev& P = a.P[p];
        const int nghost = 4 * (P.fw + 4) + 4 * P.fh;
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nghost; g += gridDim.x * blockDim.x) {
            const int rowlen = P.fw + 4;
            int fi, fj;
            if (g < 2LL * rowlen) {                       // two rows below
                fj = int(g / rowlen) - 2;
                fi = int(g % rowlen) - 2;
            } else if (g < 4LL * rowlen) {                // two rows above
                const long long h = g - 2LL * rowlen;
                fj = P.fh + int(h / rowlen);
                fi = int(h % rowlen) - 2;
            } else {                                      // two columns each side of the interior rows
                const long long h = g - 4LL * rowlen;
                fj = int(h >> 2);
                const int k = int(h & 3);
                fi = k < 2 ? k - 2 : P.fw + k - 2;
            }
            const int gx = a.ratio * P.ci0 + fi, gy = a.ratio * P.cj0 + fj;
            T* dst = static_cast<T*>(P.q[a.cur]) + (long long)(fj + 2) * P.ld_x + a.x_offset + fi;
            // another patch covering this fine cell? (only the neighbours can)
            int src = -1, si = 0, sj = 0;
            for (int n = 0; n < P.nb_count && src < 0; n++) {
                const int q = a.nb[P.nb_begin + n];
                const int qi = gx - a.ratio * a.P[q].ci0, qj = gy - a.ratio * a.P[q].cj0;
                if (qi >= 0 && qi < a.P[q].fw && qj >= 0 && qj < a.P[q].fh) {
                    src = q;
                    si = qi;
                    sj = qj;
                }
            }
            if (src >= 0) {
                const AmrPatchDev& Q = a.P[src];
                const T* s0 = static_cast<const T*>(Q.q[a.cur]) + (long long)(sj + 2) * Q.ld_x + a.x_offset + si;
                for (int m = 0; m < a.nplane; m++) dst[m * P.ld_field] = s0[m * Q.ld_field];
                continue;
            }
            // the coarse reconstruction at the fine cell centre
            const int cx = floordiv_(gx, a.ratio), cy = floordiv_(gy, a.ratio);
            const T ox = (T(gx - a.ratio * cx) + T(0.5)) / T(a.ratio) - T(0.5);
            const T oy = (T(gy - a.ratio * cy) + T(0.5)) / T(a.ratio) - T(0.5);
            const long long c = (long long)(cy + 2) * a.c_ldx + a.x_offset + cx;
            for (int m = 0; m < a.nplane; m++) {
                const long long b = m * a.c_ldf + c;
                auto qt = [&](long long o) { return (T(1) - alpha) * qc0[b + o] + alpha * qc1[b + o]; };
                const T q = qt(0);
                const T sx = mc_slope(q - qt(-1), qt(1) - q);
                const T sy = mc_slope(q - qt(-a.c_ldx), qt(a.c_ldx) - q);
                dst[m * P.ld_field] = q + ox * sx + oy * sy;
            }
        }
    }
}

template <typename T>
__global__ void amr_average_kernel(const AmrArgs a)
{
    T* qc = static_cast<T*>(const_cast<void*>(a.qc1));
    for (int p = blockIdx.y; p < a.npatch; p += gridDim.y) {
        const AmrPatchDev& P = a.P[p];
        const int ncell = P.cw * P.ch;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ncell; k += gridDim.x * blockDim.x) {
            const int ci = k % P.cw, cj = k / P.cw;
            const T* f = static_cast<const T*>(P.q[a.cur]);
            const T inv = T(1) / T(a.ratio * a.ratio);
            for (int m = 0; m < a.nplane; m++) {
                T s = T(0);
                const long long base = m * P.ld_field + (long long)(a.ratio * cj + 2) * P.ld_x + a.x_offset +
                                       a.ratio * ci;
                bool done = false;
                if constexpr (sizeof(T) == 4) {
                    if (a.ratio == 2) {
                        // the fine pair of a row in one 8-byte load: rows are
                        // 128-byte padded and cell 0 sits at element 4, so base
                        // is even; the same summation order as the loop
                        const float2 u = *reinterpret_cast<const float2*>(f + base);
                        const float2 w = *reinterpret_cast<const float2*>(f + base + P.ld_x);
                        s += u.x;
                        s += u.y;
                        s += w.x;
                        s += w.y;
                        done = true;
                    }
                }
                if (!done)
                    for (int bj = 0; bj < a.ratio; bj++)
                        for (int bi = 0; bi < a.ratio; bi++) s += f[base + (long long)bj * P.ld_x + bi];
                qc[m * a.c_ldf + (long long)(P.cj0 + cj + 2) * a.c_ldx + a.x_offset + P.ci0 + ci] = s * inv;
            }
        }
    }
}

}  // namespace mc

using namespace mc;

struct mc_amr {
    mc_problem coarse, fine;      // fine: the patches' scheme (sizes per patch)
    mc_layout clay;
    int ratio;
    mc_ctx* cctx;
    std::vector<mc_amr_patch> patches;
    std::vector<AmrPatchDev> host_desc;
    AmrPatchDev* desc = nullptr;
    int* nb = nullptr;            // neighbour lists of the patches (AmrPatchDev::nb_begin)
    MultiGrid* grids = nullptr;   // the patches for the multi-grid fused step
    CUtensorMap* maps = nullptr;  // two per patch (64-byte aligned device array)
    long long* prefix = nullptr;
    int* status = nullptr;
    int max_ghost = 0, max_cell = 0;   // largest per-patch ghost and covered-cell counts
    long long ntask = 0;
    int fine_in_b = 0;   // which buffer of every patch holds its current state
    int reflux = 0;
    RefluxEdge* edges = nullptr;  // corrected edges, grouped by (dir, sgn) class
    int nedge = 0;
    int cls[5] = {0, 0, 0, 0, 0}; // class boundaries in edges
    double* D = nullptr;          // nedge x meqn flux differences
};

namespace {

bool covered_by(const std::vector<mc_amr_patch>& P, int i, int j)
{
    for (const auto& a : P)
        if (i >= a.ci0 && i < a.ci0 + a.cw && j >= a.cj0 && j < a.cj0 + a.ch) return true;
    return false;
}

// the corrected edges of all patches, grouped by (dir, sgn): x-edges whose
// outside cell lies below in x (+1), above (-1), then the y-edges alike
std::vector<RefluxEdge> reflux_edges(const mc_problem& pc, int ratio, const std::vector<mc_amr_patch>& P,
                                     int* cls)
{
    std::vector<RefluxEdge> out;
    for (int c = 0; c < 4; c++) {
        cls[c] = (int)out.size();
        const int dir = c / 2, sgn = c % 2 == 0 ? 1 : -1;
        for (int p = 0; p < (int)P.size(); p++) {
            const mc_amr_patch& a = P[p];
            const int len = dir == 0 ? a.ch : a.cw;
            for (int k = 0; k < len; k++) {
                RefluxEdge e;
                e.dir = dir;
                e.sgn = sgn;
                e.patch = p;
                if (dir == 0) {
                    e.cj = e.oj = a.cj0 + k;
                    e.ci = sgn > 0 ? a.ci0 : a.ci0 + a.cw;
                    e.oi = sgn > 0 ? a.ci0 - 1 : a.ci0 + a.cw;
                    e.fi = sgn > 0 ? 0 : ratio * a.cw;
                    e.fj = ratio * k;
                } else {
                    e.ci = e.oi = a.ci0 + k;
                    e.cj = sgn > 0 ? a.cj0 : a.cj0 + a.ch;
                    e.oj = sgn > 0 ? a.cj0 - 1 : a.cj0 + a.ch;
                    e.fi = ratio * k;
                    e.fj = sgn > 0 ? 0 : ratio * a.ch;
                }
                if (e.oi < 0 || e.oi >= pc.mx || e.oj < 0 || e.oj >= pc.my) continue;
                if (covered_by(P, e.oi, e.oj)) continue;
                out.push_back(e);
            }
        }
    }
    cls[4] = (int)out.size();
    return out;
}

int grid_of(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : int(b);
}

// coarse (record the coarse step's fluxes from its filled input q) or fine
// (subtract the fluxes of every patch's current buffer `cur`)
template <class RP>
cudaError_t flux_launch_t(const mc_amr* A, bool coarse, const void* q, int cur, double dt, cudaStream_t s)
{
    using T = typename RP::real;
    RP rp;
    rp.setup(A->coarse.param, A->coarse.efix);
    const EdgeScheme S{A->coarse.limiter, A->coarse.order >= 2, A->coarse.transverse};
    const int blocks = grid_of(A->nedge, 128);
    if (coarse) {
        const StateView<T> V{static_cast<const T*>(q), A->clay.ld_x, A->clay.ld_field, A->clay.x_offset};
        amr_coarse_flux_kernel<RP><<<blocks, 128, 0, s>>>(rp, V, A->edges, A->nedge, T(dt / A->coarse.dx),
                                                           T(dt / A->coarse.dy), S, A->D);
    } else {
        amr_fine_flux_kernel<RP><<<blocks, 128, 0, s>>>(rp, A->desc, cur, A->clay.x_offset, A->edges, A->nedge,
                                                         A->ratio, T(dt / A->ratio / A->fine.dx),
                                                         T(dt / A->ratio / A->fine.dy), S, A->D);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t flux_launch_dtype(const mc_amr* A, bool coarse, const void* q, int cur, double dt, cudaStream_t s)
{
    switch (A->coarse.solver) {
    case MC_ACOUSTICS: return flux_launch_t<AcousticsRP<T>>(A, coarse, q, cur, dt, s);
    case MC_SWE_ROE: return flux_launch_t<SweRP<T>>(A, coarse, q, cur, dt, s);
    case MC_ADVECTION: return flux_launch_t<AdvectionRP<T>>(A, coarse, q, cur, dt, s);
    case MC_EULER_GODUNOV: return flux_launch_t<EulerGodunovRP<T>>(A, coarse, q, cur, dt, s);
    default: return flux_launch_t<EulerRP<T>>(A, coarse, q, cur, dt, s);
    }
}

cudaError_t flux_launch(const mc_amr* A, bool coarse, const void* q, int cur, double dt, cudaStream_t s)
{
    if (A->nedge == 0) return cudaSuccess;
    return A->clay.elem_bytes == 8 ? flux_launch_dtype<double>(A, coarse, q, cur, dt, s)
                                   : flux_launch_dtype<float>(A, coarse, q, cur, dt, s);
}

cudaError_t reflux_apply(const mc_amr* A, void* qc, double dt, cudaStream_t s)
{
    const int meqn = solver_meqn(A->coarse.solver);
    for (int c = 0; c < 4; c++) {
        const int b = A->cls[c], e = A->cls[c + 1];
        if (e <= b) continue;
        const int blocks = grid_of(e - b, 128);
        if (A->clay.elem_bytes == 8)
            amr_reflux_kernel<double><<<blocks, 128, 0, s>>>(static_cast<double*>(qc), A->clay.ld_x, A->clay.ld_field,
                                                             A->clay.x_offset, A->edges, b, e, meqn,
                                                             dt / A->coarse.dx, dt / A->coarse.dy, A->D);
        else
            amr_reflux_kernel<float><<<blocks, 128, 0, s>>>(static_cast<float*>(qc), A->clay.ld_x, A->clay.ld_field,
                                                            A->clay.x_offset, A->edges, b, e, meqn,
                                                            dt / A->coarse.dx, dt / A->coarse.dy, A->D);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace

static void amr_free(mc_amr* a)
{
    if (!a) return;
    if (a->cctx) mc_destroy(a->cctx);
    cudaFree(a->desc);
    cudaFree(a->nb);
    cudaFree(a->grids);
    cudaFree(a->maps);
    cudaFree(a->prefix);
    cudaFree(a->status);
    cudaFree(a->edges);
    cudaFree(a->D);
    delete a;
}

static cudaError_t multi_launch(const MultiLaunch& L)
{
    switch (L.prob.solver) {
    case MC_ACOUSTICS: return multi_launch_acoustics(L);
    case MC_SWE_ROE: return multi_launch_swe(L);
    case MC_ADVECTION: return multi_launch_advection(L);
    case MC_EULER_GODUNOV: return multi_launch_euler_godunov(L);
    default: return multi_launch_euler(L);
    }
}

extern "C" {

mc_status mc_amr_fine_problem(const mc_problem* coarse, int32_t ratio, const mc_amr_patch* patch,
                              mc_problem* out)
{
    if (!coarse || !patch || !out) return set_error(MC_EINVAL, "NULL argument");
    if (ratio < 1 || ratio > 16) return set_error(MC_EINVAL, "refinement ratio %d out of range", ratio);
    *out = *coarse;
    out->mx = ratio * patch->cw;
    out->my = ratio * patch->ch;
    out->dx = coarse->dx / ratio;
    out->dy = coarse->dy / ratio;
    for (int k = 0; k < 4; k++) out->bc[k] = MC_BC_EXTRAP;   // ghosts come from the coupling
    mc_layout lay;
    return mc_layout_of(out, &lay);
}

mc_status mc_amr_create(const mc_problem* coarse, int32_t ratio, const mc_amr_patch* patches,
                        int32_t npatch, mc_amr** out)
{
    if (!out || !coarse || (npatch > 0 && !patches)) return set_error(MC_EINVAL, "NULL argument");
    *out = nullptr;
    if (npatch < 0 || npatch > 4096) return set_error(MC_EINVAL, "npatch out of range");
    if (coarse->solver == MC_ACOUSTICS_VAR)
        return set_error(MC_ENOTSUP, "refined patches do not carry material planes");
    for (int k = 0; k < 4; k++)
        if (coarse->bc[k] == MC_BC_GIVEN)
            return set_error(MC_EINVAL, "the coarse grid's ghosts must come from its boundary kinds "
                             "(MC_BC_GIVEN sides need a fill before every coarse step)");
    mc_layout clay;
    mc_status st = mc_layout_of(coarse, &clay);
    if (st != MC_OK) return st;
    for (int p = 0; p < npatch; p++) {
        const mc_amr_patch& a = patches[p];
        if (a.cw < 1 || a.ch < 1 || a.ci0 < 0 || a.cj0 < 0 || a.ci0 + a.cw > coarse->mx ||
            a.cj0 + a.ch > coarse->my)
            return set_error(MC_EINVAL, "patch %d leaves the coarse interior", p);
        for (int q = 0; q < p; q++) {
            const mc_amr_patch& b = patches[q];
            if (a.ci0 < b.ci0 + b.cw && b.ci0 < a.ci0 + a.cw && a.cj0 < b.cj0 + b.ch && b.cj0 < a.cj0 + a.ch)
                return set_error(MC_EINVAL, "patches %d and %d overlap", q, p);
        }
        if (!a.qa || !a.qb || a.qa == a.qb) return set_error(MC_EINVAL, "patch %d needs two buffers", p);
    }
    mc_amr* A = new (std::nothrow) mc_amr();
    if (!A) return set_error(MC_ENOMEM, "allocation failed");
    A->coarse = *coarse;
    A->clay = clay;
    A->ratio = ratio;
    A->patches.assign(patches, patches + npatch);
    st = mc_create(coarse, &A->cctx);
    if (st != MC_OK) {
        amr_free(A);
        return st;
    }
    long long tk = 0;
    std::vector<MultiGrid> grids;
    std::vector<CUtensorMap> maps(2 * (size_t)(npatch > 0 ? npatch : 1));
    std::vector<long long> prefix(1, 0);
    for (int p = 0; p < npatch; p++) {
        mc_problem fp;
        st = mc_amr_fine_problem(coarse, ratio, &patches[p], &fp);
        if (st != MC_OK) {
            amr_free(A);
            return st;
        }
        A->fine = fp;
        mc_layout fl;
        mc_layout_of(&fp, &fl);
        MultiGrid mg;
        mg.mx = fp.mx;
        mg.my = fp.my;
        mg.nbands = (fp.mx + BAND_W - 1) / BAND_W;
        mg.tile_rows = fp.my < DEFAULT_TILE_ROWS ? fp.my : DEFAULT_TILE_ROWS;
        mg.ld_x = fl.ld_x;
        mg.ld_field = fl.ld_field;
        mg.q[0] = patches[p].qa;
        mg.q[1] = patches[p].qb;
        grids.push_back(mg);
        tk += (long long)mg.nbands * ((fp.my + mg.tile_rows - 1) / mg.tile_rows);
        prefix.push_back(tk);
        for (int k = 0; k < 2; k++) {
            cudaError_t e = encode_state_map(&maps[2 * p + k], mg.q[k], (int)fl.elem_bytes, (int)fl.meqn,
                                             fl.ld_x, fp.my, fl.ld_field);
            if (e != cudaSuccess) {
                amr_free(A);
                return set_error(MC_EINVAL, "tensor map of patch %d buffer %d (16-byte aligned?)", p, k);
            }
        }
        AmrPatchDev d;
        d.ci0 = patches[p].ci0;
        d.cj0 = patches[p].cj0;
        d.cw = patches[p].cw;
        d.ch = patches[p].ch;
        d.fw = fp.mx;
        d.fh = fp.my;
        d.ld_x = fl.ld_x;
        d.ld_field = fl.ld_field;
        d.q[0] = patches[p].qa;
        d.q[1] = patches[p].qb;
        d.nb_begin = d.nb_count = 0;
        A->max_ghost = std::max(A->max_ghost, 4 * (fp.mx + 4) + 4 * fp.my);
        A->max_cell = std::max(A->max_cell, d.cw * d.ch);
        A->host_desc.push_back(d);
    }
    A->ntask = tk;
    // neighbour lists: the patches whose cells fall in a patch's two fine
    // ghost layers, in ascending index order
    std::vector<int> nbl;
    for (int p = 0; p < npatch; p++) {
        AmrPatchDev& d = A->host_desc[p];
        d.nb_begin = (int)nbl.size();
        const long long x0 = (long long)ratio * d.ci0 - 2, x1 = (long long)ratio * d.ci0 + d.fw + 2;
        const long long y0 = (long long)ratio * d.cj0 - 2, y1 = (long long)ratio * d.cj0 + d.fh + 2;
        for (int q = 0; q < npatch; q++) {
            if (q == p) continue;
            const AmrPatchDev& e = A->host_desc[q];
            const long long u0 = (long long)ratio * e.ci0, u1 = u0 + e.fw;
            const long long v0 = (long long)ratio * e.cj0, v1 = v0 + e.fh;
            if (u0 < x1 && x0 < u1 && v0 < y1 && y0 < v1) nbl.push_back(q);
        }
        d.nb_count = (int)nbl.size() - d.nb_begin;
    }
    cudaError_t e0 = cudaMalloc(&A->status, sizeof(int));
    if (e0 == cudaSuccess) e0 = cudaMemset(A->status, 0, sizeof(int));
    if (e0 != cudaSuccess) {
        amr_free(A);
        return cuda_error(e0, "status word");
    }
    if (npatch > 0) {
        cudaError_t e = cudaMalloc(&A->desc, sizeof(AmrPatchDev) * npatch);
        if (e == cudaSuccess)
            e = cudaMemcpy(A->desc, A->host_desc.data(), sizeof(AmrPatchDev) * npatch, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&A->nb, sizeof(int) * (nbl.size() + 1));
        if (e == cudaSuccess && !nbl.empty())
            e = cudaMemcpy(A->nb, nbl.data(), sizeof(int) * nbl.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&A->grids, sizeof(MultiGrid) * npatch);
        if (e == cudaSuccess)
            e = cudaMemcpy(A->grids, grids.data(), sizeof(MultiGrid) * npatch, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&A->maps, sizeof(CUtensorMap) * 2 * npatch);
        if (e == cudaSuccess)
            e = cudaMemcpy(A->maps, maps.data(), sizeof(CUtensorMap) * 2 * npatch, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&A->prefix, sizeof(long long) * (npatch + 1));
        if (e == cudaSuccess)
            e = cudaMemcpy(A->prefix, prefix.data(), sizeof(long long) * (npatch + 1), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            amr_free(A);
            return cuda_error(e, "patch descriptors");
        }
    }
    {
        std::vector<RefluxEdge> edges = reflux_edges(*coarse, ratio, A->patches, A->cls);
        A->nedge = (int)edges.size();
        if (A->nedge > 0) {
            const int meqn = solver_meqn(coarse->solver);
            cudaError_t e = cudaMalloc(&A->edges, sizeof(RefluxEdge) * A->nedge);
            if (e == cudaSuccess)
                e = cudaMemcpy(A->edges, edges.data(), sizeof(RefluxEdge) * A->nedge, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMalloc(&A->D, sizeof(double) * (size_t)A->nedge * meqn);
            if (e != cudaSuccess) {
                amr_free(A);
                return cuda_error(e, "reflux edges");
            }
        }
    }
    *out = A;
    return MC_OK;
}

mc_status mc_amr_set_reflux(mc_amr* A, int32_t on)
{
    if (!A) return set_error(MC_EINVAL, "NULL argument");
    if (on != 0 && on != 1) return set_error(MC_EINVAL, "reflux must be 0 or 1");
    A->reflux = on;
    return MC_OK;
}

mc_status mc_amr_destroy(mc_amr* A)
{
    amr_free(A);
    return MC_OK;
}

mc_status mc_amr_advance(mc_amr* A, void* qc_a, void* qc_b, int32_t nsteps, double dt,
                         int32_t* coarse_in_b, int32_t* fine_in_b, void* stream)
{
    if (!A || !qc_a || !qc_b || qc_a == qc_b) return set_error(MC_EINVAL, "NULL or equal coarse buffers");
    if (nsteps < 0 || !(dt >= 0.0) || !isfinite(dt)) return set_error(MC_EINVAL, "bad nsteps or dt");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int np = (int)A->patches.size();
    const int es = (int)A->clay.elem_bytes;
    int cb = 0, fb = A->fine_in_b;
    MultiLaunch M{A->fine, A->grids, A->maps, A->prefix, np, 0, A->ntask, A->clay.x_offset,
                  dt / A->ratio / A->fine.dx, dt / A->ratio / A->fine.dy, A->status, s};
    AmrArgs a;
    a.P = A->desc;
    a.npatch = np;
    a.ratio = A->ratio;
    a.nplane = (int)A->clay.meqn;
    a.nb = A->nb;
    a.x_offset = A->clay.x_offset;
    a.c_ldx = A->clay.ld_x;
    a.c_ldf = A->clay.ld_field;
    // one grid row of blocks per patch (patches beyond 65535 wrap), enough
    // blocks along x for the largest patch
    const dim3 ggrid((unsigned)std::max(1, std::min(64, (A->max_ghost + 255) / 256)),
                     (unsigned)std::max(1, std::min(np, 65535)));
    const dim3 agrid((unsigned)std::max(1, std::min(64, (A->max_cell + 255) / 256)),
                     (unsigned)std::max(1, std::min(np, 65535)));
    for (int n = 0; n < nsteps; n++) {
        void* qin = cb ? qc_b : qc_a;
        void* qout = cb ? qc_a : qc_b;
        const bool rf = A->reflux && np > 0 && A->nedge > 0;
        mc_status st = mc_step(A->cctx, qin, qout, dt, nullptr, stream);   // fills qin's ghosts
        if (st == MC_OK) st = mc_bc_fill(A->cctx, qout, stream);
        if (st != MC_OK) return st;
        if (rf) {
            cudaError_t e = flux_launch(A, true, qin, 0, dt, s);
            if (e != cudaSuccess) return cuda_error(e, "coarse boundary fluxes");
        }
        a.qc0 = qin;
        a.qc1 = qout;
        for (int sub = 0; sub < A->ratio && np > 0; sub++) {
            a.cur = fb;
            a.alpha = double(sub) / A->ratio;
            if (es == 8) amr_ghost_kernel<double><<<ggrid, 256, 0, s>>>(a);
            else amr_ghost_kernel<float><<<ggrid, 256, 0, s>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_error(e, "patch ghost fill");
            if (rf) {
                e = flux_launch(A, false, nullptr, fb, dt, s);
                if (e != cudaSuccess) return cuda_error(e, "fine boundary fluxes");
            }
            M.cur = fb;
            e = multi_launch(M);
            if (e != cudaSuccess) return cuda_error(e, "patch steps");
            fb ^= 1;
        }
        if (np > 0) {
            a.cur = fb;
            if (es == 8) amr_average_kernel<double><<<agrid, 256, 0, s>>>(a);
            else amr_average_kernel<float><<<agrid, 256, 0, s>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_error(e, "average down");
            if (rf) {
                e = reflux_apply(A, qout, dt, s);
                if (e != cudaSuccess) return cuda_error(e, "flux correction");
            }
            st = mc_bc_fill(A->cctx, qout, stream);
            if (st != MC_OK) return st;
        }
        cb ^= 1;
    }
    A->fine_in_b = fb;
    mc_status st = ctx_check_status(A->cctx, stream);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, A->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(A->status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "patch status");
    if (st == MC_OK && (h & ST_BADARG)) st = set_error(MC_EINVAL, "a patch's tensor map or box is misaligned");
    if (st == MC_OK && (h & ST_TIMEOUT)) st = set_error(MC_ETIMEOUT, "a bounded device wait gave up");
    if (st == MC_OK && (h & ST_NONPHYS)) st = set_error(MC_ENONPHYS, "non-physical state met on a patch");
    if (coarse_in_b) *coarse_in_b = cb;
    if (fine_in_b) *fine_in_b = A->fine_in_b;
    return st;
}

}  // extern "C"
