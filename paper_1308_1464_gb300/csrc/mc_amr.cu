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
// the mean of its fine cells.  There is no refluxing.  Everything is enqueued
// on the caller's stream; the only synchronisation is the status check at
// the end.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "mc_internal.h"
#include "mc_multi.cuh"

namespace mc {

struct AmrPatchDev {
    int ci0, cj0, cw, ch;        // coarse cells covered
    int fw, fh;                  // fine interior size (ratio cw x ratio ch)
    long long ld_x, ld_field;    // fine layout
    void* q[2];                  // the patch's two state buffers
    long long ghost_begin;       // first ghost cell of this patch in the flat count
    long long cell_begin;        // first covered coarse cell in the flat count
};

struct AmrArgs {
    const AmrPatchDev* P;
    int npatch, ratio, nplane, cur;
    long long nghost, ncell;
    long long x_offset;          // element offset of cell 0 within a row (same for all layouts)
    const void* qc0;             // coarse state before its step (ghosts filled)
    const void* qc1;             // ... after its step (ghosts filled); average-down target
    long long c_ldx, c_ldf;
    double alpha;
};

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
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < a.nghost;
         t += (long long)gridDim.x * blockDim.x) {
        int p = 0;
        while (p + 1 < a.npatch && a.P[p + 1].ghost_begin <= t) p++;
        const AmrPatchDev& P = a.P[p];
        const long long g = t - P.ghost_begin;
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
        // another patch covering this fine cell?
        int src = -1, si = 0, sj = 0;
        for (int q = 0; q < a.npatch && src < 0; q++) {
            if (q == p) continue;
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

template <typename T>
__global__ void amr_average_kernel(const AmrArgs a)
{
    T* qc = static_cast<T*>(const_cast<void*>(a.qc1));
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < a.ncell;
         t += (long long)gridDim.x * blockDim.x) {
        int p = 0;
        while (p + 1 < a.npatch && a.P[p + 1].cell_begin <= t) p++;
        const AmrPatchDev& P = a.P[p];
        const long long k = t - P.cell_begin;
        const int ci = int(k % P.cw), cj = int(k / P.cw);
        const T* f = static_cast<const T*>(P.q[a.cur]);
        const T inv = T(1) / T(a.ratio * a.ratio);
        for (int m = 0; m < a.nplane; m++) {
            T s = T(0);
            for (int bj = 0; bj < a.ratio; bj++)
                for (int bi = 0; bi < a.ratio; bi++)
                    s += f[m * P.ld_field + (long long)(a.ratio * cj + bj + 2) * P.ld_x + a.x_offset +
                           a.ratio * ci + bi];
            qc[m * a.c_ldf + (long long)(P.cj0 + cj + 2) * a.c_ldx + a.x_offset + P.ci0 + ci] = s * inv;
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
    MultiGrid* grids = nullptr;   // the patches for the multi-grid fused step
    CUtensorMap* maps = nullptr;  // two per patch (64-byte aligned device array)
    long long* prefix = nullptr;
    int* status = nullptr;
    long long nghost = 0, ncell = 0, ntask = 0;
    int fine_in_b = 0;   // which buffer of every patch holds its current state
};

static void amr_free(mc_amr* a)
{
    if (!a) return;
    if (a->cctx) mc_destroy(a->cctx);
    cudaFree(a->desc);
    cudaFree(a->grids);
    cudaFree(a->maps);
    cudaFree(a->prefix);
    cudaFree(a->status);
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
    long long g = 0, c = 0, tk = 0;
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
        d.ghost_begin = g;
        d.cell_begin = c;
        g += 4LL * (fp.mx + 4) + 4LL * fp.my;
        c += (long long)d.cw * d.ch;
        A->host_desc.push_back(d);
    }
    A->nghost = g;
    A->ncell = c;
    A->ntask = tk;
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
    *out = A;
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
    a.nghost = A->nghost;
    a.ncell = A->ncell;
    a.x_offset = A->clay.x_offset;
    a.c_ldx = A->clay.ld_x;
    a.c_ldf = A->clay.ld_field;
    const int gblocks = (int)((A->nghost + 255) / 256 > 4096 ? 4096 : (A->nghost + 255) / 256);
    const int ablocks = (int)((A->ncell + 255) / 256 > 4096 ? 4096 : (A->ncell + 255) / 256);
    for (int n = 0; n < nsteps; n++) {
        void* qin = cb ? qc_b : qc_a;
        void* qout = cb ? qc_a : qc_b;
        mc_status st = mc_step(A->cctx, qin, qout, dt, nullptr, stream);   // fills qin's ghosts
        if (st == MC_OK) st = mc_bc_fill(A->cctx, qout, stream);
        if (st != MC_OK) return st;
        a.qc0 = qin;
        a.qc1 = qout;
        for (int sub = 0; sub < A->ratio && np > 0; sub++) {
            a.cur = fb;
            a.alpha = double(sub) / A->ratio;
            if (es == 8) amr_ghost_kernel<double><<<gblocks > 0 ? gblocks : 1, 256, 0, s>>>(a);
            else amr_ghost_kernel<float><<<gblocks > 0 ? gblocks : 1, 256, 0, s>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_error(e, "patch ghost fill");
            M.cur = fb;
            e = multi_launch(M);
            if (e != cudaSuccess) return cuda_error(e, "patch steps");
            fb ^= 1;
        }
        if (np > 0) {
            a.cur = fb;
            if (es == 8) amr_average_kernel<double><<<ablocks > 0 ? ablocks : 1, 256, 0, s>>>(a);
            else amr_average_kernel<float><<<ablocks > 0 ? ablocks : 1, 256, 0, s>>>(a);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_error(e, "average down");
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
