// mc_batch.cu -- C ABI of the batched form: many uneven wall-bounded
// patches, each with its own time step, advanced by one persistent launch
// captured in a CUDA graph (mc_batch_advance), or by one launch per patch per
// step for comparison (mc_batch_advance_plain).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "mc_batch.cuh"
#include "mc_internal.h"

namespace mc {

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                             const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                             const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// dt of one patch for the per-patch launch loop
__global__ void patch_dt_kernel(const unsigned long long* smax_prev, double cfl, double* dt,
                                double* dt_used)
{
    const double s = __longlong_as_double((long long)*smax_prev);
    const double v = s > 0.0 ? cfl / s : 0.0;
    *dt = v;
    *dt_used = v;
}

static int default_patch_rows(int my)
{
    // about two row tasks per patch, at least 16 rows
    int rows = 16;
    while (rows < 128 && rows * 2 < my) rows *= 2;
    return rows;
}

}  // namespace mc

using namespace mc;

struct mc_batch {
    mc_problem proto;
    int npatch;
    long long x_offset;
    std::vector<mc_patch> host_patches;
    std::vector<PatchDesc> desc;
    std::vector<long long> prefix;
    PatchDesc* d_patches = nullptr;
    CUtensorMap* d_maps = nullptr;
    long long* d_prefix = nullptr;
    unsigned int* d_done = nullptr;
    unsigned long long* d_next = nullptr;
    int* d_status = nullptr;
    unsigned long long* d_smax = nullptr;
    double* d_dt = nullptr;         // npatch x nsteps (dt used)
    double* d_dtcur = nullptr;      // npatch (plain form)
    int cap_steps = 0;              // nsteps the smax / dt arrays hold
    int blocks = 0;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_steps = -1;
    double exec_cfl = 0.0;
    cudaGraphExec_t exec_ps = nullptr;   // the one-launch-per-step form
    int exec_ps_steps = -1;
    double exec_ps_cfl = 0.0;
    int stall_patch = -1;           // fault injection for the next advance
};

// Uploads the patch descriptors; with stall >= 0 that patch's descriptor
// claims one task more than the work tables hand out, so its next-step tasks
// wait for a completion that never comes.
static cudaError_t upload_desc(mc_batch* b, int stall)
{
    std::vector<PatchDesc> d = b->desc;
    if (stall >= 0) d[stall].ntasks += 1;
    return cudaMemcpy(b->d_patches, d.data(), sizeof(PatchDesc) * b->npatch, cudaMemcpyHostToDevice);
}

static cudaError_t solver_batch_launch(const BatchLaunch& L)
{
    switch (L.proto.solver) {
    case MC_ACOUSTICS: return batch_launch_acoustics(L);
    case MC_SWE_ROE: return batch_launch_swe(L);
    case MC_ADVECTION: return batch_launch_advection(L);
    case MC_ACOUSTICS_VAR: return batch_launch_acoustics_var(L);
    case MC_EULER_GODUNOV: return batch_launch_euler_godunov(L);
    default: return batch_launch_euler(L);
    }
}

static cudaError_t solver_batch_init(const BatchLaunch& L)
{
    switch (L.proto.solver) {
    case MC_ACOUSTICS: return batch_init_acoustics(L);
    case MC_SWE_ROE: return batch_init_swe(L);
    case MC_ADVECTION: return batch_init_advection(L);
    case MC_ACOUSTICS_VAR: return batch_init_acoustics_var(L);
    case MC_EULER_GODUNOV: return batch_init_euler_godunov(L);
    default: return batch_init_euler(L);
    }
}

static cudaError_t solver_batch_occupancy(const mc_problem& p, int* ctas)
{
    switch (p.solver) {
    case MC_ACOUSTICS: return batch_occupancy_acoustics(p.dtype, ctas);
    case MC_SWE_ROE: return batch_occupancy_swe(p.dtype, ctas);
    case MC_ADVECTION: return batch_occupancy_advection(p.dtype, ctas);
    case MC_ACOUSTICS_VAR: return batch_occupancy_acoustics_var(p.dtype, ctas);
    case MC_EULER_GODUNOV: return batch_occupancy_euler_godunov(p.dtype, ctas);
    default: return batch_occupancy_euler(p.dtype, ctas);
    }
}

// dynamic shared-memory limits of the per-patch (plain) form's fused step
static cudaError_t solver_sweep_prepare(const mc_problem& p)
{
    switch (p.solver) {
    case MC_ACOUSTICS: return sweep_prepare_acoustics(p.dtype);
    case MC_SWE_ROE: return sweep_prepare_swe(p.dtype);
    case MC_ADVECTION: return sweep_prepare_advection(p.dtype);
    case MC_ACOUSTICS_VAR: return sweep_prepare_acoustics_var(p.dtype);
    case MC_EULER_GODUNOV: return sweep_prepare_euler_godunov(p.dtype);
    default: return sweep_prepare_euler(p.dtype);
    }
}

static void drop_exec(mc_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->exec_ps) cudaGraphExecDestroy(b->exec_ps);
    b->exec = b->exec_ps = nullptr;
    b->exec_steps = b->exec_ps_steps = -1;
}

static void free_batch(mc_batch* b)
{
    drop_exec(b);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->d_patches);
    cudaFree(b->d_maps);
    cudaFree(b->d_prefix);
    cudaFree(b->d_done);
    cudaFree(b->d_next);
    cudaFree(b->d_status);
    cudaFree(b->d_smax);
    cudaFree(b->d_dt);
    cudaFree(b->d_dtcur);
    delete b;
}

static mc_status upload_tables(mc_batch* b)
{
    b->prefix.assign(b->npatch + 1, 0);
    for (int p = 0; p < b->npatch; p++) b->prefix[p + 1] = b->prefix[p] + b->desc[p].ntasks;
    cudaError_t e = cudaMemcpy(b->d_patches, b->desc.data(), sizeof(PatchDesc) * b->npatch,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_prefix, b->prefix.data(), sizeof(long long) * (b->npatch + 1),
                       cudaMemcpyHostToDevice);
    drop_exec(b);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "uploading patch tables");
}

static mc_status ensure_steps(mc_batch* b, int nsteps)
{
    if (nsteps <= b->cap_steps) return MC_OK;
    cudaFree(b->d_smax);
    cudaFree(b->d_dt);
    cudaFree(b->d_next);
    b->d_smax = nullptr;
    b->d_dt = nullptr;
    b->d_next = nullptr;
    cudaError_t e = cudaMalloc(&b->d_smax, sizeof(unsigned long long) * (size_t)b->npatch * (nsteps + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_dt, sizeof(double) * (size_t)b->npatch * nsteps);
    // one work counter per launch of the one-launch-per-step form
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned long long) * (size_t)nsteps);
    if (e != cudaSuccess) return cuda_error(e, "allocating per-step arrays");
    b->cap_steps = nsteps;
    drop_exec(b);
    return MC_OK;
}

static BatchLaunch make_launch(mc_batch* b, int nsteps, double cfl, cudaStream_t s)
{
    BatchLaunch L;
    L.proto = b->proto;
    L.patches = b->d_patches;
    L.maps = b->d_maps;
    L.prefix = b->d_prefix;
    L.npatch = b->npatch;
    L.nsteps = nsteps;
    L.step0 = 0;
    L.nsteps_all = nsteps;
    L.tasks_per_step = b->prefix[b->npatch];
    L.x_offset = b->x_offset;
    L.cfl = cfl;
    L.smax = b->d_smax;
    L.dt_used = b->d_dt;
    L.done = b->d_done;
    L.next_item = b->d_next;
    L.status = b->d_status;
    L.blocks = b->blocks;
    L.stream = s;
    return L;
}

static mc_status finish(mc_batch* b, int nsteps, double* t_out, cudaStream_t s)
{
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "batched advance");
    if (status & ST_BADARG) return set_error(MC_EINVAL, "misaligned tensor map or box");
    if (status & ST_TIMEOUT) return set_error(MC_ETIMEOUT, "a bounded patch wait gave up");
    if (status & ST_NONPHYS) return set_error(MC_ENONPHYS, "non-physical state in a patch");
    if (t_out) {
        std::vector<double> dts((size_t)b->npatch * nsteps);
        e = cudaMemcpy(dts.data(), b->d_dt, sizeof(double) * dts.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_error(e, "reading time steps");
        for (int p = 0; p < b->npatch; p++) {
            double t = 0.0;
            for (int k = 0; k < nsteps; k++) t += dts[(size_t)p * nsteps + k];
            t_out[p] = t;
        }
    }
    return MC_OK;
}

extern "C" {

mc_status mc_batch_create(const mc_problem* proto, const mc_patch* patches, int32_t npatch,
                          mc_batch** out)
{
    if (!out || !proto || !patches) return set_error(MC_EINVAL, "NULL argument");
    *out = nullptr;
    if (npatch < 1 || npatch > (1 << 20)) return set_error(MC_EINVAL, "npatch out of range");
    for (int k = 0; k < 4; k++)
        if (proto->bc[k] != MC_BC_WALL)
            return set_error(MC_ENOTSUP, "batched patches support reflecting walls only");
    if (proto->solver == MC_ACOUSTICS_VAR)
        return set_error(MC_ENOTSUP, "batched patches do not carry material planes");
    mc_batch* b = new (std::nothrow) mc_batch();
    if (!b) return set_error(MC_ENOMEM, "batch allocation failed");
    b->proto = *proto;
    b->npatch = npatch;
    b->host_patches.assign(patches, patches + npatch);
    b->desc.resize(npatch);
    for (int p = 0; p < npatch; p++) {
        const mc_patch& P = patches[p];
        mc_problem q = *proto;
        q.mx = P.mx;
        q.my = P.my;
        q.dx = P.dx;
        q.dy = P.dy;
        mc_layout lay;
        mc_status st = mc_layout_of(&q, &lay);
        if (st != MC_OK) {
            free_batch(b);
            return set_error(st, "patch %d: %s", p, "invalid size or spacing");
        }
        if (P.mx < 4 || P.my < 4) {
            free_batch(b);
            return set_error(MC_EINVAL, "patch %d smaller than 4 x 4", p);
        }
        if (!P.qa || !P.qb || P.qa == P.qb || reinterpret_cast<uintptr_t>(P.qa) % 16 ||
            reinterpret_cast<uintptr_t>(P.qb) % 16) {
            free_batch(b);
            return set_error(MC_EINVAL, "patch %d: two distinct 16-byte aligned buffers needed", p);
        }
        b->x_offset = lay.x_offset;
        PatchDesc& d = b->desc[p];
        d.qa = P.qa;
        d.qb = P.qb;
        d.ld_x = lay.ld_x;
        d.ld_field = lay.ld_field;
        d.dx = P.dx;
        d.dy = P.dy;
        d.mx = P.mx;
        d.my = P.my;
        d.tile_rows = default_patch_rows(P.my);
        d.ntasks = ntasks_for(q, d.tile_rows, &d.nbands);
        d.pad = 0;
    }
    cudaError_t e = cudaMalloc(&b->d_patches, sizeof(PatchDesc) * npatch);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * 2 * npatch);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_prefix, sizeof(long long) * (npatch + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(unsigned int) * npatch);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_dtcur, sizeof(double) * npatch);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_error(e, "batch allocation");
    }
    // tensor maps of both buffers of every patch
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
        free_batch(b);
        return set_error(MC_ECUDA, "driver entry point cuTensorMapEncodeTiled unavailable");
    }
    EncodeFn encode = reinterpret_cast<EncodeFn>(fn);
    const int es = proto->dtype == MC_F64 ? 8 : 4;
    const int meqn = solver_meqn(proto->solver);
    std::vector<CUtensorMap> maps(2 * (size_t)npatch);
    for (int p = 0; p < npatch; p++) {
        const PatchDesc& d = b->desc[p];
        cuuint64_t dims[3] = {(cuuint64_t)d.ld_x, (cuuint64_t)(d.my + 4), (cuuint64_t)meqn};
        cuuint64_t strides[2] = {(cuuint64_t)(d.ld_x * es), (cuuint64_t)(d.ld_field * es)};
        cuuint32_t box[3] = {(cuuint32_t)box_w(es), (cuuint32_t)stage_rows(es), (cuuint32_t)meqn};
        cuuint32_t estr[3] = {1, 1, 1};
        for (int k = 0; k < 2; k++) {
            CUresult r = encode(&maps[2 * p + k],
                                es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                3, k ? d.qb : d.qa, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                free_batch(b);
                return set_error(MC_ECUDA, "cuTensorMapEncodeTiled failed for patch %d (%d)", p, (int)r);
            }
        }
    }
    e = cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
    int ctas = 0, dev = 0, sms = 0;
    if (e == cudaSuccess) e = solver_batch_occupancy(*proto, &ctas);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = solver_sweep_prepare(*proto);   // the plain form's smem limits
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_error(e, "batch set-up");
    }
    b->blocks = (ctas > 0 ? ctas : 1) * sms;
    mc_status st = upload_tables(b);
    if (st != MC_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return MC_OK;
}

mc_status mc_batch_destroy(mc_batch* b)
{
    if (b) free_batch(b);
    return MC_OK;
}

mc_status mc_batch_set_tile_rows(mc_batch* b, const int32_t* rows)
{
    if (!b || !rows) return set_error(MC_EINVAL, "NULL argument");
    for (int p = 0; p < b->npatch; p++) {
        if (rows[p] < 1 || rows[p] > 4096) return set_error(MC_EINVAL, "patch %d: rows out of range", p);
    }
    for (int p = 0; p < b->npatch; p++) {
        mc_problem q = b->proto;
        q.mx = b->desc[p].mx;
        q.my = b->desc[p].my;
        b->desc[p].tile_rows = rows[p];
        b->desc[p].ntasks = ntasks_for(q, rows[p], &b->desc[p].nbands);
    }
    return upload_tables(b);
}

mc_status mc_batch_advance(mc_batch* b, int32_t nsteps, double cfl, double* t_out,
                           int* result_in_b, void* stream)
{
    if (!b) return set_error(MC_EINVAL, "NULL batch");
    if (nsteps < 1 || nsteps > 100000) return set_error(MC_EINVAL, "nsteps out of range");
    if (!(cfl > 0.0 && cfl <= 1.0)) return set_error(MC_EINVAL, "need 0 < cfl <= 1");
    mc_status st = ensure_steps(b, nsteps);
    if (st != MC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->exec || b->exec_steps != nsteps || b->exec_cfl != cfl) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_error(e, "begin capture");
        BatchLaunch L = make_launch(b, nsteps, cfl, b->capture);
        cudaError_t e2 = cudaMemsetAsync(b->d_smax, 0,
                                         sizeof(unsigned long long) * (size_t)b->npatch * (nsteps + 1),
                                         b->capture);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * b->npatch, b->capture);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), b->capture);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->capture);
        if (e2 == cudaSuccess) e2 = solver_batch_init(L);
        if (e2 == cudaSuccess) e2 = solver_batch_launch(L);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->capture, &graph);
        if (e2 != cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_error(e, "capturing the batched step");
        }
        b->exec_steps = nsteps;
        b->exec_cfl = cfl;
    }
    const int stall = b->stall_patch;
    b->stall_patch = -1;
    cudaError_t e = cudaSuccess;
    if (stall >= 0) e = upload_desc(b, stall);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_error(e, "batched graph launch");
    st = finish(b, nsteps, t_out, s);
    if (stall >= 0) {
        cudaError_t e2 = upload_desc(b, -1);
        if (e2 != cudaSuccess && st == MC_OK) st = cuda_error(e2, "restoring patch descriptors");
    }
    if (st == MC_OK && result_in_b) *result_in_b = nsteps & 1;
    return st;
}

mc_status mc_batch_advance_steps(mc_batch* b, int32_t nsteps, double cfl, double* t_out,
                                 int* result_in_b, void* stream)
{
    if (!b) return set_error(MC_EINVAL, "NULL batch");
    if (nsteps < 1 || nsteps > 100000) return set_error(MC_EINVAL, "nsteps out of range");
    if (!(cfl > 0.0 && cfl <= 1.0)) return set_error(MC_EINVAL, "need 0 < cfl <= 1");
    mc_status st = ensure_steps(b, nsteps);
    if (st != MC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->exec_ps || b->exec_ps_steps != nsteps || b->exec_ps_cfl != cfl) {
        if (b->exec_ps) cudaGraphExecDestroy(b->exec_ps);
        b->exec_ps = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_error(e, "begin capture");
        BatchLaunch L = make_launch(b, nsteps, cfl, b->capture);
        cudaError_t e2 = cudaMemsetAsync(b->d_smax, 0,
                                         sizeof(unsigned long long) * (size_t)b->npatch * (nsteps + 1),
                                         b->capture);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * b->npatch, b->capture);
        if (e2 == cudaSuccess)
            e2 = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long) * (size_t)nsteps, b->capture);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->capture);
        if (e2 == cudaSuccess) e2 = solver_batch_init(L);
        // one launch per step over all patches, each with its own counter
        L.nsteps = 1;
        for (int k = 0; k < nsteps && e2 == cudaSuccess; k++) {
            L.step0 = k;
            e2 = solver_batch_launch(L);
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->capture, &graph);
        if (e2 != cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec_ps, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec_ps = nullptr;
            return cuda_error(e, "capturing the per-step launches");
        }
        b->exec_ps_steps = nsteps;
        b->exec_ps_cfl = cfl;
    }
    cudaError_t e = cudaGraphLaunch(b->exec_ps, s);
    if (e != cudaSuccess) return cuda_error(e, "per-step graph launch");
    st = finish(b, nsteps, t_out, s);
    if (st == MC_OK && result_in_b) *result_in_b = nsteps & 1;
    return st;
}

mc_status mc_batch_inject_stall(mc_batch* b, int32_t patch)
{
    if (!b) return set_error(MC_EINVAL, "NULL batch");
    if (patch < 0 || patch >= b->npatch) return set_error(MC_EINVAL, "patch %d out of range", patch);
    b->stall_patch = patch;
    return MC_OK;
}

mc_status mc_batch_advance_plain(mc_batch* b, int32_t nsteps, double cfl, double* t_out,
                                 int* result_in_b, void* stream)
{
    if (!b) return set_error(MC_EINVAL, "NULL batch");
    if (nsteps < 1 || nsteps > 100000) return set_error(MC_EINVAL, "nsteps out of range");
    if (!(cfl > 0.0 && cfl <= 1.0)) return set_error(MC_EINVAL, "need 0 < cfl <= 1");
    mc_status st = ensure_steps(b, nsteps);
    if (st != MC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchLaunch L = make_launch(b, nsteps, cfl, s);
    cudaError_t e = cudaMemsetAsync(b->d_smax, 0, sizeof(unsigned long long) * (size_t)b->npatch * (nsteps + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = solver_batch_init(L);
    if (e != cudaSuccess) return cuda_error(e, "plain batch set-up");
    const int stride = nsteps + 1;
    for (int k = 0; k < nsteps && e == cudaSuccess; k++) {
        for (int p = 0; p < b->npatch && e == cudaSuccess; p++) {
            const PatchDesc& d = b->desc[p];
            mc_problem q = b->proto;
            q.mx = d.mx;
            q.my = d.my;
            q.dx = d.dx;
            q.dy = d.dy;
            mc_layout lay;
            mc_layout_of(&q, &lay);
            void* qin = (k & 1) ? d.qb : d.qa;
            void* qout = (k & 1) ? d.qa : d.qb;
            unsigned long long* sm = b->d_smax + (size_t)p * stride;
            patch_dt_kernel<<<1, 1, 0, s>>>(sm + k, cfl, b->d_dtcur + p, b->d_dt + (size_t)p * nsteps + k);
            e = cudaGetLastError();
            if (e == cudaSuccess && k > 0) e = bc_launch(q, lay, qin, qin, nullptr, s);
            if (e != cudaSuccess) break;
            SweepLaunch S{q, lay, b->d_maps + 2 * p + (k & 1), b->d_maps + 2 * p + (k & 1), qin, qout,
                          nullptr, b->d_dtcur + p, 0.0, sm + k + 1, b->d_status, d.tile_rows, 0, s};
            switch (q.solver) {
            case MC_ACOUSTICS: e = sweep_launch_acoustics(S); break;
            case MC_SWE_ROE: e = sweep_launch_swe(S); break;
            case MC_ADVECTION: e = sweep_launch_advection(S); break;
            case MC_ACOUSTICS_VAR: e = sweep_launch_acoustics_var(S); break;
            case MC_EULER_GODUNOV: e = sweep_launch_euler_godunov(S); break;
            default: e = sweep_launch_euler(S); break;
            }
        }
    }
    if (e != cudaSuccess) return cuda_error(e, "per-patch launches");
    st = finish(b, nsteps, t_out, s);
    if (st == MC_OK && result_in_b) *result_in_b = nsteps & 1;
    return st;
}

}  // extern "C"
