// mc_capi.cu -- the C ABI of the wave-propagation library (include/manyclaw.h):
// problem validation and layout, contexts, tensor maps, the CUDA-graph step
// loop with the device-side time-step rule, host<->device copies.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "mc_internal.h"
#include "mc_sweep.cuh"
#include "mc_tile.h"

namespace mc {

static thread_local char g_msg[512] = "";
static thread_local int g_last = MC_OK;

mc_status set_error(mc_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    g_last = st;
    return st;
}

mc_status cuda_error(cudaError_t e, const char* what)
{
    return set_error(e == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

int ntasks_for(const mc_problem& p, int tile_rows, int* nbands)
{
    const int nb = (p.mx + BAND_W - 1) / BAND_W;
    const int nr = (p.my + tile_rows - 1) / tile_rows;
    *nbands = nb;
    return nb * nr;
}

int ntasks_split(const mc_problem& p, int tile_rows, int split, int* nbands, int* nbig)
{
    if (split <= 0) {
        *nbig = 0;
        return ntasks_for(p, tile_rows, nbands);
    }
    const int nb = (p.mx + BAND_W - 1) / BAND_W;
    *nbands = nb;
    *nbig = nb * (split / (TALL_TILES * tile_rows));
    return *nbig + nb * ((p.my - split + tile_rows - 1) / tile_rows);
}

static int meqn_of(int solver) { return solver_meqn(solver); }

static mc_status validate(const mc_problem* p)
{
    if (!p) return set_error(MC_EINVAL, "problem is NULL");
    if (p->solver < MC_ACOUSTICS || p->solver > MC_EULER_GODUNOV)
        return set_error(MC_EINVAL, "unknown solver %d", p->solver);
    if (p->dtype != MC_F32 && p->dtype != MC_F64)
        return set_error(MC_EINVAL, "unknown dtype %d", p->dtype);
    if (p->mx < 1 || p->my < 1 || p->mx > (1 << 28) || p->my > (1 << 28))
        return set_error(MC_EINVAL, "grid %d x %d out of range", p->mx, p->my);
    if ((long long)p->mx * p->my > (1LL << 40))
        return set_error(MC_EINVAL, "grid %d x %d too large", p->mx, p->my);
    if (p->mbc != 2) return set_error(MC_EINVAL, "mbc must be 2 (got %d)", p->mbc);
    if (p->limiter < MC_LIM_NONE || p->limiter > MC_LIM_MC)
        return set_error(MC_EINVAL, "unknown limiter %d", p->limiter);
    if (p->order != 1 && p->order != 2) return set_error(MC_EINVAL, "order must be 1 or 2");
    if (p->transverse < 0 || p->transverse > 2)
        return set_error(MC_EINVAL, "transverse must be 0, 1 or 2");
    if (p->efix != 0 && p->efix != 1) return set_error(MC_EINVAL, "efix must be 0 or 1");
    for (int k = 0; k < 4; k++)
        if (p->bc[k] < MC_BC_PERIODIC || p->bc[k] > MC_BC_GIVEN)
            return set_error(MC_EINVAL, "unknown boundary kind %d on side %d", p->bc[k], k);
    for (int k = 0; k < 4; k++)
        if (p->bc[k] == MC_BC_GIVEN && (p->mx < 2 || p->my < 2))
            return set_error(MC_EINVAL, "a grid with caller-filled ghost sides needs at least 2 x 2 cells");
    if ((p->bc[0] == MC_BC_PERIODIC) != (p->bc[1] == MC_BC_PERIODIC) ||
        (p->bc[2] == MC_BC_PERIODIC) != (p->bc[3] == MC_BC_PERIODIC))
        return set_error(MC_EINVAL, "periodic boundaries must be paired");
    if (!(p->dx > 0.0) || !(p->dy > 0.0) || !isfinite(p->dx) || !isfinite(p->dy))
        return set_error(MC_EINVAL, "cell sizes must be positive");
    if (p->solver == MC_ACOUSTICS && !(p->param[0] > 0.0 && p->param[1] > 0.0))
        return set_error(MC_EINVAL, "acoustics needs rho > 0 and K > 0");
    if (p->solver == MC_SWE_ROE && !(p->param[0] > 0.0))
        return set_error(MC_EINVAL, "shallow water needs g > 0");
    if ((p->solver == MC_EULER_ROE || p->solver == MC_EULER_GODUNOV) && !(p->param[0] > 1.0))
        return set_error(MC_EINVAL, "Euler needs gamma > 1");
    if (p->solver == MC_ADVECTION && !(isfinite(p->param[0]) && isfinite(p->param[1])))
        return set_error(MC_EINVAL, "advection needs finite velocities");
    return MC_OK;
}

static void layout_unchecked(const mc_problem* p, mc_layout* L)
{
    const int es = p->dtype == MC_F64 ? 8 : 4;
    L->elem_bytes = es;
    L->meqn = meqn_of(p->solver);
    L->x_offset = 16 / es;
    const long long row = L->x_offset + p->mx + 2;
    const long long pad = 128 / es;
    L->ld_x = (row + pad - 1) / pad * pad;
    L->ld_field = L->ld_x * (long long)(p->my + 4);
    L->bytes = L->meqn * L->ld_field * es;
}

static cudaError_t sweep_launch(const SweepLaunch& L)
{
    switch (L.prob.solver) {
    case MC_ACOUSTICS: return sweep_launch_acoustics(L);
    case MC_SWE_ROE: return sweep_launch_swe(L);
    case MC_ADVECTION: return sweep_launch_advection(L);
    case MC_ACOUSTICS_VAR: return sweep_launch_acoustics_var(L);
    case MC_EULER_GODUNOV: return sweep_launch_euler_godunov(L);
    default: return sweep_launch_euler(L);
    }
}

static cudaError_t sweep_prepare(const mc_problem& p)
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

// resident CTAs per SM of the problem's fused step (1 if unknown)
static int sweep_ctas_per_sm(const mc_problem& p)
{
    int ctas = 0;
    cudaError_t e;
    switch (p.solver) {
    case MC_ACOUSTICS: e = sweep_occupancy_acoustics(p, &ctas); break;
    case MC_SWE_ROE: e = sweep_occupancy_swe(p, &ctas); break;
    case MC_ADVECTION: e = sweep_occupancy_advection(p, &ctas); break;
    case MC_ACOUSTICS_VAR: e = sweep_occupancy_acoustics_var(p, &ctas); break;
    case MC_EULER_GODUNOV: e = sweep_occupancy_euler_godunov(p, &ctas); break;
    default: e = sweep_occupancy_euler(p, &ctas); break;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    return ctas > 0 ? ctas : 1;
}

static cudaError_t maxspeed_launch(const mc_problem& p, const mc_layout& lay, const void* q,
                                   unsigned long long* out, cudaStream_t s)
{
    switch (p.solver) {
    case MC_ACOUSTICS: return maxspeed_launch_acoustics(p, lay, q, out, s);
    case MC_SWE_ROE: return maxspeed_launch_swe(p, lay, q, out, s);
    case MC_ADVECTION: return maxspeed_launch_advection(p, lay, q, out, s);
    case MC_ACOUSTICS_VAR: return maxspeed_launch_acoustics_var(p, lay, q, out, s);
    case MC_EULER_GODUNOV: return maxspeed_launch_euler_godunov(p, lay, q, out, s);
    default: return maxspeed_launch_euler(p, lay, q, out, s);
    }
}

static bool has_given_side(const mc_problem& p)
{
    for (int k = 0; k < 4; k++)
        if (p.bc[k] == MC_BC_GIVEN) return true;
    return false;
}

cudaError_t bc_launch(const mc_problem& p, const mc_layout& lay, void* qa, void* qb,
                      const int* cur_dev, cudaStream_t s)
{
    if (has_given_side(p)) {
        // leave the caller's sides alone: x ghosts of the interior rows, then
        // y ghosts across the full width, physical sides only
        cudaError_t e = bc_dir_launch(p, lay, qa, qb, cur_dev, 0, s);
        return e == cudaSuccess ? bc_dir_launch(p, lay, qa, qb, cur_dev, 1, s) : e;
    }
    const long long total = 4LL * (p.mx + 4) + 4LL * p.my;
    int blocks = int((total + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    if (p.dtype == MC_F64) {
        BcArgs<double> a{static_cast<double*>(qa), static_cast<double*>(qb), cur_dev, p.mx, p.my,
                         (int)lay.meqn, lay.ld_x, lay.ld_field, lay.x_offset,
                         {p.bc[0], p.bc[1], p.bc[2], p.bc[3]}};
        bc_fill_kernel<double><<<blocks, 256, 0, s>>>(a);
    } else {
        BcArgs<float> a{static_cast<float*>(qa), static_cast<float*>(qb), cur_dev, p.mx, p.my,
                        (int)lay.meqn, lay.ld_x, lay.ld_field, lay.x_offset,
                        {p.bc[0], p.bc[1], p.bc[2], p.bc[3]}};
        bc_fill_kernel<float><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// Time-step rule of one attempt, run by one thread after the fused step:
// Courant number = dt * smax; reject (retake with dt = cfl_desired / smax)
// above cfl_max, otherwise accept (advance t, flip the buffer index) and
// propose dt = cfl_desired / smax.  Resets smax for the next attempt.
// The speed maximum is the context's own (smax_ext null) or a caller's
// device scalar, e.g. the maximum over the blocks of a decomposed grid.
__global__ void dt_update_kernel(DevState* st, double cfl_desired, double cfl_max,
                                 unsigned long long* smax_ext)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    dt_rule_apply(st, cfl_desired, cfl_max, smax_ext ? smax_ext : &st->smax_bits);
}

// Default rows per warp task: enough tasks to fill the GPU several times
// over, with short tiles only where the grid is small.  A grid whose 8-row
// tasks do not even fill one wave of CTAs (SWEEP_WARPS warps on every SM)
// takes the shortest tiles that still fit in one wave: such a step is
// latency-bound (a warp marches its rows one after another, rows + 3
// iterations), so fewer rows per task shorten it.  Measured on the 128^2
// FP64 acoustics step: 2 rows 39 us, 8 rows 78 us.
static int default_tile_rows(const mc_problem& p)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = 8LL * sms * SWEEP_WARPS;
    const long long nb = (p.mx + BAND_W - 1) / BAND_W;
    auto tasks = [&](int rows) { return nb * ((p.my + rows - 1) / rows); };
    int rows = DEFAULT_TILE_ROWS;
    while (rows > 8 && tasks(rows) < want) rows /= 2;
    const long long wave = (long long)sms * SWEEP_WARPS;
    if (rows == 8 && tasks(8) <= wave)
        while (rows > 1 && tasks(rows - 1) <= wave) rows--;
    return rows;
}

// Rows [0, split) of the default layout go in tasks of TALL_TILES tiles
// (fewer halo rows re-read: a task of r rows marches r + 3), the rest in
// tasks of tile rows, launched last: on a grid with several waves of tasks
// the last wave is then made of short tasks, so the SMs finish together.
// The short part holds about one wave (the kernel's resident warps on every
// SM); grids of fewer than four waves keep uniform tiles (split 0).
static int default_tile_split(const mc_problem& p, int rows, int sms, int ctas_per_sm)
{
    const long long nb = (p.mx + BAND_W - 1) / BAND_W;
    const long long wave = (long long)ctas_per_sm * (sms > 0 ? sms : 152) * SWEEP_WARPS;
    if (nb * ((p.my + rows - 1) / rows) < 4 * wave) return 0;
    long long shortr = (wave * rows + nb - 1) / nb;            // rows of about one wave
    shortr = (shortr + rows - 1) / rows * rows;
    long long split = (long long)p.my - shortr;
    split = split / (TALL_TILES * rows) * (TALL_TILES * rows);
    return split > 0 ? int(split) : 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct MapEntry {
    const void* ptr;
    int slot;      // index in the context's device array of tensor maps
};
constexpr int MAP_SLOTS = 16;

struct GraphEntry {
    const void* qa;
    const void* qb;
    int nsteps;
    double cfl_desired, cfl_max;
    cudaGraphExec_t exec;
};

}  // namespace mc

using namespace mc;

struct mc_ctx {
    mc_problem p;
    mc_layout lay;
    int tile_rows;
    int tile_split = 0;            // rows in tasks of TALL_TILES tiles (default layout), or 0
    int ctas_per_sm = 1;           // resident CTAs of the fused step's kernel
    DevState* dev;                 // device scratch: time-step scalars and status
    CUtensorMap* dmaps;            // device array of MAP_SLOTS tensor maps
    cudaStream_t capture;          // private stream used to capture graphs
    EncodeTiledFn encode;
    std::vector<MapEntry> maps;
    std::vector<GraphEntry> graphs;
    int next_slot;
    const mc_mlp* seed_net = nullptr;   // pressure seeds of the exact-solution solver, or none
    int sms = 0;                        // SMs of the context's device
    int* gq_tasks = nullptr;            // task list of the FP64 guard's queue (FP32 pair solvers)
    int gq_cap = 0;
};

// FP32 shallow-water and Euler steps carry the FP64 guard
static bool has_guard(const mc_problem& p)
{
    return p.dtype == MC_F32 && (p.solver == MC_SWE_ROE || p.solver == MC_EULER_ROE);
}

// The guard queue's task list holds one entry per task of the current tile
// shape; without it the guard kernel recomputes every task of a step that
// queued one.
static void ensure_guard_list(mc_ctx* c)
{
    if (!has_guard(c->p)) return;
    int nb = 0, nbig = 0;
    const int need = ntasks_split(c->p, c->tile_rows, c->tile_split, &nb, &nbig);
    if (need <= c->gq_cap) return;
    if (c->gq_tasks) cudaFree(c->gq_tasks);
    c->gq_tasks = nullptr;
    c->gq_cap = 0;
    if (cudaMalloc(&c->gq_tasks, sizeof(int) * (size_t)need) == cudaSuccess) c->gq_cap = need;
    else (void)cudaGetLastError();
}

// the context's extras for every fused-step launch
static void launch_extras(const mc_ctx* c, SweepLaunch& L)
{
    L.seed_net = c->seed_net ? c->seed_net->dev : nullptr;
    L.newton = c->dev->newton;
    L.guard = &c->dev->guard;
    if (has_guard(c->p)) {
        L.gq = &c->dev->gq;
        L.gq_tasks = c->gq_tasks;
    }
    L.sms = c->sms;
    L.tile_split = c->tile_split;
}

static void drop_graphs(mc_ctx* c)
{
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

// Device pointer to the tensor map of state buffer q; a buffer seen for the
// first time gets its map encoded on the host and copied (synchronously)
// into a slot of the context's device array.
static mc_status get_map(mc_ctx* c, const void* q, const CUtensorMap** out)
{
    for (auto& e : c->maps)
        if (e.ptr == q) {
            *out = c->dmaps + e.slot;
            return MC_OK;
        }
    if (reinterpret_cast<uintptr_t>(q) % 16 != 0)
        return set_error(MC_EINVAL, "state pointer %p is not 16-byte aligned", q);
    const int es = (int)c->lay.elem_bytes;
    cuuint64_t dims[3] = {(cuuint64_t)c->lay.ld_x, (cuuint64_t)(c->p.my + 4),
                          (cuuint64_t)c->lay.meqn};
    cuuint64_t strides[2] = {(cuuint64_t)(c->lay.ld_x * es), (cuuint64_t)(c->lay.ld_field * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_w(es), (cuuint32_t)stage_rows(es),
                         (cuuint32_t)c->lay.meqn};
    cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap host_map;
    CUresult r = c->encode(&host_map,
                           es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           3, const_cast<void*>(q), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(MC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    MapEntry e{q, 0};
    if ((int)c->maps.size() >= MAP_SLOTS) {
        // reuse the oldest slot; cached graphs may point at it
        e.slot = c->maps.front().slot;
        c->maps.erase(c->maps.begin());
        drop_graphs(c);
    } else {
        e.slot = c->next_slot++;
    }
    cudaError_t ce = cudaMemcpy(c->dmaps + e.slot, &host_map, sizeof(CUtensorMap),
                                cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_error(ce, "uploading a tensor map");
    c->maps.push_back(e);
    *out = c->dmaps + e.slot;
    return MC_OK;
}

extern "C" {

const char* mc_status_string(int status)
{
    switch (status) {
    case MC_OK: return "MC_OK";
    case MC_EINVAL: return "MC_EINVAL: invalid argument";
    case MC_ECUDA: return "MC_ECUDA: CUDA call failed";
    case MC_ENOMEM: return "MC_ENOMEM: allocation failed";
    case MC_ECFL: return "MC_ECFL: step rejected (Courant number too large)";
    case MC_ENONPHYS: return "MC_ENONPHYS: non-physical state";
    case MC_ETIMEOUT: return "MC_ETIMEOUT: bounded device wait gave up";
    case MC_ENOTSUP: return "MC_ENOTSUP: not supported";
    default: return "unknown status";
    }
}

int mc_last_error(char* buf, size_t n)
{
    if (buf && n) {
        strncpy(buf, g_msg, n - 1);
        buf[n - 1] = '\0';
    }
    return g_last;
}

mc_status mc_layout_of(const mc_problem* p, mc_layout* out)
{
    mc_status st = validate(p);
    if (st != MC_OK) return st;
    if (!out) return set_error(MC_EINVAL, "layout output is NULL");
    layout_unchecked(p, out);
    return MC_OK;
}

mc_status mc_create(const mc_problem* p, mc_ctx** out)
{
    if (!out) return set_error(MC_EINVAL, "output is NULL");
    *out = nullptr;
    mc_status st = validate(p);
    if (st != MC_OK) return st;
    mc_ctx* c = new (std::nothrow) mc_ctx();
    if (!c) return set_error(MC_ENOMEM, "context allocation failed");
    c->p = *p;
    layout_unchecked(p, &c->lay);
    c->tile_rows = default_tile_rows(*p);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            c->sms = 0;
    }

    cudaError_t e = cudaMalloc(&c->dev, sizeof(DevState));
    if (e != cudaSuccess) {
        delete c;
        return cuda_error(e, "cudaMalloc(device state)");
    }
    e = cudaMalloc(&c->dmaps, sizeof(CUtensorMap) * MAP_SLOTS);
    if (e != cudaSuccess) {
        cudaFree(c->dev);
        delete c;
        return cuda_error(e, "cudaMalloc(tensor maps)");
    }
    e = cudaMemset(c->dev, 0, sizeof(DevState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = sweep_prepare(c->p);
    if (e != cudaSuccess) {
        cudaFree(c->dmaps);
        cudaFree(c->dev);
        delete c;
        return cuda_error(e, "context set-up");
    }
    c->ctas_per_sm = sweep_ctas_per_sm(c->p);
    c->tile_split = default_tile_split(c->p, c->tile_rows, c->sms, c->ctas_per_sm);
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        cudaStreamDestroy(c->capture);
        cudaFree(c->dmaps);
        cudaFree(c->dev);
        delete c;
        return set_error(MC_ECUDA, "driver entry point cuTensorMapEncodeTiled unavailable");
    }
    c->encode = reinterpret_cast<EncodeTiledFn>(fn);
    ensure_guard_list(c);
    *out = c;
    return MC_OK;
}

mc_status mc_destroy(mc_ctx* c)
{
    if (!c) return MC_OK;
    drop_graphs(c);
    cudaStreamDestroy(c->capture);
    cudaFree(c->dmaps);
    cudaFree(c->dev);
    if (c->gq_tasks) cudaFree(c->gq_tasks);
    delete c;
    return MC_OK;
}

mc_status mc_set_tile_rows(mc_ctx* c, int rows)
{
    if (!c) return set_error(MC_EINVAL, "context is NULL");
    int split = 0;
    if (rows == 0) {
        rows = default_tile_rows(c->p);
        split = default_tile_split(c->p, rows, c->sms, c->ctas_per_sm);
    }
    if (rows < 1 || rows > 4096) return set_error(MC_EINVAL, "tile rows %d out of range", rows);
    if (rows != c->tile_rows || split != c->tile_split) drop_graphs(c);
    c->tile_rows = rows;
    c->tile_split = split;
    ensure_guard_list(c);
    return MC_OK;
}

mc_status mc_set_seed_net(mc_ctx* c, const mc_mlp* net)
{
    if (!c) return set_error(MC_EINVAL, "context is NULL");
    if (net && c->p.solver != MC_EULER_GODUNOV)
        return set_error(MC_ENOTSUP, "pressure seeds apply to the exact-solution Euler solver only");
    if (net != c->seed_net) drop_graphs(c);   // captured launches hold the old pointer
    c->seed_net = net;
    return MC_OK;
}

mc_status mc_newton_stats(mc_ctx* c, int64_t* updates, int64_t* solves, int32_t reset, void* stream)
{
    if (!c || !updates || !solves) return set_error(MC_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, c->dev->newton, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(c->dev->newton, 0, sizeof(h), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "Newton counters");
    *updates = (int64_t)h[0];
    *solves = (int64_t)h[1];
    return MC_OK;
}

mc_status mc_guard_stats(mc_ctx* c, int64_t* edges, int32_t reset, void* stream)
{
    if (!c || !edges) return set_error(MC_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, &c->dev->guard, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(&c->dev->guard, 0, sizeof(h), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "guard counter");
    *edges = (int64_t)h;
    return MC_OK;
}

static mc_status copy_dense(mc_ctx* c, const void* src, void* dst, bool upload, cudaStream_t s)
{
    const long long es = c->lay.elem_bytes;
    const size_t width = (size_t)c->p.mx * es;
    for (int m = 0; m < c->lay.meqn; m++) {
        const long long dense_off = (long long)m * c->p.mx * c->p.my * es;
        const long long lay_off = (m * c->lay.ld_field + 2 * c->lay.ld_x + c->lay.x_offset) * es;
        cudaError_t e;
        if (upload)
            e = cudaMemcpy2DAsync(static_cast<char*>(dst) + lay_off, c->lay.ld_x * es,
                                  static_cast<const char*>(src) + dense_off, width, width, c->p.my,
                                  cudaMemcpyHostToDevice, s);
        else
            e = cudaMemcpy2DAsync(static_cast<char*>(dst) + dense_off, width,
                                  static_cast<const char*>(src) + lay_off, c->lay.ld_x * es, width,
                                  c->p.my, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_error(e, upload ? "upload" : "download");
    }
    return MC_OK;
}

mc_status mc_upload(mc_ctx* c, const void* host_dense, void* q_dev, void* stream)
{
    if (!c || !host_dense || !q_dev) return set_error(MC_EINVAL, "NULL argument");
    return copy_dense(c, host_dense, q_dev, true, static_cast<cudaStream_t>(stream));
}

mc_status mc_download(mc_ctx* c, const void* q_dev, void* host_dense, void* stream)
{
    if (!c || !host_dense || !q_dev) return set_error(MC_EINVAL, "NULL argument");
    return copy_dense(c, q_dev, host_dense, false, static_cast<cudaStream_t>(stream));
}

mc_status mc_repack(mc_ctx* c, const void* src, void* dst, int32_t to_layout, void* stream)
{
    if (!c || !src || !dst) return set_error(MC_EINVAL, "NULL argument");
    if (src == dst) return set_error(MC_EINVAL, "src and dst must differ");
    cudaError_t e = dense_repack_launch(c->p, c->lay, src, dst, to_layout != 0,
                                        c->sms > 0 ? c->sms : 152, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "repack launch");
}

mc_status mc_bc_fill(mc_ctx* c, void* q, void* stream)
{
    if (!c || !q) return set_error(MC_EINVAL, "NULL argument");
    cudaError_t e = bc_launch(c->p, c->lay, q, q, nullptr, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "ghost fill launch");
}

mc_status mc_bc_fill_dir(mc_ctx* c, void* q, int32_t dir, void* stream)
{
    if (!c || !q) return set_error(MC_EINVAL, "NULL argument");
    if (dir != 0 && dir != 1) return set_error(MC_EINVAL, "direction must be 0 (x) or 1 (y)");
    cudaError_t e = bc_dir_launch(c->p, c->lay, q, q, nullptr, dir, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "directional ghost fill launch");
}

mc_status mc_halo_elems(const mc_problem* p, int32_t side, int64_t* elems)
{
    if (!elems) return set_error(MC_EINVAL, "NULL argument");
    mc_status st = validate(p);
    if (st != MC_OK) return st;
    if (side < 0 || side > 3) return set_error(MC_EINVAL, "side must be 0..3");
    if (p->mx < 2 || p->my < 2) return set_error(MC_EINVAL, "halo strips need at least 2 x 2 cells");
    *elems = halo_elems(*p, side);
    return MC_OK;
}

static mc_status halo_call(mc_ctx* c, const void* src, void* dst, int32_t side, bool pack,
                           void* stream)
{
    if (!c || !src || !dst) return set_error(MC_EINVAL, "NULL argument");
    if (side < 0 || side > 3) return set_error(MC_EINVAL, "side must be 0..3");
    if (c->p.mx < 2 || c->p.my < 2) return set_error(MC_EINVAL, "halo strips need at least 2 x 2 cells");
    cudaError_t e = halo_launch(c->p, c->lay, src, dst, side, pack, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, pack ? "halo pack launch" : "halo unpack launch");
}

mc_status mc_halo_pack(mc_ctx* c, const void* q, int32_t side, void* buf, void* stream)
{
    return halo_call(c, q, buf, side, true, stream);
}

mc_status mc_halo_unpack(mc_ctx* c, const void* buf, int32_t side, void* q, void* stream)
{
    return halo_call(c, buf, q, side, false, stream);
}

static mc_status read_status(mc_ctx* c, DevState* h, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(h, c->dev, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "reading device state");
    if (h->status & ST_BADARG)
        return set_error(MC_EINVAL, "the fused step found a misaligned tensor map or box");
    if (h->status & ST_TIMEOUT) return set_error(MC_ETIMEOUT, "a bounded device wait gave up");
    if (h->status & ST_NONPHYS)
        return set_error(MC_ENONPHYS, "non-physical state (depth/density <= 0 or NaN) met");
    return MC_OK;
}

}  // extern "C"

namespace mc {
cudaError_t encode_state_map(CUtensorMap* out, const void* q, int es, int nplane, long long ld_x, int my,
                             long long ld_field)
{
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &qr);
        if (e != cudaSuccess) return e;
        if (qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    cuuint64_t dims[3] = {(cuuint64_t)ld_x, (cuuint64_t)(my + 4), (cuuint64_t)nplane};
    cuuint64_t strides[2] = {(cuuint64_t)(ld_x * es), (cuuint64_t)(ld_field * es)};
    cuuint32_t box[3] = {(cuuint32_t)box_w(es), (cuuint32_t)stage_rows(es), (cuuint32_t)nplane};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(out, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                        const_cast<void*>(q), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

mc_status ctx_check_status(mc_ctx* c, void* stream)
{
    DevState h;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    mc_status st = read_status(c, &h, s);
    if (h.status) cudaMemsetAsync(&c->dev->status, 0, sizeof(int), s);
    return st;
}
}  // namespace mc

extern "C" {

mc_status mc_step(mc_ctx* c, void* q_in, void* q_out, double dt, double* smax_out, void* stream)
{
    if (!c || !q_in || !q_out) return set_error(MC_EINVAL, "NULL argument");
    if (q_in == q_out) return set_error(MC_EINVAL, "q_in and q_out must differ");
    if (!(dt >= 0.0) || !isfinite(dt)) return set_error(MC_EINVAL, "dt must be finite and >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const CUtensorMap* map;
    mc_status st = get_map(c, q_in, &map);
    if (st != MC_OK) return st;
    if (reinterpret_cast<uintptr_t>(q_out) % 16 != 0)
        return set_error(MC_EINVAL, "q_out is not 16-byte aligned");
    cudaError_t e = bc_launch(c->p, c->lay, q_in, q_in, nullptr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->dev->smax_bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_error(e, "step set-up");
    SweepLaunch L{c->p, c->lay, map, map, q_in, q_out, nullptr, nullptr, dt,
                  &c->dev->smax_bits, &c->dev->status, c->tile_rows, 0, s};
    launch_extras(c, L);
    e = sweep_launch(L);
    if (e != cudaSuccess) return cuda_error(e, "sweep launch");
    if (smax_out) {
        DevState h;
        st = read_status(c, &h, s);
        *smax_out = __builtin_bit_cast(double, h.smax_bits);
        if (st != MC_OK) {
            cudaMemsetAsync(&c->dev->status, 0, sizeof(int), s);
            return st;
        }
    }
    return MC_OK;
}

mc_status mc_sweep(mc_ctx* c, const void* q_in, void* q_out, double dt, void* stream)
{
    if (!c || !q_in || !q_out) return set_error(MC_EINVAL, "NULL argument");
    if (q_in == q_out) return set_error(MC_EINVAL, "q_in and q_out must differ");
    if (!(dt >= 0.0) || !isfinite(dt)) return set_error(MC_EINVAL, "dt must be finite and >= 0");
    if (reinterpret_cast<uintptr_t>(q_out) % 16 != 0)
        return set_error(MC_EINVAL, "q_out is not 16-byte aligned");
    const CUtensorMap* map;
    mc_status st = get_map(c, q_in, &map);
    if (st != MC_OK) return st;
    SweepLaunch L{c->p, c->lay, map, map, const_cast<void*>(q_in), q_out, nullptr, nullptr, dt,
                  &c->dev->smax_bits, &c->dev->status, c->tile_rows, 0,
                  static_cast<cudaStream_t>(stream)};
    launch_extras(c, L);
    cudaError_t e = sweep_launch(L);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "sweep launch");
}

mc_status mc_max_cell_speed(mc_ctx* c, const void* q, double* smax_out, void* stream)
{
    if (!c || !q || !smax_out) return set_error(MC_EINVAL, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long* d = &c->dev->smax_bits;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), s);
    if (e == cudaSuccess) e = maxspeed_launch(c->p, c->lay, q, d, s);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(*d), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "cell-speed reduction");
    *smax_out = __builtin_bit_cast(double, h);
    return MC_OK;
}

// enqueue `attempts` step attempts (ghost fill, fused step, time-step rule)
static cudaError_t enqueue_attempts(mc_ctx* c, const CUtensorMap* ma, const CUtensorMap* mb,
                                    void* qa, void* qb, int attempts, double cfl_desired,
                                    double cfl_max, cudaStream_t s)
{
    SweepLaunch L{c->p, c->lay, ma, mb, qa, qb, &c->dev->cur, &c->dev->dt, 0.0,
                  &c->dev->smax_bits, &c->dev->status, c->tile_rows, 0, s};
    launch_extras(c, L);
    // where the FP64 guard's kernel follows the step, it applies the rule
    // (one launch fewer per attempt)
    bool folded = false;
    L.dt_state = c->dev;
    L.cfl_desired = cfl_desired;
    L.cfl_max = cfl_max;
    L.dt_folded = &folded;
    for (int k = 0; k < attempts; k++) {
        cudaError_t e = bc_launch(c->p, c->lay, qa, qb, &c->dev->cur, s);
        if (e == cudaSuccess) e = sweep_launch(L);
        if (e != cudaSuccess) return e;
        if (!folded) {
            dt_update_kernel<<<1, 32, 0, s>>>(c->dev, cfl_desired, cfl_max, nullptr);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// cached graph of `len` attempts for this buffer pair and CFL pair
static mc_status get_graph(mc_ctx* c, const CUtensorMap* ma, const CUtensorMap* mb, void* qa,
                           void* qb, int len, double cfl_desired, double cfl_max,
                           cudaGraphExec_t* out)
{
    for (auto& g : c->graphs)
        if (g.qa == qa && g.qb == qb && g.nsteps == len && g.cfl_desired == cfl_desired &&
            g.cfl_max == cfl_max) {
            *out = g.exec;
            return MC_OK;
        }
    cudaError_t e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "begin capture");
    cudaError_t e2 = enqueue_attempts(c, ma, mb, qa, qb, len, cfl_desired, cfl_max, c->capture);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->capture, &graph);
    if (e2 != cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "capturing the step graph");
    if (c->graphs.size() >= 8) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({qa, qb, len, cfl_desired, cfl_max, exec});
    *out = exec;
    return MC_OK;
}

mc_status mc_advance(mc_ctx* c, void* qa, void* qb, int nsteps, double cfl_desired,
                     double cfl_max, double* t_inout, double* dt_inout, int* result_in_b,
                     int* nrejected, void* stream)
{
    if (!c || !qa || !qb || !t_inout || !dt_inout || !result_in_b)
        return set_error(MC_EINVAL, "NULL argument");
    if (qa == qb) return set_error(MC_EINVAL, "qa and qb must differ");
    if (has_given_side(c->p))
        return set_error(MC_EINVAL, "sides of kind MC_BC_GIVEN need their ghosts written before "
                         "every step: use mc_step");
    if (nsteps < 0 || nsteps > 1000000) return set_error(MC_EINVAL, "nsteps out of range");
    if (!(cfl_desired > 0.0) || !(cfl_max >= cfl_desired))
        return set_error(MC_EINVAL, "need 0 < cfl_desired <= cfl_max");
    if (!(*dt_inout > 0.0) || !isfinite(*dt_inout)) return set_error(MC_EINVAL, "dt must be > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const CUtensorMap *ma, *mb;
    mc_status st = get_map(c, qa, &ma);
    if (st == MC_OK) st = get_map(c, qb, &mb);
    if (st != MC_OK) return st;

    DevState h;
    memset(&h, 0, sizeof(h));
    h.dt = *dt_inout;
    h.t = *t_inout;
    cudaError_t e = cudaMemcpyAsync(c->dev, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "device state upload");

    if (nsteps > 0) {
        // The attempt sequence runs as graphs of up to GRAPH_CHUNK attempts,
        // launched back to back; dt, t and the buffer index stay on the device.
        const int chunk = nsteps < GRAPH_CHUNK ? nsteps : GRAPH_CHUNK;
        const int full = nsteps / chunk, rest = nsteps - full * chunk;
        for (int part = 0; part < 2; part++) {
            const int len = part == 0 ? chunk : rest;
            const int times = part == 0 ? full : (rest > 0 ? 1 : 0);
            if (times == 0) continue;
            cudaGraphExec_t exec = nullptr;
            st = get_graph(c, ma, mb, qa, qb, len, cfl_desired, cfl_max, &exec);
            if (st != MC_OK) return st;
            for (int k = 0; k < times; k++) {
                e = cudaGraphLaunch(exec, s);
                if (e != cudaSuccess) return cuda_error(e, "graph launch");
            }
        }
        st = read_status(c, &h, s);
        // rejected attempts: retake one at a time until nsteps are accepted
        int extra = 0;
        while (st == MC_OK && h.nacc < nsteps) {
            if (++extra > 10 * nsteps + 10) {
                st = set_error(MC_ECFL, "step rejected repeatedly (Courant %.3g)", h.cfl_last);
                break;
            }
            e = enqueue_attempts(c, ma, mb, qa, qb, 1, cfl_desired, cfl_max, s);
            if (e != cudaSuccess) return cuda_error(e, "retake");
            st = read_status(c, &h, s);
        }
        if (st != MC_OK) {
            cudaMemsetAsync(&c->dev->status, 0, sizeof(int), s);
            return st;
        }
    }
    *t_inout = h.t;
    *dt_inout = h.dt;
    *result_in_b = h.cur;
    if (nrejected) *nrejected = h.nrej;
    return MC_OK;
}

// ---- A block of a decomposed grid stepped with its time-step state on the
// device: dt, t, the buffer index and the counters live in the context's
// device state between mc_block_begin and mc_block_end, so a rank enqueues
// attempt after attempt (halo exchange, step, a max-reduction of the speed
// maximum over the ranks, the dt rule) without reading anything back.

mc_status mc_block_begin(mc_ctx* c, double t, double dt, void* stream)
{
    if (!c) return set_error(MC_EINVAL, "NULL context");
    if (!(dt > 0.0) || !isfinite(dt) || !isfinite(t)) return set_error(MC_EINVAL, "need finite t and dt > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevState h;
    memset(&h, 0, sizeof(h));
    h.dt = dt;
    h.t = t;
    // the counters of the other entry points stay as they were
    cudaError_t e = cudaMemcpyAsync(c->dev, &h, offsetof(DevState, newton), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "block state upload");
}

mc_status mc_block_pack(mc_ctx* c, const void* qa, const void* qb, int32_t side, void* buf, void* stream)
{
    if (!c || !qa || !qb || !buf) return set_error(MC_EINVAL, "NULL argument");
    if (side < 0 || side > 3) return set_error(MC_EINVAL, "side must be 0..3");
    if (c->p.mx < 2 || c->p.my < 2) return set_error(MC_EINVAL, "halo strips need at least 2 x 2 cells");
    cudaError_t e = halo_launch_cur(c->p, c->lay, const_cast<void*>(qa), const_cast<void*>(qb),
                                    &c->dev->cur, buf, side, true, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "halo pack launch");
}

mc_status mc_block_unpack(mc_ctx* c, const void* buf, int32_t side, void* qa, void* qb, void* stream)
{
    if (!c || !qa || !qb || !buf) return set_error(MC_EINVAL, "NULL argument");
    if (side < 0 || side > 3) return set_error(MC_EINVAL, "side must be 0..3");
    if (c->p.mx < 2 || c->p.my < 2) return set_error(MC_EINVAL, "halo strips need at least 2 x 2 cells");
    cudaError_t e = halo_launch_cur(c->p, c->lay, qa, qb, &c->dev->cur, const_cast<void*>(buf), side,
                                    false, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "halo unpack launch");
}

mc_status mc_block_fill_dir(mc_ctx* c, void* qa, void* qb, int32_t dir, void* stream)
{
    if (!c || !qa || !qb) return set_error(MC_EINVAL, "NULL argument");
    if (dir != 0 && dir != 1) return set_error(MC_EINVAL, "direction must be 0 (x) or 1 (y)");
    cudaError_t e = bc_dir_launch(c->p, c->lay, qa, qb, &c->dev->cur, dir, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MC_OK : cuda_error(e, "directional ghost fill launch");
}

mc_status mc_block_sweep(mc_ctx* c, void* qa, void* qb, uint64_t* smax_dev, void* stream)
{
    if (!c || !qa || !qb || !smax_dev) return set_error(MC_EINVAL, "NULL argument");
    if (qa == qb) return set_error(MC_EINVAL, "qa and qb must differ");
    if (reinterpret_cast<uintptr_t>(qa) % 16 || reinterpret_cast<uintptr_t>(qb) % 16)
        return set_error(MC_EINVAL, "states must be 16-byte aligned");
    const CUtensorMap *ma, *mb;
    mc_status st = get_map(c, qa, &ma);
    if (st == MC_OK) st = get_map(c, qb, &mb);
    if (st != MC_OK) return st;
    SweepLaunch L{c->p, c->lay, ma, mb, qa, qb, &c->dev->cur, &c->dev->dt, 0.0,
                  reinterpret_cast<unsigned long long*>(smax_dev), &c->dev->status, c->tile_rows, 0,
                  static_cast<cudaStream_t>(stream)};
    launch_extras(c, L);
    cudaError_t e = sweep_launch(L);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "sweep launch");
}

mc_status mc_block_dt_rule(mc_ctx* c, uint64_t* smax_dev, double cfl_desired, double cfl_max,
                           void* stream)
{
    if (!c || !smax_dev) return set_error(MC_EINVAL, "NULL argument");
    if (!(cfl_desired > 0.0) || !(cfl_max >= cfl_desired))
        return set_error(MC_EINVAL, "need 0 < cfl_desired <= cfl_max");
    dt_update_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        c->dev, cfl_desired, cfl_max, reinterpret_cast<unsigned long long*>(smax_dev));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MC_OK : cuda_error(e, "dt rule launch");
}

mc_status mc_block_end(mc_ctx* c, double* t, double* dt, int32_t* cur, int32_t* naccepted,
                       int32_t* nrejected, void* stream)
{
    if (!c) return set_error(MC_EINVAL, "NULL context");
    DevState h;
    mc_status st = read_status(c, &h, static_cast<cudaStream_t>(stream));
    if (t) *t = h.t;
    if (dt) *dt = h.dt;
    if (cur) *cur = h.cur;
    if (naccepted) *naccepted = h.nacc;
    if (nrejected) *nrejected = h.nrej;
    if (st != MC_OK) cudaMemsetAsync(&c->dev->status, 0, sizeof(int), static_cast<cudaStream_t>(stream));
    return st;
}

mc_status mc_advance_host(mc_ctx* c, const void* host_q0, void* host_q, void* qa, void* qb,
                          int nsteps, double cfl_desired, double cfl_max, double* t_inout,
                          double* dt_inout, int* nrejected, void* stream)
{
    if (!c || !host_q0 || !host_q || !qa || !qb) return set_error(MC_EINVAL, "NULL argument");
    if (qa == qb) return set_error(MC_EINVAL, "qa and qb must differ");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The buffer that does not hold the state stages it densely, so each
    // direction moves one contiguous block over the host link (a row-pitched
    // copy moves one row at a time) and a kernel repacks it on the device.
    const size_t dense = (size_t)c->lay.meqn * c->p.mx * c->p.my * c->lay.elem_bytes;
    const int sms = c->sms > 0 ? c->sms : 152;
    cudaError_t e = cudaMemcpyAsync(qb, host_q0, dense, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = dense_repack_launch(c->p, c->lay, qb, qa, true, sms, s);
    if (e != cudaSuccess) return cuda_error(e, "upload");
    int inb = 0;
    mc_status st = mc_advance(c, qa, qb, nsteps, cfl_desired, cfl_max, t_inout, dt_inout, &inb,
                              nrejected, stream);
    if (st != MC_OK) return st;
    void* res = inb ? qb : qa;
    void* spare = inb ? qa : qb;
    e = dense_repack_launch(c->p, c->lay, res, spare, false, sms, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_q, spare, dense, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MC_OK : cuda_error(e, "download");
}

}  // extern "C"
