// mc_batch.cuh -- many uneven patches advanced together in one persistent
// launch (batched form of the fused step).
//
// The paper motivates this with its execution model (§1.2): larger threads
// schedule pieces of work to finer-grained ones, and each refined grid keeps
// its own time step ("local precision with minimal effects to global time
// stepping"; Table 1, dynamic time stepping).  Here every patch is an
// independent grid with reflecting walls and its own dt = cfl / smax of its
// previous step.  Work items are (step, patch, task) in step-major order,
// handed out by one global counter; a task of step s waits (bounded) until all
// tasks of step s-1 of its patch are done, which also makes the ping-pong
// buffers safe to overwrite.  Because items are taken in increasing order,
// every item a task waits for was taken earlier by a running warp, so the
// scheme cannot deadlock whatever the grid size.  Ghost cells of the next
// step are written by the tasks themselves (wall epilogue of sweep_task).
#pragma once

#include "mc_sweep.cuh"

namespace mc {

constexpr int BC_WALL_KIND = 2;   // reflecting wall in bc_map's numbering

struct PatchDesc {
    void* qa;
    void* qb;
    long long ld_x, ld_field;
    double dx, dy;
    int mx, my, nbands, tile_rows, ntasks, pad;
};

template <class RP>
struct BatchArgs {
    RP rp;
    const PatchDesc* patches;
    const CUtensorMap* maps;        // two per patch: [2p] of qa, [2p + 1] of qb
    const long long* prefix;        // npatch + 1 cumulative task counts
    int npatch, nsteps;             // steps of this launch
    int step0, nsteps_all;          // its first step; steps of the whole advance
    long long tasks_per_step;
    long long x_offset;
    double cfl;
    int limiter, order, transverse;
    unsigned long long* smax;       // npatch x (nsteps_all + 1): [p][0] initial cell speeds, [p][s+1] step s
    double* dt_used;                // npatch x nsteps_all
    unsigned int* done;             // npatch: tasks completed so far
    unsigned long long* next_item;  // work counters, one per launch (indexed by step0)
    int* status;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until *counter >= target (acquire); false after WAIT_CYCLES.
__device__ __forceinline__ bool wait_counter(const unsigned* counter, unsigned target)
{
    if (ld_acquire_u32(counter) >= target) return true;
    const long long t0 = clock64();
    unsigned ns = 32;
    while (ld_acquire_u32(counter) < target) {
        if (clock64() - t0 > WAIT_CYCLES) return false;
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
    return true;
}

template <class RP, int MODE>
__global__ void __launch_bounds__(SWEEP_WARPS * 32, min_ctas<RP>::value) batch_sweep_kernel(const BatchArgs<RP> a)
{
    using T = typename RP::real;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    WarpRing W = warp_ring(smem, sizeof(T), RP::NPLANE);
    const bool second = a.order >= 2;
    // items of this launch: steps [step0, step0 + nsteps), in step order
    const long long first = (long long)a.step0 * a.tasks_per_step;
    const long long total = first + (long long)a.nsteps * a.tasks_per_step;
    const int stride = a.nsteps_all + 1;
    bool dep_failed = false, tma_failed = false, bad = false;

    for (;;) {
        long long item = 0;
        if (lane == 0) item = first + (long long)atomicAdd(&a.next_item[a.step0], 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int s = int(item / a.tasks_per_step);
        const long long r = item - (long long)s * a.tasks_per_step;
        int lo = 0, hi = a.npatch;   // prefix[lo] <= r < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.prefix[mid] <= r) lo = mid;
            else hi = mid;
        }
        const int p = lo;
        const int t = int(r - a.prefix[p]);
        const PatchDesc d = a.patches[p];
        if (s > 0) {
            int ok = 1;
            if (lane == 0) ok = wait_counter(&a.done[p], unsigned(s) * unsigned(d.ntasks));
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                dep_failed = true;   // between tasks: no copies in flight
                break;
            }
        }
        // the previous step's stores (generic proxy, acquired above) must be
        // visible to this task's TMA reads (async proxy)
        fence_proxy_async_global();
        const double sprev = __longlong_as_double((long long)__ldcg(&a.smax[(long long)p * stride + s]));
        const double dt = sprev > 0.0 ? a.cfl / sprev : 0.0;
        const int cur = s & 1;
        const CUtensorMap* map = a.maps + 2 * p + cur;
        T* qout = static_cast<T*>(cur ? d.qa : d.qb);
        if ((reinterpret_cast<uintptr_t>(map) & 63) != 0) {
            if (lane == 0) atomicOr(a.status, ST_BADARG);
            break;
        }
        if (lane == 0) acquire_tensormap(map);
        __syncwarp();
        const int i0 = (t % d.nbands) * BAND_W;
        const int j0 = (t / d.nbands) * d.tile_rows;
        const int jend = min(j0 + d.tile_rows, d.my);
        T smx = T(0), smy = T(0);
        if (!sweep_task<RP, true, MODE>(a.rp, map, qout, d.mx, d.my, d.ld_x, d.ld_field, a.x_offset, i0,
                                  j0, jend, T(dt / d.dx), T(dt / d.dy), a.limiter, second, a.transverse,
                                  W, bad, smx, smy, a.status)) {
            tma_failed = true;
            break;
        }
        double v = fmax(double(smx) / d.dx, double(smy) / d.dy);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) {
            atomic_max_nonneg(&a.smax[(long long)p * stride + s + 1], v);
            if (t == 0) a.dt_used[(long long)p * a.nsteps_all + s] = dt;
            __threadfence();
            atomicAdd(&a.done[p], 1u);
        }
        __syncwarp();
    }
    if (tma_failed) drain_ring(W);
    if ((tma_failed || dep_failed) && lane == 0) atomicOr(a.status, ST_TIMEOUT);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, ST_NONPHYS);
}

// Initial ghost fill (walls) and cell-speed maximum of every patch: a row
// of gridDim.x blocks per patch (patches beyond gridDim.y wrap around),
// which share its ghost cells and its rows.
template <class RP>
__global__ void batch_init_kernel(const RP rp, const PatchDesc* patches, int npatch,
                                  long long x_offset, int stride, unsigned long long* smax)
{
    using T = typename RP::real;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int wid = blockIdx.x * nw + (threadIdx.x >> 5), nwarp = gridDim.x * nw;
    for (int pi = blockIdx.y; pi < npatch; pi += gridDim.y) {
        const PatchDesc d = patches[pi];
        T* q = static_cast<T*>(d.qa);
        // ghosts: x of interior rows, then y over the full width (corners)
        const int W = d.mx + 4;
        const int nghost = 4 * W + 4 * d.my;
        for (int g = tid; g < nghost; g += nthr) {
            int i, j;
            if (g < 4 * W) {
                const int jr = g / W;
                j = jr < 2 ? jr - 2 : d.my + jr - 2;
                i = g - jr * W - 2;
            } else {
                const int u = g - 4 * W;
                j = u >> 2;
                const int ir = u & 3;
                i = ir < 2 ? ir - 2 : d.mx + ir - 2;
            }
            bool fx = false, fy = false;
            const int si = bc_map(i, d.mx, BC_WALL_KIND, BC_WALL_KIND, fx);
            const int sj = bc_map(j, d.my, BC_WALL_KIND, BC_WALL_KIND, fy);
            for (int m = 0; m < RP::NPLANE; m++) {
                T v = q[m * d.ld_field + (long long)(sj + 2) * d.ld_x + x_offset + si];
                if ((m == 1 && fx) || (m == 2 && fy)) v = -v;
                q[m * d.ld_field + (long long)(j + 2) * d.ld_x + x_offset + i] = v;
            }
        }
        // cell-speed maxima (see max_cell_speed_kernel): warps take rows
        T msx = T(0), msy = T(0);
        for (int j = wid; j < d.my; j += nwarp) {
            const T* row = q + (long long)(j + 2) * d.ld_x + x_offset;
            for (int i = lane; i < d.mx; i += 32) {
                T qq[RP::NPLANE];
                for (int m = 0; m < RP::NPLANE; m++) qq[m] = row[m * d.ld_field + i];
                T sx, sy;
                rp.cell_speeds(qq, sx, sy);
                msx = fmax(msx, sx);
                msy = fmax(msy, sy);
            }
        }
        double v = fmax(double(msx) / d.dx, double(msy) / d.dy);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomic_max_nonneg(&smax[(long long)pi * stride], v);
    }
}

}  // namespace mc
