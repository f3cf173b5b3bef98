// mc_multi.cuh -- the fused step over many grids of one size class in one
// launch: every warp task is (grid, band, row tile), mapped from a prefix of
// the grids' task counts; the per-warp march is sweep_task, unchanged.  Used
// for the refined patches of mc_amr_advance, whose ghost layers are filled
// before the launch and all advance by the same dt.
#pragma once

#include "mc_sweep.cuh"

namespace mc {

struct MultiGrid {
    int mx, my, nbands, tile_rows;
    long long ld_x, ld_field;
    void* q[2];
};

template <class RP>
struct MultiArgs {
    RP rp;
    const MultiGrid* grids;
    const CUtensorMap* maps;     // two per grid: [2g] of q[0], [2g + 1] of q[1]
    const long long* prefix;     // ngrid + 1 cumulative task counts
    int ngrid, cur;              // the step reads q[cur] and writes q[cur ^ 1]
    long long total;
    long long x_offset;
    double nux, nuy;             // dt/dx, dt/dy (the same on every grid)
    int limiter, order, transverse;
    int* status;
};

template <class RP, int MODE>
__global__ void __launch_bounds__(SWEEP_WARPS * 32, min_ctas<RP>::value) multi_sweep_kernel(const MultiArgs<RP> a)
{
    using T = typename RP::real;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpRing W = warp_ring(smem, sizeof(T), RP::NPLANE);
    const bool second = a.order >= 2;
    bool failed = false, bad = false;
    for (long long task = (long long)blockIdx.x * SWEEP_WARPS + warp; task < a.total && !failed;
         task += (long long)gridDim.x * SWEEP_WARPS) {
        int lo = 0, hi = a.ngrid;   // prefix[lo] <= task < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.prefix[mid] <= task) lo = mid;
            else hi = mid;
        }
        const MultiGrid g = a.grids[lo];
        const int t = int(task - a.prefix[lo]);
        const CUtensorMap* map = a.maps + 2 * lo + a.cur;
        if ((reinterpret_cast<uintptr_t>(map) & 63) != 0) {
            if (lane == 0) atomicOr(a.status, ST_BADARG);
            break;
        }
        if (lane == 0) acquire_tensormap(map);
        __syncwarp();
        const int i0 = (t % g.nbands) * BAND_W;
        const int j0 = (t / g.nbands) * g.tile_rows;
        const int jend = min(j0 + g.tile_rows, g.my);
        T smx = T(0), smy = T(0);
        failed = !sweep_task<RP, false, MODE>(a.rp, map, static_cast<T*>(g.q[a.cur ^ 1]), g.mx, g.my,
                                              g.ld_x, g.ld_field, a.x_offset, i0, j0, jend, T(a.nux),
                                              T(a.nuy), a.limiter, second, a.transverse, W, bad, smx,
                                              smy, a.status);
    }
    if (failed) {
        drain_ring(W);
        if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, ST_NONPHYS);
}

}  // namespace mc
