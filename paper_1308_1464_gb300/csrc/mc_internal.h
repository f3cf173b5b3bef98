// mc_internal.h -- host-side declarations shared by the library's
// translation units (not part of the public C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/manyclaw.h"

namespace mc {

// planes of a solver's state array (acoustics (p, u, v) and shallow water
// (h, hu, hv): 3; Euler (rho, rho u, rho v, E): 4; advection (q): 1;
// variable-coefficient acoustics (p, u, v, rho, c): 5)
inline int solver_meqn(int solver)
{
    switch (solver) {
    case MC_EULER_ROE:
    case MC_EULER_GODUNOV: return 4;
    case MC_ADVECTION: return 1;
    case MC_ACOUSTICS_VAR: return 5;
    default: return 3;
    }
}

struct DevState;

// One launch of the fused step (and its companions) for one problem.
struct SweepLaunch {
    mc_problem prob;
    mc_layout lay;
    const CUtensorMap* map_a;  // device pointers to 64-byte aligned tensor maps
    const CUtensorMap* map_b;
    void* qa;
    void* qb;
    const int* cur_dev;        // device buffer index, or null (qa -> qb)
    const double* dt_dev;      // device dt, or null (use dt)
    double dt;
    unsigned long long* smax_bits;
    int* status;
    int tile_rows;
    int max_blocks;            // 0: one warp per task
    cudaStream_t stream;
    const void* seed_net = nullptr;            // MlpDev of a pressure-seed network (SEEDED solvers)
    unsigned long long* newton = nullptr;      // Newton update / solve counters, or null
    unsigned long long* guard = nullptr;       // FP64-guard edge counter, or null
    void* gq = nullptr;                        // GuardQueue of the FP64 guard, or null (no guard)
    int* gq_tasks = nullptr;                   // its task list (ntasks entries), or null: all tasks
    // A loop of attempts may fold its time-step rule into the guard kernel:
    // dt_state (the context's DevState) and the CFL pair.  The rule is applied
    // there only when the guard kernel runs; the launch reports in *dt_folded
    // (if given) whether it was, so that the caller applies it otherwise.
    DevState* dt_state = nullptr;
    double cfl_desired = 0.0, cfl_max = 0.0;
    bool* dt_folded = nullptr;
    int tile_split = 0;                        // rows in tasks of TALL_TILES tiles, launched first (0: none)
    int sms = 0;                               // SMs of the device (0: unknown, full CTAs)
};

// One launch of the fused step over many grids (mc_multi.cuh); grids and
// prefix are device arrays (MultiGrid, ngrid + 1 task offsets).
struct MultiLaunch {
    mc_problem prob;             // scheme and parameters (sizes come from the grids)
    const void* grids;
    const CUtensorMap* maps;     // two per grid
    const long long* prefix;
    int ngrid, cur;
    long long total, x_offset;
    double nux, nuy;
    int* status;
    cudaStream_t stream;
};
cudaError_t multi_launch_acoustics(const MultiLaunch& L);
cudaError_t multi_launch_swe(const MultiLaunch& L);
cudaError_t multi_launch_euler(const MultiLaunch& L);
cudaError_t multi_launch_advection(const MultiLaunch& L);
cudaError_t multi_launch_acoustics_var(const MultiLaunch& L);
cudaError_t multi_launch_euler_godunov(const MultiLaunch& L);
// a tensor map of a state array in the library layout (the box of the fused step)
cudaError_t encode_state_map(CUtensorMap* out, const void* q, int elem_bytes, int nplane,
                             long long ld_x, int my, long long ld_field);

// the status word of a context's fused steps (synchronises; cleared after)
mc_status ctx_check_status(mc_ctx* c, void* stream);

// per-solver launchers (mc_sweep_<solver>.cu), dispatching on dtype
cudaError_t sweep_launch_acoustics(const SweepLaunch& L);
cudaError_t sweep_launch_swe(const SweepLaunch& L);
cudaError_t sweep_launch_euler(const SweepLaunch& L);
cudaError_t sweep_launch_advection(const SweepLaunch& L);
cudaError_t sweep_launch_acoustics_var(const SweepLaunch& L);
cudaError_t sweep_launch_euler_godunov(const SweepLaunch& L);
cudaError_t sweep_prepare_acoustics(int dtype);
cudaError_t sweep_prepare_swe(int dtype);
cudaError_t sweep_prepare_euler(int dtype);
cudaError_t sweep_prepare_advection(int dtype);
cudaError_t sweep_prepare_acoustics_var(int dtype);
cudaError_t sweep_prepare_euler_godunov(int dtype);
// resident CTAs per SM of the problem's fused-step kernel (after its prepare)
cudaError_t sweep_occupancy_acoustics(const mc_problem& p, int* ctas);
cudaError_t sweep_occupancy_swe(const mc_problem& p, int* ctas);
cudaError_t sweep_occupancy_euler(const mc_problem& p, int* ctas);
cudaError_t sweep_occupancy_advection(const mc_problem& p, int* ctas);
cudaError_t sweep_occupancy_acoustics_var(const mc_problem& p, int* ctas);
cudaError_t sweep_occupancy_euler_godunov(const mc_problem& p, int* ctas);
cudaError_t maxspeed_launch_acoustics(const mc_problem& p, const mc_layout& lay, const void* q,
                                      unsigned long long* out, cudaStream_t s);
cudaError_t maxspeed_launch_swe(const mc_problem& p, const mc_layout& lay, const void* q,
                                unsigned long long* out, cudaStream_t s);
cudaError_t maxspeed_launch_euler(const mc_problem& p, const mc_layout& lay, const void* q,
                                  unsigned long long* out, cudaStream_t s);
cudaError_t maxspeed_launch_advection(const mc_problem& p, const mc_layout& lay, const void* q,
                                      unsigned long long* out, cudaStream_t s);
cudaError_t maxspeed_launch_acoustics_var(const mc_problem& p, const mc_layout& lay, const void* q,
                                          unsigned long long* out, cudaStream_t s);
cudaError_t maxspeed_launch_euler_godunov(const mc_problem& p, const mc_layout& lay, const void* q,
                                          unsigned long long* out, cudaStream_t s);

// ghost fill (mc_capi.cu)
cudaError_t bc_launch(const mc_problem& p, const mc_layout& lay, void* qa, void* qb,
                      const int* cur_dev, cudaStream_t s);

// halo strips and directional ghost fills of a decomposed grid's block (mc_halo.cu)
long long halo_elems(const mc_problem& p, int side);
cudaError_t halo_launch(const mc_problem& p, const mc_layout& lay, const void* src, void* dst,
                        int side, bool pack, cudaStream_t s);
// the same on q[cur]: qa, or qb when *cur_dev == 1
cudaError_t halo_launch_cur(const mc_problem& p, const mc_layout& lay, void* qa, void* qb,
                            const int* cur_dev, void* buf, int side, bool pack, cudaStream_t s);
// Copies a whole interior between the dense [meqn][my][mx] order (src or
// dst, device memory) and the padded layout; the two must not overlap.
cudaError_t dense_repack_launch(const mc_problem& p, const mc_layout& lay, const void* src,
                                void* dst, bool to_layout, int sms, cudaStream_t s);
cudaError_t bc_dir_launch(const mc_problem& p, const mc_layout& lay, void* qa, void* qb,
                          const int* cur_dev, int dir, cudaStream_t s);

int ntasks_for(const mc_problem& p, int tile_rows, int* nbands);
// tasks of the layout with rows [0, split) in tiles of TALL_TILES tile_rows
// (nbig of them, first) and the rest in tiles of tile_rows; split 0: uniform
int ntasks_split(const mc_problem& p, int tile_rows, int split, int* nbands, int* nbig);

// error reporting
mc_status set_error(mc_status st, const char* fmt, ...);
mc_status cuda_error(cudaError_t e, const char* what);

}  // namespace mc

namespace mc {

struct PatchDesc;

// One launch of the batched persistent step (mc_batch.cu builds it).
struct BatchLaunch {
    mc_problem proto;
    const PatchDesc* patches;
    const CUtensorMap* maps;
    const long long* prefix;
    int npatch, nsteps;
    int step0 = 0, nsteps_all = 0;   // first step of the launch; steps of the whole advance
    long long tasks_per_step;
    long long x_offset;
    double cfl;
    unsigned long long* smax;
    double* dt_used;
    unsigned int* done;
    unsigned long long* next_item;
    int* status;
    int blocks;
    cudaStream_t stream;
};

cudaError_t batch_launch_acoustics(const BatchLaunch& L);
cudaError_t batch_launch_swe(const BatchLaunch& L);
cudaError_t batch_launch_euler(const BatchLaunch& L);
cudaError_t batch_launch_advection(const BatchLaunch& L);
cudaError_t batch_launch_acoustics_var(const BatchLaunch& L);
cudaError_t batch_launch_euler_godunov(const BatchLaunch& L);
cudaError_t batch_init_acoustics(const BatchLaunch& L);
cudaError_t batch_init_swe(const BatchLaunch& L);
cudaError_t batch_init_euler(const BatchLaunch& L);
cudaError_t batch_init_advection(const BatchLaunch& L);
cudaError_t batch_init_acoustics_var(const BatchLaunch& L);
cudaError_t batch_init_euler_godunov(const BatchLaunch& L);
// resident CTAs per SM of the batched kernel (also raises its smem limit)
cudaError_t batch_occupancy_acoustics(int dtype, int* ctas);
cudaError_t batch_occupancy_swe(int dtype, int* ctas);
cudaError_t batch_occupancy_euler(int dtype, int* ctas);
cudaError_t batch_occupancy_advection(int dtype, int* ctas);
cudaError_t batch_occupancy_acoustics_var(int dtype, int* ctas);
cudaError_t batch_occupancy_euler_godunov(int dtype, int* ctas);

}  // namespace mc
